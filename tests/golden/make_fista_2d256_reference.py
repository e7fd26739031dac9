"""Writes the FP64 oracle's reconstruction of the 256x256 FISTA workload
(seeded synthetic slice, oracle-built A_g, oracle compression, 20 power
iterations from E_c^H S', FISTA l1-Haar 50 iterations) to
fista_2d256_ref.npz.  Calls only the oracle and the input generators.

    python tests/golden/make_fista_2d256_reference.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle as O  # noqa: E402
from paper_2601_05418_gb300 import synth  # noqa: E402


def main():
    wl = synth.workload("2d256")
    g = wl.geom
    c = synth.make_case(wl)
    S = O.simulate(g, c.coils, c.rho, c.noise)
    As, evs, _ = O.build_groups(g, c.coils, c.roi)
    Sc = O.compress(g, As, S)
    pb = O.Problem(g, c.coils, As)
    b = pb.EcH(Sc)
    L = O.power_lipschitz(pb.normal_c, b, 20)
    x = O.fista(pb.normal_c, b, L, wl.lam, wl.haar_levels, wl.iters)
    np.savez_compressed(os.path.join(HERE, "fista_2d256_ref.npz"), x=x, L=L,
                        nrmse_vs_phantom=O.nrmse(x, c.rho))
    print("L", L, "nrmse vs phantom", O.nrmse(x, c.rho))


if __name__ == "__main__":
    main()
