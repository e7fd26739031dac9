"""The plain-PyTorch FP32 operator that bench.py times as a sanity floor
(--torch-floor) computes the same E_c / E_c^H as the FP64 oracle: checked on
the CPU so that its timings compare like with like."""
import numpy as np
import pytest

import oracle as O
from paper_2601_05418_gb300 import synth

torch = pytest.importorskip("torch")


def _rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


@pytest.mark.parametrize("geom", ["2d128", "ragged"])
def test_torch_floor_matches_oracle(geom):
    import bench

    if geom == "2d128":
        g = synth.workload("2d128").geom
    else:  # non-square, several groups, oversampling 3, uniform keep
        g = synth.tiny_geometry(nx=40, ny=36, nz=1, nc=5, os=3, cycles=4.0, kappa_y=1.7, n_groups=3, keep=4,
                                lines="regular", r=2)
    coils = synth.coil_maps(g.nx, g.ny, g.nz, g.nc, 51)
    rho = synth.phantom(g.nx, g.ny, g.nz)
    As, _, _ = O.build_groups(g, coils, synth.roi_mask(rho))
    tf = bench.TorchFloor(g, coils, As, torch.device("cpu"))
    x = synth.complex_normal(g.shape, 52)
    y = tf.E(torch.from_numpy(x.astype(np.complex64))).numpy().astype(np.complex128)
    y_ref = O.Ec_apply(g, coils, As, x)
    assert y.shape == y_ref.shape
    assert _rel(y, y_ref) < 1e-5
    v = synth.complex_normal(y_ref.shape, 53)
    xa = tf.EH(torch.from_numpy(v.astype(np.complex64))).numpy().astype(np.complex128)
    assert _rel(xa, O.EcH_apply(g, coils, As, v)) < 1e-5
