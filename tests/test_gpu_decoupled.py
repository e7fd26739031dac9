"""Hybrid-space reconstruction (Sec. 3.4, algorithm #1) on the device.

1. The aliased sets of the mask, computed by the library at plan creation,
   are bit-exact against the oracle's connected components of
   F^H M^T M F (integer bookkeeping): regular masks with and without
   R | N_y, 3x3 CAIPI on a lattice and off it, a variable-density mask.
2. Per-set CG (GPJC_DECOUPLED) against the oracle's per-set CG on the same
   compression matrices and data, FP32 path: images within NRMSE 1e-5 plus
   the element-wise bound (tests/_checks.py), like the global CG.
"""
import numpy as np
import pytest

import oracle as O
from _checks import check_image
from paper_2601_05418_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module")
def gp():
    import __graft_entry__ as ge

    ge.build()
    from paper_2601_05418_gb300 import gpjc

    return gpjc


def to_dev(a, dtype=np.complex64):
    return torch.from_numpy(np.ascontiguousarray(a.astype(dtype))).to(DEV)


def to_np(t):
    return t.detach().cpu().numpy().astype(np.complex128)


def oracle_labels(g):
    sets, _, _ = O.aliased_sets(g)
    lab = np.zeros(g.ny * g.nz, np.int32)
    for k, Y in enumerate(sorted(sets, key=min)):
        lab[np.asarray(Y)] = k
    return len(sets), lab


def geoms():
    out = {}
    for r in (2, 3, 4):
        out[f"2d64_R{r}"] = synth._geom_2d(64, 8, 4, 8, 2.5, 16, 4.0, r)
    out["2d128_R3"] = synth.workload("2d128").geom  # 128 / 3: no lattice, one set
    g = synth._geom_2d(64, 8, 4, 8, 2.5, 16, 4.0, 3)
    g.line_ky, g.line_kz = synth.lines_variable_density(64, 3.0, 81, center=12)
    out["2d64_vd"] = g  # random samples: no lattice, one set
    # 3x3 CAIPI closes into a lattice when N_y is a multiple of 3 and N_z of 9
    out["3d_caipi_lattice"] = synth.geom_3d(24, 24, 18, 4, 4, 3, 1.5, 1.1, 8, 8.0)
    out["3d56_caipi"] = synth.workload("3d56").geom
    return out


@pytest.mark.parametrize("name", list(geoms().keys()))
def test_aliased_sets_bit_exact(gp, name):
    g = geoms()[name]
    n, lab = gp.Plan(g).sets()
    n_ref, lab_ref = oracle_labels(g)
    assert n == n_ref
    assert np.array_equal(lab, lab_ref)
    if name.startswith("2d64_R") and 64 % int(name[-1]) == 0:
        assert n == 64 // int(name[-1])  # R-row sets
    if name == "3d_caipi_lattice":
        assert n == 24 * 18 // 9  # nine rows per set


@pytest.mark.parametrize("name,iters", [("2d64_R4", 12), ("2d64_R2", 6), ("3d_caipi_lattice", 10)])
def test_decoupled_cg_matches_oracle(gp, name, iters):
    g = geoms()[name]
    coils = synth.coil_maps(g.nx, g.ny, g.nz, g.nc, 82)
    rho = synth.phantom(g.nx, g.ny, g.nz)
    roi = synth.roi_mask(rho)
    As, _, _ = O.build_groups(g, coils, roi)
    S = O.simulate(g, coils, rho, synth.complex_normal((g.n_lines, g.nc, g.ntx), 83, 1e-3))
    Sc = O.compress(g, As, S)
    x_ref = O.decoupled_cg(g, coils, As, Sc, iters)
    op = gp.Operator(gp.Groups.from_matrices(gp.Plan(g), As), to_dev(coils))
    x, info = op.recon(to_dev(Sc), alg=gp.DECOUPLED, iters=iters, history=True)
    assert info["status"] == 0
    check_image(to_np(x), x_ref, 1e-5, f"decoupled CG {name}")
    # the per-set iterates differ from the global CG's when there are several sets
    n_sets, _ = gp.Plan(g).sets()
    if n_sets > 1:
        pb = O.Problem(g, coils, As)
        x_glob, _ = O.cg(pb.normal_c, pb.EcH(Sc), iters)
        assert O.nrmse(x_glob, x_ref) > 1e-5


def test_decoupled_with_one_set_is_the_global_cg(gp):
    """128 rows with R = 3 form one aliased set: the decoupled loop then runs
    the global CG's recurrences."""
    g = geoms()["2d128_R3"]
    coils = synth.coil_maps(g.nx, g.ny, g.nz, g.nc, 84)
    rho = synth.phantom(g.nx, g.ny, g.nz)
    As, _, _ = O.build_groups(g, coils, synth.roi_mask(rho))
    Sc = O.compress(g, As, O.simulate(g, coils, rho, synth.complex_normal((g.n_lines, g.nc, g.ntx), 85, 1e-3)))
    op = gp.Operator(gp.Groups.from_matrices(gp.Plan(g), As), to_dev(coils))
    xd, _ = op.recon(to_dev(Sc), alg=gp.DECOUPLED, iters=15)
    xc, _ = op.recon(to_dev(Sc), alg=gp.CG, iters=15)
    pb = O.Problem(g, coils, As)
    x_ref, _ = O.cg(pb.normal_c, pb.EcH(Sc), 15)
    check_image(to_np(xd), x_ref, 1e-5, "decoupled, one set")
    check_image(to_np(xc), x_ref, 1e-5, "global CG")
