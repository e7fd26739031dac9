"""Tensor-core (tcgen05) compression and operator: BF16 / FP16 operands,
FP32 accumulation, against the FP64 oracle.

Tolerances.  FP16 rounds each operand once (relative error 2^-12); a
contraction over N_s terms with random phases keeps the relative error of
each output at that order, so single FP16 applications are held to a
relative L2 error of 2e-3.  BF16 carries every operand as a head and a
remainder (both BF16, three MMAs per K step), so each product keeps about
2 x 8 mantissa bits (relative error ~2^-16 plus the dropped
remainder x remainder term, ~2^-18): single BF16 applications are held to
1e-4.  Images: the compressed hybrid data entering A_g^H are always split
into two 16-bit parts; both formats are held to the NRMSE 1e-3 bar of the
16-bit path against the FP64 oracle.  Every check also bounds the largest
element error (tests/_checks.py).
"""
import numpy as np
import pytest

import oracle as O
from _checks import check_close, check_image
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




TOL = {1: 1e-4, 2: 2e-3}  # BF16 (split), FP16: single applications
IMG = {1: 1e-3, 2: 1e-3}  # BF16, FP16: reconstructed images


def geoms():
    return {"2d128": synth.workload("2d128").geom, "3d56": synth.workload("3d56").geom,
            "2d64": synth._geom_2d(64, 8, 4, 8, 2.5, 16, 8.0, 3)}


def case(g, seed):
    coils = synth.coil_maps(g.nx, g.ny, g.nz, g.nc, seed)
    rho = synth.phantom(g.nx, g.ny, g.nz)
    return coils, rho, synth.roi_mask(rho)


@pytest.mark.parametrize("prec", [1, 2])
@pytest.mark.parametrize("name", ["2d128", "3d56"])
def test_tc_compress_matches_oracle(gp, name, prec):
    g = geoms()[name]
    coils, rho, roi = case(g, 41)
    As, _, _ = O.build_groups(g, coils, roi)
    S = synth.complex_normal((g.n_lines, g.nc, g.ntx), 42)
    grp = gp.Groups.from_matrices(gp.Plan(g), As)
    Sc = to_np(gp.compress(grp, to_dev(S), prec))
    check_close(Sc, O.compress(g, As, S), TOL[prec])


@pytest.mark.parametrize("prec", [1, 2])
@pytest.mark.parametrize("name", ["2d128", "3d56"])
def test_tc_operator_matches_oracle(gp, name, prec):
    g = geoms()[name]
    coils, rho, roi = case(g, 43)
    As, _, _ = O.build_groups(g, coils, roi)
    op = gp.Operator(gp.Groups.from_matrices(gp.Plan(g), As), to_dev(coils), prec)
    x = synth.complex_normal(g.shape, 44)
    y = to_np(op.E(to_dev(x)))
    y_ref = O.Ec_apply(g, coils, As, x)
    check_close(y, y_ref, TOL[prec])
    v = synth.complex_normal(y_ref.shape, 45)
    xa = to_np(op.EH(to_dev(v)))
    check_close(xa, O.EcH_apply(g, coils, As, v), TOL[prec])


def test_tc_unsupported_group_map_is_rejected(gp):
    g = synth.tiny_geometry(nx=40, ny=36, nz=1, nc=5, os=3, cycles=4.0, kappa_y=1.7, n_groups=3,
                            lines="regular", r=2)
    coils, rho, roi = case(g, 46)
    As, _, _ = O.build_groups(g, coils, roi)
    grp = gp.Groups.from_matrices(gp.Plan(g), As)
    with pytest.raises(gp.GpjcError) as ei:
        gp.Operator(grp, to_dev(coils), gp.BF16)
    assert ei.value.status == gp.GPJC_EUNSUPPORTED


@pytest.mark.parametrize("prec", [1, 2])
def test_tc_cg_image_within_1e3(gp, prec):
    wl = synth.workload("2d128")
    g = wl.geom
    c = synth.make_case(wl)
    S = O.simulate(g, c.coils, c.rho, c.noise)
    As, _, _ = O.build_groups(g, c.coils, c.roi)
    x_ref, _ = O.reconstruct(g, c.coils, As, O.compress(g, As, S), "cg", wl.iters)
    plan = gp.Plan(g)
    c_d = to_dev(c.coils)
    grp = gp.Groups.build(plan, c_d, to_dev(c.roi, np.uint8))
    op = gp.Operator(grp, c_d, prec)
    x, info = op.recon(gp.compress(grp, to_dev(S), prec), alg=gp.CG, iters=wl.iters)
    assert info["status"] == 0
    e, m = check_image(to_np(x), x_ref, IMG[prec])
    print(f"precision {prec}: NRMSE {e:.3e}, max element error {m:.3e}")


@pytest.mark.parametrize("prec", [1, 2])
def test_tc_fista_image_within_1e3(gp, prec):
    g = geoms()["2d64"]
    coils, rho, roi = case(g, 47)
    S = O.simulate(g, coils, rho, synth.complex_normal((g.n_lines, g.nc, g.ntx), 48, 1e-3))
    As, _, _ = O.build_groups(g, coils, roi)
    Sc = O.compress(g, As, S)
    pb = O.Problem(g, coils, As)
    b = pb.EcH(Sc)
    L = O.power_lipschitz(pb.normal_c, b, 20)
    x_ref = O.fista(pb.normal_c, b, L, 1e-3, 3, 30)
    op = gp.Operator(gp.Groups.from_matrices(gp.Plan(g), As), to_dev(coils), prec)
    x, _ = op.recon(gp.compress(op.groups, to_dev(S), prec), alg=gp.FISTA, iters=30, lam=1e-3, lipschitz=L,
                    haar_levels=3)
    e, m = check_image(to_np(x), x_ref, IMG[prec])
    print(f"precision {prec}: NRMSE {e:.3e}, max element error {m:.3e}")


@pytest.mark.parametrize("prec", [0, 2, 1])
def test_fista_2d256_full_size_vs_stored_oracle(gp, prec):
    """The benchmark workload at full size (256x256, 32 coils, 8x, 16x
    compression, FISTA-50), groups built on the GPU, against the oracle's
    image stored by tests/golden/make_fista_2d256_reference.py."""
    import os

    ref = np.load(os.path.join(os.path.dirname(__file__), "golden", "fista_2d256_ref.npz"))
    wl = synth.workload("2d256")
    g = wl.geom
    c = synth.make_case(wl)
    S = O.simulate(g, c.coils, c.rho, c.noise)
    plan = gp.Plan(g)
    c_d = to_dev(c.coils)
    grp = gp.Groups.build(plan, c_d, to_dev(c.roi, np.uint8))
    op = gp.Operator(grp, c_d, prec)
    Sc = gp.compress(grp, to_dev(S), prec)
    x, info = op.recon(Sc, alg=gp.FISTA, iters=wl.iters, lam=wl.lam, lipschitz=float(ref["L"]),
                       haar_levels=wl.haar_levels)
    assert info["status"] == 0
    bound = {0: 1e-5, 2: 1e-3, 1: 1e-3}[prec]
    e, m = check_image(to_np(x), ref["x"], bound)
    print(f"2d256 FISTA precision {prec}: NRMSE vs oracle {e:.3e}, max element error {m:.3e}")


@pytest.mark.parametrize("prec", [1, 2])
@pytest.mark.parametrize("name,pieces", [("2d128", 3), ("3d56", 4)])
def test_tc_adjoint_row_pieces_bit_exact(gp, name, pieces, prec, monkeypatch):
    """The 16-bit adjoint runs its tensor-core expansion and inverse readout
    FFT in row pieces of whole expansion row tiles (here with a ragged last
    piece: 128 rows in pieces of 48 / 48 / 32, 2240 rows in pieces of 640 x 3
    + 320); every row goes through the same arithmetic whatever the split, so
    the image must be bit-identical to the one-piece result."""
    g = geoms()[name]
    coils, rho, roi = case(g, 47)
    As, _, _ = O.build_groups(g, coils, roi)
    grp = gp.Groups.from_matrices(gp.Plan(g), As)
    c_d = to_dev(coils)
    monkeypatch.setenv("GPJC_ADJ_PIECES", "1")
    op1 = gp.Operator(grp, c_d, prec)
    monkeypatch.setenv("GPJC_ADJ_PIECES", str(pieces))
    opn = gp.Operator(grp, c_d, prec)
    y_shape = tuple(op1.E(to_dev(synth.complex_normal(g.shape, 48))).shape)
    v = to_dev(synth.complex_normal(y_shape, 49))
    x1 = op1.EH(v)
    xn = opn.EH(v)
    torch.cuda.synchronize()
    assert torch.equal(x1, xn)
    check_close(to_np(xn), O.EcH_apply(g, coils, As, v.cpu().numpy().astype(np.complex128)), TOL[prec])
