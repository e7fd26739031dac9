"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances: the FP32 path must reproduce the oracle's images within
NRMSE 1e-5 (range-normalised, Sec. 3.4); single operator applications are
held to a relative L2 error of 1e-5 (FP32 rounding over a few FFT stages and
a length-N_s contraction stays well below that).  Every such check also
bounds the largest element error (tests/_checks.py).  Integer bookkeeping is
compared bit for bit.
"""
import math

import numpy as np
import pytest

import oracle as O
from _checks import check_close, check_image
from paper_2601_05418_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gp():
    import __graft_entry__ as ge

    ge.build()
    from paper_2601_05418_gb300 import gpjc

    assert torch.cuda.is_available()
    return gpjc


DEV = "cuda:0"


def to_dev(a, dtype=np.complex64):
    return torch.from_numpy(np.ascontiguousarray(a.astype(dtype))).to(DEV)


def to_np(t):
    return t.detach().cpu().numpy().astype(np.complex128)




def ragged_geometry():
    """nx, ny not multiples of the tile sizes, uneven keep per group."""
    g = synth.tiny_geometry(nx=40, ny=36, nz=1, nc=5, os=3, cycles=4.0, kappa_y=1.7, n_groups=3,
                            lines="regular", r=2)
    g.keep = np.array([7, 2, 11], np.int32)
    return g


def geometries():
    wl = synth.workload("2d128")
    g3 = synth.workload("3d56").geom
    # keep 16 on every patch (offsets on 16-component boundaries): the
    # adjoint stages H2 in its paired layout; periodic groups (full column
    # blocks, pair loads) and contiguous groups (one patch per group and row:
    # column blocks with one column, the one-component loop on that layout)
    k16 = synth.tiny_geometry(nx=64, ny=48, nz=1, nc=8, os=4, cycles=4.0, kappa_y=1.5, n_groups=8, keep=16,
                              lines="regular", r=2)
    k16c = synth.tiny_geometry(nx=64, ny=40, nz=1, nc=6, os=4, cycles=4.0, kappa_y=1.5, n_groups=16, keep=16,
                               grouping="contiguous", lines="regular", r=2)
    return {"2d128": wl.geom, "ragged": ragged_geometry(), "3d56": g3, "keep16": k16, "keep16c": k16c}


def case_for(g, seed):
    coils = synth.coil_maps(g.nx, g.ny, g.nz, g.nc, seed)
    rho = synth.phantom(g.nx, g.ny, g.nz)
    return coils, rho, synth.roi_mask(rho)


# ------------------------------------------------------------ bookkeeping --

@pytest.mark.parametrize("name", ["2d128", "ragged", "3d56"])
def test_plan_tables_bit_exact(gp, name):
    g = geometries()[name]
    plan = gp.Plan(g)
    off, ref, lof = plan.tables()
    assert np.array_equal(off, O.patch_offsets(g.patch_group, g.keep).astype(np.int32))
    assert np.array_equal(ref, O.reference_patch(g.patch_group, g.n_groups).astype(np.int32))
    assert plan.ntx_c == O.ntx_compressed(g.patch_group, g.keep)
    exp = np.full(g.nz * g.ny, -1, np.int32)
    exp[g.line_kz * g.ny + g.line_ky] = np.arange(g.n_lines)
    assert np.array_equal(lof, exp)


def test_random_group_map_bit_exact(gp):
    rng = np.random.default_rng(7)
    g = synth.tiny_geometry(nx=16, ny=8, nc=3, os=4, cycles=2.0, n_groups=4)
    pg = rng.integers(0, 5, size=g.ntx // g.w).astype(np.int32)
    pg[:5] = np.arange(5)
    g.patch_group, g.n_groups = pg, 5
    g.keep = rng.integers(1, g.ns + 1, size=5).astype(np.int32)
    plan = gp.Plan(g)
    off, ref, _ = plan.tables()
    assert np.array_equal(off, O.patch_offsets(pg, g.keep).astype(np.int32))
    assert np.array_equal(ref, O.reference_patch(pg, 5).astype(np.int32))


@pytest.mark.parametrize("name", ["2d128", "3d56"])
def test_roi_compaction_bit_exact(gp, name):
    g = geometries()[name]
    coils, rho, roi = case_for(g, 3)
    plan = gp.Plan(g)
    grp = gp.Groups.build(plan, to_dev(coils), to_dev(roi, np.uint8), eig_iters=2)
    assert np.array_equal(grp.roi(), O.roi_pixels(roi, coils).astype(np.int32))


def test_roi_drops_uncovered_pixels(gp):
    g = synth.tiny_geometry(nx=16, ny=16, nc=2, os=2, cycles=2.0, n_groups=2, keep=2)
    coils = synth.coil_maps(16, 16, 1, 2, 5)
    coils[:, 0, 3:6, 4:9] = 0
    roi = np.ones((1, 16, 16), np.uint8)
    grp = gp.Groups.build(gp.Plan(g), to_dev(coils), to_dev(roi, np.uint8), eig_iters=2)
    assert np.array_equal(grp.roi(), O.roi_pixels(roi, coils).astype(np.int32))


def test_empty_roi_is_rejected(gp):
    g = synth.tiny_geometry(nx=8, ny=8, nc=2, os=2, cycles=2.0, n_groups=2, keep=2)
    coils = synth.coil_maps(8, 8, 1, 2, 5)
    with pytest.raises(gp.GpjcError) as ei:
        gp.Groups.build(gp.Plan(g), to_dev(coils), to_dev(np.zeros((1, 8, 8)), np.uint8))
    assert ei.value.status == gp.GPJC_EINVAL


# ------------------------------------------------------------ operators --

@pytest.mark.parametrize("name", ["2d128", "ragged", "3d56"])
def test_simulate_matches_oracle(gp, name):
    g = geometries()[name]
    coils, rho, roi = case_for(g, 4)
    x = synth.complex_normal(g.shape, 5)
    plan = gp.Plan(g)
    A = [np.eye(int(k), g.ns, dtype=complex) for k in g.keep]
    op = gp.Operator(gp.Groups.from_matrices(plan, A), to_dev(coils))
    S = to_np(op.simulate(to_dev(x)))
    S_ref = O.E_apply(g, coils, x)
    check_close(S, S_ref, 1e-5)
    y = synth.complex_normal(S_ref.shape, 6)
    xa = to_np(op.simulate_adjoint(to_dev(y)))
    check_close(xa, O.EH_apply(g, coils, y), 1e-5)


@pytest.mark.parametrize("name", ["2d128", "ragged", "3d56", "keep16", "keep16c"])
def test_compressed_operator_matches_oracle(gp, name):
    g = geometries()[name]
    coils, rho, roi = case_for(g, 7)
    As, _, _ = O.build_groups(g, coils, roi)
    plan = gp.Plan(g)
    op = gp.Operator(gp.Groups.from_matrices(plan, As), to_dev(coils))
    x = synth.complex_normal(g.shape, 8)
    y = to_np(op.E(to_dev(x)))
    y_ref = O.Ec_apply(g, coils, As, x)
    check_close(y, y_ref, 1e-5)
    v = synth.complex_normal(y_ref.shape, 9)
    xa = to_np(op.EH(to_dev(v)))
    check_close(xa, O.EcH_apply(g, coils, As, v), 1e-5)
    # adjoint identity of the GPU pair itself
    lhs = np.vdot(y, v)
    rhs = np.vdot(x, xa)
    assert abs(lhs - rhs) < 1e-5 * abs(lhs)
    # normal operator and ||E_c x||^2
    qq = torch.zeros(1, dtype=torch.float64, device=DEV)
    n = to_np(op.normal(to_dev(x), qq=qq))
    check_close(n, O.EcH_apply(g, coils, As, y_ref), 1e-5)
    assert abs(qq.item() - np.vdot(y_ref, y_ref).real) < 1e-5 * np.vdot(y_ref, y_ref).real


@pytest.mark.parametrize("balance", ["1", "0"])
def test_balanced_forward_readout_matches_oracle(gp, balance, monkeypatch):
    """192 rows x 4 groups of 4 coils: 768 (row, coil group) units, enough
    for every resident block of the device to take at least two, so the
    forward readout runs its one-wave balanced launch (rows cut between
    blocks sum into up to three planes); GPJC_READOUT_BALANCE=0 keeps the
    row x coil-chunk grid.  Both against the oracle."""
    monkeypatch.setenv("GPJC_READOUT_BALANCE", balance)
    g = synth.tiny_geometry(nx=128, ny=192, nz=1, nc=16, os=4, cycles=4.0, kappa_y=1.5, n_groups=8, keep=12,
                            lines="regular", r=3)
    coils, rho, roi = case_for(g, 41)
    As, _, _ = O.build_groups(g, coils, roi)
    plan = gp.Plan(g)
    op = gp.Operator(gp.Groups.from_matrices(plan, As), to_dev(coils))
    x = synth.complex_normal(g.shape, 42)
    y_ref = O.Ec_apply(g, coils, As, x)
    check_close(to_np(op.E(to_dev(x))), y_ref, 1e-5)
    qq = torch.zeros(1, dtype=torch.float64, device=DEV)
    n = to_np(op.normal(to_dev(x), qq=qq))
    check_close(n, O.EcH_apply(g, coils, As, y_ref), 1e-5)
    assert abs(qq.item() - np.vdot(y_ref, y_ref).real) < 1e-5 * np.vdot(y_ref, y_ref).real


@pytest.mark.parametrize("nchunk", [1, 2, 3, 8])
def test_coil_chunking_is_exact(gp, nchunk):
    g = geometries()["2d128"]
    coils, rho, roi = case_for(g, 10)
    As, _, _ = O.build_groups(g, coils, roi)
    plan = gp.Plan(g)
    op = gp.Operator(gp.Groups.from_matrices(plan, As), to_dev(coils), nchunk=nchunk)
    x = synth.complex_normal(g.shape, 11)
    check_close(to_np(op.E(to_dev(x))), O.Ec_apply(g, coils, As, x), 1e-5)


def test_keep_all_is_lossless(gp):
    g = synth.tiny_geometry(nx=16, ny=12, nc=3, os=2, cycles=2.0, kappa_y=1.2, n_groups=2, lines="regular")
    coils, rho, roi = case_for(g, 12)
    As, _, _ = O.build_groups(g, coils, roi)
    plan = gp.Plan(g)
    op = gp.Operator(gp.Groups.from_matrices(plan, As), to_dev(coils))
    x = synth.complex_normal(g.shape, 13)
    a = np.linalg.norm(to_np(op.E(to_dev(x))))
    b = np.linalg.norm(to_np(op.simulate(to_dev(x))))
    assert abs(a - b) < 1e-5 * b


@pytest.mark.parametrize("name", ["2d128", "ragged"])
def test_compress_matches_oracle(gp, name):
    g = geometries()[name]
    coils, rho, roi = case_for(g, 14)
    As, _, _ = O.build_groups(g, coils, roi)
    S = synth.complex_normal((g.n_lines, g.nc, g.ntx), 15)
    plan = gp.Plan(g)
    grp = gp.Groups.from_matrices(plan, As)
    Sc = to_np(gp.compress(grp, to_dev(S)))
    check_close(Sc, O.compress(g, As, S), 1e-5)


# ------------------------------------------------------------ groups --

@pytest.mark.parametrize("simt", [False, True])
@pytest.mark.parametrize("name", ["2d128", "ragged", "3d56"])
def test_gram_matches_oracle(gp, name, simt, monkeypatch):
    """Both Gram kernels: the tensor-core one (FP16 head/remainder split) and
    the FFMA one (GPJC_SIMT_GRAM=1)."""
    if simt:
        monkeypatch.setenv("GPJC_SIMT_GRAM", "1")
    g = geometries()[name]
    coils, rho, roi = case_for(g, 16)
    plan = gp.Plan(g)
    grp = gp.Groups.build(plan, to_dev(coils), to_dev(roi, np.uint8), keep_gram=True)
    P = grp.gram()
    idx = O.roi_pixels(roi, coils)
    for gi in range(g.n_groups):
        Pr = O.gram(g, coils, idx, gi)
        assert np.linalg.norm(P[gi] - Pr) < 1e-5 * np.linalg.norm(Pr)
        assert abs(np.trace(P[gi]).real - len(idx)) < 1e-5 * len(idx)


@pytest.mark.parametrize("name", ["2d128", "ragged", "3d56"])
def test_compression_subspace_matches_oracle(gp, name):
    g = geometries()[name]
    coils, rho, roi = case_for(g, 17)
    plan = gp.Plan(g)
    grp = gp.Groups.build(plan, to_dev(coils), to_dev(roi, np.uint8))
    A, ritz = grp.matrices()
    As, evs, _ = O.build_groups(g, coils, roi)
    assert grp.info().max_residual < 1e-6
    for gi in range(g.n_groups):
        a = A[gi].astype(np.complex128)
        assert np.abs(a @ a.conj().T - np.eye(a.shape[0])).max() < 1e-5
        k = a.shape[0]
        dist = np.linalg.norm(a.conj().T @ a - As[gi].conj().T @ As[gi], 2)
        gap = (evs[gi][k - 1] - evs[gi][k]) / evs[gi][0] if k < len(evs[gi]) else 1.0
        assert dist < max(1e-5, 1e-6 / gap), (gi, dist, gap)
        np.testing.assert_allclose(ritz[gi][:k], evs[gi][:k], rtol=1e-5, atol=1e-6 * evs[gi][0])


def test_whitened_groups_match_oracle(gp):
    g = synth.tiny_geometry(nx=16, ny=16, nc=3, os=2, cycles=2.0, kappa_y=1.1, n_groups=2, keep=4)
    coils, rho, roi = case_for(g, 18)
    psi = synth.random_psd(g.nc, 19)
    T = np.linalg.inv(np.linalg.cholesky(psi))
    grp = gp.Groups.build(gp.Plan(g), to_dev(coils), to_dev(roi, np.uint8), T=T)
    A, _ = grp.matrices()
    As, _, _ = O.build_groups(g, coils, roi, T=T.astype(np.complex64).astype(np.complex128))
    for a, b in zip(A, As):
        # A_g = U^H (T (x) I): compare the row spaces (unitary freedom within the kept subspace)
        pa = np.linalg.pinv(a.astype(np.complex128)) @ a
        pb = np.linalg.pinv(b) @ b
        assert np.linalg.norm(pa - pb, 2) < 1e-4


# ------------------------------------------------------------ reconstruction --

def _oracle_pipeline(g, coils, rho, roi, seed, alg, iters, lam=0.0, levels=4, L=None):
    S = O.simulate(g, coils, rho, synth.complex_normal((g.n_lines, g.nc, g.ntx), seed, 1e-3))
    As, _, _ = O.build_groups(g, coils, roi)
    Sc = O.compress(g, As, S)
    x, Lo = O.reconstruct(g, coils, As, Sc, alg, iters, lam, levels, L=L)
    return S, As, Sc, x


@pytest.mark.parametrize("name", ["2d128", "ragged"])
def test_cg_matches_oracle_same_matrices(gp, name):
    g = geometries()[name]
    coils, rho, roi = case_for(g, 20)
    S, As, Sc, x_ref = _oracle_pipeline(g, coils, rho, roi, 21, "cg", 20)
    op = gp.Operator(gp.Groups.from_matrices(gp.Plan(g), As), to_dev(coils))
    x, info = op.recon(to_dev(Sc), alg=gp.CG, iters=20, history=True)
    assert info["status"] == 0
    check_image(to_np(x), x_ref, 1e-5)
    pb = O.Problem(g, coils, As)
    _, hist = O.cg(None, pb.EcH(Sc), 20, fwd=pb.Ec, adj=pb.EcH)
    np.testing.assert_allclose(info["history"][:len(hist)], hist, rtol=1e-3)


def test_cg_end_to_end_2d128(gp):
    """Groups, compression and CG all on the GPU vs the oracle pipeline."""
    wl = synth.workload("2d128")
    g = wl.geom
    case = synth.make_case(wl)
    S = O.simulate(g, case.coils, case.rho, case.noise)
    As, _, _ = O.build_groups(g, case.coils, case.roi)
    x_ref, _ = O.reconstruct(g, case.coils, As, O.compress(g, As, S), "cg", wl.iters)
    plan = gp.Plan(g)
    c_d = to_dev(case.coils)
    grp = gp.Groups.build(plan, c_d, to_dev(case.roi, np.uint8))
    Sc_d = gp.compress(grp, to_dev(S))
    op = gp.Operator(grp, c_d)
    x, info = op.recon(Sc_d, alg=gp.CG, iters=wl.iters)
    check_image(to_np(x), x_ref, 1e-5)


def test_cg_warm_start_and_zero_iterations(gp):
    g = geometries()["ragged"]
    coils, rho, roi = case_for(g, 22)
    S, As, Sc, _ = _oracle_pipeline(g, coils, rho, roi, 23, "cg", 1)
    op = gp.Operator(gp.Groups.from_matrices(gp.Plan(g), As), to_dev(coils))
    x0, _ = op.recon(to_dev(Sc), alg=gp.CG, iters=0)
    assert float(x0.abs().max()) == 0.0
    pb = O.Problem(g, coils, As)
    xs = synth.complex_normal(g.shape, 24) * 0.1
    ref, _ = O.cg(pb.normal_c, pb.EcH(Sc), 6, x0=xs, fwd=pb.Ec, adj=pb.EcH)
    x, _ = op.recon(to_dev(Sc), alg=gp.CG, iters=6, x0=to_dev(xs))
    check_image(to_np(x), ref, 1e-5)


def test_fista_matches_oracle_small(gp):
    g = synth._geom_2d(64, 8, 4, 8, 2.5, 16, 8.0, 3)
    coils, rho, roi = case_for(g, 25)
    S = O.simulate(g, coils, rho, synth.complex_normal((g.n_lines, g.nc, g.ntx), 26, 1e-3))
    As, _, _ = O.build_groups(g, coils, roi)
    Sc = O.compress(g, As, S)
    pb = O.Problem(g, coils, As)
    b = pb.EcH(Sc)
    L = O.power_lipschitz(pb.normal_c, b, 20)
    x_ref = O.fista(pb.normal_c, b, L, 1e-3, 3, 30)
    op = gp.Operator(gp.Groups.from_matrices(gp.Plan(g), As), to_dev(coils))
    # power iteration from E_c^H S' on the device reproduces the oracle's L
    _, info = op.recon(to_dev(Sc), alg=gp.FISTA, iters=1, lam=1e-3, haar_levels=3, power_iters=20)
    assert abs(info["lipschitz"] - L) < 1e-5 * L
    x, info = op.recon(to_dev(Sc), alg=gp.FISTA, iters=30, lam=1e-3, lipschitz=L, haar_levels=3)
    check_image(to_np(x), x_ref, 1e-5)


def test_graph_and_eager_agree(gp):
    g = geometries()["2d128"]
    coils, rho, roi = case_for(g, 27)
    S, As, Sc, _ = _oracle_pipeline(g, coils, rho, roi, 28, "cg", 1)
    op = gp.Operator(gp.Groups.from_matrices(gp.Plan(g), As), to_dev(coils))
    a, _ = op.recon(to_dev(Sc), alg=gp.CG, iters=15, use_graph=True)
    b, _ = op.recon(to_dev(Sc), alg=gp.CG, iters=15, use_graph=False)
    c, _ = op.recon(to_dev(Sc), alg=gp.CG, iters=15, use_graph=True)  # cached graph replay
    assert torch.equal(a, b) and torch.equal(a, c)


def test_3d_cg_end_to_end(gp):
    wl = synth.workload("3d56")
    g = wl.geom
    case = synth.make_case(wl)
    S = O.simulate(g, case.coils, case.rho, case.noise)
    As, _, _ = O.build_groups(g, case.coils, case.roi)
    x_ref, _ = O.reconstruct(g, case.coils, As, O.compress(g, As, S), "cg", wl.iters)
    plan = gp.Plan(g)
    c_d = to_dev(case.coils)
    grp = gp.Groups.build(plan, c_d, to_dev(case.roi, np.uint8))
    op = gp.Operator(grp, c_d)
    x, _ = op.recon(gp.compress(grp, to_dev(S)), alg=gp.CG, iters=wl.iters)
    check_image(to_np(x), x_ref, 1e-5)


# ------------------------------------------------------------ FFT lengths --

@pytest.mark.parametrize("n", [40, 56, 160, 192, 224, 240, 288, 320])
def test_two_pass_fft_lengths_match_oracle(gp, n):
    """Every transform length with a two-pass plan (n = 8 x {5, 7} or
    16 x {10, 12, 14, 15, 18, 20}) along both the readout and the
    phase-encode axis: the uncompressed model, E_c and E_c^H against the
    FP64 oracle."""
    g = synth.tiny_geometry(nx=n, ny=n, nz=1, nc=2, os=2, cycles=2.0, kappa_y=1.9, n_groups=n // 8, keep=4,
                            lines="regular", r=2)
    coils, rho, roi = case_for(g, 30)
    x = synth.complex_normal(g.shape, 31)
    As, _, _ = O.build_groups(g, coils, roi)
    plan = gp.Plan(g)
    op = gp.Operator(gp.Groups.from_matrices(plan, As), to_dev(coils))
    check_close(to_np(op.simulate(to_dev(x))), O.E_apply(g, coils, x), 1e-5)
    check_close(to_np(op.E(to_dev(x))), O.Ec_apply(g, coils, As, x), 1e-5)
    v = synth.complex_normal((g.n_lines, plan.ntx_c), 32)
    check_close(to_np(op.EH(to_dev(v))), O.EcH_apply(g, coils, As, v), 1e-5)
