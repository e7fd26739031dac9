"""Pins for the FP64 oracle: brute force, closed forms, invariants and the
paper's printed bookkeeping.  CPU only; none of these calls the CUDA path."""
import json
import math
import os

import numpy as np
import pytest

import oracle as O
from paper_2601_05418_gb300 import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _rand(shape, seed):
    return synth.complex_normal(shape, seed)


def _tiny2d(**kw):
    g = synth.tiny_geometry(**kw)
    c = synth.coil_maps(g.nx, g.ny, g.nz, g.nc, 11)
    return g, c


def _tiny3d(**kw):
    base = dict(nx=6, ny=4, nz=4, nc=2, os=2, cycles=2.0, kappa_y=1.1,
                kappa_z=0.7, n_groups=3, grouping="contiguous")
    base.update(kw)
    g = synth.tiny_geometry(**base)
    c = synth.coil_maps(g.nx, g.ny, g.nz, g.nc, 12)
    return g, c


# ---------------------------------------------------------------- encoding --

@pytest.mark.parametrize("dim", [2, 3])
def test_factorised_E_equals_dense_E(dim):
    g, c = _tiny2d() if dim == 2 else _tiny3d()
    rho = _rand(g.shape, 3)
    E = O.dense_E(g, c)
    s_dense = (E @ rho.ravel()).reshape(g.n_lines, g.nc, g.ntx)
    s_fact = O.E_apply(g, c, rho)
    assert np.abs(s_dense - s_fact).max() < 1e-12 * np.abs(s_dense).max()
    y = _rand(s_fact.shape, 4)
    x_dense = (E.conj().T @ y.ravel()).reshape(g.shape)
    assert np.abs(x_dense - O.EH_apply(g, c, y)).max() < 1e-12 * np.abs(x_dense).max()


@pytest.mark.parametrize("dim", [2, 3])
def test_adjoint_identity(dim):
    g, c = _tiny2d(lines="regular") if dim == 2 else _tiny3d(lines="caipi")
    rho = _rand(g.shape, 5)
    y = _rand((g.n_lines, g.nc, g.ntx), 6)
    lhs = np.vdot(O.E_apply(g, c, rho), y)
    rhs = np.vdot(rho, O.EH_apply(g, c, y))
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)
    roi = np.ones(g.shape, np.uint8)
    g.keep[:] = max(1, g.ns // 3)
    As, _, _ = O.build_groups(g, c, roi)
    yc = _rand((g.n_lines, O.ntx_compressed(g.patch_group, g.keep)), 7)
    lhs = np.vdot(O.Ec_apply(g, c, As, rho), yc)
    rhs = np.vdot(rho, O.EcH_apply(g, c, As, yc))
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def test_zero_wave_is_fft_sense():
    """kappa = 0: E reduces to SENSE on an x-zero-padded grid, written here
    with numpy's 2D FFT (no readout / phase-encode factorisation)."""
    g, c = _tiny2d(nx=8, ny=6, os=3, cycles=3.0, kappa_y=0.0, n_groups=2,
                   lines="regular", r=2)
    rho = _rand(g.shape, 8)
    ntx = g.ntx
    pad = np.zeros((g.nc, g.ny, ntx), complex)
    s0 = ntx // 2 - g.nx // 2
    pad[:, :, s0:s0 + g.nx] = (c * rho[None])[:, 0]
    k = np.fft.fftshift(np.fft.fft2(np.fft.ifftshift(pad, axes=(1, 2)),
                                    norm="ortho"), axes=(1, 2))
    ref = np.transpose(k[:, g.line_ky, :], (1, 0, 2))
    assert np.abs(ref - O.E_apply(g, c, rho)).max() < 1e-12


def test_wave_is_phase_encode_shift():
    """Linear wave gradient (Eq. 3): at a sample where the excursion a_y is an
    integer m, the modulated sample equals the unmodulated sample of line
    ky + m (the B0 kernel is an off-centre point, Eq. 5)."""
    g0, c = _tiny2d(nx=4, ny=8, os=2, cycles=1.0, kappa_y=0.0, n_groups=1)
    g2, _ = _tiny2d(nx=4, ny=8, os=2, cycles=1.0, kappa_y=2.0, n_groups=1)
    rho = _rand(g0.shape, 9)
    s0, s2 = O.E_apply(g0, c, rho), O.E_apply(g2, c, rho)
    t_star = g0.ntx // 2  # theta = pi, a_y = kappa_y = 2
    ay, _ = O.wave_coeffs(g2.ntx, g2.cycles, g2.kappa_y, 0.0)
    assert abs(ay[t_star] - 2.0) < 1e-12
    for ky in range(g0.ny - 2):
        np.testing.assert_allclose(s2[ky, :, t_star], s0[ky + 2, :, t_star],
                                   atol=1e-12)
    assert ay[0] == 0.0
    np.testing.assert_allclose(s2[:, :, 0], s0[:, :, 0], atol=1e-12)


# ---------------------------------------------------------------- gram --

def test_gram_trace_hermitian_psd():
    g, c = _tiny2d(nx=8, ny=8, nc=3, os=2, cycles=2.0, n_groups=2)
    roi = synth.roi_mask(synth.phantom(g.nx, g.ny))
    idx = O.roi_pixels(roi, c)
    for gi in range(g.n_groups):
        P = O.gram(g, c, idx, gi)
        assert abs(np.trace(P).real - len(idx)) < 1e-12 * len(idx)
        assert np.abs(P - P.conj().T).max() < 1e-13 * len(idx)
        assert np.linalg.eigvalsh(P).min() > -1e-12 * len(idx)


def test_gram_matches_rows_of_dense_E():
    """P_g (Eq. 9) built from the rows of the brute-force E for one patch and
    one line: the phase-encode factor is a per-pixel unit scalar."""
    g, c = _tiny2d(nx=6, ny=4, nc=2, os=2, cycles=2.0, kappa_y=1.7, n_groups=2)
    idx = np.arange(g.nx * g.ny)
    E = O.dense_E(g, c).reshape(g.n_lines, g.nc, g.ntx, -1)
    for gi in range(g.n_groups):
        p = int(O.reference_patch(g.patch_group, g.n_groups)[gi])
        for line in (0, g.n_lines - 1):
            Eg = E[line, :, p * g.w:(p + 1) * g.w, :].reshape(g.ns, -1)
            nrm = np.sum(np.abs(Eg) ** 2, axis=0)
            P_ref = (Eg / nrm[None]) @ Eg.conj().T
            assert np.abs(P_ref - O.gram(g, c, idx, gi)).max() < 1e-12 * len(idx)


def test_gram_dirichlet_closed_form():
    """One uniform coil, no wave, full ROI: P[tau, tau'] = (Ny Nz / w)
    e^{i pi d / Ntx} sin(pi d Nx / Ntx) / sin(pi d / Ntx), d = tau - tau'."""
    g = synth.tiny_geometry(nx=8, ny=4, nc=1, os=4, cycles=2.0, kappa_y=0.0,
                            n_groups=2)
    c = np.ones((1, 1, g.ny, g.nx), complex)
    idx = np.arange(g.nx * g.ny)
    P = O.gram(g, c, idx, 1)
    w, ntx, nx = g.w, g.ntx, g.nx
    ref = np.empty((w, w), complex)
    for a in range(w):
        for b in range(w):
            d = a - b
            ref[a, b] = nx if d == 0 else (np.exp(1j * math.pi * d / ntx)
                                          * math.sin(math.pi * d * nx / ntx)
                                          / math.sin(math.pi * d / ntx))
    ref *= g.ny * g.nz / w
    assert np.abs(P - ref).max() < 1e-12 * len(idx)


def test_gram_w1_is_rf_only():
    """w = 1: every group's P_g is the RF-only matrix sum c c^H / ||c||^2,
    independent of the B0 phase (Sec. 2.4, RF-only special case)."""
    g = synth.tiny_geometry(nx=8, ny=8, nc=4, os=2, cycles=2.0, kappa_y=2.3,
                            n_groups=8)
    assert g.w == 1
    c = synth.coil_maps(g.nx, g.ny, 1, g.nc, 13)
    roi = synth.roi_mask(synth.phantom(g.nx, g.ny))
    idx = O.roi_pixels(roi, c)
    cm = c.reshape(g.nc, -1)[:, idx]
    ref = (cm / np.sum(np.abs(cm) ** 2, axis=0)) @ cm.conj().T
    for gi in range(g.n_groups):
        assert np.abs(O.gram(g, c, idx, gi) - ref).max() < 1e-12 * len(idx)


def test_gram_periodicity():
    """Per-period groups: the Gram from any occurrence of g equals the first
    (the readout shift by a whole period is a per-pixel phase)."""
    g, c = _tiny2d(nx=8, ny=6, nc=2, os=4, cycles=4.0, kappa_y=1.5, n_groups=2)
    idx = np.arange(g.nx * g.ny)
    for gi in range(g.n_groups):
        occ = np.flatnonzero(g.patch_group == gi)
        assert len(occ) > 1
        P0 = O.gram(g, c, idx, gi)
        for p in occ[1:]:
            assert np.abs(O.gram(g, c, idx, gi, patch=int(p)) - P0).max() < 1e-11 * len(idx)
    # a non-periodic split is rejected by the validator
    assert O.periodic_grouping_ok(g.patch_group, g.w, g.ntx // int(g.cycles))
    bad = g.patch_group.copy()
    bad[[0, 1]] = bad[[1, 0]]
    assert not O.periodic_grouping_ok(bad, g.w, g.ntx // int(g.cycles))


# ---------------------------------------------------------------- eig / A --

def test_compression_matrix_orthonormal_and_spectrum():
    g, c = _tiny2d(nx=8, ny=8, nc=3, os=2, cycles=2.0, n_groups=2, keep=3)
    roi = np.ones(g.shape, np.uint8)
    As, evs, Ps = O.build_groups(g, c, roi)
    for A, ev, P in zip(As, evs, Ps):
        assert np.abs(A @ A.conj().T - np.eye(A.shape[0])).max() < 1e-12
        assert abs(ev.sum() - g.nx * g.ny) < 1e-10
        assert np.all(np.diff(ev) <= 1e-12)
        # rows of A are eigenvectors: A P = diag(ev[:k]) A
        assert np.abs(A @ P - ev[:A.shape[0], None] * A).max() < 1e-10


def test_keep_from_energy_geometric_closed_form():
    """lambda_i = r^i (i < n): the leading k hold (1 - r^k) / (1 - r^n) of the
    total, so keep = ceil(log(1 - tau (1 - r^n)) / log r)."""
    for r, n, tau in [(0.5, 20, 0.9), (0.8, 64, 0.99), (0.3, 10, 0.5), (0.95, 200, 0.999)]:
        ev = r ** np.arange(n, dtype=np.float64)
        k = math.ceil(math.log(1 - tau * (1 - r ** n)) / math.log(r))
        assert O.keep_from_energy(ev[None], tau)[0] == k
        # the same with the trace passed explicitly and the tail cut off
        tr = (1 - r ** n) / (1 - r)
        assert O.keep_from_energy(ev[None, :k + 1], tau, trace=tr)[0] == k
        # fewer leading values than needed: -1
        if k > 1:
            assert O.keep_from_energy(ev[None, :k - 1], tau, trace=tr)[0] == -1


def test_keep_from_energy_brute_force():
    """Against a direct search over k on random spectra (ties, zeros and
    tiny negative rounding values included)."""
    rng = np.random.default_rng(7)
    for _ in range(200):
        m = int(rng.integers(1, 12))
        ev = np.sort(np.round(rng.exponential(1.0, m), 1))[::-1]
        ev[-1] -= 1e-15 * rng.integers(0, 2)
        tau = float(rng.choice([0.3, 0.5, 0.9, 1.0]))
        pos = np.maximum(ev, 0.0)
        total = sum(float(v) for v in pos)
        want = -1
        for k in range(1, m + 1):
            if sum(float(v) for v in pos[:k]) >= tau * total:
                want = k
                break
        assert O.keep_from_energy(ev[None], tau)[0] == want
    # negative (rounding) eigenvalues add nothing to the total either: the
    # default trace of [1, 0.5, -0.5] is 1.5, so the whole energy needs k = 2
    assert O.keep_from_energy(np.array([[1.0, 0.5, -0.5]]), 1.0)[0] == 2


def test_keep_from_energy_is_the_encoding_energy_kept():
    """With trace(P_g) = |ROI| (one unit per normalised encoding vector,
    Eq. 11), the energy left out by the first k eigenvectors is the squared
    residual of the normalised encoding vectors outside their span (Eq. 8):
    the chosen keep is the smallest k whose residual is at most
    (1 - tau) |ROI|."""
    g, c = _tiny2d(nx=8, ny=8, nc=3, os=2, cycles=2.0, n_groups=2)
    roi = synth.roi_mask(synth.phantom(g.nx, g.ny))
    idx = O.roi_pixels(roi, c)
    for gi in range(g.n_groups):
        P = O.gram(g, c, idx, gi)
        _, ev = O.compression_matrix(P, g.nc * g.w, g.nc, g.w)
        U = O.compression_matrix(P, g.nc * g.w, g.nc, g.w)[0].conj().T  # columns: eigenvectors, descending
        V = O.encoding_vectors(g, c, idx, int(O.reference_patch(g.patch_group, g.n_groups)[gi]))
        V = V / np.linalg.norm(V, axis=0, keepdims=True)
        resid = [float(np.sum(np.abs(V - U[:, :k] @ (U[:, :k].conj().T @ V)) ** 2)) for k in range(len(ev) + 1)]
        for tau in (0.5, 0.9, 0.99, 0.999):
            k = O.keep_from_energy(ev[None], tau, trace=len(idx))[0]
            assert 1 <= k <= len(ev)
            assert resid[k] <= (1 - tau) * len(idx) + 1e-9 * len(idx)
            assert resid[k - 1] > (1 - tau) * len(idx) - 1e-9 * len(idx)


def test_keep_all_is_lossless():
    """keep = N_s: A_g unitary, ||E' x|| = ||E x||, CG on E' equals CG on E."""
    g, c = _tiny2d(nx=8, ny=6, nc=2, os=2, cycles=2.0, n_groups=2,
                   lines="regular", r=2)
    roi = np.ones(g.shape, np.uint8)
    As, _, _ = O.build_groups(g, c, roi)
    rho = _rand(g.shape, 14)
    pb = O.Problem(g, c, As)
    assert abs(np.linalg.norm(pb.Ec(rho)) - np.linalg.norm(pb.E(rho))) < 1e-12 * np.linalg.norm(pb.E(rho))
    S = pb.E(rho) + synth.complex_normal((g.n_lines, g.nc, g.ntx), 15, 1e-2)
    Sc = O.compress(g, As, S)
    xc, _ = O.cg(None, pb.EcH(Sc), 8, fwd=pb.Ec, adj=pb.EcH)
    xu, _ = O.cg(None, pb.EH(S), 8, fwd=pb.E, adj=pb.EH)
    assert np.abs(xc - xu).max() < 1e-11 * np.abs(xu).max()


def test_rotation_invariance_of_image():
    """Replacing A_g by Q A_g (Q unitary) leaves the CG image unchanged."""
    g, c = _tiny2d(nx=8, ny=6, nc=2, os=2, cycles=2.0, n_groups=2, keep=5,
                   lines="regular", r=2)
    roi = np.ones(g.shape, np.uint8)
    As, _, _ = O.build_groups(g, c, roi)
    rng = np.random.default_rng(3)
    Qs = [np.linalg.qr(rng.normal(size=(5, 5)) + 1j * rng.normal(size=(5, 5)))[0]
          for _ in As]
    As2 = [Q @ A for Q, A in zip(Qs, As)]
    rho = _rand(g.shape, 16)
    S = O.E_apply(g, c, rho)
    x1, _ = O.reconstruct(g, c, As, O.compress(g, As, S), "cg", 6)
    x2, _ = O.reconstruct(g, c, As2, O.compress(g, As2, S), "cg", 6)
    assert np.abs(x1 - x2).max() < 1e-11 * np.abs(x1).max()


def test_dense_compressed_model():
    """E' = A E (Eq. 14) as a dense matrix equals the matrix-free E_c."""
    g, c = _tiny2d(nx=6, ny=4, nc=2, os=2, cycles=2.0, n_groups=2, keep=3)
    roi = np.ones(g.shape, np.uint8)
    As, _, _ = O.build_groups(g, c, roi)
    rho = _rand(g.shape, 17)
    Ed = O.dense_Ec(g, c, As)
    ref = (Ed @ rho.ravel()).reshape(g.n_lines, -1)
    assert np.abs(ref - O.Ec_apply(g, c, As, rho)).max() < 1e-12


def test_whitening():
    """keep = N_s with T = Q^{-1}, Psi = Q Q^H: ||E' x||^2 =
    x^H E^H (Psi^{-1} (x) I) E x (Eq. 12's noise decorrelation)."""
    g, c = _tiny2d(nx=6, ny=4, nc=3, os=2, cycles=2.0, n_groups=2)
    psi = synth.random_psd(g.nc, 18)
    T = np.linalg.inv(np.linalg.cholesky(psi))
    roi = np.ones(g.shape, np.uint8)
    As, _, _ = O.build_groups(g, c, roi, T=T)
    rho = _rand(g.shape, 19)
    s = O.E_apply(g, c, rho)
    lhs = np.linalg.norm(O.compress(g, As, s)) ** 2
    sw = np.einsum("nm,lmt->lnt", np.linalg.inv(psi), s)
    rhs = np.vdot(s, sw).real
    assert abs(lhs - rhs) < 1e-11 * rhs


# ---------------------------------------------------------------- recon --

def test_readout_rows_assemble_the_compressed_model():
    """The per-row compressed readout matrices, followed by the sampled rows
    of the centred phase-encode DFT, reproduce E_c (Eq. 14-15)."""
    g, c = _tiny2d(nx=8, ny=12, nc=3, os=2, cycles=2.0, kappa_y=1.3, n_groups=2, keep=5,
                   lines="regular", r=3)
    As, _, _ = O.build_groups(g, c, np.ones(g.shape, np.uint8))
    x = _rand(g.shape, 61)
    H = np.stack([O.readout_Ec_row(g, c, As, y) @ x[0, y] for y in range(g.ny)])  # [y][N'_tx]
    ky = np.asarray(g.line_ky)
    F = np.exp(-2j * np.pi * np.outer(ky - g.ny // 2, O.centred(g.ny)) / g.ny) / math.sqrt(g.ny)
    ref = O.Ec_apply(g, c, As, x)
    assert np.linalg.norm(F @ H - ref) < 1e-12 * np.linalg.norm(ref)


@pytest.mark.parametrize("r,keep", [(3, 8), (2, 6), (1, 3)])
def test_decoupled_ls_is_the_global_least_squares(r, keep):
    """Algorithm #1 (Sec. 3.4) on a regular mask with R | N_y returns the
    least-squares solution of the whole compressed model (dense E' of
    Eq. 14 solved by numpy's lstsq), noisy data included."""
    g, c = _tiny2d(nx=8, ny=12, nc=3, os=2, cycles=2.0, kappa_y=1.3, n_groups=2, keep=keep,
                   lines="regular", r=r)
    As, _, _ = O.build_groups(g, c, np.ones(g.shape, np.uint8))
    Sc = O.compress(g, As, O.E_apply(g, c, _rand(g.shape, 62))) + 0.05 * _rand((g.n_lines, O.ntx_compressed(g.patch_group, g.keep)), 63)
    D = O.dense_Ec(g, c, As).reshape(-1, g.nx * g.ny)
    x_ls = np.linalg.lstsq(D, Sc.ravel(), rcond=None)[0]
    x_dec = O.decoupled_ls(g, c, As, Sc).ravel()
    assert np.linalg.norm(x_dec - x_ls) < 1e-8 * np.linalg.norm(x_ls)
    sets, _, _ = O.aliased_sets(g)
    assert sorted(len(Y) for Y in sets) == [r] * (g.ny // r)


def test_decoupled_ls_3d_caipi_is_the_global_least_squares():
    """3x3 CAIPI on a 6 x 18 phase-encode grid (the shift pattern 0, 1, 2
    closes within N_z, so the samples form a lattice): twelve aliased sets
    of nine rows, and algorithm #1 equals the least-squares solution of the
    dense 3D compressed model."""
    g, c = _tiny3d(nx=6, ny=6, nz=18, nc=4, os=4, n_groups=2, lines="caipi", r=3)
    As, _, _ = O.build_groups(g, c, np.ones(g.shape, np.uint8))
    sets, _, _ = O.aliased_sets(g)
    assert sorted(len(Y) for Y in sets) == [9] * 12
    Sc = O.compress(g, As, O.E_apply(g, c, _rand(g.shape, 64))) + 0.05 * _rand((g.n_lines, O.ntx_compressed(g.patch_group, g.keep)), 65)
    D = O.dense_Ec(g, c, As).reshape(-1, g.nx * g.ny * g.nz)
    x_ls = np.linalg.lstsq(D, Sc.ravel(), rcond=None)[0]
    x_dec = O.decoupled_ls(g, c, As, Sc).ravel()
    assert np.linalg.norm(x_dec - x_ls) < 1e-8 * np.linalg.norm(x_ls)


def test_decoupled_cg_converges_to_decoupled_ls():
    """Per-set CG (algorithm #1 with an iterative subproblem solver) reaches
    the exact per-set least squares of `decoupled_ls` once the iterations
    reach the set's unknown count (2 rows x 8 pixels = 16)."""
    g, c = _tiny2d(nx=8, ny=12, nc=3, os=2, cycles=2.0, kappa_y=1.3, n_groups=2, keep=5,
                   lines="regular", r=2)
    As, _, _ = O.build_groups(g, c, np.ones(g.shape, np.uint8))
    Sc = O.compress(g, As, O.E_apply(g, c, _rand(g.shape, 66))) + 0.05 * _rand((g.n_lines, O.ntx_compressed(g.patch_group, g.keep)), 67)
    x_ls = O.decoupled_ls(g, c, As, Sc)
    x_cg = O.decoupled_cg(g, c, As, Sc, 16)
    assert np.linalg.norm(x_cg - x_ls) < 1e-8 * np.linalg.norm(x_ls)
    # fewer iterations than unknowns: not yet there (the test would pass
    # trivially if the iteration count were ignored)
    assert np.linalg.norm(O.decoupled_cg(g, c, As, Sc, 3) - x_ls) > 1e-4 * np.linalg.norm(x_ls)


def test_decoupled_cg_with_one_set_is_global_cg():
    """A mask whose samples form no lattice (R = 5 on 12 rows) couples all
    rows into one aliased set: per-set CG is then the global CG of
    Eq. 16 (same recurrences, same iterates)."""
    g, c = _tiny2d(nx=8, ny=12, nc=3, os=2, cycles=2.0, kappa_y=1.3, n_groups=2, keep=4,
                   lines="regular", r=5)
    sets, _, _ = O.aliased_sets(g)
    assert len(sets) == 1
    As, _, _ = O.build_groups(g, c, np.ones(g.shape, np.uint8))
    Sc = O.compress(g, As, O.E_apply(g, c, _rand(g.shape, 68)))
    pb = O.Problem(g, c, As)
    x_glob, _ = O.cg(pb.normal_c, pb.EcH(Sc), 7)
    x_dec = O.decoupled_cg(g, c, As, Sc, 7)
    assert np.linalg.norm(x_dec - x_glob) < 1e-10 * np.linalg.norm(x_glob)


def test_cg_reaches_least_squares():
    g, c = _tiny2d(nx=4, ny=4, nc=2, os=2, cycles=2.0, n_groups=2, keep=3)
    roi = np.ones(g.shape, np.uint8)
    As, _, _ = O.build_groups(g, c, roi)
    Ed = O.dense_Ec(g, c, As)
    rho = _rand(g.shape, 20)
    Sc = (Ed @ rho.ravel()).reshape(g.n_lines, -1) + _rand((g.n_lines, Ed.shape[0] // g.n_lines), 21) * 0.05
    ref = np.linalg.lstsq(Ed, Sc.ravel(), rcond=None)[0].reshape(g.shape)
    x, hist = O.reconstruct(g, c, As, Sc, "cg", 16)
    assert np.abs(x - ref).max() < 1e-8 * np.abs(ref).max()


def test_haar_orthonormal_and_closed_form():
    img = _rand((1, 16, 32), 22)[0]
    c = O.haar_fwd(img, 3)
    assert abs(np.linalg.norm(c) - np.linalg.norm(img)) < 1e-12 * np.linalg.norm(img)
    assert np.abs(O.haar_inv(c, 3) - img).max() < 1e-13
    # one level on a 2x2 block [[a, b], [c, d]]
    a, b, cc, d = 1.0, 2.0, 4.0, 8.0
    one = O.haar_fwd(np.array([[a, b], [cc, d]]), 1)
    ref = 0.5 * np.array([[a + b + cc + d, a - b + cc - d],
                          [a + b - cc - d, a - b - cc + d]])
    assert np.abs(one - ref).max() < 1e-14
    # constant image: only the coarsest approximation survives
    const = np.full((16, 16), 3.0 + 1.0j)
    cf = O.haar_fwd(const, 4)
    assert abs(cf[0, 0] - (3.0 + 1.0j) * 16) < 1e-12
    cf[0, 0] = 0
    assert np.abs(cf).max() < 1e-12


def test_soft_threshold_closed_form():
    z = np.array([0.0, 0.5, -2.0, 3.0 + 4.0j, 1e-3j])
    out = O.soft(z, 1.0)
    ref = np.array([0.0, 0.0, -1.0, (3.0 + 4.0j) * 0.8, 0.0])
    assert np.abs(out - ref).max() < 1e-15


def test_power_iteration_and_fista():
    g, c = _tiny2d(nx=8, ny=8, nc=2, os=2, cycles=2.0, n_groups=2, keep=4,
                   lines="regular", r=2)
    roi = np.ones(g.shape, np.uint8)
    As, _, _ = O.build_groups(g, c, roi)
    Ed = O.dense_Ec(g, c, As)
    lmax = np.linalg.eigvalsh(Ed.conj().T @ Ed).max()
    pb = O.Problem(g, c, As)
    L = O.power_lipschitz(pb.normal_c, _rand(g.shape, 23), 3000)
    assert abs(L - lmax) < 1e-8 * lmax
    rho = _rand(g.shape, 24)
    Sc = pb.Ec(rho)
    # lambda = 0: FISTA tends to the least-squares solution
    ref = np.linalg.lstsq(Ed, Sc.ravel(), rcond=None)[0].reshape(g.shape)
    x = O.fista(pb.normal_c, pb.EcH(Sc), L, 0.0, 2, 3000)
    assert np.abs(x - ref).max() < 1e-5 * np.abs(ref).max()
    # lambda > 0: FISTA and plain ISTA reach the same minimiser
    lam = 0.05
    b = pb.EcH(Sc)
    xf = O.fista(pb.normal_c, b, L, lam, 2, 4000)
    xi = np.zeros_like(b)
    for _ in range(20000):
        z = xi - (pb.normal_c(xi) - b) / L
        xi = O.wavelet_prox(z[0], lam / L, 2)[None]
    assert np.abs(xf - xi).max() < 1e-6 * np.abs(xi).max()


def test_tv_smooth_closed_forms_and_adjoint():
    """Constant image: every term is eps.  Vertical edge (0 left, 1 right of
    column c): the N_y terms at column c - 1 are sqrt(1 + eps^2), the rest
    eps.  D^H is the adjoint of the forward differences."""
    eps = 1e-2
    ny, nx, c = 6, 9, 4
    assert abs(O.tv_smooth(np.full((ny, nx), 2.5 + 1j), eps) - ny * nx * eps) < 1e-12
    u = np.zeros((ny, nx), np.complex128)
    u[:, c:] = 1.0
    want = ny * math.sqrt(1 + eps * eps) + (ny * nx - ny) * eps
    assert abs(O.tv_smooth(u, eps) - want) < 1e-12
    v, px, py = _rand((ny, nx), 81), _rand((ny, nx), 82), _rand((ny, nx), 83)
    dx, dy = O.tv_diff(v)
    lhs = np.vdot(px, dx) + np.vdot(py, dy)
    rhs = np.vdot(O.tv_diff_adj(px, py), v)
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def test_tv_smooth_gradient_and_lipschitz():
    """The gradient matches central differences of the function along random
    complex directions, and never changes faster than 8 / eps."""
    eps = 0.05
    u = _rand((7, 8), 84)
    gr = O.tv_smooth_grad(u, eps)
    for seed in range(5):
        d = _rand((7, 8), 90 + seed)
        h = 1e-6
        fd = (O.tv_smooth(u + h * d, eps) - O.tv_smooth(u - h * d, eps)) / (2 * h)
        assert abs(fd - np.vdot(gr, d).real) < 1e-6 * max(1.0, abs(fd))
    rng = np.random.default_rng(85)
    for _ in range(50):
        a = _rand((7, 8), int(rng.integers(1 << 30)))
        b = a + 0.01 * _rand((7, 8), int(rng.integers(1 << 30)))
        ratio = np.linalg.norm(O.tv_smooth_grad(a, eps) - O.tv_smooth_grad(b, eps)) / np.linalg.norm(a - b)
        assert ratio <= 8 / eps * (1 + 1e-9)


def test_fista_with_tv_reaches_its_optimality_condition():
    """Wavelet weight 0, TV weight > 0: the objective is smooth and strongly
    convex here (full-rank E'), and FISTA's limit zeroes its gradient
    E'^H (E' x - S') + lam_tv grad TV_eps(x); with lam_tv = 0 it is the
    plain FISTA iteration."""
    g, c = _tiny2d(nx=8, ny=8, nc=2, os=2, cycles=2.0, n_groups=2, keep=4, lines="regular", r=2)
    As, _, _ = O.build_groups(g, c, np.ones(g.shape, np.uint8))
    pb = O.Problem(g, c, As)
    Sc = pb.Ec(_rand(g.shape, 86))
    b = pb.EcH(Sc)
    L0 = O.power_lipschitz(pb.normal_c, _rand(g.shape, 87), 500)
    assert np.array_equal(O.fista(pb.normal_c, b, L0, 0.01, 2, 30),
                          O.fista(pb.normal_c, b, L0, 0.01, 2, 30, lam_tv=0.0))
    lam_tv, eps = 0.02, 0.1
    L = 1.01 * L0 + 8 * lam_tv / eps
    x = O.fista(pb.normal_c, b, L, 0.0, 2, 4000, lam_tv=lam_tv, eps_tv=eps)
    grad = pb.normal_c(x) - b + lam_tv * O.tv_smooth_grad(x[0], eps)[None]
    assert np.linalg.norm(grad) < 1e-7 * np.linalg.norm(b)
    assert np.linalg.norm(lam_tv * O.tv_smooth_grad(x[0], eps)) > 1e-3 * np.linalg.norm(b)  # the TV term acts


def test_nrmse_closed_form():
    ref = np.zeros((1, 4, 4), complex)
    ref[0, 0, 0] = 2.0
    x = ref + 0.1
    assert abs(O.nrmse(x, ref) - 0.1 / 2.0) < 1e-15


# ---------------------------------------------------------------- bookkeeping --

def test_offsets_and_compressed_length():
    pg = np.array([0, 1, 2, 0, 1, 2, 1], np.int32)
    keep = np.array([3, 1, 2], np.int32)
    assert list(O.patch_offsets(pg, keep)) == [0, 3, 4, 6, 9, 10, 12]
    assert O.ntx_compressed(pg, keep) == 13
    assert list(O.reference_patch(pg, 3)) == [0, 1, 2]


def test_table_s2_readout_matrix_sizes():
    """SI Table S2: the explicitly stored readout encoding matrix is 298.6 GB
    with 3.2x RF-only and 53.1 GB with 18x joint compression."""
    gold = json.load(open(os.path.join(GOLD, "table_s2_sizes.json")))
    nx, ny, nz = gold["matrix"]
    nc, os_ = gold["coils"], gold["oversampling"]
    ntx = nx * os_
    # RF-only: every readout sample is its own patch, one shared group
    pg_rf = np.zeros(ntx, np.int32)
    k_rf = np.array([gold["rf_only"]["virtual_coils"]], np.int32)
    rf = O.readout_matrix_bytes(O.ntx_compressed(pg_rf, k_rf), nx, ny, nz)
    assert round(rf / 1e9, 1) == gold["rf_only"]["readout_matrix_GB"]
    # joint: 45-sample period, 5 groups of 9 samples, keep 16 of 288
    w, pg = synth.grouping_periodic(ntx, ntx / gold["period_samples"],
                                    gold["joint"]["groups_per_period"])
    assert w == gold["joint"]["samples_per_patch"]
    assert round(nc * w / gold["joint"]["keep"]) == 18
    keep = np.full(5, gold["joint"]["keep"], np.int32)
    ntxc = O.ntx_compressed(pg, keep)
    assert ntxc == 2560
    jt = O.readout_matrix_bytes(ntxc, nx, ny, nz)
    assert round(jt / 1e9, 1) == gold["joint"]["readout_matrix_GB"]
    assert round(rf / jt, 1) == gold["readout_matrix_ratio_printed"]
    assert O.periodic_grouping_ok(pg, w, gold["period_samples"])


def test_sampling_lines():
    ky, kz = synth.lines_regular(256, 3)
    assert len(ky) == 86 and ky[0] == 0 and ky[-1] == 255
    ky, kz = synth.lines_caipi(9, 6, 3, 3)
    pairs = set(zip(kz.tolist(), ky.tolist()))
    assert (0, 0) in pairs and (3, 1) in pairs and (0, 1) not in pairs
    assert all(k % 3 == 0 for k in kz)
    order = np.lexsort((ky, kz))
    assert np.all(order == np.arange(len(ky)))


def test_roi_pixels_raster_and_coverage():
    roi = np.zeros((1, 3, 4), np.uint8)
    roi[0, 1, 2] = roi[0, 2, 0] = roi[0, 0, 3] = 1
    c = np.ones((2, 1, 3, 4), complex)
    c[:, 0, 2, 0] = 0  # a pixel no coil sees
    assert list(O.roi_pixels(roi, c)) == [3, 6]


def test_variable_density_lines():
    """Seeded variable-density mask: reproducible, sorted and unique, the
    requested count, the centre always sampled, denser near the centre."""
    ny, accel = 256, 4
    a = synth.lines_variable_density(ny, accel, 5)
    b = synth.lines_variable_density(ny, accel, 5)
    assert np.array_equal(a[0], b[0]) and np.all(a[1] == 0)
    ky = a[0]
    assert len(ky) == 64 and np.all(np.diff(ky) > 0) and ky.min() >= 0 and ky.max() < ny
    assert set(range(ny // 2 - 8, ny // 2 + 8)) <= set(ky.tolist())
    kyc = np.abs(ky - ny // 2)
    assert np.sum(kyc < ny // 8) > np.sum(kyc >= 3 * ny // 8)
    assert not np.array_equal(ky, synth.lines_variable_density(ny, accel, 6)[0])


def _wave_as_field(g):
    """The linear wave of Eq. 3 written as one local field 2 pi y_c / N_y
    driven by a_y(t): the general-phase functions must reduce to the wave
    ones."""
    ay, _ = O.wave_coeffs(g.ntx, g.cycles, g.kappa_y, g.kappa_z)
    field = np.broadcast_to((2 * np.pi * O.centred(g.ny) / g.ny)[None, None, :, None],
                            (1, g.nz, g.ny, g.nx)).copy()
    return O.local_b0_phase(field, ay[None, :])


def test_general_phase_reduces_to_the_wave():
    g, c = _tiny2d(nx=8, ny=6, nc=3, os=2, cycles=2.0, kappa_y=1.3, n_groups=2, keep=4, lines="regular", r=2)
    phi = _wave_as_field(g)
    assert np.abs(phi[:, :, :, 3] - O.wave_phase(g)).max() < 1e-12
    roi = synth.roi_mask(synth.phantom(g.nx, g.ny))
    As, _, Ps = O.build_groups(g, c, roi)
    idx = O.roi_pixels(roi, c)
    for gi in range(g.n_groups):
        assert np.abs(O.gram_phase(g, c, idx, gi, phi) - Ps[gi]).max() < 1e-11 * len(idx)
    x = _rand(g.shape, 101)
    ref = O.Ec_apply(g, c, As, x)
    assert np.linalg.norm(O.Ec_apply_phase(g, c, As, phi, x) - ref) < 1e-12 * np.linalg.norm(ref)
    # the dense compressed matrix of the general phase is the same model
    D = O.dense_Ec_phase(g, c, As, phi)
    assert np.linalg.norm(D @ x.ravel() - ref.ravel()) < 1e-12 * np.linalg.norm(ref)


def test_dense_compressed_general_phase_reduces_to_the_wave():
    """With the wave phase written as a general phase, dense_Ec_phase is the
    wave model's dense_Ec."""
    g, c = _tiny2d(nx=8, ny=6, nc=2, os=2, cycles=2.0, kappa_y=1.3, n_groups=2, keep=3, lines="regular", r=2)
    As, _, _ = O.build_groups(g, c, np.ones(g.shape, np.uint8))
    D1 = O.dense_Ec_phase(g, c, As, _wave_as_field(g))
    D0 = O.dense_Ec(g, c, As)
    assert np.linalg.norm(D1 - D0) < 1e-12 * np.linalg.norm(D0)


def test_nonlinear_local_b0_model_equals_dense_E():
    """Three synthetic local B0 coils (x-dependent phase): the stored
    per-row readout matrices with the phase-encode DFT equal the compressed
    brute-force E (Eq. 1, 4, 13-14); the Gram keeps trace |ROI|."""
    g, c = _tiny2d(nx=8, ny=6, nc=3, os=2, cycles=2.0, kappa_y=0.0, n_groups=2, keep=4, lines="regular", r=2)
    phi = O.local_b0_phase(synth.local_b0_fields(g.nx, g.ny, 1, 3, 102), synth.local_b0_amplitudes(g.ntx, 2.0, 3, 103))
    assert np.ptp(phi[:, 0, 2, :], axis=1).max() > 0.5  # the phase varies along the readout
    roi = synth.roi_mask(synth.phantom(g.nx, g.ny))
    idx = O.roi_pixels(roi, c)
    Ps = [O.gram_phase(g, c, idx, gi, phi) for gi in range(g.n_groups)]
    As = [O.compression_matrix(P, int(g.keep[gi]), g.nc, g.w)[0] for gi, P in enumerate(Ps)]
    for P in Ps:
        assert abs(np.trace(P).real - len(idx)) < 1e-12 * len(idx)
        assert np.linalg.eigvalsh(P).min() > -1e-12 * len(idx)
    x = _rand(g.shape, 104)
    S = (O.dense_E_phase(g, c, phi) @ x.ravel()).reshape(g.n_lines, g.nc, g.ntx)
    ref = O.compress(g, As, S)
    assert np.linalg.norm(O.Ec_apply_phase(g, c, As, phi, x) - ref) < 1e-12 * np.linalg.norm(ref)
