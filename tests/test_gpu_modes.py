"""Compression modes and diagnostics on the device (Sec. 2.4):

* RF-only compression, the special case E_g = E_RF (one sample per patch,
  one group): every P_g is the coil-only Gram sum_r c c^H / ||c||^2 and A_g
  is the classic coil-compression matrix;
* the eigen-spectrum of P_g at the 256 x 256 workload (the leading Ritz
  values the group build returns) against the oracle's full eigenvalue
  list, and the energy-threshold keep decided from either;
* the 3D volume with per-period groups (14 cycles over the readout give an
  integer period, 48 groups of w = 2), at its reduced size, FP32 and the
  16-bit tensor-core paths against the oracle.
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


def rf_only_geometry(keep):
    nx = ny = 64
    os = 2
    ky, kz = synth.lines_regular(ny, 2)
    return synth.Geometry(nx=nx, ny=ny, nz=1, nc=8, os=os, cycles=4.0, kappa_y=2.0, kappa_z=0.0, w=1, n_groups=1,
                          patch_group=np.zeros(os * nx, np.int32), keep=np.array([keep], np.int32),
                          line_ky=ky, line_kz=kz)


def test_rf_only_compression_on_the_device(gp):
    g = rf_only_geometry(4)
    coils = synth.coil_maps(g.nx, g.ny, g.nz, g.nc, 101)
    rho = synth.phantom(g.nx, g.ny)
    roi = synth.roi_mask(rho)
    grp = gp.Groups.build(gp.Plan(g), to_dev(coils), to_dev(roi, np.uint8))
    A, ritz = grp.matrices()
    # the coil-only Gram, written out: sum over the ROI of c c^H / ||c||^2
    idx = O.roi_pixels(roi, coils)
    c = coils.reshape(g.nc, -1)[:, idx]
    P = (c / np.sum(np.abs(c) ** 2, axis=0)) @ c.conj().T
    ev, U = np.linalg.eigh(P)
    Uk = U[:, ::-1][:, :4]
    a = A[0].astype(np.complex128)
    assert np.linalg.norm(a.conj().T @ a - Uk @ Uk.conj().T, 2) < 1e-5
    np.testing.assert_allclose(ritz[0][:4], ev[::-1][:4], rtol=1e-5)
    # and the oracle's group build (w = 1) is the same compression
    As, _, _ = O.build_groups(g, coils, roi)
    assert np.linalg.norm(As[0].conj().T @ As[0] - Uk @ Uk.conj().T, 2) < 1e-10
    # reconstruction with it
    S = O.simulate(g, coils, rho, synth.complex_normal((g.n_lines, g.nc, g.ntx), 102, 1e-3))
    Sc = O.compress(g, As, S)
    x_ref, _ = O.reconstruct(g, coils, As, Sc, "cg", 15)
    op = gp.Operator(gp.Groups.from_matrices(gp.Plan(g), As), to_dev(coils))
    x, _ = op.recon(to_dev(Sc), alg=gp.CG, iters=15)
    check_image(to_np(x), x_ref, 1e-5, "RF-only CG")


def test_spectrum_2d256_matches_oracle_eigenvalues(gp):
    """Leading Ritz values of four groups of the 256 x 256 workload against
    numpy's full eigenvalue list of the oracle's P_g; the energy-threshold
    keep (90%, 95%, 99% of trace(P_g) = |ROI|) from either list agrees."""
    wl = synth.workload("2d256")
    g = wl.geom
    case = synth.make_case(wl, with_noise=False)
    grp = gp.Groups.build(gp.Plan(g), to_dev(case.coils), to_dev(case.roi, np.uint8))
    _, ritz = grp.matrices()
    idx = O.roi_pixels(case.roi, case.coils)
    b = ritz.shape[1]
    for gi in (0, 7, 16, 31):
        ev = np.linalg.eigvalsh(O.gram(g, case.coils, idx, gi))[::-1]
        assert abs(ev.sum() - len(idx)) < 1e-9 * len(idx)
        k = int(g.keep[gi])
        np.testing.assert_allclose(ritz[gi][:k], ev[:k], rtol=1e-5, atol=1e-7 * ev[0])
        for thr in (0.9, 0.95, 0.99):
            k_ref = O.keep_from_energy(ev[None, :], thr, len(idx))[0]
            if k_ref <= b - 8:  # decided well inside the returned Ritz values
                k_gpu = gp.keep_from_energy(ritz[gi:gi + 1], thr, float(len(idx)))[0]
                assert k_gpu == k_ref, (gi, thr, k_gpu, k_ref)


@pytest.fixture(scope="module")
def periodic_3d():
    """The reduced periodic-group 3D case and its oracle image (computed once)."""
    wl = synth.workload("3d56r1")
    g = wl.geom
    case = synth.make_case(wl)
    S = O.simulate(g, case.coils, case.rho, case.noise)
    As, _, _ = O.build_groups(g, case.coils, case.roi)
    x_ref, _ = O.reconstruct(g, case.coils, As, O.compress(g, As, S), "cg", wl.iters)
    return wl, case, S, x_ref


@pytest.mark.parametrize("prec,tc", [(0, None), (1, None), (2, None), (1, "1"), (2, "1")])
def test_3d_periodic_groups_end_to_end(gp, prec, tc, periodic_3d, monkeypatch):
    """w = 2: the 16-bit operators keep the FP32 readout kernels by default
    (no spectra buffer in their workspace); GPJC_TC_READOUT=1 forces the
    tensor-core readout, which must agree as well."""
    wl, case, S, x_ref = periodic_3d
    g = wl.geom
    assert (g.w, g.n_groups, g.ntx // g.w) == (2, 12, 168)
    if tc is not None:
        monkeypatch.setenv("GPJC_TC_READOUT", tc)
    plan = gp.Plan(g)
    c_d = to_dev(case.coils)
    grp = gp.Groups.build(plan, c_d, to_dev(case.roi, np.uint8))
    spectra = g.ny * g.nz * g.nc * g.ntx * 8
    ws = grp.query(prec)[1] - grp.query(0)[1]
    assert ws == (spectra if (prec and tc == "1") else 0)
    op = gp.Operator(grp, c_d, prec)
    x, info = op.recon(gp.compress(grp, to_dev(S), prec), alg=gp.CG, iters=wl.iters)
    assert info["status"] == 0
    check_image(to_np(x), x_ref, 1e-5 if prec == 0 else 1e-3, f"3d56r1 precision {prec} tc {tc}")
