"""TV-regularised FISTA on the device (Eq. 17: Haar l1 + smoothed isotropic
TV, the TV term in the gradient step) against the FP64 oracle's FISTA, on a
regular R = 3 mask and on a seeded variable-density random mask (the
stand-in for the paper's Poisson-disc variable-density masks).

Tolerance: FP32 path, images within NRMSE 1e-5 of the oracle (and the
element-wise bound of tests/_checks.py), as for the l1-only FISTA.  The
step size 1/L with L = L(E_c^H E_c) + 8 lambda_tv / eps is passed to both
sides; the device's own power iteration must reproduce it."""
import numpy as np
import pytest

import oracle as O
from _checks import check_image
from paper_2601_05418_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"
LAM, LAM_TV, EPS = 1e-3, 2e-3, 0.05


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


def _geom(mask):
    g = synth._geom_2d(64, 8, 4, 8, 2.5, 16, 8.0, 3)
    if mask == "vd":
        ky, kz = synth.lines_variable_density(g.ny, 3.0, 71, center=12)
        g.line_ky, g.line_kz = ky, kz
    return g


def _problem(g, seed):
    coils = synth.coil_maps(g.nx, g.ny, g.nz, g.nc, seed)
    rho = synth.phantom(g.nx, g.ny)
    roi = synth.roi_mask(rho)
    S = O.simulate(g, coils, rho, synth.complex_normal((g.n_lines, g.nc, g.ntx), seed + 1, 1e-3))
    As, _, _ = O.build_groups(g, coils, roi)
    Sc = O.compress(g, As, S)
    pb = O.Problem(g, coils, As)
    return coils, As, Sc, pb


@pytest.mark.parametrize("mask", ["regular", "vd"])
def test_tv_fista_matches_oracle(gp, mask):
    g = _geom(mask)
    coils, As, Sc, pb = _problem(g, 72)
    b = pb.EcH(Sc)
    L = O.power_lipschitz(pb.normal_c, b, 20) + 8.0 * LAM_TV / EPS
    x_ref = O.fista(pb.normal_c, b, L, LAM, 3, 30, lam_tv=LAM_TV, eps_tv=EPS)
    op = gp.Operator(gp.Groups.from_matrices(gp.Plan(g), As), to_dev(coils))
    x, info = op.recon(to_dev(Sc), alg=gp.FISTA, iters=30, lam=LAM, lipschitz=L, haar_levels=3, lam_tv=LAM_TV,
                       tv_eps=EPS)
    assert info["status"] == 0
    check_image(to_np(x), x_ref, 1e-5, f"TV-FISTA ({mask} mask)")
    # the TV term changes the image (it is not silently dropped)
    x_l1 = O.fista(pb.normal_c, b, L, LAM, 3, 30)
    assert O.nrmse(x_ref, x_l1) > 1e-3


def test_tv_fista_step_size_from_device_power_iteration(gp):
    g = _geom("regular")
    coils, As, Sc, pb = _problem(g, 73)
    b = pb.EcH(Sc)
    L = O.power_lipschitz(pb.normal_c, b, 20) + 8.0 * LAM_TV / EPS
    op = gp.Operator(gp.Groups.from_matrices(gp.Plan(g), As), to_dev(coils))
    _, info = op.recon(to_dev(Sc), alg=gp.FISTA, iters=1, lam=LAM, haar_levels=3, power_iters=20, lam_tv=LAM_TV,
                       tv_eps=EPS)
    assert abs(info["lipschitz"] - L) < 1e-5 * L


def test_tv_fista_rejects_bad_parameters(gp):
    g = _geom("regular")
    coils, As, Sc, _ = _problem(g, 74)
    op = gp.Operator(gp.Groups.from_matrices(gp.Plan(g), As), to_dev(coils))
    for kw in ({"lam_tv": -1.0}, {"lam_tv": 1e-3, "tv_eps": 0.0}, {"lam_tv": 1e-3, "tv_eps": 1e-30}):
        with pytest.raises(gp.GpjcError) as ei:
            op.recon(to_dev(Sc), alg=gp.FISTA, iters=2, lam=LAM, haar_levels=3, **kw)
        assert ei.value.status == gp.GPJC_EINVAL
