"""Failure paths and supporting calls of the C ABI on the device, all made
on the host side (no GPU fault is provoked): a NaN planted in the compressed
data S', an allocation failure injected into the library's allocator, and
the workspace query.  Also the smoothed-TV gradient kernel against the
oracle (Eq. 17's TV term)."""
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


def _small_problem(gp, seed=61):
    g = synth.tiny_geometry(nx=40, ny=36, nz=1, nc=5, os=3, cycles=4.0, kappa_y=1.7, n_groups=3,
                            lines="regular", r=2)
    coils = synth.coil_maps(g.nx, g.ny, g.nz, g.nc, seed)
    rho = synth.phantom(g.nx, g.ny)
    roi = synth.roi_mask(rho)
    As, _, _ = O.build_groups(g, coils, roi)
    S = O.simulate(g, coils, rho, synth.complex_normal((g.n_lines, g.nc, g.ntx), seed + 1, 1e-3))
    Sc = O.compress(g, As, S)
    op = gp.Operator(gp.Groups.from_matrices(gp.Plan(g), As), to_dev(coils))
    return g, coils, As, Sc, op


@pytest.mark.parametrize("alg", ["cg", "fista"])
def test_nan_in_data_reports_nonfinite_and_device_stays_usable(gp, alg):
    g, coils, As, Sc, op = _small_problem(gp)
    bad = Sc.copy()
    bad[g.n_lines // 2, 3] = np.nan  # planted on the host
    a = gp.CG if alg == "cg" else gp.FISTA
    kw = {} if alg == "cg" else {"lam": 1e-3, "haar_levels": 2}
    # gpjc_recon returns the device-side verdict as its status
    with pytest.raises(gp.GpjcError) as ei:
        op.recon(to_dev(bad), alg=a, iters=5, **kw)
    assert ei.value.status == gp.GPJC_ENONFINITE
    # the same operator and device still reconstruct the clean data correctly
    x, info = op.recon(to_dev(Sc), alg=gp.CG, iters=10)
    assert info["status"] == 0
    pb = O.Problem(g, coils, As)
    ref, _ = O.cg(pb.normal_c, pb.EcH(Sc), 10, fwd=pb.Ec, adj=pb.EcH)
    check_image(to_np(x), ref, 1e-5)


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_query_matches_operator_workspace(gp, prec):
    """gpjc_query reports N'_tx and the device bytes gpjc_op_create takes;
    the device's free memory drops by that much (plus cudaMalloc's
    rounding of each of the ~20 buffers to 2 MiB pages) when the operator
    is created, and comes back when it is destroyed."""
    wl = synth.workload("2d128")
    g = wl.geom
    case = synth.make_case(wl, with_noise=False)
    As, _, _ = O.build_groups(g, case.coils, case.roi)
    plan = gp.Plan(g)
    grp = gp.Groups.from_matrices(plan, As)
    ntxc, nbytes = grp.query(prec)
    assert ntxc == plan.ntx_c == int(O.ntx_compressed(g.patch_group, g.keep))
    coils = to_dev(case.coils)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    op = gp.Operator(grp, coils, prec)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    used = free0 - free1
    assert nbytes <= used <= nbytes + 24 * (2 << 20) + (16 << 20), (nbytes, used)
    del op
    torch.cuda.synchronize()
    free2, _ = torch.cuda.mem_get_info()
    assert abs(free2 - free0) <= (4 << 20)


def test_query_rejects_bad_arguments(gp):
    g = synth.workload("2d128").geom
    grp = gp.Groups.from_matrices(gp.Plan(g), [np.eye(int(k), g.ns, dtype=np.complex64) for k in g.keep])
    with pytest.raises(gp.GpjcError) as ei:
        grp.query(7)
    assert ei.value.status == gp.GPJC_EINVAL
    with pytest.raises(gp.GpjcError) as ei:
        grp.query(0, nchunk=g.nc + 1)
    assert ei.value.status == gp.GPJC_EINVAL


@pytest.mark.parametrize("budget", [0, 3, 9])
def test_injected_allocation_failure_reports_enomem_without_leaks(gp, budget):
    g, coils, As, Sc, _ = _small_problem(gp)
    plan = gp.Plan(g)
    grp = gp.Groups.from_matrices(plan, As)
    c_d = to_dev(coils)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    gp.debug_fail_allocations(budget)
    try:
        with pytest.raises(gp.GpjcError) as ei:
            gp.Operator(grp, c_d)
        assert ei.value.status == gp.GPJC_ENOMEM
    finally:
        gp.debug_fail_allocations(-1)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert abs(free1 - free0) <= (4 << 20)
    op = gp.Operator(grp, c_d)  # allocation works again
    x, info = op.recon(to_dev(Sc), alg=gp.CG, iters=3)
    assert info["status"] == 0


def test_tv_gradient_matches_oracle(gp):
    """Three ragged slices (13 x 19), eps 0.05: FP32 differences and one
    rsqrt per pixel, relative error ~1e-7 per term."""
    nz, ny, nx, eps = 3, 13, 19, 0.05
    u = synth.complex_normal((nz, ny, nx), 62)
    ref = np.stack([O.tv_smooth_grad(u[k], eps) for k in range(nz)])
    got = to_np(gp.tv_grad(to_dev(u), eps))
    check_close(got, ref, 1e-5, "tv gradient")
    # one 256 x 256 slice: the grid-stride loop covers more pixels than threads
    u2 = synth.complex_normal((1, 256, 256), 63)
    check_close(to_np(gp.tv_grad(to_dev(u2), eps)), O.tv_smooth_grad(u2[0], eps)[None], 1e-5, "tv 256")


def test_tv_gradient_rejects_underflowing_eps(gp):
    u = to_dev(synth.complex_normal((1, 8, 8), 64))
    with pytest.raises(gp.GpjcError) as ei:
        gp.tv_grad(u, 1e-30)
    assert ei.value.status == gp.GPJC_EINVAL
