"""The allocation-free adjoint (gpjc_apply_EH_static) through the C ABI.

It serves callers that cannot allocate device memory where they apply
E_c^H (for example code running inside a component that forbids
cudaMalloc after start-up: cudaMalloc and cudaFree synchronise the device
and can fail under a fixed memory budget); its scratch is a fixed array
inside the library.  Two calls in a row must both agree with the ordinary
adjoint (gpjc_apply_EH) and with the FP64 oracle's E_c^H, in 2D and in 3D
(where the phase-encode intermediate sits behind the hybrid matrix in the
array): the shared scratch keeps the previous call's contents, which must not
leak into the next result.  This file is collected last so that a run
stopping at the first failure has run every other test before it."""
import numpy as np
import pytest

import oracle as O
from _checks import check_close
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


@pytest.mark.parametrize("name", ["2d128", "3d56"])
def test_static_adjoint_matches_adjoint_and_oracle_twice(gp, name):
    wl = synth.workload(name)
    g = wl.geom
    case = synth.make_case(wl, with_noise=False)
    As, _, _ = O.build_groups(g, case.coils, case.roi)
    plan = gp.Plan(g)
    grp = gp.Groups.from_matrices(plan, As)
    coils = torch.from_numpy(case.coils.astype(np.complex64)).to(DEV)
    op = gp.Operator(grp, coils)
    ys = [synth.complex_normal((g.n_lines, plan.ntx_c), s) for s in (31, 32)]
    for y in ys:  # the second call sees the first call's scratch contents
        y_d = torch.from_numpy(y.astype(np.complex64)).to(DEV)
        ref = op.EH(y_d)
        got = gp.apply_EH_static(grp, coils, y_d)
        torch.cuda.synchronize()
        got_np = got.cpu().numpy().astype(np.complex128)
        check_close(got_np, ref.cpu().numpy().astype(np.complex128), 1e-5, "static vs gpjc_apply_EH")
        check_close(got_np, O.EcH_apply(g, case.coils, As, y.astype(np.complex64).astype(np.complex128)), 1e-5,
                    "static vs oracle")


def test_static_adjoint_rejects_oversized_geometry(gp):
    # 3D: two 2048-row x 1536-column complex64 matrices = 48 MiB > 32 MiB of scratch
    big = synth.geom_3d(64, 64, 32, 8, 6, 12, 1.0, 1.0, 12, 2.0)
    plan = gp.Plan(big)
    A = [np.eye(int(k), big.ns, dtype=np.complex64) for k in big.keep]
    grp = gp.Groups.from_matrices(plan, A)
    coils = torch.zeros((big.nc, big.nz, big.ny, big.nx), dtype=torch.complex64, device=DEV)
    y = torch.zeros((big.n_lines, plan.ntx_c), dtype=torch.complex64, device=DEV)
    with pytest.raises(gp.GpjcError) as ei:
        gp.apply_EH_static(grp, coils, y)
    assert ei.value.status == gp.GPJC_EINVAL
    assert "static scratch" in str(ei.value)


def test_static_adjoint_rejects_wrong_buffers(gp):
    """Shapes are checked by the binding; a buffer that is not device memory
    of the current device is refused by the C entry point before any launch."""
    import ctypes

    g = synth.workload("2d128").geom
    plan = gp.Plan(g)
    grp = gp.Groups.from_matrices(plan, [np.eye(int(k), g.ns, dtype=np.complex64) for k in g.keep])
    coils = torch.zeros((g.nc, g.nz, g.ny, g.nx), dtype=torch.complex64, device=DEV)
    y = torch.zeros((g.n_lines, plan.ntx_c), dtype=torch.complex64, device=DEV)
    with pytest.raises(ValueError):
        gp.apply_EH_static(grp, coils, y[:-1])
    with pytest.raises(ValueError):
        gp.apply_EH_static(grp, coils[:-1], y)
    with pytest.raises(ValueError):
        gp.apply_EH_static(grp, coils, y, out=torch.zeros((g.nz, g.ny, g.nx - 1), dtype=torch.complex64,
                                                         device=DEV))
    host_x = np.zeros((g.nz, g.ny, g.nx), np.complex64)
    out = torch.zeros((g.nz, g.ny, g.nx), dtype=torch.complex64, device=DEV)
    st = gp.lib().gpjc_apply_EH_static(grp.h, ctypes.c_void_p(coils.data_ptr()), ctypes.c_void_p(y.data_ptr()),
                                       ctypes.c_void_p(host_x.ctypes.data), None)
    assert st == gp.GPJC_EINVAL
    # the device is still usable and the entry point still works
    gp.apply_EH_static(grp, coils, y, out=out)
    torch.cuda.synchronize()
    assert float(out.abs().max()) == 0.0
