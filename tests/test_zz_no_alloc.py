"""The allocation-free adjoint (gpjc_apply_EH_static) against the ordinary
adjoint (gpjc_apply_EH), through the C ABI.

It serves callers that cannot allocate device memory where they apply
E_c^H: its scratch is a fixed array inside the library.  Two calls in a
row must both agree with the operator's adjoint (the shared scratch keeps the
previous call's contents, which must not leak into the next result).  This
file is collected last so that a run stopping at the first failure has run
every other test before it."""
import numpy as np
import pytest

import oracle as O
from paper_2601_05418_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _rel(a, b):
    return float(torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b))


def test_static_adjoint_matches_operator_adjoint_twice():
    import __graft_entry__ as ge

    ge.build()
    from paper_2601_05418_gb300 import gpjc

    dev = "cuda:0"
    wl = synth.workload("2d128")
    g = wl.geom
    case = synth.make_case(wl, with_noise=False)
    As, _, _ = O.build_groups(g, case.coils, case.roi)
    plan = gpjc.Plan(g)
    grp = gpjc.Groups.from_matrices(plan, As)
    coils = torch.from_numpy(case.coils.astype(np.complex64)).to(dev)
    op = gpjc.Operator(grp, coils)
    ys = [torch.from_numpy(synth.complex_normal((g.n_lines, plan.ntx_c), s).astype(np.complex64)).to(dev)
          for s in (31, 32)]
    for y in ys:  # second call sees the first call's scratch contents
        ref = op.EH(y)
        got = gpjc.apply_EH_static(grp, coils, y)
        torch.cuda.synchronize()
        assert _rel(got, ref) < 1e-5


def test_static_adjoint_rejects_oversized_geometry():
    import __graft_entry__ as ge

    ge.build()
    from paper_2601_05418_gb300 import gpjc

    # 3D: two 2048-row x 1536-column complex64 matrices = 48 MiB > 32 MiB of scratch
    big = synth.geom_3d(64, 64, 32, 8, 6, 12, 1.0, 1.0, 12, 2.0)
    plan = gpjc.Plan(big)
    A = [np.eye(int(k), big.ns, dtype=np.complex64) for k in big.keep]
    grp = gpjc.Groups.from_matrices(plan, A)
    coils = torch.zeros((big.nc, big.nz, big.ny, big.nx), dtype=torch.complex64, device="cuda:0")
    y = torch.zeros((big.n_lines, plan.ntx_c), dtype=torch.complex64, device="cuda:0")
    with pytest.raises(gpjc.GpjcError) as ei:
        gpjc.apply_EH_static(grp, coils, y)
    assert ei.value.status == gpjc.GPJC_EINVAL
    assert "static scratch" in str(ei.value)
