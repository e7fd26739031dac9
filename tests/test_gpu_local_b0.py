"""Nonlinear local-B0 modulation on the device (Sec. 2.1-2.2, Eq. 2-3, 14):
the stored compressed readout matrices G_row (built on the device from A_g,
the coil maps and the local-B0 phase sum_l a_l(t) B_l(r)) against the
oracle's dense compressed model of the same phase.

Compression matrices come from the oracle's Gram of the general phase
(gram_phase, Eq. 7-12).  Tolerance: FP32 path, 1e-5 relative L2 with the
element-wise bound of tests/_checks.py for single applications, NRMSE
1e-5 for the CG image.  The fields are rounded to FP32 before the oracle
uses them (the device reads FP32 fields); the drive is rounded to FP32 on
the device (relative change ~6e-8)."""
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


def case(name):
    if name == "2d":  # nx = 40: two x tiles of the build, the second ragged
        g = synth.tiny_geometry(nx=40, ny=24, nz=1, nc=4, os=2, cycles=2.0, kappa_y=0.0, n_groups=5, keep=10,
                                lines="regular", r=2)
    else:
        g = synth.tiny_geometry(nx=16, ny=12, nz=6, nc=3, os=2, cycles=2.0, kappa_y=0.0, n_groups=4, keep=8,
                                grouping="contiguous", lines="caipi", r=2)
    coils = synth.coil_maps(g.nx, g.ny, g.nz, g.nc, 91)
    fields = synth.local_b0_fields(g.nx, g.ny, g.nz, 3, 92).astype(np.float32)
    amps = synth.local_b0_amplitudes(g.ntx, 2.0, 3, 93)
    phi = O.local_b0_phase(fields.astype(np.float64), amps)
    rho = synth.phantom(g.nx, g.ny, g.nz)
    roi = synth.roi_mask(rho)
    idx = O.roi_pixels(roi, coils)
    As = [O.compression_matrix(O.gram_phase(g, coils, idx, gi, phi), int(g.keep[gi]), g.nc, g.w)[0]
          for gi in range(g.n_groups)]
    D = O.dense_Ec_phase(g, coils, As, phi)
    return g, coils, fields, amps, As, D, rho


@pytest.mark.parametrize("name", ["2d", "3d"])
def test_local_b0_operator_matches_dense_model(gp, name):
    g, coils, fields, amps, As, D, rho = case(name)
    plan = gp.Plan(g)
    grp = gp.Groups.from_matrices(plan, As)
    op = gp.Operator.local_b0(grp, to_dev(coils), torch.from_numpy(fields).to(DEV), amps)
    x = synth.complex_normal(g.shape, 94)
    y = to_np(op.E(to_dev(x)))
    check_close(y.ravel(), D @ x.ravel(), 1e-5, "local-B0 E_c")
    v = synth.complex_normal((g.n_lines, plan.ntx_c), 95)
    xa = to_np(op.EH(to_dev(v)))
    check_close(xa.ravel(), D.conj().T @ v.ravel(), 1e-5, "local-B0 E_c^H")
    # CG-SENSE with the stored-matrix operator
    Sc = (D @ rho.ravel()).reshape(g.n_lines, -1) + synth.complex_normal((g.n_lines, plan.ntx_c), 96, 1e-3)
    ref, _ = O.cg(lambda u: (D.conj().T @ (D @ u.ravel())).reshape(g.shape), (D.conj().T @ Sc.ravel()).reshape(g.shape),
                  12)
    xr, info = op.recon(to_dev(Sc), alg=gp.CG, iters=12)
    assert info["status"] == 0
    check_image(to_np(xr), ref, 1e-5, "local-B0 CG")
    # the x-dependent phase matters: the wave operator of the same groups differs
    assert np.linalg.norm(y.ravel() - to_np(gp.Operator(grp, to_dev(coils)).E(to_dev(x))).ravel()) > \
        0.1 * np.linalg.norm(y)


def test_local_b0_operator_refuses_the_uncompressed_model(gp):
    g, coils, fields, amps, As, D, rho = case("2d")
    grp = gp.Groups.from_matrices(gp.Plan(g), As)
    op = gp.Operator.local_b0(grp, to_dev(coils), torch.from_numpy(fields).to(DEV), amps)
    with pytest.raises(gp.GpjcError) as ei:
        op.simulate(to_dev(rho))
    assert ei.value.status == gp.GPJC_EUNSUPPORTED
    bad = amps.copy()
    bad[0, 3] = np.inf
    with pytest.raises(gp.GpjcError) as ei:
        gp.Operator.local_b0(grp, to_dev(coils), torch.from_numpy(fields).to(DEV), bad)
    assert ei.value.status == gp.GPJC_EINVAL
