"""E_c as a torch.autograd.Function: backward is the E_c^H kernel, checked
by finite differences and against the FP64 oracle's adjoint; unrolled,
checkpointed CG differentiates through the operator kernels."""
import numpy as np
import pytest

import oracle as O
from paper_2601_05418_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module")
def mods():
    import __graft_entry__ as ge

    ge.build()
    from paper_2601_05418_gb300 import autograd as AG
    from paper_2601_05418_gb300 import gpjc

    return gpjc, AG


def to_dev(a, dtype=np.complex64):
    return torch.from_numpy(np.ascontiguousarray(a.astype(dtype))).to(DEV)


def to_np(t):
    return t.detach().cpu().numpy().astype(np.complex128)


def setup(gpjc, name, seed=60):
    g = synth.workload(name).geom
    coils = synth.coil_maps(g.nx, g.ny, g.nz, g.nc, seed)
    rho = synth.phantom(g.nx, g.ny, g.nz)
    As, _, _ = O.build_groups(g, coils, synth.roi_mask(rho))
    op = gpjc.Operator(gpjc.Groups.from_matrices(gpjc.Plan(g), As), to_dev(coils))
    return g, coils, As, op


def redot(a, b):
    return float(torch.sum(a.real.double() * b.real.double() + a.imag.double() * b.imag.double()))


@pytest.mark.parametrize("name", ["2d128", "3d56"])
def test_ec_backward_is_fp64_adjoint_and_matches_fd(mods, name):
    gpjc, AG = mods
    g, coils, As, op = setup(gpjc, name)
    x = to_dev(synth.complex_normal(g.shape, 61)).requires_grad_(True)
    v_np = synth.complex_normal((g.n_lines, op.plan.ntx_c), 62)
    v = to_dev(v_np)
    y = AG.Ec.apply(x, op)
    L = torch.sum(y.real * v.real + y.imag * v.imag)  # Re <v, E_c x>
    L.backward()
    # the gradient is E_c^H v; compare with the FP64 oracle's adjoint
    ref = O.EcH_apply(g, coils, As, v_np)
    grad = to_np(x.grad)
    assert np.linalg.norm(grad - ref) < 1e-5 * np.linalg.norm(ref)
    # finite differences along random directions (L is linear: exact up to rounding)
    with torch.no_grad():
        for s in range(3):
            d = to_dev(synth.complex_normal(g.shape, 70 + s))
            eps = 1e-2
            lp = redot(AG.Ec.apply(x + eps * d, op), v)
            lm = redot(AG.Ec.apply(x - eps * d, op), v)
            fd = (lp - lm) / (2 * eps)
            an = redot(x.grad, d)
            assert abs(fd - an) < 1e-4 * (abs(an) + 1e-12) + 1e-6 * np.linalg.norm(grad) * np.linalg.norm(to_np(d))


def test_unrolled_cg_matches_library_cg_and_fd(mods):
    gpjc, AG = mods
    g, coils, As, op = setup(gpjc, "2d128", 63)
    rho = synth.phantom(g.nx, g.ny)
    S = O.simulate(g, coils, rho, synth.complex_normal((g.n_lines, g.nc, g.ntx), 64, 1e-3))
    Sc = to_dev(O.compress(g, As, S))
    iters = 6
    x_lib, _ = op.recon(Sc, alg=gpjc.CG, iters=iters)
    Sc_req = Sc.clone().requires_grad_(True)
    x_ag = AG.unrolled_cg(op, Sc_req, iters, use_checkpoint=True)
    assert torch.linalg.vector_norm(x_ag - x_lib) < 1e-4 * torch.linalg.vector_norm(x_lib)
    w = to_dev(synth.complex_normal(g.shape, 65))
    L = torch.sum(x_ag.real * w.real + x_ag.imag * w.imag)
    L.backward()
    g_ck = Sc_req.grad.clone()
    # the same without checkpointing gives the same gradient
    Sc2 = Sc.clone().requires_grad_(True)
    L2 = AG.unrolled_cg(op, Sc2, iters, use_checkpoint=False)
    torch.sum(L2.real * w.real + L2.imag * w.imag).backward()
    assert torch.linalg.vector_norm(Sc2.grad - g_ck) < 1e-4 * torch.linalg.vector_norm(g_ck)
    # finite difference of the (nonlinear in Sc) unrolled map along one direction
    with torch.no_grad():
        d = to_dev(synth.complex_normal(tuple(Sc.shape), 66)) * (torch.linalg.vector_norm(Sc) / np.sqrt(Sc.numel()))
        eps = 1e-3
        lp = redot(AG.unrolled_cg(op, Sc + eps * d, iters), w)
        lm = redot(AG.unrolled_cg(op, Sc - eps * d, iters), w)
        fd = (lp - lm) / (2 * eps)
        an = redot(g_ck, d)
        assert abs(fd - an) < 2e-2 * abs(an), (fd, an)
