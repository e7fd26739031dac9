"""Batched persistent CG (one cooperative launch for many uneven slices)
against the single-slice path and the FP64 oracle, and the bounded-wait
failure path.  Slices differ in matrix size, coil count, oversampling and
group count, like the uneven batch workload (at sizes the oracle finishes
in seconds)."""
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


SPECS = [  # (N, coils, os, groups)
    (32, 4, 4, 4), (48, 6, 6, 6), (64, 8, 8, 8), (40, 5, 4, 4), (56, 4, 8, 7), (64, 6, 4, 8),
]


def make_slices(gp, iters):
    out = []
    for i, (n, nc, os_, G) in enumerate(SPECS):
        g = synth._geom_2d(n, nc, os_, 8, 2.5, G, 6.0, 3)
        coils = synth.coil_maps(n, n, 1, nc, 100 + i)
        rho = synth.phantom(n, n)
        roi = synth.roi_mask(rho)
        S = O.simulate(g, coils, rho, synth.complex_normal((g.n_lines, nc, g.ntx), 200 + i, 1e-3))
        As, _, _ = O.build_groups(g, coils, roi)
        Sc = O.compress(g, As, S)
        x_ref, _ = O.reconstruct(g, coils, As, Sc, "cg", iters)
        grp = gp.Groups.from_matrices(gp.Plan(g), As)
        op = gp.Operator(grp, to_dev(coils))
        out.append((g, op, to_dev(Sc), x_ref))
    return out


def test_batched_cg_matches_single_and_oracle(gp):
    iters = 12
    sl = make_slices(gp, iters)
    batch = gp.Batch([s[1] for s in sl], iters)
    grid, items = batch.info()
    assert grid >= 152 and items > 0
    xs, status = batch.recon([s[2] for s in sl])
    assert status == 0
    for (g, op, Sc, x_ref), xb in zip(sl, xs):
        xs1, _ = op.recon(Sc, alg=gp.CG, iters=iters, use_graph=False)
        a, b = to_np(xb), to_np(xs1)
        check_close(a, b, 1e-5, 'batch vs single slice')
        check_image(a, x_ref, 1e-5)
    # graph replay with the same pointers gives the same images
    xs2, status = batch.recon([s[2] for s in sl], xs)
    assert status == 0


def test_batched_cg_wait_budget_runs_out(gp):
    """A wait budget of 0 cycles makes the first dependent wait give up: the
    launch must abort cleanly with GPJC_ETIMEOUT and leave the device usable."""
    sl = make_slices(gp, 2)
    batch = gp.Batch([s[1] for s in sl], 2)
    batch.set_wait_budget(0)
    with pytest.raises(gp.GpjcError) as ei:
        batch.recon([s[2] for s in sl], use_graph=False)
    assert ei.value.status == gp.GPJC_ETIMEOUT
    torch.cuda.synchronize()
    batch.set_wait_budget(4_000_000_000)
    xs, status = batch.recon([s[2] for s in sl], use_graph=False)
    assert status == 0
    g, op, Sc, x_ref = sl[0]
    check_image(to_np(xs[0]), x_ref, 1e-5)


def test_multi_slice_graph_matches_single_slice_and_oracle(gp):
    """The multi-slice graph (slices on parallel branches of one CUDA graph)
    runs each slice's reconstruction with the single-slice kernels: the images
    are bit-identical to gpjc_recon's, and within the FP32 bound of the
    oracle; a 3D slice and a BF16 slice ride along."""
    iters = 12
    sl = make_slices(gp, iters)
    wl = synth.workload("3d56")
    g3 = wl.geom
    c3 = synth.make_case(wl)
    As3, _, _ = O.build_groups(g3, c3.coils, c3.roi)
    Sc3 = O.compress(g3, As3, O.simulate(g3, c3.coils, c3.rho, c3.noise))
    x3_ref, _ = O.reconstruct(g3, c3.coils, As3, Sc3, "cg", iters)
    op3 = gp.Operator(gp.Groups.from_matrices(gp.Plan(g3), As3), to_dev(c3.coils))
    g, op0, Sc0, x0_ref = sl[2]
    op16 = gp.Operator(op0.groups, op0.coil, gp.BF16)
    ops = [s[1] for s in sl] + [op3, op16]
    scs = [s[2] for s in sl] + [to_dev(Sc3), Sc0]
    refs = [s[3] for s in sl] + [x3_ref, x0_ref]
    multi = gp.Multi(ops, n_branches=3)
    xs, status = multi.recon(scs, iters=iters)
    assert status == 0
    for k, (op, sc, xm, ref) in enumerate(zip(ops, scs, xs, refs)):
        x1, _ = op.recon(sc, alg=gp.CG, iters=iters, use_graph=False)
        torch.cuda.synchronize()
        assert torch.equal(xm, x1), k
        check_image(to_np(xm), ref, 1e-5 if op is not op16 else 1e-3, f"multi slice {k}")
    # replay of the cached graph gives the same images
    xs2, status = multi.recon(scs, xs, iters=iters)
    assert status == 0 and all(torch.equal(a, b) for a, b in zip(xs, xs2))


def test_multi_slice_graph_rejects_a_repeated_operator(gp):
    sl = make_slices(gp, 2)
    with pytest.raises(gp.GpjcError) as ei:
        gp.Multi([sl[0][1], sl[1][1], sl[0][1]])
    assert ei.value.status == gp.GPJC_EINVAL


def test_uneven_batch_workload_sizes_vs_oracle(gp):
    """Slices of the uneven batch workload itself (matrix 192-320, 16-32
    coils, 6-8x oversampling, 16-48 groups; the two with the least readout
    work, so the oracle finishes in seconds): the persistent batch and the
    multi-slice graph against the FP64 oracle, CG-SENSE 5 iterations."""
    iters = 5
    wls = synth.batch_workloads(64)
    wls = sorted(wls, key=lambda w: w.geom.nx * w.geom.ny * w.geom.nc * w.geom.os)[:2]
    ops, scs, refs = [], [], []
    for wl in wls:
        g = wl.geom
        assert 192 <= g.nx <= 320 and 16 <= g.nc <= 32
        coils = synth.coil_maps(g.nx, g.ny, 1, g.nc, wl.seed)
        rho = synth.phantom(g.nx, g.ny)
        roi = synth.roi_mask(rho)
        S = O.simulate(g, coils, rho, synth.complex_normal((g.n_lines, g.nc, g.ntx), wl.seed + 1, wl.sigma))
        As, _, _ = O.build_groups(g, coils, roi)
        Sc = O.compress(g, As, S)
        x_ref, _ = O.reconstruct(g, coils, As, Sc, "cg", iters)
        ops.append(gp.Operator(gp.Groups.from_matrices(gp.Plan(g), As), to_dev(coils)))
        scs.append(to_dev(Sc))
        refs.append(x_ref)
    xb, status = gp.Batch(ops, iters).recon(scs)
    assert status == 0
    xm, status = gp.Multi(ops, n_branches=2).recon(scs, iters=iters)
    assert status == 0
    for a, b, ref in zip(xb, xm, refs):
        check_image(to_np(a), ref, 1e-5, "persistent batch, uneven-batch slice")
        check_image(to_np(b), ref, 1e-5, "multi-slice graph, uneven-batch slice")
