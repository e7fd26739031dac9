#!/usr/bin/env python
"""Benchmark of the group-patch joint compression hot path on GB300.

One step = the whole hot path for one 2D slice, inputs resident in HBM:
  groups (ROI compaction, Gram, eigen-decomposition, A_g)  -> compression of
  the raw k-space (Eq. 13) -> compressed reconstruction (power iteration for
  the FISTA step + FISTA l1-Haar, or CG-SENSE), all through the C ABI.

Metric: E_c+E_c^H pairs per second over the whole step (every pair of the
power iteration and the reconstruction counted; the group build and the
compression add to the time, not to the count), with the per-slice time
reported beside it.  N > 1 GPUs: one rank per GPU, each on its own slice
(weak scaling, no collective on the data path).

--impl reference times the FP64 CPU oracle on the host cores on a bounded
sample of the same workload (the reference arm for this method).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "E_c+E_c^H pairs/s and recon s/slice vs plain FP32 GPU at NRMSE<=1e-3"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpjc", choices=["gpjc", "reference"])
    ap.add_argument("--workload", default="2d256", choices=["2d256", "2d256h", "2d256bf", "2d128", "batch64"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--torch-floor", action="store_true",
                    help="time the plain-PyTorch FP32 operator beside the library's (2D workloads)")
    ap.add_argument("--no-compare", action="store_true",
                    help="skip the BF16 tensor-core step timed beside the FP32 one (2d256)")
    return ap.parse_args()


def dist_info():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ---------------------------------------------------------------- ranks --
def max_over_ranks(ms: float, world: int, dev) -> float:
    """The slowest rank's time: the job is only as fast as its slowest
    replica (all_reduce MAX over the process group; a no-op for one rank)."""
    if world <= 1:
        return float(ms)
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(ms)], device=dev, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_step: float, steps: int, world: int, total_ms: float) -> float:
    """Whole-job throughput: the units every rank processed over the slowest
    rank's time (each rank runs its own slice: weak scaling)."""
    return units_per_step * steps * world / (total_ms / 1e3)


def rank_barrier(world: int) -> None:
    if world > 1:
        import torch.distributed as dist

        dist.barrier()


# ---------------------------------------------------------------- clocks --
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.path = tempfile.mktemp(prefix="gpjc_clocks_", suffix=".csv")
        self.idx = gpu_index
        self.proc = None

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        if self.proc is None:
            return out
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        os.unlink(self.path)
        if sm:
            out = {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                   "samples": len(sm)}
        return out


# ---------------------------------------------------------------- roofline --
def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


# DRAM bytes (read + write) per launch of the adjoint readout kernel, from
# the ncu capture summarised in profiles/k1_readout_2d256_fp32.md; to be
# retaken whenever that kernel changes.  (The forward kernel's traffic
# depends on the autotuned coil-chunk count, so it is not recorded.)
DRAM_TRAFFIC = {("2d256", 2): 30536448}


def k1_flops(g, ntxc, keep_avg, contraction=True):
    """Algorithmic FP32 flops of one readout-stage launch (all rows, all
    coils): coil multiply (6 N_x), pre-twiddle (6 N_tx), os FFTs of N_x
    points (5 N_x log2 N_x each), wave/centring post-multiply (6 N_tx) and,
    with `contraction`, the A_g contraction (8 flops per complex MAC,
    N_s'_g x w per patch and coil)."""
    rows = g.ny * g.nz
    per_coil_row = (6 * g.nx + 6 * g.ntx + g.os * 5 * g.nx * math.log2(g.nx) + 6 * g.ntx
                    + (8 * ntxc * g.w if contraction else 0))
    return rows * g.nc * per_coil_row


# ---------------------------------------------------------------- gpjc arm --
def run_gpjc(args, rank, world, local):
    import numpy as np
    import torch

    import __graft_entry__ as ge

    ge.build()
    from paper_2601_05418_gb300 import gpjc, synth

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=dev)
    wl = synth.workload(args.workload)
    g = wl.geom
    case = synth.make_case(wl)
    prec = {"fp32": gpjc.FP32, "bf16": gpjc.BF16, "fp16": gpjc.FP16}[wl.precision]
    plan = gpjc.Plan(g)
    coils_h = torch.from_numpy(case.coils.astype(np.complex64)).pin_memory()
    roi_h = torch.from_numpy(case.roi).pin_memory()
    coils = coils_h.to(dev)
    roi = roi_h.to(dev)
    rho = torch.from_numpy(case.rho.astype(np.complex64)).to(dev)
    noise = torch.from_numpy(case.noise.astype(np.complex64)).to(dev)
    grp = gpjc.Groups.build(plan, coils, roi)
    op = gpjc.Operator(grp, coils, prec)
    op.autotune()
    S = op.simulate(rho) + noise  # raw k-space of this slice, resident in HBM
    torch.cuda.synchronize()
    S_h = S.cpu().pin_memory()
    Sc = torch.empty((g.n_lines, plan.ntx_c), dtype=torch.complex64, device=dev)
    x = torch.empty(g.shape, dtype=torch.complex64, device=dev)
    power_iters = 20
    pairs_per_step = wl.iters + (power_iters if wl.alg == "fista" else 0)

    def step():
        grp.rebuild(coils, roi)
        gpjc.compress(grp, S, prec, out=Sc)
        if wl.alg == "fista":
            op.recon(Sc, alg=gpjc.FISTA, iters=wl.iters, lam=wl.lam, power_iters=power_iters,
                     haar_levels=wl.haar_levels, out=x, sync=False)
        else:
            op.recon(Sc, alg=gpjc.CG, iters=wl.iters, out=x, sync=False)

    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)  # > 129 MB L2
    stream = torch.cuda.current_stream()
    op.profile(True)  # stage events are part of the captured graph from the first call on
    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()

    def barrier():
        rank_barrier(world)

    # ---- timed region (device events per step; L2 flushed between steps)
    sampler = ClockSampler(local)
    sampler.start()
    launches0 = gpjc.launch_count()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    prof = {s: [0.0, 0] for s in (gpjc.STAGE_READOUT_FWD, gpjc.STAGE_PHASE_ENCODE, gpjc.STAGE_READOUT_ADJ)}
    barrier()
    torch.cuda.synchronize()
    wall0 = time.perf_counter()
    for i in range(args.steps):
        flush.zero_()
        ev[i][0].record(stream)
        step()
        ev[i][1].record(stream)
        torch.cuda.synchronize()
        for s in prof:
            ms, n = op.profile_read(s)
            prof[s][0] += ms
            prof[s][1] += n
    torch.cuda.synchronize()
    barrier()
    wall = time.perf_counter() - wall0
    launches = gpjc.launch_count() - launches0
    clocks = sampler.stop()
    op.profile(False)
    ms_steps = [a.elapsed_time(b) for a, b in ev]
    total_ms = max_over_ranks(sum(ms_steps), world, dev)
    ms_per_step = total_ms / args.steps
    value = job_rate(pairs_per_step, args.steps, world, total_ms)

    # ---- dominant kernel and its roofline (FP32 ALU bound)
    fp32 = prec == gpjc.FP32
    names = {gpjc.STAGE_READOUT_FWD: ("k1f_tiled (coil x image, readout FFT, wave PSF, A_g)" if fp32 else
                                      "k1_sim_fwd2 + k_tc_compress (16-bit spectra, tcgen05 A_g)"),
             gpjc.STAGE_PHASE_ENCODE: "k2 (phase-encode FFT / mask projection)",
             gpjc.STAGE_READOUT_ADJ: ("k1a_tiled (A_g^H, inverse readout FFT, coil sum)" if fp32 else
                                      "k_tc_expand + k1_sim_adj2 (tcgen05 A_g^H, inverse FFT, coil sum)")}
    dom = max(prof, key=lambda s: prof[s][0])
    dom_ms = prof[dom][0] / max(prof[dom][1], 1)
    keep_avg = float(np.mean(g.keep))
    # 16-bit operators: the A_g contraction runs on the tensor cores, so the
    # FP32 ALU roofline of their readout stage counts the rest only
    fl = k1_flops(g, plan.ntx_c, keep_avg, contraction=fp32)
    sm_mhz = clocks["sm_mhz"] or 2070.0
    alu_peak = 152 * 128 * 2 * sm_mhz * 1e6 / 1e12  # TFLOP/s at the sampled SM clock
    achieved = fl / (dom_ms * 1e-3) / 1e12
    traffic = DRAM_TRAFFIC.get((wl.name, dom)) if fp32 else None
    roofline = {"kernel": names[dom], "bound": "alu", "achieved": round(achieved, 3), "peak": round(alu_peak, 2),
                "unit": "TFLOP/s", "frac": round(achieved / alu_peak, 4), "traffic": traffic,
                "peak_source": f"152 SMs x 128 FP32 lanes x 2 flop x {sm_mhz:.0f} MHz (median sampled SM clock)",
                "launch_ms": round(dom_ms, 5),
                "stage_share": {names[s]: round(prof[s][0] / max(total_ms, 1e-9), 4) for s in prof}}
    if not fp32:
        roofline["alu_work"] = ("coil multiply, pre / post factors and readout FFTs; the A_g contraction "
                                "(tensor_flop_per_launch) runs on the tensor cores")
        roofline["tensor_flop_per_launch"] = k1_flops(g, plan.ntx_c, keep_avg) - fl

    # ---- end to end through the C ABI with host buffers
    e2e = None
    if not args.no_e2e:
        x_h = torch.empty(g.shape, dtype=torch.complex64).pin_memory()
        e2e_steps = args.steps
        torch.cuda.synchronize()
        barrier()
        t0 = time.perf_counter()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(e2e_steps):
            coils.copy_(coils_h, non_blocking=True)
            roi.copy_(roi_h, non_blocking=True)
            S.copy_(S_h, non_blocking=True)
            step()
            x_h.copy_(x, non_blocking=True)
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        e2e_ms = max_over_ranks(e0.elapsed_time(e1), world, dev)
        h2d = coils_h.numel() * 8 + roi_h.numel() + S_h.numel() * 8
        e2e = {"value": round(job_rate(pairs_per_step, e2e_steps, world, e2e_ms), 2), "unit": "pairs/s",
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(x_h.numel() * 8),
               "s_per_slice": round(e2e_ms / 1e3 / e2e_steps, 6)}

    # ---- the same step with the BF16 tensor-core operator, timed the same
    # way: the metric compares it with the plain FP32 step
    bf16 = None
    if fp32 and wl.name == "2d256" and not args.no_compare:
        x32 = x.clone()
        op16 = gpjc.Operator(grp, coils, gpjc.BF16)
        op16.autotune()
        op16.profile(True)  # the same stage events as the FP32 step, so the two times compare like for like
        Sc16 = torch.empty_like(Sc)
        x16 = torch.empty_like(x)

        def step16():
            grp.rebuild(coils, roi)
            gpjc.compress(grp, S, gpjc.BF16, out=Sc16)
            op16.recon(Sc16, alg=gpjc.FISTA, iters=wl.iters, lam=wl.lam, power_iters=power_iters,
                       haar_levels=wl.haar_levels, out=x16, sync=False)

        for _ in range(max(3, args.warmup)):
            step16()
        torch.cuda.synchronize()
        barrier()
        ev16 = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                for _ in range(args.steps)]
        for i in range(args.steps):
            flush.zero_()
            ev16[i][0].record(stream)
            step16()
            ev16[i][1].record(stream)
        torch.cuda.synchronize()
        barrier()
        op16.profile(False)
        ms16 = max_over_ranks(sum(a.elapsed_time(b) for a, b in ev16), world, dev)
        v16 = job_rate(pairs_per_step, args.steps, world, ms16)
        # NRMSE (complex, full grid) of the BF16 image against this run's FP32 image
        ref_abs = x32.abs()
        nr = float((x16 - x32).abs().pow(2).mean().sqrt() / (ref_abs.max() - ref_abs.min()))
        bf16 = {"dtype": "bf16", "value": round(v16, 2), "unit": "pairs/s",
                "ms_per_step": round(ms16 / args.steps, 4), "speedup_vs_fp32": round(v16 / value, 3),
                "nrmse_vs_fp32_image": float(f"{nr:.3e}"),
                "note": "same workload, inputs, stage events and timing as the FP32 step; NRMSE against "
                        "the FP64 oracle is checked by the tests"}

    out = {
        "metric": METRIC, "value": round(value, 2), "unit": "pairs/s", "n_gpus": world, "steps": args.steps,
        "warmup": max(3, args.warmup), "ms_per_step": round(ms_per_step, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": {gpjc.FP32: "f32", gpjc.BF16: "bf16", gpjc.FP16: "f16"}[prec],
        "data": "synthetic (seeded phantom, Gaussian-phase coils, regular R=3 mask, sigma 1e-3 noise)",
        "config": {"workload": wl.name, "matrix": [g.nz, g.ny, g.nx], "coils": g.nc, "os": g.os,
                   "groups": g.n_groups, "w": g.w, "keep": int(g.keep[0]), "ntx_c": plan.ntx_c,
                   "n_lines": g.n_lines, "alg": wl.alg, "iters": wl.iters,
                   "power_iters": power_iters if wl.alg == "fista" else 0, "pairs_per_step": pairs_per_step,
                   "slices_per_step_per_gpu": 1, "l2": "flushed (256 MB write) between timed steps",
                   "parallelism": f"replicas x{world} (one slice per GPU)"},
        "recon_s_per_slice": round(ms_per_step / 1e3, 6),
        "wall_s": round(wall, 3),
        "clocks": clocks,
        "roofline": roofline,
        "gpu_launches": int(launches),
        "e2e": e2e,
    }
    if bf16 is not None:
        out["bf16_tensor_core_step"] = bf16
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(wl, pairs_per_step, power_iters)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


# ---------------------------------------------------------------- oracle arm --
def _oracle_sample(wl, pairs_per_step, power_iters, n_groups_sample=1, n_iters_sample=1):
    """Time the FP64 oracle on a bounded sample of one step and extrapolate:
    Gram + eigen-decomposition of `n_groups_sample` groups, compression of
    the slice, E_c^H S' and `n_iters_sample` E_c^H E_c applications plus the
    FISTA proximal step.  Returns (seconds per full step, sample description)."""
    import numpy as np

    import oracle as O
    from paper_2601_05418_gb300 import synth

    g = wl.geom
    case = synth.make_case(wl)
    S = O.simulate(g, case.coils, case.rho, case.noise)
    idx = O.roi_pixels(case.roi, case.coils)
    t0 = time.perf_counter()
    As = []
    for gi in range(n_groups_sample):
        P = O.gram(g, case.coils, idx, gi)
        A, _ = O.compression_matrix(P, int(g.keep[gi]), g.nc, g.w)
        As.append(A)
    t_groups = (time.perf_counter() - t0) / n_groups_sample * g.n_groups
    As = As + [As[0]] * (g.n_groups - len(As))
    t0 = time.perf_counter()
    Sc = O.compress(g, As, S)
    t_comp = time.perf_counter() - t0
    pb = O.Problem(g, case.coils, As)
    t0 = time.perf_counter()
    b = pb.EcH(Sc)
    t_b = time.perf_counter() - t0
    t0 = time.perf_counter()
    y = b.copy()
    for _ in range(n_iters_sample):
        z = y - (pb.normal_c(y) - b) / 1.0
        if wl.alg == "fista":
            y = np.stack([O.wavelet_prox(z[k], wl.lam, wl.haar_levels) for k in range(z.shape[0])])
    t_it = (time.perf_counter() - t0) / n_iters_sample
    total = t_groups + t_comp + t_b + t_it * pairs_per_step
    sample = (f"oracle on {n_groups_sample}/{g.n_groups} groups (Gram+eigh) and {n_iters_sample} of "
              f"{pairs_per_step} normal-operator iterations of one {wl.name} slice, plus compression and "
              f"E_c^H S'; extrapolated linearly to the full step")
    return total, sample


def _blas_threads():
    try:
        from threadpoolctl import threadpool_info

        return max([i.get("num_threads", 1) for i in threadpool_info()] or [1])
    except Exception:
        return os.cpu_count() or 1


def cpu_baseline(wl, pairs_per_step, power_iters):
    t, sample = _oracle_sample(wl, pairs_per_step, power_iters)
    return {"value": round(pairs_per_step / t, 4), "unit": "pairs/s", "cores": _blas_threads(), "kind": "oracle",
            "sample": sample + " (numpy FFT single-threaded, BLAS threaded)", "s_per_slice": round(t, 3)}


def run_reference(args, rank, world):
    if rank != 0:
        return
    from paper_2601_05418_gb300 import synth

    wl = synth.workload(args.workload)
    power_iters = 20
    pairs_per_step = wl.iters + (power_iters if wl.alg == "fista" else 0)
    for _ in range(args.warmup):
        _oracle_sample(wl, pairs_per_step, power_iters)
    ts, sample = [], ""
    for _ in range(args.steps):
        t, sample = _oracle_sample(wl, pairs_per_step, power_iters)
        ts.append(t)
    t = sum(ts) / len(ts)
    value = pairs_per_step / t
    out = {"metric": METRIC, "value": round(value, 4), "unit": "pairs/s", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": round(t * 1e3, 2), "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": wl.name, "pairs_per_step": pairs_per_step}, "impl": "reference",
           "cpu_baseline": {"value": round(value, 4), "unit": "pairs/s", "cores": _blas_threads(), "kind": "oracle",
                            "sample": sample},
           "e2e": {"value": round(value, 4), "unit": "pairs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def run_batch(args, rank, world, local):
    """64 uneven 2D slices, CG-SENSE 30 iterations each, in one persistent
    launch replayed from a CUDA graph; the same slices reconstructed one
    after another with the single-slice path are timed beside it."""
    import numpy as np
    import torch

    import __graft_entry__ as ge

    ge.build()
    from paper_2601_05418_gb300 import gpjc, synth

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=dev)
    wls = synth.batch_workloads(64)
    ops, scs, xs, keep = [], [], [], []
    gen = torch.Generator(device=dev).manual_seed(4)
    for wl in wls:
        g = wl.geom
        rho = synth.phantom(g.nx, g.ny)
        coils = synth.coil_maps(g.nx, g.ny, 1, g.nc, wl.seed)
        plan = gpjc.Plan(g)
        c_d = torch.from_numpy(coils.astype(np.complex64)).to(dev)
        grp = gpjc.Groups.build(plan, c_d, torch.from_numpy(synth.roi_mask(rho)).to(dev))
        op = gpjc.Operator(grp, c_d)
        op.autotune()
        S = op.simulate(torch.from_numpy(rho.astype(np.complex64)).to(dev))
        S += wl.sigma / np.sqrt(2) * torch.complex(torch.randn(S.shape, generator=gen, device=dev),
                                                    torch.randn(S.shape, generator=gen, device=dev))
        scs.append(gpjc.compress(grp, S))
        xs.append(torch.empty(g.shape, dtype=torch.complex64, device=dev))
        ops.append(op)
        keep.append((plan, grp, c_d))
    iters = wls[0].iters
    batch = gpjc.Batch(ops, iters)
    grid, items = batch.info()
    for _ in range(max(3, args.warmup)):
        batch.recon(scs, xs, sync=False)
    torch.cuda.synchronize()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()
    sampler = ClockSampler(local)
    sampler.start()
    l0 = gpjc.launch_count()
    tot = 0.0
    rank_barrier(world)
    for _ in range(args.steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        batch.recon(scs, xs, sync=False)
        e1.record(stream)
        torch.cuda.synchronize()
        tot += e0.elapsed_time(e1)
    clocks = sampler.stop()
    launches = gpjc.launch_count() - l0
    # the same work through the single-slice entry point, one slice after another
    for op, sc, x in zip(ops, scs, xs):
        op.recon(sc, alg=gpjc.CG, iters=iters, out=x, sync=False)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for op, sc, x in zip(ops, scs, xs):
        op.recon(sc, alg=gpjc.CG, iters=iters, out=x, sync=False)
    e1.record(stream)
    torch.cuda.synchronize()
    seq_ms = e0.elapsed_time(e1)
    tot = max_over_ranks(tot, world, dev)
    ms = tot / args.steps
    pairs = len(ops) * iters
    out = {"metric": METRIC + " (uneven 64-slice batch, CG-SENSE 30)",
           "value": round(job_rate(pairs, args.steps, world, tot), 2),
           "unit": "pairs/s", "n_gpus": world, "steps": args.steps, "warmup": max(3, args.warmup),
           "ms_per_step": round(ms, 3), "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "f32", "data": "synthetic",
           "config": {"workload": "batch64", "slices": len(ops), "iters": iters,
                      "sizes": sorted(set(int(w.geom.nx) for w in wls)),
                      "coils": sorted(set(int(w.geom.nc) for w in wls)),
                      "os": sorted(set(int(w.geom.os) for w in wls)),
                      "groups": sorted(set(int(w.geom.n_groups) for w in wls)),
                      "persistent_grid": grid, "work_items": items,
                      "l2": "flushed (256 MB write) between timed steps"},
           "sequential_single_slice_ms": round(seq_ms, 3),
           "speedup_vs_sequential": round(seq_ms / ms, 3),
           "recon_s_per_slice": round(ms / 1e3 / len(ops), 6),
           "clocks": clocks, "gpu_launches": int(launches)}
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


# ---------------------------------------------------------- torch floor --
class TorchFloor:
    """Plain-PyTorch FP32 E_c and E_c^H of a 2D slice (torch.fft and complex64
    batched matmul), the sanity floor the hand-written kernels are compared
    with; not part of the library.  Same model and conventions as the
    library (Eq. 1-4, 13-15): coil multiply, centred zero-padded unitary
    readout DFT, wave phase exp(-i 2 pi a_y(t) y_c / N_y), patch compression
    by A_{g(p)} on the coil-major patch vector (n w + tau), centred unitary
    phase-encode DFT, line gather.  The group map may be any, the kept
    dimension must be the same for every group."""

    def __init__(self, g, coils, As, dev):
        import numpy as np
        import torch

        assert g.nz == 1, "2D slices only"
        keep = {int(k) for k in g.keep}
        assert len(keep) == 1, "uniform kept dimension"
        self.g, self.k = g, keep.pop()
        self.np_ = g.ntx // g.w
        t = np.arange(g.ntx, dtype=np.float64)
        ay = g.kappa_y * (1 - np.cos(2 * np.pi * g.cycles * t / g.ntx)) / 2
        yc = (np.arange(g.ny) - g.ny // 2) / g.ny
        self.psf = torch.from_numpy(np.exp(-2j * np.pi * yc[:, None] * ay[None, :]).astype(np.complex64)).to(dev)
        self.coils = torch.as_tensor(coils).to(dev, torch.complex64).reshape(g.nc, g.ny, g.nx)
        self.Ap = torch.from_numpy(np.stack([np.asarray(As[int(q)]) for q in g.patch_group]).astype(np.complex64)).to(dev)
        self.lines = torch.as_tensor(np.asarray(g.line_ky, dtype=np.int64)).to(dev)
        self.s0 = g.ntx // 2 - g.nx // 2

    def E(self, rho):
        import torch

        g, fft = self.g, torch.fft
        U = torch.zeros((g.nc, g.ny, g.ntx), dtype=torch.complex64, device=rho.device)
        U[..., self.s0:self.s0 + g.nx] = self.coils * rho.reshape(1, g.ny, g.nx)
        U = fft.fftshift(fft.fft(fft.ifftshift(U, dim=-1), dim=-1, norm="ortho"), dim=-1) * self.psf
        V = U.reshape(g.nc, g.ny, self.np_, g.w).permute(1, 2, 0, 3).reshape(g.ny, self.np_, g.nc * g.w)
        H = torch.einsum("pki,ypi->ypk", self.Ap, V).reshape(g.ny, self.np_ * self.k)
        K = fft.fftshift(fft.fft(fft.ifftshift(H, dim=0), dim=0, norm="ortho"), dim=0)
        return K[self.lines]

    def EH(self, Sc):
        import torch

        g, fft = self.g, torch.fft
        K = torch.zeros((g.ny, self.np_ * self.k), dtype=torch.complex64, device=Sc.device)
        K[self.lines] = Sc
        H = fft.fftshift(fft.ifft(fft.ifftshift(K, dim=0), dim=0, norm="ortho"), dim=0)
        V = torch.einsum("pki,ypk->ypi", self.Ap.conj(), H.reshape(g.ny, self.np_, self.k))
        U = V.reshape(g.ny, self.np_, g.nc, g.w).permute(2, 0, 1, 3).reshape(g.nc, g.ny, g.ntx) * self.psf.conj()
        u = fft.fftshift(fft.ifft(fft.ifftshift(U, dim=-1), dim=-1, norm="ortho"), dim=-1)
        return (self.coils.conj() * u[..., self.s0:self.s0 + g.nx]).sum(0).reshape(1, g.ny, g.nx)


def run_torch_floor(args):
    """E_c + E_c^H pairs per second of the plain-PyTorch FP32 operator and of
    the library's FP32 operator in the same loop (same A_g, inputs resident,
    CUDA events around 200 pairs after 20 warm-up pairs, L2 not flushed for
    either)."""
    import numpy as np
    import torch

    import __graft_entry__ as ge

    ge.build()
    from paper_2601_05418_gb300 import gpjc, synth

    dev = torch.device("cuda", 0)
    wl = synth.workload(args.workload)
    g = wl.geom
    case = synth.make_case(wl)
    plan = gpjc.Plan(g)
    coils = torch.from_numpy(case.coils.astype(np.complex64)).to(dev)
    roi = torch.from_numpy(case.roi).to(dev)
    grp = gpjc.Groups.build(plan, coils, roi)
    As, _ = grp.matrices()
    op = gpjc.Operator(grp, coils, gpjc.FP32)
    op.autotune()
    tf = TorchFloor(g, case.coils, As, dev)
    x = torch.from_numpy(case.rho.astype(np.complex64)).to(dev).reshape(g.shape)

    def timed(pair, n=200, warm=20):
        for _ in range(warm):
            pair()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(n):
            pair()
        e1.record()
        torch.cuda.synchronize()
        return n / (e0.elapsed_time(e1) / 1e3)

    a = tf.EH(tf.E(x))
    b = op.EH(op.E(x))
    torch.cuda.synchronize()
    rel = float((a - b).abs().pow(2).sum().sqrt() / b.abs().pow(2).sum().sqrt())
    v_torch = timed(lambda: tf.EH(tf.E(x)))
    v_gpjc = timed(lambda: op.EH(op.E(x)))
    out = {"impl": "torch-floor", "metric": "E_c+E_c^H pairs/s (single pairs, plain PyTorch FP32)",
           "value": round(v_torch, 2), "unit": "pairs/s", "higher_is_better": True, "dtype": "f32",
           "gpjc_fp32_same_loop": round(v_gpjc, 2), "gpjc_over_torch": round(v_gpjc / v_torch, 3),
           "rel_l2_diff_EH_E": float(f"{rel:.3e}"),
           "config": {"workload": wl.name, "matrix": [g.nz, g.ny, g.nx], "coils": g.nc, "os": g.os,
                      "pairs": 200, "warmup_pairs": 20, "l2": "not flushed (both operators)"}}
    print(json.dumps(out), flush=True)


def main():
    args = parse()
    rank, world, local = dist_info()
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.workload == "batch64":
        run_batch(args, rank, world, local)
        return
    if args.torch_floor:
        if rank == 0:
            run_torch_floor(args)
        return
    run_gpjc(args, rank, world, local)


if __name__ == "__main__":
    main()
