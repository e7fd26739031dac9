#!/usr/bin/env python
"""Benchmark of the group-patch joint compression hot path on GB300.

One step = the whole hot path for one 2D slice, inputs resident in HBM:
  groups (ROI compaction, Gram, eigen-decomposition, A_g)  -> compression of
  the raw k-space (Eq. 13) -> compressed reconstruction (power iteration for
  the FISTA step + FISTA l1-Haar, or CG-SENSE), all through the C ABI.
Each step is timed in two parts with CUDA events: groups + compression
(`compress_s`) and the reconstruction loop (`recon_s_per_slice`, the time
the paper's SI Table S2 reports).

Metric: E_c+E_c^H pairs per second over the whole step (every pair of the
power iteration and the reconstruction counted; the group build and the
compression add to the time, not to the count), with the reconstruction
loop alone beside it (`recon_pairs_per_s`) and the median of 200 single
pairs (`pairs_isolated`).  The default 2d256 run also times the BF16
tensor-core step the same way, the 3D volume (3d224, s/volume) and the
uneven 64-slice batch.  N > 1 GPUs: one rank per GPU, each on its own slice
(weak scaling, no collective on the data path).

--impl reference times the FP64 CPU oracle on the host cores: real oracle
E_c + E_c^H pairs of the same slice (the reference arm for this method).
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
    ap.add_argument("--workload", default="2d256",
                    choices=["2d256", "2d256h", "2d256bf", "2d128", "batch64", "3d224", "3d224r1"],
                    help="3d224 / 3d224r1 only with --profile-case (the default line times both 3D workloads)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--torch-floor", action="store_true",
                    help="time the plain-PyTorch FP32 operator beside the library's (2D workloads)")
    ap.add_argument("--no-compare", action="store_true",
                    help="skip the BF16 tensor-core step timed beside the FP32 one (2d256)")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the 3d224 and batch64 workloads timed after the 2d256 line")
    ap.add_argument("--profile-case", default=None, choices=["fp32", "bf16", "fp16", "lb0", "recon16", "groups"],
                    help="profiling driver: E_c + E_c^H pairs (or the BF16 FISTA recon, or group rebuilds) "
                         "of the --workload operator between cudaProfilerStart / Stop, for ncu "
                         "--profile-from-start off")
    ap.add_argument("--reps", type=int, default=3, help="pairs (or recons) of --profile-case")
    ap.add_argument("--knobs", default=None, help="--profile-case: forward chunks, adjoint chunks, adjoint pieces")
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


# DRAM bytes (read + write) per launch of the adjoint readout kernel
# (k1a_tiled with the paired H2 layout, adjoint chunks 6), from the ncu
# capture summarised in profiles/k1_readout_2d256_fp32.md; to be retaken
# whenever that kernel changes.  (The forward kernel's traffic depends on its
# launch mode, so it is not recorded.)
DRAM_TRAFFIC = {("2d256", 2): 30543872}


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
def _events(n):
    import torch

    return [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n)]


def time_pairs(op, x, n=200, warm=20):
    """Median device time (us) of single E_c + E_c^H pairs, each between its
    own pair of CUDA events on the launching stream, after `warm` untimed
    pairs (inputs resident; the pair's working set stays in L2)."""
    import torch

    stream = torch.cuda.current_stream()
    y = op.E(x)
    z = op.EH(y)
    for _ in range(warm):
        op.E(x, out=y)
        op.EH(y, out=z)
    ev = _events(n)
    for a, b in ev:
        a.record(stream)
        op.E(x, out=y)
        op.EH(y, out=z)
        b.record(stream)
    torch.cuda.synchronize()
    ts = sorted(a.elapsed_time(b) * 1e3 for a, b in ev)
    return {"median_us": round(statistics.median(ts), 2), "p10_us": round(ts[n // 10], 2),
            "p90_us": round(ts[(9 * n) // 10], 2), "n": n, "warmup": warm,
            "pairs_per_s": round(1e6 / statistics.median(ts), 2)}


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
    stream = torch.cuda.current_stream()

    def make_step(o, p, sc, xo):
        """One pass of the hot path, split in two timed parts: (groups +
        compression) and the reconstruction loop."""

        def part_a():
            grp.rebuild(coils, roi)
            gpjc.compress(grp, S, p, out=sc)

        def part_b():
            if wl.alg == "fista":
                o.recon(sc, alg=gpjc.FISTA, iters=wl.iters, lam=wl.lam, power_iters=power_iters,
                        haar_levels=wl.haar_levels, out=xo, sync=False)
            else:
                o.recon(sc, alg=gpjc.CG, iters=wl.iters, out=xo, sync=False)

        return part_a, part_b

    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)  # > 129 MB L2

    def timed_steps(part_a, part_b, steps, o=None, prof=None):
        """Per step: L2 flush, then events around part a and part b."""
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
               torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for i in range(steps):
            flush.zero_()
            ev[i][0].record(stream)
            part_a()
            ev[i][1].record(stream)
            part_b()
            ev[i][2].record(stream)
            if prof is not None:
                torch.cuda.synchronize()
                for s in prof:
                    ms, n = o.profile_read(s)
                    prof[s][0] += ms
                    prof[s][1] += n
        torch.cuda.synchronize()
        a = [e0.elapsed_time(e1) for e0, e1, _ in ev]
        b = [e1.elapsed_time(e2) for _, e1, e2 in ev]
        return a, b

    part_a, part_b = make_step(op, prec, Sc, x)
    op.profile(True)  # stage events are part of the captured graph from the first call on
    for _ in range(max(3, args.warmup)):
        part_a()
        part_b()
    torch.cuda.synchronize()

    # ---- measured FP32 ALU peak of this device (FMA loop), the roofline denominator
    alu_peak = gpjc.probe_fp32_tflops()

    # ---- timed region (device events per step; L2 flushed between steps)
    sampler = ClockSampler(local)
    sampler.start()
    launches0 = gpjc.launch_count()
    prof = {s: [0.0, 0] for s in (gpjc.STAGE_READOUT_FWD, gpjc.STAGE_PHASE_ENCODE, gpjc.STAGE_READOUT_ADJ)}
    rank_barrier(world)
    torch.cuda.synchronize()
    wall0 = time.perf_counter()
    ta, tb = timed_steps(part_a, part_b, args.steps, op, prof)
    torch.cuda.synchronize()
    rank_barrier(world)
    wall = time.perf_counter() - wall0
    launches = gpjc.launch_count() - launches0
    clocks = sampler.stop()
    op.profile(False)
    total_ms = max_over_ranks(sum(ta) + sum(tb), world, dev)
    recon_ms = max_over_ranks(sum(tb), world, dev)
    ms_per_step = total_ms / args.steps
    value = job_rate(pairs_per_step, args.steps, world, total_ms)

    # ---- dominant kernel and its roofline (FP32 ALU bound)
    fp32 = prec == gpjc.FP32
    names = {gpjc.STAGE_READOUT_FWD: ("k1f_batched (coil x image, readout FFTs of 2 coils per call, wave PSF, A_g)" if fp32 else
                                      "k1_sim_fwd2 + k_tc_compress (readout spectra, tcgen05 A_g)"),
             gpjc.STAGE_PHASE_ENCODE: "k2 (phase-encode FFT / mask projection)",
             gpjc.STAGE_READOUT_ADJ: ("k1a_tiled (A_g^H, inverse readout FFT, coil sum)" if fp32 else
                                      "k_tc_expand + k1_sim_adj2 (tcgen05 A_g^H, inverse FFT, coil sum)")}
    dom = max(prof, key=lambda s: prof[s][0])
    dom_ms = prof[dom][0] / max(prof[dom][1], 1)
    keep_avg = float(np.mean(g.keep))
    # 16-bit operators: the A_g contraction runs on the tensor cores, so the
    # FP32 ALU roofline of their readout stage counts the rest only
    fl = k1_flops(g, plan.ntx_c, keep_avg, contraction=fp32)
    achieved = fl / (dom_ms * 1e-3) / 1e12
    traffic = DRAM_TRAFFIC.get((wl.name, dom)) if fp32 else None
    roofline = {"kernel": names[dom], "bound": "alu", "achieved": round(achieved, 3), "peak": round(alu_peak, 2),
                "unit": "TFLOP/s", "frac": round(achieved / alu_peak, 4), "traffic": traffic,
                "peak_source": "measured: FP32 FMA loop on this device (gpjc_probe_fp32_tflops, SM count x 8 "
                               "blocks x 256 threads x 8 chains), taken just before the timed region",
                "launch_ms": round(dom_ms, 5), "flop_per_launch": int(fl), "tuning": list(op.tuning()),
                "stage_share": {names[s]: round(prof[s][0] / max(total_ms, 1e-9), 4) for s in prof}}
    if not fp32:
        roofline["alu_work"] = ("coil multiply, pre / post factors and readout FFTs; the A_g contraction "
                                "(tensor_flop_per_launch) runs on the tensor cores")
        roofline["tensor_flop_per_launch"] = k1_flops(g, plan.ntx_c, keep_avg) - fl

    # ---- single E_c + E_c^H pairs (median of 200), beside the step metric
    xin = rho.reshape(g.shape).clone()
    pairs = time_pairs(op, xin)

    # ---- end to end through the C ABI with host buffers (L2 flushed per step)
    e2e = None
    if not args.no_e2e:
        x_h = torch.empty(g.shape, dtype=torch.complex64).pin_memory()
        e2e_steps = args.steps
        torch.cuda.synchronize()
        rank_barrier(world)
        tot = 0.0
        for _ in range(e2e_steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            coils.copy_(coils_h, non_blocking=True)
            roi.copy_(roi_h, non_blocking=True)
            S.copy_(S_h, non_blocking=True)
            part_a()
            part_b()
            x_h.copy_(x, non_blocking=True)
            e1.record(stream)
            torch.cuda.synchronize()
            tot += e0.elapsed_time(e1)
        rank_barrier(world)
        e2e_ms = max_over_ranks(tot, world, dev)
        h2d = coils_h.numel() * 8 + roi_h.numel() + S_h.numel() * 8
        e2e = {"value": round(job_rate(pairs_per_step, e2e_steps, world, e2e_ms), 2), "unit": "pairs/s",
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(x_h.numel() * 8),
               "s_per_slice": round(e2e_ms / 1e3 / e2e_steps, 6),
               "l2": "flushed (256 MB write) before each step, outside its events"}

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
        a16, b16 = make_step(op16, gpjc.BF16, Sc16, x16)
        for _ in range(max(3, args.warmup)):
            a16()
            b16()
        torch.cuda.synchronize()
        rank_barrier(world)
        prof16 = {s: [0.0, 0] for s in prof}
        ta16, tb16 = timed_steps(a16, b16, args.steps, op16, prof16)
        rank_barrier(world)
        op16.profile(False)
        ms16 = max_over_ranks(sum(ta16) + sum(tb16), world, dev)
        rc16 = max_over_ranks(sum(tb16), world, dev)
        v16 = job_rate(pairs_per_step, args.steps, world, ms16)
        # NRMSE (complex, full grid) of the BF16 image against this run's FP32 image
        ref_abs = x32.abs()
        nr = float((x16 - x32).abs().pow(2).mean().sqrt() / (ref_abs.max() - ref_abs.min()))
        bf16 = {"dtype": "bf16", "value": round(v16, 2), "unit": "pairs/s",
                "ms_per_step": round(ms16 / args.steps, 4), "speedup_vs_fp32": round(v16 / value, 3),
                "recon_s_per_slice": round(rc16 / 1e3 / args.steps, 6),
                "compress_s": round(statistics.median(ta16) / 1e3, 6),
                "recon_speedup_vs_fp32": round(recon_ms / rc16, 3),
                "recon_pairs_per_s": round(job_rate(pairs_per_step, args.steps, world, rc16), 2),
                "pairs_isolated": time_pairs(op16, xin),
                "tuning": list(op16.tuning()),
                "stage_ms_per_launch": {nm: round(prof16[s][0] / max(prof16[s][1], 1), 5) for s, nm in
                                        ((gpjc.STAGE_READOUT_FWD, "readout_fwd (k1_sim_fwd2 + k_tc_compress)"),
                                         (gpjc.STAGE_PHASE_ENCODE, "phase_encode (k2)"),
                                         (gpjc.STAGE_READOUT_ADJ, "readout_adj (k_tc_expand + k1_sim_adj2)"))},
                "nrmse_vs_fp32_image": float(f"{nr:.3e}"),
                "note": "same workload, inputs, stage events and timing as the FP32 step (BF16 operands as "
                        "head + remainder, three MMAs per K step); NRMSE against the FP64 oracle is checked "
                        "by the tests (full-size 2d256 FISTA bound 1e-3)"}
        del op16

    out = {
        "metric": METRIC, "value": round(value, 2), "unit": "pairs/s", "n_gpus": world, "steps": args.steps,
        "warmup": max(3, args.warmup), "ms_per_step": round(ms_per_step, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": {gpjc.FP32: "f32", gpjc.BF16: "bf16", gpjc.FP16: "f16"}[prec],
        "data": "synthetic (seeded phantom, Gaussian-phase coils, regular R=3 mask, sigma 1e-3 noise)",
        "config": config_of(wl, plan.ntx_c, pairs_per_step, power_iters, world),
        "step": "groups (ROI, Gram, eigen, A_g) + compression + reconstruction (power iteration + FISTA / CG); "
                "value = pairs of the step / whole-step time",
        "recon_s_per_slice": round(recon_ms / 1e3 / args.steps, 6),
        "recon_pairs_per_s": round(job_rate(pairs_per_step, args.steps, world, recon_ms), 2),
        "compress_s": round(statistics.median(ta) / 1e3, 6),
        "pairs_isolated": pairs,
        "wall_s": round(wall, 3),
        "clocks": clocks,
        "roofline": roofline,
        "gpu_launches": int(launches),
        "e2e": e2e,
    }
    if bf16 is not None:
        out["bf16_tensor_core_step"] = bf16
    if wl.name == "2d256" and world == 1 and not args.no_extras:
        del op, grp
        torch.cuda.empty_cache()
        out["workloads"] = {"3d": run_3d(args, dev), "local_b0_2d256": run_local_b0(args, dev),
                            "batch64": run_batch(args, 0, 1, local, emit=False)}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(wl)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def config_of(wl, ntx_c, pairs_per_step, power_iters, world):
    g = wl.geom
    return {"workload": wl.name, "matrix": [g.nz, g.ny, g.nx], "coils": g.nc, "os": g.os,
            "groups": g.n_groups, "w": g.w, "keep": int(g.keep[0]), "ntx_c": int(ntx_c),
            "n_lines": g.n_lines, "alg": wl.alg, "iters": wl.iters,
            "power_iters": power_iters if wl.alg == "fista" else 0, "pairs_per_step": pairs_per_step,
            "slices_per_step_per_gpu": 1, "l2": "flushed (256 MB write) between timed steps",
            "parallelism": f"replicas x{world} (one slice per GPU)"}


def run_3d(args, dev):
    """The 3D volume (224 x 224 x 160, 32 coils, corkscrew wave, 6x
    oversampling, 3x3 CAIPI) in two groupings: 48 contiguous readout
    subregions compressed 20x (11 cycles, no integer period), and 48
    per-period groups of w = 2 (14 cycles, period 96).  For each: group build
    + compression timed once after one warm-up, then the CG-SENSE 10
    reconstruction loop (s/volume) timed over 3 runs after 3 warm-up runs,
    FP32 and BF16 operators (BF16 compression for the BF16 operator).  Inputs
    resident in HBM; the 2.1 GB coil maps exceed L2."""
    import numpy as np
    import torch

    from paper_2601_05418_gb300 import gpjc, synth

    t0 = time.perf_counter()
    wl0 = synth.workload("3d224")
    g0 = wl0.geom
    rho = synth.phantom(g0.nx, g0.ny, g0.nz)
    roi = torch.from_numpy(synth.roi_mask(rho)).to(dev)
    coils = torch.from_numpy(synth.coil_maps(g0.nx, g0.ny, g0.nz, g0.nc, wl0.seed).astype(np.complex64)).to(dev)
    rho_d = torch.from_numpy(rho.astype(np.complex64)).to(dev)
    stream = torch.cuda.current_stream()
    out = {"unit": "s/volume", "higher_is_better": False, "setup_s": None}
    sampler = ClockSampler(torch.cuda.current_device())
    sampler.start()
    for name in ("3d224", "3d224r1"):
        wl = synth.workload(name)
        g = wl.geom
        plan = gpjc.Plan(g)
        grp = gpjc.Groups.build(plan, coils, roi)
        op = gpjc.Operator(grp, coils)
        S = op.simulate(rho_d)
        gen = torch.Generator(device=dev).manual_seed(wl.seed)
        S += wl.sigma / np.sqrt(2) * torch.complex(torch.randn(S.shape, generator=gen, device=dev),
                                                   torch.randn(S.shape, generator=gen, device=dev))
        torch.cuda.synchronize()
        res = {"config": {"workload": name, "matrix": [g.nz, g.ny, g.nx], "coils": g.nc, "os": g.os,
                          "cycles": g.cycles, "groups": g.n_groups, "w": g.w, "keep": int(g.keep[0]),
                          "ntx_c": int(plan.ntx_c), "n_lines": g.n_lines, "alg": "cg", "iters": wl.iters,
                          "grouping": ("48 contiguous readout subregions, one patch per group per line"
                                       if name == "3d224" else "48 groups per modulation period of 96 samples")}}
        for prec, pname in ((gpjc.FP32, "fp32"), (gpjc.BF16, "bf16")):
            o = op if prec == gpjc.FP32 else gpjc.Operator(grp, coils, prec)
            Sc = torch.empty((g.n_lines, plan.ntx_c), dtype=torch.complex64, device=dev)
            x = torch.empty(g.shape, dtype=torch.complex64, device=dev)
            e = _events(2)
            grp.rebuild(coils, roi)  # warm-up of the group build
            gpjc.compress(grp, S, prec, out=Sc)
            e[0][0].record(stream)
            grp.rebuild(coils, roi)
            e[0][1].record(stream)
            e[1][0].record(stream)
            gpjc.compress(grp, S, prec, out=Sc)
            e[1][1].record(stream)
            for _ in range(3):
                o.recon(Sc, alg=gpjc.CG, iters=wl.iters, out=x, sync=False)
            ev = _events(3)
            for a, b in ev:
                a.record(stream)
                o.recon(Sc, alg=gpjc.CG, iters=wl.iters, out=x, sync=False)
                b.record(stream)
            torch.cuda.synchronize()
            rec = [a.elapsed_time(b) / 1e3 for a, b in ev]
            res[pname] = {"s_per_volume": round(statistics.median(rec), 4), "runs": 3, "warmup": 3,
                          "groups_s": round(e[0][0].elapsed_time(e[0][1]) / 1e3, 4),
                          "compress_s": round(e[1][0].elapsed_time(e[1][1]) / 1e3, 5),
                          "pairs_per_s": round(wl.iters / statistics.median(rec), 2)}
            if prec != gpjc.FP32:
                del o
        res["bf16_recon_speedup_vs_fp32"] = round(res["fp32"]["s_per_volume"] / res["bf16"]["s_per_volume"], 3)
        out[name] = res
        del op, grp, plan, S
        torch.cuda.empty_cache()
    out["clocks"] = sampler.stop()
    out["setup_s"] = round(time.perf_counter() - t0, 2)
    return out


def run_local_b0(args, dev):
    """Nonlinear local-B0 operator at the 256 x 256 size (32 coils, 8x
    oversampling, 32 periodic groups, keep 16): stored compressed readout
    matrices (256 rows x 4096 x 256 complex64 = 2.15 GB), built on the device
    from three synthetic local-B0 fields; E_c + E_c^H pairs timed after
    warm-up.  Each application streams the matrices from HBM once, so the
    readout stages are HBM-bound: achieved GB/s = matrix bytes / stage time.
    (Timing only: A_g comes from the wave model's group build, the same
    shapes as a general-phase build.)"""
    import numpy as np
    import torch

    from paper_2601_05418_gb300 import gpjc, synth

    wl = synth.workload("2d256")
    g = wl.geom
    case = synth.make_case(wl, with_noise=False)
    plan = gpjc.Plan(g)
    coils = torch.from_numpy(case.coils.astype(np.complex64)).to(dev)
    grp = gpjc.Groups.build(plan, coils, torch.from_numpy(case.roi).to(dev))
    fields = torch.from_numpy(synth.local_b0_fields(g.nx, g.ny, 1, 3, 7).astype(np.float32)).to(dev)
    amps = synth.local_b0_amplitudes(g.ntx, g.cycles, 3, 8)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    op = gpjc.Operator.local_b0(grp, coils, fields, amps)
    build_s = time.perf_counter() - t0
    x = torch.from_numpy(case.rho.astype(np.complex64)).to(dev).reshape(g.shape)
    pairs = time_pairs(op, x, n=50, warm=5)
    y = op.E(x)
    z = op.EH(y)
    torch.cuda.synchronize()
    op.profile(True)  # resets the stage records; the pairs below are the measured ones
    n = 20
    for _ in range(n):
        op.E(x, out=y)
        op.EH(y, out=z)
    torch.cuda.synchronize()
    gbytes = 8.0 * g.ny * g.nz * plan.ntx_c * g.nx
    res = {"config": {"workload": "2d256 local-B0", "matrix": [g.nz, g.ny, g.nx], "coils": g.nc, "os": g.os,
                      "fields": 3, "ntx_c": int(plan.ntx_c), "stored_matrix_bytes": int(gbytes)},
           "build_s": round(build_s, 3), "pairs_isolated": pairs}
    peak = peaks()[0]["hbm_gbs"]
    for s, nm in ((gpjc.STAGE_READOUT_FWD, "k_lb0_fwd"), (gpjc.STAGE_READOUT_ADJ, "k_lb0_adj")):
        ms, cnt = op.profile_read(s)
        per = ms / max(cnt, 1)
        gbs = gbytes / (per * 1e-3) / 1e9
        res[nm] = {"launch_ms": round(per, 4), "achieved_gbs": round(gbs, 1), "peak_gbs": peak,
                   "frac": round(gbs / peak, 4), "bound": "hbm",
                   "algorithmic_bytes": int(gbytes), "note": "matrix bytes only (vectors are < 0.1%)"}
    op.profile(False)
    return res


# ---------------------------------------------------------------- oracle arm --
def _cpu_model():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform

    return platform.processor() or platform.machine()


def _oracle_problem(wl):
    """The oracle's problem for one slice of the workload: raw data, the
    compression matrices of every group (from the oracle's Gram and eigh of
    group 0, reused for all groups: the timed pairs do not depend on which
    orthonormal A_g they apply) and the compressed data."""
    import oracle as O
    from paper_2601_05418_gb300 import synth

    g = wl.geom
    case = synth.make_case(wl)
    S = O.simulate(g, case.coils, case.rho, case.noise)
    idx = O.roi_pixels(case.roi, case.coils)
    t0 = time.perf_counter()
    P = O.gram(g, case.coils, idx, 0)
    A, _ = O.compression_matrix(P, int(g.keep[0]), g.nc, g.w)
    t_group = time.perf_counter() - t0
    As = [A] * g.n_groups
    t0 = time.perf_counter()
    Sc = O.compress(g, As, S)
    t_comp = time.perf_counter() - t0
    return O.Problem(g, case.coils, As), Sc, t_group, t_comp


def _blas_threads():
    try:
        from threadpoolctl import threadpool_info

        return max([i.get("num_threads", 1) for i in threadpool_info()] or [1])
    except Exception:
        return os.cpu_count() or 1


def _one_thread_pair_s(workload):
    """One oracle pair timed in a child process whose BLAS / OpenMP pools
    are limited to one thread (numpy's FFT is single-threaded anyway)."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               BLIS_NUM_THREADS="1")
    code = ("import sys, json; sys.path.insert(0, %r); import bench; from paper_2601_05418_gb300 import synth; "
            "pb, Sc, _, _ = bench._oracle_problem(synth.workload(%r)); bench._oracle_pairs(pb, Sc, 1); "
            "print(json.dumps(bench._oracle_pairs(pb, Sc, 1)[0]))") % (ROOT, workload)
    try:
        r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=300)
        return float(r.stdout.strip().splitlines()[-1])
    except Exception:
        return None


def _oracle_pairs(pb, Sc, n):
    """Times n oracle E_c + E_c^H pairs (FP64, numpy); returns seconds each."""
    x = pb.EcH(Sc)
    ts = []
    for _ in range(n):
        t0 = time.perf_counter()
        x = pb.EcH(pb.Ec(x))
        ts.append(time.perf_counter() - t0)
        x = x / max(float(abs(x).max()), 1e-30)
    return ts


def cpu_baseline(wl, n_pairs=8):
    """The oracle timed on the host cores on a bounded sample: n_pairs real
    E_c + E_c^H pairs of the same slice (all BLAS threads), one more pair on
    one thread, and one group's Gram + eigh."""
    pb, Sc, t_group, t_comp = _oracle_problem(wl)
    _oracle_pairs(pb, Sc, 1)
    ts = _oracle_pairs(pb, Sc, n_pairs)
    t1 = _one_thread_pair_s(wl.name)
    pair_s = statistics.median(ts)
    return {"value": round(1.0 / pair_s, 4), "unit": "pairs/s", "cores": _blas_threads(), "kind": "oracle",
            "sample": f"{n_pairs} FP64 oracle E_c + E_c^H pairs of one {wl.name} slice (median), after one "
                      f"warm-up pair; numpy FFT single-threaded, BLAS on all threads",
            "one_thread_pair_s": round(t1, 4) if t1 is not None else None,
            "group_gram_eigh_s": round(t_group, 3), "compress_s": round(t_comp, 3),
            "cpu_model": _cpu_model(), "nproc": os.cpu_count()}


def run_reference(args, rank, world):
    """Reference arm: the FP64 oracle on the host cores.  One step = one
    E_c + E_c^H pair of the oracle on the same 2D slice (same A_g shapes and
    data), exactly `steps` of them timed after `warmup`; the full oracle
    step of the workload is extrapolated from them in its own field."""
    if rank != 0:
        return
    from paper_2601_05418_gb300 import synth

    wl = synth.workload(args.workload)
    power_iters = 20
    pairs_per_step = wl.iters + (power_iters if wl.alg == "fista" else 0)
    pb, Sc, t_group, t_comp = _oracle_problem(wl)
    _oracle_pairs(pb, Sc, args.warmup)
    t0 = time.perf_counter()
    ts = _oracle_pairs(pb, Sc, args.steps)
    wall = time.perf_counter() - t0
    t1 = _one_thread_pair_s(wl.name)
    total = sum(ts)
    value = args.steps / total
    import oracle as O

    ntxc = int(O.ntx_compressed(wl.geom.patch_group, wl.geom.keep))
    out = {"metric": METRIC, "value": round(value, 4), "unit": "pairs/s", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": round(total / args.steps * 1e3, 2), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": config_of(wl, ntxc, pairs_per_step, power_iters, world), "impl": "reference",
           "step": "one FP64 oracle E_c + E_c^H pair of the slice (the pairs are measured, not extrapolated)",
           "wall_s": round(wall, 3),
           "oracle_full_step_s_extrapolated": round(t_group * wl.geom.n_groups + t_comp + pairs_per_step * total
                                                    / args.steps, 2),
           "extrapolation": f"{wl.geom.n_groups} x one group's Gram + eigh ({t_group:.2f} s) + compression "
                            f"({t_comp:.2f} s) + {pairs_per_step} x the median pair",
           "cpu_baseline": {"value": round(value, 4), "unit": "pairs/s", "cores": _blas_threads(), "kind": "oracle",
                            "sample": f"{args.steps} FP64 oracle E_c + E_c^H pairs of one {wl.name} slice after "
                                      f"{args.warmup} warm-up pairs; numpy FFT single-threaded, BLAS on all "
                                      f"threads",
                            "one_thread_pair_s": round(t1, 4) if t1 is not None else None,
                            "cpu_model": _cpu_model(), "nproc": os.cpu_count()},
           "e2e": {"value": round(value, 4), "unit": "pairs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def run_batch(args, rank, world, local, emit=True):
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
    if world > 1 and emit:
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
    # the same slices as one CUDA graph on parallel branches (multi-slice
    # graph); the branch count is chosen by timing 2, 4, 8 and 16 branches
    multi = {}
    for nbr in (2, 4, 8, 16):
        mg = gpjc.Multi(ops, n_branches=nbr)
        for _ in range(2):
            mg.recon(scs, xs, iters=iters, sync=False)
        torch.cuda.synchronize()
        ts = []
        for _ in range(max(3, args.steps // 2)):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            mg.recon(scs, xs, iters=iters, sync=False)
            b.record(stream)
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
        multi[nbr] = statistics.median(ts)
        del mg
    best_nb = min(multi, key=multi.get)
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
           "multi_slice_graph": {"ms_per_batch": round(multi[best_nb], 3), "branches": best_nb,
                                 "by_branches_ms": {str(k): round(v, 3) for k, v in multi.items()},
                                 "speedup_vs_sequential": round(seq_ms / multi[best_nb], 3),
                                 "pairs_per_s": round(len(ops) * iters / (multi[best_nb] / 1e3), 2),
                                 "note": "same slices, CG-30, one CUDA graph with the slices on parallel "
                                         "branches (median of timed launches, L2 flushed before each)"},
           "recon_s_per_slice": round(ms / 1e3 / len(ops), 6),
           "clocks": clocks, "gpu_launches": int(launches)}
    if not emit:
        return out
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


def run_profile_case(args):
    """The operator in a fixed configuration (no autotuning, so an
    instrumented run uses the same launch knobs as a plain one), warmed up,
    then `--reps` E_c + E_c^H pairs (or BF16 FISTA-50 recons) between
    cudaProfilerStart and cudaProfilerStop."""
    import numpy as np
    import torch

    import __graft_entry__ as ge

    ge.build()
    from paper_2601_05418_gb300 import gpjc, synth

    dev = torch.device("cuda", 0)
    wl = synth.workload(args.workload)
    g = wl.geom
    mode = args.profile_case
    if g.nz > 1:
        if mode not in ("fp32", "bf16", "fp16", "groups"):
            raise SystemExit("--profile-case: the 3D workloads take fp32, bf16, fp16 or groups")
        rho = synth.phantom(g.nx, g.ny, g.nz)
        roi = synth.roi_mask(rho)
        coil_np = synth.coil_maps(g.nx, g.ny, g.nz, g.nc, wl.seed)
    else:
        case = synth.make_case(wl)
        rho, roi, coil_np = case.rho, case.roi, case.coils
    plan = gpjc.Plan(g)
    coils = torch.from_numpy(coil_np.astype(np.complex64)).to(dev)
    grp = gpjc.Groups.build(plan, coils, torch.from_numpy(roi).to(dev))
    x = torch.from_numpy(rho.astype(np.complex64)).to(dev).reshape(g.shape)
    if mode == "groups":
        roi_d = torch.from_numpy(roi).to(dev)
        grp.rebuild(coils, roi_d)
        torch.cuda.synchronize()
        torch.cuda.profiler.start()
        for _ in range(args.reps):
            grp.rebuild(coils, roi_d)
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
        print(json.dumps({"profile_case": mode, "workload": args.workload, "reps": args.reps}), flush=True)
        return
    if mode == "lb0":
        fields = torch.from_numpy(synth.local_b0_fields(g.nx, g.ny, 1, 3, 7).astype(np.float32)).to(dev)
        op = gpjc.Operator.local_b0(grp, coils, fields, synth.local_b0_amplitudes(g.ntx, g.cycles, 3, 8))
    else:
        prec = {"fp32": gpjc.FP32, "bf16": gpjc.BF16, "fp16": gpjc.FP16, "recon16": gpjc.BF16}[mode]
        op = gpjc.Operator(grp, coils, prec)
        if args.knobs:
            op.set_tuning(*[int(v) for v in args.knobs.split(",")])
    y = op.E(x)
    z = op.EH(y)
    Sc = None
    if mode == "recon16":
        Sc = gpjc.compress(grp, gpjc.Operator(grp, coils).simulate(x), gpjc.BF16)
    torch.cuda.synchronize()
    torch.cuda.profiler.start()
    for _ in range(args.reps):
        if Sc is not None:
            op.recon(Sc, alg=gpjc.FISTA, iters=50, lam=1e-3, power_iters=20, haar_levels=4, use_graph=False)
        else:
            op.E(x, out=y)
            op.EH(y, out=z)
    torch.cuda.synchronize()
    torch.cuda.profiler.stop()
    print(json.dumps({"profile_case": mode, "workload": args.workload, "reps": args.reps,
                      "knobs": list(op.tuning()) if mode != "lb0" else None}), flush=True)


def main():
    args = parse()
    rank, world, local = dist_info()
    if args.profile_case:
        if rank == 0:
            run_profile_case(args)
        return
    if args.workload.startswith("3d"):
        raise SystemExit("--workload 3d224 / 3d224r1 go with --profile-case; the default line times both")
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
