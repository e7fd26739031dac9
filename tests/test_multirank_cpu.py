"""The multi-process path of bench.py on CPU: two ranks over gloo (the
data path has no collective; ranks meet only for the timing barrier and the
max-over-ranks of the timed duration), and the reference arm under a
2-rank launch (rank 0 alone prints, the others exit without work)."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    import bench

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    bench.rank_barrier(world)
    ms = 10.0 + 5.0 * rank  # rank 1 is the slow replica
    slowest = bench.max_over_ranks(ms, world, torch.device("cpu"))
    rate = bench.job_rate(70, 4, world, slowest)
    dist.destroy_process_group()
    with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
        json.dump({"slowest": slowest, "rate": rate}, f)


def test_two_rank_timing_aggregation(tmp_path):
    import torch.multiprocessing as mp

    world, port = 2, _free_port()
    mp.spawn(_rank_main, args=(world, port, str(tmp_path)), nprocs=world, join=True)
    for r in range(world):
        d = json.load(open(tmp_path / f"rank{r}.json"))
        assert d["slowest"] == 15.0  # every rank sees the slowest rank's time
        # 70 pairs x 4 steps on each of 2 ranks in 15 ms
        assert abs(d["rate"] - 70 * 4 * 2 / 0.015) < 1e-6


def test_reference_arm_other_ranks_exit_quietly():
    env = dict(os.environ, RANK="1", LOCAL_RANK="1", WORLD_SIZE="2")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr[-2000:]
    assert r.stdout.strip() == ""


def test_single_rank_helpers_need_no_process_group():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.max_over_ranks(12.5, 1, None) == 12.5
    bench.rank_barrier(1)
    assert abs(bench.job_rate(70, 10, 1, 1000.0) - 700.0) < 1e-9
