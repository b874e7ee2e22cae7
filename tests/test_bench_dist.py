"""The multi-process (N > 1) host logic of bench.py on CPU ranks (gloo, world size 2): the
max-over-ranks step time, the weak-scaling aggregate, per-rank batch seeds, and the reference
arm printing on rank 0 only."""
import json
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = [12.5, 20.0][rank]  # the slower rank decides
    ms_max = bench.world_max(dist, ms, "cpu")
    val = bench.weak_value(1e12, world, ms_max)
    seeds = [None] * world
    dist.all_gather_object(seeds, bench.rank_batch_seed(rank))
    dist.barrier()
    out[rank] = (ms_max, val, seeds)
    dist.destroy_process_group()


def test_world_max_and_weak_value_over_two_gloo_ranks():
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank_main, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    for r in (0, 1):
        ms_max, val, seeds = res[r]
        assert ms_max == 20.0
        assert val == pytest.approx(2 * 1e12 / 0.020 / 1e12)  # both ranks' flops over the slowest time
        assert len(set(seeds)) == 2  # independent batches per rank


def test_single_process_helpers():
    import bench
    assert bench.world_max(None, 3.5, "cpu") == 3.5
    assert bench.weak_value(2e12, 1, 1000.0) == pytest.approx(2.0)


def test_reference_arm_prints_on_rank0_only():
    env = dict(os.environ, RANK="1", LOCAL_RANK="1", WORLD_SIZE="2")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and r.stdout.strip() == ""


def test_reference_arm_line_on_rank0():
    env = dict(os.environ, RANK="0", LOCAL_RANK="0", WORLD_SIZE="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0", "--count", "64"], env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0 and line["e2e"]["h2d_bytes_per_step"] == 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
