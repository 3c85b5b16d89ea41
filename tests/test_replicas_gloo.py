"""Multi-process host logic of the benchmark on CPU (gloo, world size 2).

The method does not shard (one global wavefront per sweep), so N GPUs run N independent
replicas; what crosses ranks is only the timing: the slowest rank's time and the whole-job
throughput (units of all ranks over that time).  These tests run that exchange with two gloo
ranks, and check that the reference arm prints on rank 0 only.
"""
import json
import os
import socket
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, local_ms, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    t = bench.max_over_ranks(local_ms[rank], dist, "cpu")
    v = bench.whole_job_value(16384, 10, world, t)
    out[rank] = (t, v)
    dist.barrier()
    dist.destroy_process_group()


def test_slowest_rank_sets_the_whole_job_time():
    world, port = 2, _free_port()
    local_ms = [80.0, 95.5]
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_rank_main, args=(world, port, local_ms, out), nprocs=world, start_method="spawn")
    (t0, v0), (t1, v1) = out[0], out[1]
    assert t0 == t1 == max(local_ms)
    assert v0 == v1 == pytest.approx(world * 16384 * 10 / (max(local_ms) / 1e3) / 1e6)


def test_reference_arm_prints_on_rank_zero_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1", MASTER_ADDR="127.0.0.1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "3"], env=env, capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert r.returncode == 0 and r.stdout.strip() == ""
    env["RANK"], env["LOCAL_RANK"] = "0", "0"
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "3"], env=env, capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert r.returncode == 0
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0
