"""The multi-rank bench path on CPU: two gloo ranks take the max of their step
times and report the whole-job rate; the reference arm prints on rank 0 only."""
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


def _worker(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local = [1.0 + rank, 10.0 - rank]  # rank 1 is slower on the first timer
    ms = bench.sync_max(local, dist, "cpu")
    rate = bench.whole_job_rate(3.0, world, ms[0])
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, ms, rate))


def test_two_gloo_ranks_take_the_max_and_aggregate():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, rate in out:
        assert ms == [2.0, 10.0]
        assert rate == pytest.approx(2 * 3.0 / 2.0e-3)


def test_single_process_helpers():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.sync_max([3.5, 1.0]) == [3.5, 1.0]
    assert bench.whole_job_rate(10.0, 1, 1000.0) == pytest.approx(10.0)


def test_reference_arm_prints_on_rank_zero_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--workload", "laplace", "--steps", "1", "--warmup", "3"],
                       capture_output=True, text=True, env=env, timeout=300)
    assert r.returncode == 0 and r.stdout.strip() == ""
    env = dict(os.environ, RANK="0", WORLD_SIZE="1", LOCAL_RANK="0")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--workload", "laplace", "--steps", "2", "--warmup", "3"],
                       capture_output=True, text=True, env=env, timeout=300)
    assert r.returncode == 0
    import json
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["cpu_baseline"]["kind"] == "oracle"
    assert line["e2e"]["h2d_bytes_per_step"] == 0


@pytest.mark.parametrize("workload,size", [
    ("dense", 600), ("dense32", 600), ("dense64", 0), ("tet", 12), ("tet32", 12), ("tetcsr", 12),
    ("hvp", 12), ("hvp32", 12), ("autograd", 12), ("autograd32", 12), ("sparse", 20000),
    ("sparse32", 20000), ("batched", 16), ("laplace", 0), ("laplace_atomic", 0)])
def test_reference_arm_covers_every_workload(workload, size):
    # the oracle arm needs no GPU: every workload prints one line with its own config and unit
    env = dict(os.environ, RANK="0", WORLD_SIZE="1", LOCAL_RANK="0")
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload", workload,
           "--steps", "1", "--warmup", "3"] + (["--size", str(size)] if size else [])
    r = subprocess.run(cmd, capture_output=True, text=True, env=env, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    import json
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0 and line["config"]["workload"]
    assert line["cpu_baseline"]["value"] == line["value"] and line["e2e"]["d2h_bytes_per_step"] == 0
