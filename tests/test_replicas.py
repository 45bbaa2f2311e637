"""The multi-GPU path of bench.py on CPU: independent replicas, one per rank,
with the whole-job rate taken over the slowest rank (gloo, world size 2).

The method has no exchange step across GPUs at this problem size (the N x N
Gram reduction and the FFT run within one GPU), so the only collective of a
run is the max over ranks of the timed region.
"""
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

torch = pytest.importorskip("torch")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    r, w, _ = bench.dist_env()
    # rank r took 10 (r + 1) ms for its 5 steps
    ms, value = bench.job_rate(10.0 * (r + 1), 5, w, device="cpu")
    q.put((r, ms, value))
    dist.barrier()
    dist.destroy_process_group()


def test_job_rate_is_over_the_slowest_rank_gloo():
    world = 2
    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    try:
        got = sorted(q.get(timeout=120) for _ in range(world))
    finally:
        for p in procs:
            p.join(timeout=60)
            if p.is_alive():
                p.kill()
    assert [g[0] for g in got] == [0, 1]
    for _, ms, value in got:
        assert ms == pytest.approx(20.0)            # the slowest rank's time
        assert value == pytest.approx(2 * 5 / 0.020)  # all ranks' steps over it


def test_single_process_rate_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    ms, value = bench.job_rate(40.0, 8, 1)
    assert ms == 40.0 and value == pytest.approx(200.0)


def test_reference_arm_prints_on_rank_0_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], capture_output=True, text=True, env=env, cwd=ROOT, timeout=120)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""
