"""The bench's N > 1 path on CPU: two gloo ranks, max-over-ranks timing, weak-scaling rate,
and the reference arm printing on rank 0 only."""
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    local_ms = 100.0 + 50.0 * rank
    m = bench.max_over_ranks(local_ms, world)
    rate = bench.whole_job_rate(640, world, 3, m / 1e3)
    q.put((rank, m, rate))
    dist.destroy_process_group()


def test_two_gloo_ranks_aggregate_like_the_bench():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [150.0, 150.0]           # both ranks see the slowest time
    assert all(abs(r[2] - 640 * 2 * 3 / 0.150) < 1e-6 for r in res)  # units of all ranks / max time


def test_reference_arm_prints_on_rank_zero_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and r.stdout.strip() == ""


def test_all_cores_oracle_baseline_uses_every_core():
    """The CPU baseline's all-cores leg runs the oracle unchanged in one spawn-started process per host
    core and returns their joint chain-rule sample rate (here on the 4-qubit ring for half a second)."""
    sys.path.insert(0, ROOT)
    import bench
    from paper_2103_17226_gb300 import inputs as I, native as N
    W = bench.make_workload("qaoa32", 100)
    c = I.workload("qaoa4_ring_p1")
    W = dict(W, circuit=c, angles=I.uniform_angles(1, c.n_angles, seed=1), seeds=I.vector_seeds(1, 1))
    rate, cores = bench.oracle_all_cores(W, N.compile(c, N.QKC_AC_DENSITY), seconds=0.5)
    assert cores == (os.cpu_count() or 1)
    assert rate > 0
