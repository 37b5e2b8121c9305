"""The multi-GPU path of bench.py is replicas only: each rank solves its own
seeded problem and the ranks meet only for the barrier and the max-over-ranks
step time.  This runs that host logic as two gloo ranks on the CPU."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        from synth import make_workload
        seed = bench.replica_seed(rank)
        w = make_workload("gp2k", N=256, d=4, seed=seed)
        # each rank reports a different step time; all must agree on the max
        mx = bench.max_over_ranks(10.0 + rank, dist, "cpu")
        dist.barrier()
        q.put((rank, seed, float(w.X[0, 0]), mx))
    finally:
        dist.destroy_process_group()


def test_two_replicas_max_over_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    out = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, s0, x0, m0), (r1, s1, x1, m1) = out
    assert (s0, s1) == (None, 101)
    assert x0 != x1                      # independent problems
    assert m0 == m1 == 11.0              # the slowest rank sets the time


def test_reference_arm_nonzero_rank_exits_without_work(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")

    class A:
        workload, warmup, steps, gpus = "gp2k", 3, 1, 2
    assert bench.run_reference(A()) == 0
