"""bench.py's multi-rank (replicas) logic on CPU: two gloo ranks; the job time is the slowest
rank's, the bytes are summed, and the reference arm runs on rank 0 only."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import bench

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    torch.distributed.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t, e, b = bench.aggregate_ranks(1.0 + rank, 2.0 + 3 * rank, 10.0 * (rank + 1), world, "cpu")
        out.put((rank, t, e, b))
    finally:
        torch.distributed.destroy_process_group()


def test_aggregate_over_two_gloo_ranks():
    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for _, t, e, b in res:  # every rank sees the same whole-job figures
        assert (t, e, b) == (2.0, 5.0, 30.0)


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.aggregate_ranks(1.5, 2.5, 7.0, 1, "cpu") == (1.5, 2.5, 7.0)


def test_reference_arm_runs_on_rank_zero_only():
    sys.path.insert(0, ROOT)
    import bench

    class A:
        steps, warmup = 1, 0

    assert bench.run_reference(A(), rank=1, world=2) is None
