"""The N > 1 path of bench.py on CPU: two ranks of a gloo process group (127.0.0.1)
run its rank set-up, its max-over-ranks timing and barrier, and the whole-job
throughput of replicas (units of all ranks over the slowest rank's time)."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "WORLD_SIZE": "2",
                       "RANK": str(rank), "LOCAL_RANK": str(rank)})
    import bench
    import torch.distributed as dist
    ws, r, local = bench.dist_setup(None, backend="gloo")
    ms = 10.0 + 5.0 * rank  # rank 1 is the slower one
    bench.barrier(ws)
    ms_max = bench.max_over_ranks(ws, ms)
    out.put((r, ws, local, ms_max, bench.replica_value(ws, 1000, 3.0, ms_max)))
    dist.destroy_process_group()


def test_two_gloo_ranks_time_by_the_slowest_and_sum_the_work():
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(out.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[0] for r in res] == [0, 1]
    for r, ws, local, ms_max, value in res:
        assert ws == 2 and local == r
        assert ms_max == 15.0
        assert value == pytest.approx(2 * 1000 * 3.0 / 15e-3 / 1e9, rel=1e-15)


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK"):
        os.environ.pop(k, None)
    assert bench.dist_setup(None) == (1, 0, 0)
    assert bench.max_over_ranks(1, 3.5) == 3.5
    assert bench.replica_value(1, 1000, 3.0, 2.0) == pytest.approx(1.5e-3)
