"""Multi-GPU runs are replicas: each rank detects its own captures and the
ranks only agree on timing (a barrier and the slowest rank's time).  This
checks that host logic with two gloo ranks on the CPU, the same helpers
bench.py uses under torchrun with NCCL."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    w, r, local = bench._dist()
    bench._init_dist(local, w)
    # ranks finish at different times: the job rate uses the slowest one
    rate, t_max = bench.replica_throughput(units_per_rank=1000, steps=10, t_local=1.0 + rank,
                                           world=w)
    bench._barrier(w)
    q.put((r, w, rate, t_max))
    torch.distributed.destroy_process_group()


def test_two_gloo_replicas_agree_on_the_slowest_rank():
    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[0] for o in out] == [0, 1] and all(o[1] == 2 for o in out)
    for _, _, rate, t_max in out:
        assert t_max == 2.0
        assert rate == 2 * 10 * 1000 / 2.0


def test_single_process_needs_no_group():
    sys.path.insert(0, ROOT)
    import bench
    rate, t_max = bench.replica_throughput(500, 4, 2.0, 1)
    assert (rate, t_max) == (1000.0, 2.0)
