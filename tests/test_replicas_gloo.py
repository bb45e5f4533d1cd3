"""Multi-process path of the replicas-only benchmark on CPU (gloo, world 2):
barrier, maximum of the per-rank times, whole-job rate."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
mp = pytest.importorskip("torch.multiprocessing")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    from paper_2209_14740_gb300 import replicas
    w, r, _ = replicas.init("gloo")
    replicas.barrier(w)
    t = replicas.max_over_ranks(1.5 + r, w, device="cpu")      # rank 1 is the slow one
    rate = replicas.whole_job_rate(10.0, t, w)
    out.put((r, w, t, rate))
    import torch.distributed as dist
    dist.destroy_process_group()


def test_two_replicas_take_the_slowest_rank():
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
    assert [r[0] for r in res] == [0, 1]
    for _, w, t, rate in res:
        assert w == 2 and t == 2.5
        assert rate == pytest.approx(2 * 10.0 / 2.5)


def test_single_process_needs_no_group():
    from paper_2209_14740_gb300 import replicas
    assert replicas.max_over_ranks(3.0, 1) == 3.0
    assert replicas.whole_job_rate(4.0, 2.0, 1) == 2.0
