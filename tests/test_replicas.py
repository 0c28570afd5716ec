"""The replica path (world size 2, gloo on CPU): every rank reports its own timed interval;
all ranks agree on the slowest, and the job rate counts both ranks' work."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, size, port, out):
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(size), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    from paper_2507_14046_gb300 import replicas
    import torch.distributed as dist
    replicas.init("gloo")
    r, s, lr = replicas.world()
    replicas.barrier()
    t = replicas.max_over_ranks(1.5 + rank)          # rank 1 is slower
    rate = replicas.job_rate(100.0, t, s)
    out.put((r, s, lr, t, rate))
    dist.destroy_process_group()


def test_two_rank_max_and_rate():
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
    for r, s, lr, t, rate in res:
        assert s == 2 and lr == r
        assert t == 2.5
        assert rate == pytest.approx(2 * 100.0 / 2.5)


def test_single_process_is_identity():
    from paper_2507_14046_gb300 import replicas
    assert replicas.max_over_ranks(3.25) == 3.25
    assert replicas.job_rate(10.0, 2.0, 1) == 5.0
