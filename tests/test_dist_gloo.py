"""The multi-rank path of the benchmark on CPU: two gloo ranks shard the
sweep's instances and reduce their timings (max time, summed work)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    from paper_1210_4090_gb300 import dist as D
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    items = list(range(11))
    mine = D.shard(items, rank, world)
    t, u = D.reduce_step(10.0 + rank, float(sum(mine)))
    q.put((rank, mine, t, u))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_shard_and_reduce():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, m0, t0, u0), (r1, m1, t1, u1) = out
    assert sorted(m0 + m1) == list(range(11)) and not set(m0) & set(m1)
    assert t0 == t1 == 11.0 and u0 == u1 == float(sum(range(11)))


def test_single_process_reduce_is_identity():
    from paper_1210_4090_gb300 import dist as D
    assert D.reduce_step(3.0, 7.0) == (3.0, 7.0)
    with pytest.raises(ValueError):
        D.shard([1, 2], 2, 2)
