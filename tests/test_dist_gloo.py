"""The multi-rank path of the batched sweep on CPU (gloo, two ranks): the
instances are assigned by LPT on their work (N_i^2 points each), every rank
computes the H-bar readout of its own instances with the oracle, the
per-instance rows are gathered in instance order, and the timings reduce to
(max time, summed work).  The gathered table equals a single-rank run.  Not
run on several GPUs (one GPU per call on this hardware)."""
import os
import socket

import numpy as np
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


def _instances():
    """Eight small 2D instances with the sweep's laws (uneven sizes)."""
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    from paper_1210_4090_gb300 import workloads as WL
    probs = []
    for i, N in enumerate((16, 24, 12, 20, 16, 8, 24, 12)):
        p = WL.sweep512(count=1, nsteps=6, sizes=(N,), seed=40 + i)[0]
        probs.append(p)
    return probs


def _hbar_rows(probs):
    """Readout of each instance after its steps: -mean((u^n - u^0)/(n h)),
    min and max over the grid (oracle)."""
    from oracle import oracle as O
    rows = []
    for p in probs:
        un = O.run(p.u0, p.dx, p.h, p.P, p.W, p.V, p.nsteps)
        r = -(un - p.u0) / (p.nsteps * p.h)
        rows.append((float(np.mean(r)), float(np.min(r)), float(np.max(r))))
    return np.array(rows)


def _worker(rank, world, port, q):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    from paper_1210_4090_gb300 import dist as D
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    probs = _instances()
    weights = [p.npts for p in probs]
    idx = D.shard_indices(len(probs), rank, world, weights)
    rows = _hbar_rows([probs[i] for i in idx])
    table = D.gather_rows(rows, idx, len(probs))
    t, u = D.reduce_step(10.0 + rank, float(sum(weights[i] for i in idx)))
    q.put((rank, idx, table.tolist(), t, u))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_lpt_gather_and_reduce():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, i0, tab0, t0, u0), (r1, i1, tab1, t1, u1) = out
    probs = _instances()
    weights = [p.npts for p in probs]
    assert sorted(i0 + i1) == list(range(len(probs))) and not set(i0) & set(i1)
    single = _hbar_rows(probs)
    assert np.array_equal(np.array(tab0), single) and np.array_equal(np.array(tab1), single)
    assert t0 == t1 == 11.0 and u0 == u1 == float(sum(weights))


def test_lpt_balance():
    """LPT on N_i^2 work: the largest rank load is within Graham's 4/3 bound
    of the best possible (the total over the ranks, or the largest item), and
    no worse than round-robin on the sweep's size mix."""
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    from paper_1210_4090_gb300 import dist as D
    rng = np.random.default_rng(4)
    sizes = rng.choice(np.arange(128, 513, 64), size=512)
    w = [int(n) * int(n) for n in sizes]
    for world in (2, 3, 4, 8):
        owner = D.lpt_assign(w, world)
        loads = np.bincount(owner, weights=w, minlength=world)
        lower = max(sum(w) / world, max(w))
        assert loads.max() <= (4 / 3 - 1 / (3 * world)) * lower + 1e-9
        rr = np.bincount(np.arange(len(w)) % world, weights=w, minlength=world)
        assert loads.max() <= rr.max()
        got = sorted(i for r in range(world) for i in D.shard_indices(len(w), r, world, w))
        assert got == list(range(len(w)))


def test_single_process_gather_and_reduce_are_identity():
    from paper_1210_4090_gb300 import dist as D
    assert D.reduce_step(3.0, 7.0) == (3.0, 7.0)
    with pytest.raises(ValueError):
        D.shard([1, 2], 2, 2)
    t = D.gather_rows([[1.0, 2.0], [3.0, 4.0]], [2, 0], 3)
    assert np.array_equal(t[[0, 2]], np.array([[3.0, 4.0], [1.0, 2.0]]))
