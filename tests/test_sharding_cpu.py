"""Sharding of independent problems over ranks: partition logic and a
2-rank gloo run on CPU (the local solver is injected; here the FP64 oracle)."""
import os
import socket

import numpy as np
import pytest

from paper_1905_12154_gb300.sharding import partition_lpt, solve_sharded


def test_partition_lpt_balances_and_covers():
    costs = [512 * 512, 64 * 64, 256 * 256, 128 * 128, 512 * 512, 64 * 64, 256 * 256]
    bins = partition_lpt(costs, 2)
    assert sorted(i for b in bins for i in b) == list(range(len(costs)))
    loads = [sum(costs[i] for i in b) for b in bins]
    assert max(loads) - min(loads) <= max(costs)
    assert partition_lpt(costs, 1) == [list(range(len(costs)))]
    assert partition_lpt([5], 3) == [[0], [], []]


def _problems():
    import synthetic_inputs as si
    rng = np.random.default_rng(40)
    out = []
    for n in (8, 12, 16, 8, 12):
        a = si.normalise(rng.uniform(0.1, 1.0, (n, n)))
        b = si.normalise(rng.uniform(0.1, 1.0, (n, n)))
        out.append((a, b))
    return out


def _oracle_solve(mus, nus, **kw):
    import oracle
    return [oracle.solve(m, v, **kw) for m, v in zip(mus, nus)]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)

    def gather(obj):
        out = [None] * world
        dist.all_gather_object(out, obj)
        return out

    probs = _problems()
    res = solve_sharded([p[0] for p in probs], [p[1] for p in probs], rank, world,
                        _oracle_solve, gather, tol=0.0, max_iter=6)
    q.put((rank, res))
    dist.destroy_process_group()


def test_two_rank_gloo_gather_matches_serial():
    import torch.multiprocessing as mp
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    probs = _problems()
    serial = _oracle_solve([p[0] for p in probs], [p[1] for p in probs], tol=0.0, max_iter=6)
    for rank in (0, 1):
        assert [r["w2sq"] for r in got[rank]] == [r["w2sq"] for r in serial]
        assert {r["rank"] for r in got[rank]} == {0, 1}        # both ranks did work
    assert got[0] == got[1]
