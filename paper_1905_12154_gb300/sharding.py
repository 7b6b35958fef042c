"""Independent problems spread over the ranks of a process group.

A batch of unrelated transport problems needs no exchange while it is being
solved: each rank solves its own share (with bfm_solve_batched on its GPU) and
only the per-problem results (W2^2, iterations, convergence) are gathered at
the end.  Shares balance the work by the longest-processing-time rule on the
cell count, the per-iteration cost of a problem.
"""
from __future__ import annotations


def partition_lpt(costs, world_size: int) -> list[list[int]]:
    """Assign item indices to `world_size` bins, largest cost first, each to
    the currently lightest bin (ties: lowest rank).  Deterministic."""
    order = sorted(range(len(costs)), key=lambda i: (-costs[i], i))
    loads = [0] * world_size
    bins: list[list[int]] = [[] for _ in range(world_size)]
    for i in order:
        r = min(range(world_size), key=lambda k: (loads[k], k))
        bins[r].append(i)
        loads[r] += costs[i]
    return [sorted(b) for b in bins]


def solve_sharded(mus, nus, rank: int, world_size: int, solve_local, gather_objects, **kw):
    """Solve this rank's share of the problems and gather every problem's
    summary on every rank.

    solve_local(mus_subset, nus_subset, **kw) -> list of result dicts;
    gather_objects(obj) -> list with one obj per rank (e.g. a wrapper of
    torch.distributed.all_gather_object).  Returns one summary per problem in
    the original order: {"w2sq", "iters", "converged", "rank"}."""
    costs = [int(getattr(m, "numel", lambda: m.size)()) for m in mus]
    shares = partition_lpt(costs, world_size)
    mine = shares[rank]
    local = solve_local([mus[i] for i in mine], [nus[i] for i in mine], **kw) if mine else []
    summary = {i: {"w2sq": float(r["w2sq"]), "iters": int(r["iters"]),
                   "converged": bool(r["converged"]), "rank": rank}
               for i, r in zip(mine, local)}
    merged = {}
    for part in gather_objects(summary):
        merged.update(part)
    return [merged[i] for i in range(len(mus))]
