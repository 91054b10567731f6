"""Star sharding across ranks (one process per GPU).

Stars are independent problems, so a batch is split across ranks with no
collective on the data path: each rank plans and searches its own stars, and
only small host-side results travel afterwards (the best record per star, the
per-rank work and time).

* ``star_cost``: relative search cost of each star, N_s * T_s * sqrt(rho_s).
  The grid of Sec. 2.1 steps by q_min(f) / (spp T) with q_min ~ rho^(-1/3)
  f^(2/3) for a/R* >> 1, so the number of trial frequencies grows as
  T rho^(1/3) (f_max^(1/3) - f_min^(1/3)) and f_max = 1/Pmin ~ rho^(1/2):
  n_f ~ T sqrt(rho) when f_max dominates; every trial frequency costs O(N).
* ``partition``: longest-processing-time-first assignment of stars to ranks.
* ``job_totals``: the job's work and its max-over-ranks time (the throughput
  rule of the bench: all ranks' units / the slowest rank's time).
* ``gather_best``: best records of every rank, in global star order, on rank 0.
* ``search_sharded``: the driver every rank calls with the whole batch.
"""
from __future__ import annotations

import heapq

import numpy as np


def star_cost(offsets, t, rho=None, rho_default: float = 1.41) -> np.ndarray:
    offsets = np.asarray(offsets, np.int64)
    t = np.asarray(t, np.float64)
    n = np.diff(offsets).astype(np.float64)
    span = np.zeros(n.shape[0])
    nz = n > 0
    span[nz] = t[offsets[1:][nz] - 1] - t[offsets[:-1][nz]]
    r = np.full(n.shape[0], rho_default) if rho is None else np.asarray(rho, np.float64).copy()
    r[~np.isfinite(r) | (r <= 0)] = rho_default
    return n * np.maximum(span, 0.0) * np.sqrt(r)


def partition(cost, world: int):
    """Stars per rank (sorted index arrays): each star, most expensive first,
    goes to the rank with the least assigned cost (ties: lowest rank)."""
    if world < 1:
        raise ValueError("world must be >= 1")
    cost = np.asarray(cost, np.float64)
    order = np.argsort(-cost, kind="stable")
    heap = [(0.0, r) for r in range(world)]
    parts = [[] for _ in range(world)]
    for s in order:
        load, r = heapq.heappop(heap)
        parts[r].append(int(s))
        heapq.heappush(heap, (load + float(cost[s]), r))
    return [np.asarray(sorted(p), np.int64) for p in parts]


def job_totals(local_work: float, local_ms: float, group=None):
    """(sum of work over ranks, max of time over ranks); no-op without a process group."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(local_work), float(local_ms)
    dev = "cuda" if dist.get_backend(group) == "nccl" else "cpu"
    w = torch.tensor([float(local_work)], dtype=torch.float64, device=dev)
    t = torch.tensor([float(local_ms)], dtype=torch.float64, device=dev)
    dist.all_reduce(w, op=dist.ReduceOp.SUM, group=group)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(w.item()), float(t.item())


def gather_best(best_local: np.ndarray, indices, n_stars: int, group=None):
    """Rank 0 gets the records of all ranks placed at their global star index
    (a structured array of n_stars entries); other ranks get None."""
    import torch.distributed as dist
    indices = np.asarray(indices, np.int64)
    if not (dist.is_available() and dist.is_initialized()):
        out = np.zeros(n_stars, best_local.dtype)
        out[indices] = best_local
        return out
    rank = dist.get_rank(group)
    world = dist.get_world_size(group)
    payload = (indices.tolist(), best_local.tobytes(), best_local.dtype.descr)
    got = [None] * world if rank == 0 else None
    dist.gather_object(payload, got, dst=0, group=group)
    if rank != 0:
        return None
    out = np.zeros(n_stars, best_local.dtype)
    seen = np.zeros(n_stars, bool)
    for idx, raw, descr in got:
        recs = np.frombuffer(raw, dtype=np.dtype(descr))
        idx = np.asarray(idx, np.int64)
        if np.any(seen[idx]):
            raise ValueError("a star was searched on two ranks")
        seen[idx] = True
        out[idx] = recs
    if not seen.all():
        raise ValueError("stars missing from the gathered results")
    return out


def _subset(offsets, arrays, stars):
    offsets = np.asarray(offsets, np.int64)
    idx = [np.arange(offsets[s], offsets[s + 1]) for s in stars]
    sel = np.concatenate(idx) if idx else np.zeros(0, np.int64)
    sub_off = np.concatenate([[0], np.cumsum([len(i) for i in idx])]).astype(np.int64)
    return sub_off, [None if a is None else np.asarray(a)[sel] for a in arrays]


def _search_library(offsets, t, y, dy, rho, rstar, params):
    from . import qlpbls
    return qlpbls.run_host(offsets, t, y, dy, rho, rstar, params)["best"]


def search_sharded(offsets, t, y, dy, rho=None, rstar=None, params=None, group=None, search_fn=None):
    """Every rank calls this with the same whole batch: each searches its
    longest-first share of the stars (one GPU per rank, no collective while
    searching) and rank 0 returns the best records of all stars in batch order
    (other ranks return None). search_fn(offsets, t, y, dy, rho, rstar, params)
    returns one record per star of its sub-batch; default: the library's
    host-buffer search (qlp_bls_run_host)."""
    import torch.distributed as dist
    on = dist.is_available() and dist.is_initialized()
    rank = dist.get_rank(group) if on else 0
    world = dist.get_world_size(group) if on else 1
    n_stars = int(np.asarray(offsets).shape[0] - 1)
    mine = partition(star_cost(offsets, t, rho), world)[rank]
    sub_off, (st, sy, sdy) = _subset(offsets, [t, y, dy], mine)
    srho = None if rho is None else np.asarray(rho)[mine]
    srs = None if rstar is None else np.asarray(rstar)[mine]
    best = (search_fn or _search_library)(sub_off, st, sy, sdy, srho, srs, params)
    return gather_best(np.asarray(best), mine, n_stars, group)
