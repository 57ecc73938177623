"""Work partitions across GPUs (one process per GPU).

Two places of the method split naturally:
  * snapshots or scenarios (the batched tracking updates, the autograd batch)
    are independent problems: they are shared out longest-processing-time
    first (LPT) over the ranks, with no collective on the data path;
  * within one Hessian the direction blocks are independent given the factors
    (Sec. III-C: the n_u HVPs reuse one factorisation): every rank solves the
    power flow and factorises (replicas), computes a contiguous range of the
    Hessian's columns, and one all-gather assembles H on every rank.
The functions here decide the split and move the columns; the columns
themselves come from the library (opf_reduced_hessian with col_begin /
col_count) or, in the CPU tests, from any function with the same contract.
"""
from __future__ import annotations

import heapq


def lpt_assign(costs, nranks):
    """Longest-processing-time-first assignment: items by descending cost (ties by index),
    each to the rank with the smallest load so far (ties by rank).  Returns one list of item
    indices per rank (in assignment order) and the per-rank loads."""
    if nranks < 1:
        raise ValueError("nranks must be >= 1")
    order = sorted(range(len(costs)), key=lambda i: (-float(costs[i]), i))
    heap = [(0.0, r) for r in range(nranks)]
    out = [[] for _ in range(nranks)]
    loads = [0.0] * nranks
    for i in order:
        load, r = heapq.heappop(heap)
        out[r].append(i)
        loads[r] = load + float(costs[i])
        heapq.heappush(heap, (loads[r], r))
    return out, loads


def column_ranges(nu, nranks, block_k=8):
    """Contiguous column ranges [begin, end) per rank, cut at multiples of block_k (whole tiles)
    with tile counts differing by at most one between ranks."""
    if nranks < 1 or block_k < 1:
        raise ValueError("nranks and block_k must be >= 1")
    tiles = -(-nu // block_k)
    base, extra = divmod(tiles, nranks)
    out, t = [], 0
    for r in range(nranks):
        n = base + (1 if r < extra else 0)
        b, e = min(nu, t * block_k), min(nu, (t + n) * block_k)
        out.append((b, e))
        t += n
    return out


def gather_hessian_columns(local_cols, ranges, group=None):
    """All-gather of Hessian column blocks: rank r holds H[:, b_r:e_r] as a (e_r - b_r, n_u)
    tensor of columns (row j = column b_r + j); returns the full (n_u, n_u) tensor of columns
    on every rank.  Blocks are padded to the largest so one all_gather moves them."""
    import torch
    import torch.distributed as dist
    nu = local_cols.shape[1]
    width = max(e - b for b, e in ranges)
    pad = torch.zeros((width, nu), dtype=local_cols.dtype, device=local_cols.device)
    pad[:local_cols.shape[0]] = local_cols
    world = dist.get_world_size(group)
    bufs = [torch.empty_like(pad) for _ in range(world)]
    dist.all_gather(bufs, pad, group=group)
    full = torch.empty((nu, nu), dtype=local_cols.dtype, device=local_cols.device)
    for (b, e), buf in zip(ranges, bufs):
        full[b:e] = buf[:e - b]
    return full


def sharded_hessian(compute_columns, nu, block_k=8, group=None):
    """The full Hessian with this rank's column range from compute_columns(begin, count) (a
    (count, n_u) tensor of columns) and the others' by one all-gather."""
    import torch.distributed as dist
    ranges = column_ranges(nu, dist.get_world_size(group), block_k)
    b, e = ranges[dist.get_rank(group)]
    return gather_hessian_columns(compute_columns(b, e - b), ranges, group)
