"""Multi-process sharding of the DBIE path (one process per GPU).

Evaluation points are independent: each rank solves a contiguous share of the points against
the same (replicated) magnetogram, with no exchange during the solve.  The one real exchange is
the backward pass: dL/dB0 = A^T gB is a sum over all points, i.e. a sum over the ranks' partial
adjoints (one all-reduce of (ny, nx, 3) FP64 at the end).

The gradient through the lambda search (DBIEField.vjp_implicit) is also a sum over points, so it
shards the same way.  The functions take the per-rank compute as a callable so that the same
host logic drives the GPU library (DBIEField.vjp / .vjp_implicit / .solve) and can be exercised
with CPU process groups.
"""
from __future__ import annotations

from typing import Callable, Sequence

import torch
import torch.distributed as dist


def partition(n: int, world: int, weights: Sequence[float] | None = None) -> list[tuple[int, int]]:
    """Contiguous [start, end) ranges of n points over `world` ranks, balanced by count (or by
    cumulative `weights`, e.g. expected objective evaluations per point)."""
    if world < 1:
        raise ValueError("world must be >= 1")
    if weights is None:
        base, extra = divmod(n, world)
        out, s = [], 0
        for r in range(world):
            e = s + base + (1 if r < extra else 0)
            out.append((s, e))
            s = e
        return out
    w = torch.as_tensor(weights, dtype=torch.float64)
    if w.numel() != n:
        raise ValueError("weights must have one entry per point")
    c = torch.cumsum(w, 0)
    total = float(c[-1]) if n else 0.0
    bounds = [0]
    for r in range(1, world):
        bounds.append(int(torch.searchsorted(c, total * r / world).item()))
    bounds.append(n)
    return [(bounds[r], max(bounds[r], bounds[r + 1])) for r in range(world)]


def shard_of(x, rank: int, world: int):
    s, e = partition(x.shape[0], world)[rank]
    return x[s:e]


def sharded_vjp(vjp_fn: Callable, xyz, lam, gB, group=None):
    """dL/dB0 summed over all ranks' points.  vjp_fn(xyz_shard, lam_shard, gB_shard) returns this
    rank's partial adjoint as a tensor; the sum is an all-reduce over the process group."""
    rank = dist.get_rank(group)
    world = dist.get_world_size(group)
    s, e = partition(xyz.shape[0], world)[rank]
    part = vjp_fn(xyz[s:e], lam[s:e], gB[s:e])
    part = part.contiguous()
    dist.all_reduce(part, op=dist.ReduceOp.SUM, group=group)
    return part


def sharded_solve(solve_fn: Callable, xyz, group=None, gather: bool = True):
    """Solve this rank's share of the points; optionally all-gather the per-point results
    (a dict of tensors with the points along dim 0) into full-size tensors on every rank."""
    rank = dist.get_rank(group)
    world = dist.get_world_size(group)
    parts = partition(xyz.shape[0], world)
    s, e = parts[rank]
    res = solve_fn(xyz[s:e])
    if not gather:
        return res
    m = max(pe - ps for ps, pe in parts)   # equal-size buffers for every backend
    out = {}
    for k, v in res.items():
        pad = torch.zeros((m,) + tuple(v.shape[1:]), dtype=v.dtype, device=v.device)
        pad[: v.shape[0]] = v
        full = [torch.empty_like(pad) for _ in parts]
        dist.all_gather(full, pad, group=group)
        out[k] = torch.cat([f[: pe - ps] for f, (ps, pe) in zip(full, parts)], 0)
    return out
