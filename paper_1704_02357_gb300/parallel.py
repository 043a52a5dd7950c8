"""Splitting one catalog's multipoles over several GPUs.

The transforms of a multipole are independent (Sec. 2.1: P_l needs the 2l+1 transforms
G_lm, each binned against the same F0), so they shard without any exchange until the end.
Every rank paints the same catalogs and builds the same F0 (one r2c, cheap next to the
harmonics), computes the raw FP64 bin sums of a contiguous range of the flat harmonic list
(pspec_multipoles_range), and one all-reduce (sum) of the (1 + n_ells) x nk bins precedes
pspec_finalize_bins. Only rank 0 contributes the l = 0 bins, so they are counted once.

Independent catalogs (mocks, the common case) need none of this: one catalog per GPU, no
collective. This module is the strong-scaling path for a single catalog with a high l_max.
"""
from __future__ import annotations

from typing import Callable, List, Optional, Sequence, Tuple


def harmonic_items(ells: Sequence[int]) -> List[Tuple[int, int]]:
    """The flat harmonic list: (l, m) for each l >= 2 of ells, in that order, m = 0, +1, -1, +2, -2, ..."""
    out = []
    for ell in ells:
        ell = int(ell)
        if ell == 0:
            continue
        out.append((ell, 0))
        for a in range(1, ell + 1):
            out.append((ell, a))
            out.append((ell, -a))
    return out


def split(n_items: int, world: int, rank: int) -> Tuple[int, int]:
    """Contiguous range [q0, q1) of rank `rank`; sizes differ by at most one, ranks in order."""
    if world < 1 or not 0 <= rank < world or n_items < 0:
        raise ValueError("bad world/rank/items")
    base, extra = divmod(n_items, world)
    q0 = rank * base + min(rank, extra)
    return q0, q0 + base + (1 if rank < extra else 0)


def sharded_multipoles(est, ells: Sequence[int], k_edges, rank: Optional[int] = None, world: Optional[int] = None,
                       group=None, all_reduce: Optional[Callable] = None) -> dict:
    """P_l of the catalogs painted on `est`, the harmonics shared across the ranks of `group`.

    `est` is an Estimator (or anything with multipoles_range / finalize_bins). The bins are
    summed with torch.distributed.all_reduce unless `all_reduce` is given. For CUDA bins the
    collective is issued on the estimator's stream, so nothing synchronises with the host.
    """
    import torch
    import torch.distributed as dist
    if world is None:
        world = dist.get_world_size(group) if dist.is_initialized() else 1
    if rank is None:
        rank = dist.get_rank(group) if dist.is_initialized() else 0
    q0, q1 = split(len(harmonic_items(ells)), world, rank)
    bins = est.multipoles_range(ells, k_edges, q0, q1, include_p0=(rank == 0))
    if world > 1:
        reduce = all_reduce or (lambda t: dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group))
        if bins.is_cuda:
            with torch.cuda.stream(est.stream):
                reduce(bins)
        else:
            reduce(bins)
    return est.finalize_bins(bins, ells, k_edges)
