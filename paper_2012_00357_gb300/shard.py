"""Merge of nearest-point searches over a data set sharded across ranks.

Each rank holds a contiguous slice [offset, offset + n) of the data points
and answers every query over its slice (dd_project_nearest on its own data
set).  The exact answer over the whole set is, per query, the smallest
squared distance over the ranks, ties to the lowest global index (the tie
rule of the exact search).  One all_gather of (d2, global index) per call;
works with gloo (host tensors) and NCCL (device tensors).
"""
from __future__ import annotations

import torch
import torch.distributed as dist


def merge_nearest(d2, idx, offset: int, group=None):
    """(d2, global index) of the nearest point over all ranks, per query.

    d2: squared distances of the local answers [m]; idx: local indices [m]
    (int); offset: global index of this rank's first point.  Every rank
    passes the same m and receives the same result.
    """
    d2 = torch.as_tensor(d2, dtype=torch.float64).contiguous()
    gi = (torch.as_tensor(idx).to(torch.int64) + int(offset)).contiguous()
    world = dist.get_world_size(group)
    all_d = [torch.empty_like(d2) for _ in range(world)]
    all_i = [torch.empty_like(gi) for _ in range(world)]
    dist.all_gather(all_d, d2, group=group)
    dist.all_gather(all_i, gi, group=group)
    D = torch.stack(all_d)
    G = torch.stack(all_i)
    best = D.min(dim=0).values
    big = torch.iinfo(torch.int64).max
    gidx = torch.where(D == best.unsqueeze(0), G, torch.full_like(G, big)).min(dim=0).values
    return best, gidx
