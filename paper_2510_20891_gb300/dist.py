"""Multi-GPU data parallelism over tracks (one process per GPU).

Tracks are independent, so each rank evaluates its own shard against its own
replica of the table and basis; the only exchange is the global top-k: every
rank contributes its local (value, global index) list and the lists are
merged with the same order as the single-GPU top-k (descending value, lower
index first, NaN last).
"""
from __future__ import annotations

import numpy as np


def merge_topk(vals_list, idx_list, k: int):
    """Merge per-rank top-k lists (values float32, global int64 indices) into the global top-k."""
    v = np.concatenate([np.asarray(a, dtype=np.float32) for a in vals_list]) if vals_list else np.zeros(0, np.float32)
    i = np.concatenate([np.asarray(a, dtype=np.int64) for a in idx_list]) if idx_list else np.zeros(0, np.int64)
    nan = np.isnan(v)
    key = np.where(nan, 0.0, -v.astype(np.float64)) + 0.0
    order = np.lexsort((i, key, nan))[: min(k, v.size)]
    return i[order], v[order]


def allgather_topk(idx, val, k: int, offset: int, group=None):
    """Global top-k over all ranks of a torch.distributed group.

    ``idx`` / ``val`` are this rank's local top-k (torch tensors, any device);
    ``offset`` is the global index of this rank's first track.
    """
    import torch
    import torch.distributed as dist

    ws = dist.get_world_size(group)
    kk = int(idx.numel())
    dev = val.device
    gi = (idx.to(torch.int64) + offset).to(dev)
    gv = val.to(torch.float32)
    counts = [torch.zeros(1, dtype=torch.int64, device=dev) for _ in range(ws)]
    dist.all_gather(counts, torch.tensor([kk], dtype=torch.int64, device=dev), group=group)
    cmax = int(max(c.item() for c in counts))
    pad_i = torch.full((cmax,), -1, dtype=torch.int64, device=dev)
    pad_v = torch.full((cmax,), float("nan"), dtype=torch.float32, device=dev)
    pad_i[:kk] = gi
    pad_v[:kk] = gv
    all_i = [torch.empty_like(pad_i) for _ in range(ws)]
    all_v = [torch.empty_like(pad_v) for _ in range(ws)]
    dist.all_gather(all_i, pad_i, group=group)
    dist.all_gather(all_v, pad_v, group=group)
    vals = [all_v[r][: int(counts[r].item())].cpu().numpy() for r in range(ws)]
    idxs = [all_i[r][: int(counts[r].item())].cpu().numpy() for r in range(ws)]
    return merge_topk(vals, idxs, k)
