"""Sharding one simulation over several ranks by history id.

Every random number of a history is addressed by (seed, history id), and
decay times are drawn over the whole run's span, so the histories of one run
can be split across ranks in any way: each rank simulates a contiguous range
(gpet_options.h_begin / h_end), per-crystal tallies are summed and the singles
concatenated.  Coincidence sorting needs the merged, time-sorted singles of the
whole run.  This module holds the host-side logic; the collectives are
torch.distributed calls (NCCL on GPUs, gloo on CPUs).
"""
from __future__ import annotations

import numpy as np

SINGLE_FIELDS = ("t_ps", "h", "unit", "panel", "e", "e_raw")


def history_range(n_decays: int, rank: int, world: int) -> tuple[int, int]:
    """Contiguous, balanced slice [h0, h1) of the n_decays histories for `rank`."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("rank outside [0, world)")
    return n_decays * rank // world, n_decays * (rank + 1) // world


def merge_tallies(parts):
    """Sum of per-crystal (count, energy) tallies of several shards."""
    counts = np.sum([np.asarray(p[0], np.uint64) for p in parts], axis=0, dtype=np.uint64)
    efx = np.sum([np.asarray(p[1], np.uint64) for p in parts], axis=0, dtype=np.uint64)
    return counts, efx


def merge_singles(parts):
    """Concatenate the singles of several shards and order them by (time, unit, history)."""
    cat = {f: np.concatenate([np.asarray(p[f]) for p in parts]) for f in SINGLE_FIELDS if f in parts[0]}
    order = np.lexsort((cat["h"], cat["unit"], cat["t_ps"]))
    return {f: v[order] for f, v in cat.items()}


def allreduce_tallies(counts, efx, group=None):
    """Sum the per-crystal tallies over all ranks (torch.distributed, int64)."""
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend(group) == "nccl" else "cpu"
    t = torch.from_numpy(np.stack([counts, efx]).astype(np.int64)).to(dev)
    dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    t = t.cpu().numpy().astype(np.uint64)
    return t[0], t[1]


def gather_singles(singles, group=None):
    """All ranks' singles, merged and time-ordered, on every rank.

    Tensor collectives, no pickling: the ranks first exchange their singles
    counts (one all-gather of an int64), then every field is all-gathered as a
    tensor padded to the largest count (64-bit unsigned fields travel as their
    int64 bit patterns), and each rank trims the padding before the merge."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    dev = "cuda" if dist.get_backend(group) == "nccl" else "cpu"
    fields = [f for f in SINGLE_FIELDS if f in singles]
    n = len(np.asarray(singles[fields[0]])) if fields else 0
    counts = [torch.zeros(1, dtype=torch.int64, device=dev) for _ in range(world)]
    dist.all_gather(counts, torch.tensor([n], dtype=torch.int64, device=dev), group=group)
    counts = [int(c.item()) for c in counts]
    cap = max(counts + [1])
    parts = [dict() for _ in range(world)]
    for f in fields:
        a = np.asarray(singles[f])
        dt = a.dtype
        wire = a.view(np.int64) if dt == np.uint64 else a
        buf = np.zeros(cap, dtype=wire.dtype)
        buf[:n] = wire
        t = torch.from_numpy(buf).to(dev)
        out = [torch.empty_like(t) for _ in range(world)]
        dist.all_gather(out, t, group=group)
        for r in range(world):
            v = out[r].cpu().numpy()[:counts[r]]
            parts[r][f] = v.view(np.uint64) if dt == np.uint64 else v
    return merge_singles(parts)
