"""Sharding the search over several GPUs, one process per GPU.

The scan needs no exchange: occurrences in different parts of a text, or in
different texts, are independent.  A text of n bytes is cut into one byte
range per rank; rank w reads [lo, hi) with hi extended by m - 1 bytes past
its own range so that every window starting in its own range [own_lo,
own_hi) lies inside what it reads, and keeps only the occurrences that start
there (each start belongs to exactly one rank).  A batch of texts is dealt
out whole, longest text first to the rank with the fewest bytes so far.
Gathering the ranks' lists is the only collective, and it sits outside the
data path (after the searches): with ranges in rank order the concatenation
is already sorted by position.

Nothing here touches a GPU; the per-rank search is whatever function the
caller passes (the library's mpm_search on a GPU).
"""
import numpy as np


def text_shards(n, m, world):
    """Per rank (lo, hi, own_lo, own_hi): bytes read and starts owned."""
    if world < 1 or m < 1 or n < 0:
        raise ValueError("bad shard request")
    out = []
    for w in range(world):
        own_lo = n * w // world
        own_hi = n * (w + 1) // world
        hi = min(n, own_hi + m - 1) if own_hi > own_lo else own_lo
        out.append((own_lo, hi, own_lo, own_hi))
    return out


def batch_shards(lengths, world):
    """Texts per rank: longest first to the rank with the fewest bytes so far
    (ties to the lowest rank); each rank's list is in increasing text order."""
    if world < 1:
        raise ValueError("bad shard request")
    load = [0] * world
    parts = [[] for _ in range(world)]
    for t in sorted(range(len(lengths)), key=lambda i: (-int(lengths[i]), i)):
        w = min(range(world), key=lambda j: (load[j], j))
        parts[w].append(t)
        load[w] += int(lengths[t])
    return [sorted(p) for p in parts]


def search_shard(search, T, m, rank, world):
    """Occurrences (pos, pid) of this rank's share of text T: search(view)
    returns (pos, pid) for a contiguous view of T; positions come back
    relative to T and only those this rank owns are kept."""
    lo, hi, own_lo, own_hi = text_shards(len(T), m, world)[rank]
    pos, pid = search(T[lo:hi])
    pos = np.asarray(pos, dtype=np.int64) + lo
    pid = np.asarray(pid, dtype=np.int64)
    keep = (pos >= own_lo) & (pos < own_hi)
    return pos[keep], pid[keep]


def gather_occurrences(pos, pid, group=None):
    """All ranks' (pos, pid) lists, concatenated in rank order (every rank
    receives the whole list)."""
    import torch.distributed as dist
    world = dist.get_world_size(group)
    parts = [None] * world
    dist.all_gather_object(parts, (np.asarray(pos, np.int64), np.asarray(pid, np.int64)), group)
    if not parts:
        return np.zeros(0, np.int64), np.zeros(0, np.int64)
    return (np.concatenate([p[0] for p in parts]), np.concatenate([p[1] for p in parts]))
