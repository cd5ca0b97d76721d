"""Sharding the search across ranks (paper_1405_5483_gb300/shard.py), on the
CPU: the range arithmetic, and world-size-2 gloo process groups whose ranks
each search their share (with the oracle's Aho-Corasick standing in for the
GPU search, which needs no GPU here) and gather the lists."""
import os
import socket

import numpy as np
import pytest

from paper_1405_5483_gb300 import shard


@pytest.mark.parametrize("n,m,world", [(0, 4, 2), (10, 4, 3), (1000, 16, 2), (1000, 16, 7),
                                       (5, 8, 4), (1 << 20, 32, 8)])
def test_text_shards_own_every_start_once_and_read_every_window(n, m, world):
    sh = shard.text_shards(n, m, world)
    owned = np.zeros(n, np.int64)
    for lo, hi, own_lo, own_hi in sh:
        assert 0 <= lo <= own_lo <= own_hi <= n and lo <= hi <= n
        owned[own_lo:own_hi] += 1
        # every window starting in the owned range that fits the text is read whole
        for i in (own_lo, own_hi - 1):
            if own_lo <= i < own_hi and i + m <= n:
                assert lo <= i and i + m <= hi
    assert np.all(owned == 1)
    # contiguous and in rank order
    assert [s[2] for s in sh[1:]] == [s[3] for s in sh[:-1]]


def test_batch_shards_balance_and_cover():
    rng = np.random.default_rng(4)
    lengths = np.exp(rng.uniform(np.log(1024), np.log(4 << 20), 500)).astype(np.int64)
    parts = shard.batch_shards(lengths, 4)
    assert sorted(t for p in parts for t in p) == list(range(500))
    loads = [int(lengths[p].sum()) for p in parts]
    # LPT: no rank exceeds the mean by more than the longest text
    assert max(loads) - sum(loads) / 4 <= lengths.max()
    assert all(p == sorted(p) for p in parts)
    assert shard.batch_shards([], 3) == [[], [], []]


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, T, P, out):
    import torch.distributed as dist
    from oracle import native
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        def search(view):
            pos, pid = native.aho_corasick(np.ascontiguousarray(view), P)
            return pos, pid
        pos, pid = shard.search_shard(search, T, P.shape[1], rank, world)
        allpos, allpid = shard.gather_occurrences(pos, pid)
        out.put((rank, allpos, allpid, pos.size))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2])
def test_sharded_search_equals_whole_text_search(world):
    import torch.multiprocessing as mp
    from oracle import native
    native.build()
    rng = np.random.default_rng(8)
    T = rng.integers(0, 4, size=200_003).astype(np.uint8) + 65
    P = rng.integers(0, 4, size=(40, 9)).astype(np.uint8) + 65
    # plant occurrences across the split point and at both ends
    mid = len(T) // 2
    for i, at in enumerate([0, mid - 4, mid - 1, mid, len(T) - 9]):
        T[at:at + 9] = P[i]
    want_pos, want_pid = native.aho_corasick(T, P)
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, T, P, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    total_local = 0
    for rank, pos, pid, nlocal in got:
        total_local += nlocal
        order = np.lexsort((pid, pos))
        assert np.array_equal(pos[order], want_pos) and np.array_equal(pid[order], want_pid)
        # rank-ordered concatenation is already sorted by position
        assert np.all(np.diff(pos) >= 0)
    assert total_local == want_pos.size
