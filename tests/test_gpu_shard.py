"""The sharded search on one GPU: G logical partitions of one text, each
searched by its own handle on its own CUDA stream (independent searches, no
kernel waits on another), kept to the starts each partition owns and
concatenated in partition order; the result must equal the oracle's list for
the whole text, element by element.  The same for a batch of texts dealt out
by batch_shards."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

from paper_1405_5483_gb300 import shard  # noqa: E402
from paper_1405_5483_gb300 import workloads as W  # noqa: E402


@pytest.fixture(scope="module")
def mpm():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_1405_5483_gb300 import build_lib
    build_lib.build()
    import paper_1405_5483_gb300 as mpm
    return mpm


@pytest.fixture(scope="module")
def native():
    from oracle import native
    native.build()
    return native


def as_u32(t):
    return t.cpu().numpy().view(np.uint32)


@pytest.mark.parametrize("world", [2, 3, 4, 7])
def test_logical_partitions_on_separate_streams_equal_the_whole_search(mpm, native, world):
    case = W.dna_case((8 << 20) + 13, 200, 16, 100, cfg=31)
    T = np.array(case.T)
    m = case.P.shape[1]
    # occurrences straddling every partition boundary
    for w in range(1, world):
        cut = len(T) * w // world
        T[cut - m // 2: cut - m // 2 + m] = case.P[w % case.P.shape[0]]
    want_pos, want_pid = native.aho_corasick(T, case.P, threads=8)
    Td = torch.from_numpy(T).cuda()
    torch.cuda.synchronize()
    streams = [torch.cuda.Stream() for _ in range(world)]
    matchers = [mpm.Matcher(case.P, sigma=4) for _ in range(world)]
    results = [None] * world
    for w in range(world):
        with torch.cuda.stream(streams[w]):
            def search(view, mt=matchers[w]):
                pos, pid = mt.search(view)
                return as_u32(pos), as_u32(pid)
            results[w] = shard.search_shard(search, Td, m, w, world)
    torch.cuda.synchronize()
    pos = np.concatenate([r[0] for r in results])
    pid = np.concatenate([r[1] for r in results])
    assert np.array_equal(pos, want_pos.astype(np.int64))
    assert np.array_equal(pid, want_pid.astype(np.int64))
    # every boundary occurrence is there exactly once
    for w in range(1, world):
        cut = len(T) * w // world
        assert np.count_nonzero(pos == cut - m // 2) >= 1


def test_batch_partitions_cover_every_text_once(mpm, native):
    rng = np.random.default_rng(5)
    case = W.protein_case(1 << 20, 100, 12, 50, cfg=32)
    lengths = rng.integers(1, 200_000, size=40)
    texts = [case.source.draw(int(n), rng) for n in lengths]
    for i in range(0, 40, 5):  # a planted occurrence in some texts
        if texts[i].size >= 12:
            texts[i][: 12] = case.P[i % case.P.shape[0]]
    mt = mpm.Matcher(case.P, sigma=20)
    parts = shard.batch_shards(lengths, 3)
    assert sorted(t for p in parts for t in p) == list(range(40))
    for p in parts:
        for t in p:
            pos, pid = mt.search(torch.from_numpy(texts[t]).cuda())
            wp, wi = native.aho_corasick(texts[t], case.P, threads=4)
            assert np.array_equal(as_u32(pos), wp) and np.array_equal(as_u32(pid), wi)
