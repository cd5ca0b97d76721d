"""GPU parity of the pipelined search (mpm_search_async): many searches in
flight on one handle, each checked against the oracle (Aho-Corasick), and
the status block's account of the cases it cannot finish by itself."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

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


@pytest.mark.parametrize("kernel", [1, 2, 3])
def test_pipelined_searches_match_oracle(mpm, native, kernel):
    rng = np.random.default_rng(kernel)
    texts, P = [], None
    case = W.protein_case(1 << 21, 300, 16, 150, cfg=9)
    P = case.P
    for i in range(12):
        n = int(rng.integers(1000, 1 << 21))
        texts.append(np.ascontiguousarray(case.T[(1 << 21) - n:]) if i % 2 else case.T[:n])
    m = mpm.Matcher(P, sigma=20, q=3, sigma_r=16, k=1, map_kind=2, kernel=kernel)
    cap = 4096
    outs = [(torch.empty(cap, dtype=torch.int32, device="cuda"),
             torch.empty(cap, dtype=torch.int32, device="cuda")) for _ in texts]
    status = torch.zeros((len(texts), 4), dtype=torch.int32, device="cuda")
    dev = [torch.from_numpy(t).cuda() for t in texts]
    for i, T in enumerate(dev):
        m.search_async(T, outs[i][0], outs[i][1], status[i])
    m.sync()
    st = status.cpu().numpy()
    for i, T in enumerate(texts):
        want = native.aho_corasick(T, P)
        z = want[0].size
        assert st[i, 1] == z and st[i, 2] == 0 and st[i, 3] == 1, (i, st[i])
        assert np.array_equal(as_u32(outs[i][0])[:z], want[0])
        assert np.array_equal(as_u32(outs[i][1])[:z], want[1])


def test_incomplete_cases_and_the_synchronous_rerun(mpm, native):
    case = W.dna_case(1 << 20, 100, 16, 50, cfg=1)
    T = torch.from_numpy(case.T).cuda()
    m = mpm.Matcher(case.P, sigma=4)
    want = native.aho_corasick(case.T, case.P)
    z = want[0].size
    assert z >= 50
    status = torch.zeros(4, dtype=torch.int32, device="cuda")
    small = torch.empty(10, dtype=torch.int32, device="cuda")
    m.search_async(T, small, small.clone(), status)
    m.sync()
    s = status.cpu().numpy()
    assert s[1] == z and s[3] == 0          # z > cap
    pos, pid = m.search(T)
    assert np.array_equal(as_u32(pos), want[0]) and np.array_equal(as_u32(pid), want[1])
    # more than 4096 occurrences (runs of one symbol): the radix sort closes
    # the search when the outputs have room; with 4096 entries they have not
    runs = np.full(20_000, 65, np.uint8)
    P = np.full((2, 8), 65, np.uint8)
    m2 = mpm.Matcher(P, sigma=2)
    big = torch.empty(1 << 16, dtype=torch.int32, device="cuda")
    bigi = big.clone()
    m2.search_async(torch.from_numpy(runs).cuda(), big, bigi, status)
    m2.sync()
    s = status.cpu().numpy()
    zr = 2 * (20_000 - 7)
    assert s[1] == zr and s[3] == 1
    wr = native.aho_corasick(runs, P)
    assert np.array_equal(as_u32(big)[:zr], wr[0]) and np.array_equal(as_u32(bigi)[:zr], wr[1])
    m2.search_async(torch.from_numpy(runs).cuda(), big[:4096], bigi[:4096], status)
    m2.sync()
    s = status.cpu().numpy()
    assert s[1] == zr and s[3] == 0
    # a text shorter than the patterns: z = 0, complete
    m.search_async(T[:5], small, small.clone(), status)
    m.sync()
    assert list(status.cpu().numpy()) == [0, 0, 0, 1]


def test_candidate_overflow_is_reported(mpm, native):
    # q = 1 over DNA with the split kernel: a candidate at nearly every byte,
    # more than the first candidate buffer (n / 64 + 1024 records) holds
    rng = np.random.default_rng(3)
    Tn = (rng.integers(0, 4, 1 << 20) + 65).astype(np.uint8)
    P = (rng.integers(0, 4, (64, 8)) + 65).astype(np.uint8)
    m = mpm.Matcher(P, sigma=4, q=1, sigma_r=4, k=1, map_kind=2, kernel=3)
    status = torch.zeros(4, dtype=torch.int32, device="cuda")
    out = torch.empty(1 << 16, dtype=torch.int32, device="cuda")
    T = torch.from_numpy(Tn).cuda()
    m.search_async(T, out, out.clone(), status)
    m.sync()
    s = status.cpu().numpy()
    want = native.aho_corasick(Tn, P)
    assert s[0] > (1 << 20) // 64 + 1024 and s[3] == 0
    pos, pid = m.search(T)   # grows the buffer
    assert np.array_equal(as_u32(pos), want[0]) and np.array_equal(as_u32(pid), want[1])
    # now the buffer is large enough for the pipelined call too
    m.search_async(T, out, out.clone(), status)
    m.sync()
    s = status.cpu().numpy()
    assert s[3] == 1 and s[1] == want[0].size


def test_mapped_status_interleaving_and_timing(mpm, native):
    case = W.protein_case(1 << 22, 1000, 32, 500, cfg=2)
    T = torch.from_numpy(case.T).cuda()
    want = native.aho_corasick(case.T, case.P)
    z = want[0].size
    m = mpm.Matcher(case.P, sigma=20)
    m.set_timing(True)
    pinned = torch.zeros((6, 4), dtype=torch.int32).pin_memory()
    pos = torch.empty(4096, dtype=torch.int32, device="cuda")
    pid = torch.empty_like(pos)
    m.reset_stats()
    for i in range(3):
        m.search_async(T, pos, pid, pinned[i])
    # a synchronous search in between gives the same answer
    p2, i2 = m.search(T)
    assert np.array_equal(as_u32(p2), want[0]) and np.array_equal(as_u32(i2), want[1])
    m.reset_stats()
    for i in range(3, 6):
        m.search_async(T, pos, pid, pinned[i])
    m.sync()
    st = m.stats
    assert st["launches"] >= 6 and st["ms_scan"] > 0 and st["n"] == 3 * case.n
    assert np.all(pinned.numpy()[:, 1] == z) and np.all(pinned.numpy()[:, 3] == 1)
    assert np.array_equal(as_u32(pos)[:z], want[0]) and np.array_equal(as_u32(pid)[:z], want[1])


def test_join_orders_later_stream_work_and_stream_switches(mpm, native):
    case = W.protein_case(1 << 21, 500, 24, 250, cfg=12)
    T = torch.from_numpy(case.T).cuda()
    want = native.aho_corasick(case.T, case.P)
    z = want[0].size
    assert 0 < z <= 4096
    m = mpm.Matcher(case.P, sigma=20)
    outs = [(torch.empty(4096, dtype=torch.int32, device="cuda"),
             torch.empty(4096, dtype=torch.int32, device="cuda")) for _ in range(5)]
    status = torch.zeros((5, 4), dtype=torch.int32, device="cuda")
    copies = []
    for i in range(3):
        m.search_async(T, outs[i][0], outs[i][1], status[i])
    m.join()
    # later work on the same stream sees the finished outputs without a host wait
    copies = [o[0][:z].clone() for o in outs[:3]] + [status[:3].clone()]
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        for i in range(3, 5):
            m.search_async(T, outs[i][0], outs[i][1], status[i])
        m.join()
        late = [o[1][:z].clone() for o in outs[3:]]
    torch.cuda.synchronize()
    for c in copies[:3]:
        assert np.array_equal(c.cpu().numpy().view(np.uint32), want[0])
    assert np.all(copies[3].cpu().numpy()[:, 1] == z)
    for c in late:
        assert np.array_equal(c.cpu().numpy().view(np.uint32), want[1])
    assert np.all(status.cpu().numpy()[:, 3] == 1)


@pytest.mark.parametrize("cap", [1 << 17, (1 << 20) + 64], ids=["one-block", "multi-block"])
@pytest.mark.parametrize("z_target", [4095, 4097, 9000, 70_000])
def test_pipelined_large_counts_through_both_buffer_sets(mpm, native, z_target, cap):
    """Counts on both sides of the rank sort's 4096, several searches in a
    row (both internal buffer sets, the closing sorts overlapping the next
    scans), each against the oracle, with the one-block and the multi-block
    closing sorts; the occurrence buffer's first size (65 536) is exceeded
    by the last count, which the synchronous search then grows for the
    pipelined calls after it."""
    rng = np.random.default_rng(z_target)
    n = 1 << 22
    T = (rng.integers(0, 4, n) + 65).astype(np.uint8)
    P = (rng.integers(0, 4, (50, 16)) + 65).astype(np.uint8)
    offs = rng.choice(n // 16, size=z_target, replace=False) * 16
    for i, o in enumerate(offs):
        T[o:o + 16] = P[i % 50]
    want = native.aho_corasick(T, P, threads=8)
    z = want[0].size
    Td = torch.from_numpy(T).cuda()
    m = mpm.Matcher(P, sigma=4)
    outs = [(torch.full((cap,), -1, dtype=torch.int32, device="cuda"),
             torch.full((cap,), -1, dtype=torch.int32, device="cuda")) for _ in range(3)]
    status = torch.zeros((3, 4), dtype=torch.int32, device="cuda")
    for attempt in range(2):
        for i in range(3):
            m.search_async(Td, outs[i][0], outs[i][1], status[i])
        m.sync()
        st = status.cpu().numpy()
        if attempt == 0 and z > 65536:
            assert np.all(st[:, 3] == 0)   # the first occurrence buffer is too small
            m.search(Td)                   # grows it
            continue
        assert np.all(st[:, 1] == z) and np.all(st[:, 2] == 0) and np.all(st[:, 3] == 1), st
        for pos, pid in outs:
            assert np.array_equal(as_u32(pos)[:z], want[0])
            assert np.array_equal(as_u32(pid)[:z], want[1])
        break
