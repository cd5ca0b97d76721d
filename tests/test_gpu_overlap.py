"""GPU parity of the overlapping-q-gram filter (Section 2's first filter,
`overlap = 1`): the scan's candidate windows equal the oracle's AOSO scan
over the text's q-gram at every byte, and full searches equal Aho-Corasick,
in the generic kernel and in both variants of the specialised one (the one
that verifies its candidates itself and the split one)."""
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

from oracle import filter as F  # noqa: E402
from paper_1405_5483_gb300 import workloads as W  # noqa: E402

KIND = {1: "rank", 2: "greedy", 3: "lowbits", 4: "qhash"}


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


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def as_u32(t):
    return t.cpu().numpy().view(np.uint32)


def windows_of(records, k, mprime):
    rec = records.cpu().numpy().view(np.uint64)
    h = (rec & np.uint64(0xFFFFFFFF)).astype(np.int64)
    fired = (rec >> np.uint64(32)).astype(np.int64)
    out = [h[((fired >> j) & 1) == 1] - (mprime - 1) * k - j for j in range(k)]
    return np.sort(np.concatenate(out)) if out else np.zeros(0, np.int64)


# (sigma, m, q, sigma_r, k, map_kind): every scan mode (2-bit and wider low
# bits, byte maps on raw and on reduced windows, q-gram hashing), every entry
# width, k from 1 to L'
SCAN_CASES = [
    (4, 16, 4, 4, 1, 3),
    (4, 16, 8, 4, 3, 3),
    (20, 32, 3, 8, 2, 2),
    (20, 32, 2, 16, 7, 1),
    (95, 64, 3, 16, 1, 2),
    (95, 64, 4, 1 << 12, 5, 4),
    (95, 40, 5, 1 << 12, 12, 4),
    (20, 80, 2, 16, 1, 2),      # 64 positions: 8-byte entries
    (4, 12, 1, 4, 4, 3),
    (95, 16, 6, 4, 2, 1),       # q = 6: reduced-symbol window
]


# mpm_scan runs the generic kernel or the specialised one that writes
# candidate records
SCAN_KERNELS = [1, 3]


@pytest.mark.parametrize("kernel", SCAN_KERNELS, ids=["generic", "specialised"])
@pytest.mark.parametrize("case", SCAN_CASES, ids=[str(c) for c in SCAN_CASES])
def test_overlap_candidates_equal_oracle(mpm, case, kernel):
    sigma, m, q, sr, k, kind = case
    rng = np.random.default_rng(sum(case))
    base = 65 if sigma <= 20 else 33
    n = 150_003
    T = (rng.integers(0, sigma, n) + base).astype(np.uint8)
    P = (rng.integers(0, sigma, (40, m)) + base).astype(np.uint8)
    for i in range(20):
        o = int(rng.integers(0, n - m + 1))
        P[i] = T[o:o + m]
    kw = dict(q=q, sigma_r=sr, k=k, map_kind=kind, overlap=1, kernel=kernel)
    if kind == 3:
        kw["map_shift"] = 0 if sigma > 4 else 1
    M = mpm.Matcher(P, sigma=sigma, **kw)
    p, info = M.params, M.info
    assert p["overlap"] == 1 and p["kernel"] == kernel
    got = windows_of(M.scan(dev(T)), k, info["mprime"])
    if kernel != 1:
        assert M.stats["specialised"] == 1
    fp = F.make_params(P, q, sr, k, KIND[kind], shift=p["map_shift"], overlap=True)
    cls = F.pattern_classes(P, fp)
    want = F.aoso_scan(F.text_codes(T, fp), F.mask_table(cls, fp), fp, len(cls))
    assert np.array_equal(got, np.array(want, np.int64))


@pytest.mark.parametrize("kernel", [1, 2, 3], ids=["generic", "verifying", "split"])
@pytest.mark.parametrize("case", SCAN_CASES[::2], ids=[str(c) for c in SCAN_CASES[::2]])
def test_overlap_search_equals_aho_corasick(mpm, native, case, kernel):
    sigma, m, q, sr, k, kind = case
    rng = np.random.default_rng(7 + sum(case))
    base = 65 if sigma <= 20 else 33
    n = (1 << 22) + 13
    T = (rng.integers(0, sigma, n) + base).astype(np.uint8)
    P = (rng.integers(0, sigma, (300, m)) + base).astype(np.uint8)
    for i in range(150):
        o = int(rng.integers(0, n - m + 1))
        P[i] = T[o:o + m]
    kw = dict(q=q, sigma_r=sr, k=k, map_kind=kind, overlap=1, kernel=kernel)
    M = mpm.Matcher(P, sigma=sigma, **kw)
    pos, pid = M.search(dev(T))
    want = native.aho_corasick(T, P, threads=8)
    assert np.array_equal(as_u32(pos), want[0]) and np.array_equal(as_u32(pid), want[1])
    # the pipelined call takes the same path
    status = torch.zeros(4, dtype=torch.int32, device="cuda")
    op = torch.empty(1 << 16, dtype=torch.int32, device="cuda")
    oi = torch.empty_like(op)
    M.search_async(dev(T), op, oi, status)
    M.sync()
    z = want[0].size
    if z <= 4096:
        assert list(status.cpu().numpy()[1:]) == [z, 0, 1]
        assert np.array_equal(as_u32(op)[:z], want[0])


def test_overlap_edges(mpm, native):
    rng = np.random.default_rng(99)
    P = (rng.integers(0, 4, (10, 9)) + 65).astype(np.uint8)
    for n in (0, 5, 8, 9, 10, 63, 64, 65, 1000, 4097):
        T = (rng.integers(0, 4, n) + 65).astype(np.uint8)
        if n >= 9:
            T[n - 9:] = P[3]
            T[:9] = P[0]
        for kw in (dict(q=9, sigma_r=4, k=1, map_kind=2),     # q = m: L' = 1
                   dict(q=2, sigma_r=4, k=8, map_kind=2),     # k = L'
                   dict(q=3, sigma_r=1 << 12, k=3, map_kind=4)):
            for kernel in (1, 2, 3):
                M = mpm.Matcher(P, sigma=4, overlap=1, kernel=kernel, **kw)
                pos, pid = M.search(T)   # host text and outputs
                want = native.aho_corasick(T, P)
                assert np.array_equal(pos, want[0]) and np.array_equal(pid, want[1]), \
                    (n, kw, kernel)


def test_overlap_rows_and_tail_edges(mpm, native):
    """Texts of a few specialised-kernel rows: occurrences planted at row and
    stage starts, across row boundaries and at both text ends, for filters
    whose first bytes come from 0, 1 and 2 words before a stage."""
    rng = np.random.default_rng(5)
    for q, k, m in ((1, 4, 12), (5, 2, 16), (8, 4, 16), (8, 3, 20)):
        P = (rng.integers(0, 4, (30, m)) + 65).astype(np.uint8)
        for n in (4 * 1024 * 1024 + 77, 2 * 1024 * 1024):
            T = (rng.integers(0, 4, n) + 65).astype(np.uint8)
            T[:m] = P[0]
            T[n - m:] = P[1]
            for at in list(range(80, n - m, n // 37))[:36]:
                # every place of a stage row: ends and middle
                for d in (-m // 2, 0, 3):
                    o = at + d
                    if 0 <= o <= n - m:
                        T[o:o + m] = P[int(rng.integers(0, 30))]
            want = native.aho_corasick(T, P, threads=8)
            for kernel in (2, 3):
                M = mpm.Matcher(P, sigma=4, q=q, sigma_r=4, k=k, map_kind=3, map_shift=1,
                                overlap=1, kernel=kernel)
                pos, pid = M.search(dev(T))
                assert np.array_equal(as_u32(pos), want[0]), (q, k, m, n, kernel)
                assert np.array_equal(as_u32(pid), want[1]), (q, k, m, n, kernel)
                # unaligned text: every byte through the plain-load path
                pos, pid = M.search(dev(np.concatenate([np.zeros(1, np.uint8), T]))[1:])
                assert np.array_equal(as_u32(pos), want[0]), (q, k, m, n, kernel, "unaligned")


def test_overlap_refused_where_unsupported(mpm):
    P = np.frombuffer(b"ACGTACGTACGTACGT", np.uint8).reshape(1, 16)
    for kw in (dict(smag=1),):
        with pytest.raises(mpm.MpmError) as e:
            mpm.Matcher(P, sigma=4, q=3, sigma_r=4, k=1, map_kind=2, overlap=1, **kw)
        assert e.value.code == mpm.MPM_ENOTSUP
    M = mpm.Matcher(P, sigma=4, q=3, sigma_r=4, k=1, map_kind=2, overlap=1)
    with pytest.raises(mpm.MpmError):
        mpm.Batch([M], [dev(np.zeros(100, np.uint8))], np.zeros(1, np.uint32))


def test_overlap_full_size_dna(mpm, native):
    """1 GiB uniform DNA, r = 100, m = 16 (config 1's patterns at scale):
    the generic kernel and the specialised one."""
    case = W.config1_scaled()
    T = dev(case.T)
    want = native.aho_corasick(case.T, case.P, threads=max(1, min(32, os.cpu_count() or 1)))
    for kw in (dict(q=8, k=1, kernel=1), dict(q=8, k=4, kernel=2), dict(q=8, k=2, kernel=3)):
        M = mpm.Matcher(case.P, sigma=4, sigma_r=4, map_kind=3, map_shift=1, overlap=1, **kw)
        pos, pid = M.search(T)
        assert np.array_equal(as_u32(pos), want[0]) and np.array_equal(as_u32(pid), want[1]), kw
        M.close()
