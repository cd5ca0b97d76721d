"""GPU parity of Shift-Or state of several 64-bit words (`wide` = 1..3,
Section 3.2's ceil((m/q)/w) words): filters of 65 to 256 positions in the
generic kernels and both variants of the specialised one, candidate windows
equal to the oracle's scan and searches equal to Aho-Corasick."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

from oracle import filter as F  # noqa: E402


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


def long_case(rng, n, r, m, sigma=4):
    T = (rng.integers(0, sigma, n) + 65).astype(np.uint8)
    P = (rng.integers(0, sigma, (r, m)) + 65).astype(np.uint8)
    for i in range(r // 2):
        o = int(rng.integers(0, n - m + 1))
        P[i] = T[o:o + m]
    # near-misses: planted copies with one byte changed late in the pattern
    for i in range(r // 2, r - 1):
        o = int(rng.integers(0, n - m + 1))
        P[i] = T[o:o + m]
        P[i, m - 3] = 65 + (P[i, m - 3] - 64) % sigma
    return T, P


CASES = [  # (m, q, k, overlap, map_kind, sigma_r, wide)
    (100, 1, 1, 0, 2, 4, 1),
    (150, 1, 2, 0, 2, 4, 1),
    (200, 2, 1, 0, 3, 4, 1),
    (260, 2, 2, 0, 2, 4, 1),
    (100, 2, 1, 1, 2, 4, 1),
    (140, 3, 1, 1, 4, 1 << 12, 1),
    (180, 1, 1, 0, 2, 4, 2),        # 180 positions: 3 words
    (300, 1, 3, 0, 3, 4, 3),        # 255 positions: 4 words
    (260, 2, 1, 1, 3, 4, 3),        # overlapping, 256 positions
    (220, 3, 2, 1, 4, 1 << 12, 2),  # q-gram hashing, 3 words
]
KERNELS = [1, 3]  # generic, specialised (candidate records)


@pytest.mark.parametrize("kernel", KERNELS, ids=["generic", "specialised"])
@pytest.mark.parametrize("case", CASES, ids=[str(c) for c in CASES])
def test_wide_candidates_equal_oracle(mpm, case, kernel):
    m, q, k, overlap, kind, sr, wide = case
    rng = np.random.default_rng(m + q + k)
    T, P = long_case(rng, 200_001, 12, m)
    kw = dict(q=q, sigma_r=sr, k=k, map_kind=kind, overlap=overlap, wide=wide, kernel=kernel)
    if kind == 3:
        kw["map_shift"] = 1
    M = mpm.Matcher(P, sigma=4, **kw)
    p, info = M.params, M.info
    assert p["wide"] == wide and info["positions"] > 64 * wide
    got = windows_of(M.scan(dev(T)), k, info["mprime"])
    assert M.stats["specialised"] == (1 if kernel != 1 else 0)
    names = {2: "greedy", 3: "lowbits", 4: "qhash"}
    fp = F.make_params(P, q, sr, k, names[kind], shift=p["map_shift"], overlap=bool(overlap),
                       max_positions=64 * (wide + 1))
    cls = F.pattern_classes(P, fp)
    want = F.aoso_scan(F.text_codes(T, fp), F.mask_table(cls, fp), fp, len(cls))
    assert np.array_equal(got, np.array(want, np.int64))
    # the wider filter is at least as selective as 64 positions
    M64 = mpm.Matcher(P, sigma=4, **dict(kw, wide=0, kernel=1))
    got64 = windows_of(M64.scan(dev(T)), k, M64.info["mprime"])
    assert set(got.tolist()) <= set(got64.tolist())


@pytest.mark.parametrize("kernel", [1, 2, 3], ids=["generic", "verifying", "split"])
@pytest.mark.parametrize("case", CASES[::2], ids=[str(c) for c in CASES[::2]])
def test_wide_search_equals_aho_corasick(mpm, native, case, kernel):
    m, q, k, overlap, kind, sr, wide = case
    rng = np.random.default_rng(7 * m + q)
    T, P = long_case(rng, (1 << 22) + 5, 60, m)
    kw = dict(q=q, sigma_r=sr, k=k, map_kind=kind, overlap=overlap, wide=wide, kernel=kernel)
    if kind == 3:
        kw["map_shift"] = 1
    M = mpm.Matcher(P, sigma=4, **kw)
    pos, pid = M.search(dev(T))
    want = native.aho_corasick(T, P, threads=8)
    assert want[0].size >= 30
    assert np.array_equal(as_u32(pos), want[0]) and np.array_equal(as_u32(pid), want[1])
    # unaligned text: every byte through the plain-load path
    pos, pid = M.search(dev(np.concatenate([np.zeros(3, np.uint8), T]))[3:])
    assert np.array_equal(as_u32(pos), want[0]) and np.array_equal(as_u32(pid), want[1])


def test_wide_refused_where_unsupported(mpm):
    P = (np.arange(200) % 4 + 65).astype(np.uint8).reshape(1, 200)
    with pytest.raises(mpm.MpmError) as e:
        mpm.Matcher(P, sigma=4, q=1, sigma_r=4, k=1, map_kind=2, wide=1, smag=1)
    assert e.value.code == mpm.MPM_ENOTSUP
