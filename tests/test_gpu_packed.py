"""GPU parity of packed mask tables: filters of at most 4 positions whose
table is too large for shared memory keep 8, 4 or 2 entries per byte, read
by the specialised kernels (both variants) from shared memory when the packed
table fits there and from L2 otherwise.  Candidate windows equal the oracle's
scan; searches equal Aho-Corasick, aligned and unaligned."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

from oracle import filter as F  # noqa: E402
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


# (m, params, bits): one position (shared-memory and global packed tables),
# two positions, four positions (overlapping q-grams)
CASES = [
    (20, dict(q=9, sigma_r=4, k=1, map_kind=3, map_shift=1), 1),
    (24, dict(q=11, sigma_r=4, k=1, map_kind=3, map_shift=1), 1),
    (27, dict(q=9, sigma_r=4, k=1, map_kind=3, map_shift=1), 2),
    (12, dict(q=9, sigma_r=4, k=1, map_kind=3, map_shift=1, overlap=1), 4),
]


def _text(rng, n, P):
    T = W.dna_source().draw(n, rng)
    for i in range(P.shape[0] // 2):
        o = int(rng.integers(0, n - P.shape[1] + 1))
        T[o:o + P.shape[1]] = P[i]
    return T


@pytest.mark.parametrize("case", CASES, ids=[str(c[2]) + "-" + str(c[0]) for c in CASES])
def test_packed_candidates_equal_oracle(mpm, case):
    m, kw, bits = case
    c = W.dna_case(1 << 12, 200, m, 100, cfg=40 + m)
    rng = np.random.default_rng(m)
    T = _text(rng, 300_007, c.P)
    M = mpm.Matcher(c.P, sigma=4, kernel=3, **kw)
    info, p = M.info, M.params
    assert info["entry_bits"] == bits
    got = windows_of(M.scan(dev(T)), p["k"], info["mprime"])
    assert M.stats["specialised"] == 1
    fp = F.make_params(c.P, p["q"], p["sigma_r"], p["k"], "lowbits", shift=p["map_shift"],
                       overlap=bool(p["overlap"]))
    cls = F.pattern_classes(c.P, fp)
    want = F.aoso_scan(F.text_codes(T, fp), F.mask_table(cls, fp), fp, len(cls))
    assert np.array_equal(got, np.array(want, np.int64))


@pytest.mark.parametrize("kernel", [2, 3], ids=["verifying", "split"])
@pytest.mark.parametrize("case", CASES, ids=[str(c[2]) + "-" + str(c[0]) for c in CASES])
def test_packed_search_equals_aho_corasick(mpm, native, case, kernel):
    m, kw, bits = case
    c = W.dna_case(1 << 12, 300, m, 150, cfg=50 + m)
    rng = np.random.default_rng(7 * m)
    T = _text(rng, (1 << 22) + 9, c.P)
    want = native.aho_corasick(T, c.P, threads=8)
    assert want[0].size >= 150
    M = mpm.Matcher(c.P, sigma=4, kernel=kernel, **kw)
    assert M.info["entry_bits"] == bits
    for Td in (dev(T), dev(np.concatenate([np.zeros(5, np.uint8), T]))[5:]):
        pos, pid = M.search(Td)
        assert np.array_equal(as_u32(pos), want[0]) and np.array_equal(as_u32(pid), want[1])
    # the generic kernel builds the same filter with whole-byte entries
    G = mpm.Matcher(c.P, sigma=4, kernel=1, **kw)
    assert G.info["entry_bits"] == 8
    pos, pid = G.search(dev(T))
    assert np.array_equal(as_u32(pos), want[0]) and np.array_equal(as_u32(pid), want[1])


def test_packed_large_set(mpm, native):
    """r = 100 000, m = 32 (the large-set configuration's patterns) on 64 MiB
    of its text: the planner's filter (one position, q = 14 on 2-bit codes), a
    packed table of one bit per entry (32 MiB) read from L2, both variants and
    the pipelined call."""
    c = W.config3(n=1 << 26)
    M = mpm.Matcher(c.P, sigma=4)
    q = M.params["q"]
    assert M.info["positions"] == 1 and M.info["entry_bits"] == 1
    assert M.info["table_bytes"] == (1 << (2 * q)) // 8 and M.info["table_bytes"] > 227 << 10
    want = native.aho_corasick(c.T, c.P, threads=16)
    T = dev(c.T)
    for kernel in (2, 3):
        M = mpm.Matcher(c.P, sigma=4, kernel=kernel, **{k: M.params[k] for k in (
            "q", "sigma_r", "k", "map_kind", "map_shift")})
        pos, pid = M.search(T)
        assert np.array_equal(as_u32(pos), want[0]) and np.array_equal(as_u32(pid), want[1])
    status = torch.zeros(4, dtype=torch.int32, device="cuda")
    op = torch.empty(1 << 17, dtype=torch.int32, device="cuda")
    oi = torch.empty_like(op)
    M.search_async(T, op, oi, status)
    M.sync()
    z = want[0].size
    assert list(status.cpu().numpy()[1:]) == [z, 0, 1]
    assert np.array_equal(as_u32(op)[:z], want[0]) and np.array_equal(as_u32(oi)[:z], want[1])
