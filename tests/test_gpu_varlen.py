"""GPU parity for patterns of different lengths (mpm_build_var): the filter
runs on every pattern's first m_min bytes and each candidate window is
verified against each pattern's own length; the occurrence lists equal the
oracle's Aho-Corasick over the same variable-length set."""
import ctypes
import os

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


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def as_u32(t):
    return t.cpu().numpy().view(np.uint32)


def var_set(rng, T, r, lo, hi, planted, src):
    """r patterns with lengths uniform in [lo, hi]; the first `planted` are
    substrings of T, some of them prefixes or extensions of one another."""
    P = []
    for i in range(r):
        L = int(rng.integers(lo, hi + 1))
        if i < planted:
            o = int(rng.integers(0, T.size - L + 1))
            P.append(T[o:o + L].tobytes())
        else:
            P.append(src.draw(L, rng).tobytes())
    # a short pattern that is a prefix of a longer planted one, and a duplicate
    P.append(P[0][:lo])
    P.append(P[1])
    return P


@pytest.mark.parametrize("kernel", [1, 2, 3])
@pytest.mark.parametrize("lo,hi,params", [
    (8, 24, dict(q=3, sigma_r=8, k=1, map_kind=2)),
    (16, 64, dict(q=4, sigma_r=1 << 12, k=2, map_kind=4)),
    (32, 40, {}),
])
def test_variable_lengths_equal_aho_corasick(mpm, native, kernel, lo, hi, params):
    rng = np.random.default_rng(lo + hi + kernel)
    src = W.protein_source()
    T = src.draw((1 << 21) + 17, rng)
    P = var_set(rng, T, 400, lo, hi, 200, src)
    M = mpm.Matcher(P, sigma=20, kernel=kernel, **params)
    assert M.m == min(len(p) for p in P)
    pos, pid = M.search(dev(T))
    want = native.AhoCorasick(P).search(T, threads=8)
    assert want[0].size >= 200
    assert np.array_equal(as_u32(pos), want[0]) and np.array_equal(as_u32(pid), want[1])
    # host text and outputs, and the pipelined call
    hp, hi_ = M.search(T)
    assert np.array_equal(hp, want[0]) and np.array_equal(hi_, want[1])
    status = torch.zeros(4, dtype=torch.int32, device="cuda")
    op = torch.empty(8192, dtype=torch.int32, device="cuda")
    oi = torch.empty_like(op)
    M.search_async(dev(T), op, oi, status)
    M.sync()
    z = want[0].size
    if z <= 4096:
        assert list(status.cpu().numpy()[1:]) == [z, 0, 1]
        assert np.array_equal(as_u32(op)[:z], want[0]) and np.array_equal(as_u32(oi)[:z], want[1])


def test_variable_lengths_at_the_end_of_the_text(mpm, native):
    # patterns that would run past the end are not reported; those that end
    # exactly there are
    T = np.frombuffer(b"xxabcdefgh", np.uint8)
    P = [b"abcdefgh", b"abcdefghij", b"efgh", b"ghij", b"ab", b"gh"]
    for kw in (dict(kernel=1), dict(kernel=2), {}):
        M = mpm.Matcher(P, sigma=256, **kw)
        pos, pid = M.search(T)
        want = native.AhoCorasick(P).search(T)
        assert np.array_equal(pos, want[0]) and np.array_equal(pid, want[1])
        assert set(zip(pos.tolist(), pid.tolist())) == {(2, 0), (6, 2), (2, 4), (8, 5)}


def test_variable_lengths_in_a_batch(mpm, native):
    rng = np.random.default_rng(5)
    src = W.english_source()
    texts = [src.draw(int(n), rng) for n in rng.integers(1000, 200_000, 40)]
    P1 = var_set(rng, texts[0], 50, 8, 20, 25, src)
    P2 = [bytes(p) for p in src.draw(30 * 16, rng).reshape(30, 16)]
    sot = rng.integers(0, 2, len(texts)).astype(np.uint32)
    ms = [mpm.Matcher(P1, sigma=95, q=3, sigma_r=16, k=1, map_kind=2),
          mpm.Matcher(P2, sigma=95)]
    b = mpm.Batch(ms, [dev(t) for t in texts], sot)
    tid, pos, pid = b.run()
    got = np.stack([as_u32(tid), as_u32(pos), as_u32(pid)], axis=1)
    want = []
    acs = [native.AhoCorasick(P1), native.AhoCorasick(P2)]
    for t, T in enumerate(texts):
        p, i = acs[sot[t]].search(T)
        want.append(np.stack([np.full(p.size, t, np.uint32), p, i], axis=1))
    want = np.concatenate(want)
    assert np.array_equal(got, want)


def test_bad_offsets_are_rejected(mpm):
    L = mpm.lib()
    P = np.frombuffer(b"abcdef", np.uint8)
    for offs in ([1, 3, 6], [0, 3, 3], [0, 4, 2]):
        off = (ctypes.c_size_t * 3)(*offs)
        assert not L.mpm_build_var(P.ctypes.data, off, 2, 256, None)
        assert L.mpm_last_error() == mpm.MPM_EINVAL


def test_variable_lengths_full_size_protein(mpm, native):
    """The 256 MiB protein text with 1000 patterns of lengths 16 .. 64."""
    case = W.config2()
    rng = np.random.default_rng(2002)
    P = var_set(rng, case.T, 1000, 16, 64, 500, case.source)
    M = mpm.Matcher(P, sigma=20)
    pos, pid = M.search(dev(case.T))
    want = native.AhoCorasick(P).search(case.T, threads=max(1, min(32, os.cpu_count() or 1)))
    assert np.array_equal(as_u32(pos), want[0]) and np.array_equal(as_u32(pid), want[1])
