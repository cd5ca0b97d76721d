"""GPU parity of the batched search (mpm_batch_*): many texts of uneven
length, each against one of several pattern sets, in one persistent launch.
Every (text, position, pattern id) triple must equal the oracle's
(Aho-Corasick per text), for graph replays, plain launches and the one-shot
call, and when the occurrences outgrow the batch's first buffers."""
import ctypes
import math

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


def small_config4(ntexts=300, nsets=8, max_log2=18, seed=7):
    """A config-4-shaped batch at a size the oracle checks in seconds."""
    src = W.english_source()
    rng = np.random.default_rng(seed)
    lens = np.exp(rng.uniform(10 * math.log(2), max_log2 * math.log(2), ntexts)).astype(int)
    texts = [src.draw(int(L), rng) for L in lens]
    set_of_text = rng.integers(0, nsets, ntexts).astype(np.uint32)
    sets = []
    for s in range(nsets):
        r = int(round(math.exp(rng.uniform(math.log(10), math.log(2000)))))
        m = int(rng.choice([8, 16, 32, 64]))
        mine = np.flatnonzero(set_of_text == s)
        P = src.draw(r * m, rng).reshape(r, m)
        for i in range(r // 2):
            if mine.size == 0:
                break
            t = texts[int(mine[rng.integers(0, mine.size)])]
            if t.size >= m:
                o = int(rng.integers(0, t.size - m + 1))
                P[i] = t[o:o + m]
        sets.append(P)
    return texts, sets, set_of_text


def expected(native, texts, sets, set_of_text):
    acs = [native.AhoCorasick(P) for P in sets]
    out = []
    for t, T in enumerate(texts):
        pos, pid = acs[set_of_text[t]].search(T)
        out.append(np.stack([np.full(pos.size, t, np.uint32), pos, pid], axis=1))
    return np.concatenate(out) if out else np.zeros((0, 3), np.uint32)


def batch_matchers(mpm, sets):
    ms = []
    for P in sets:
        m = mpm.Matcher(P, sigma=95)
        info, p = m.info, m.params
        if info["positions"] > 32 or (p["map_kind"] == 4 and p["q"] > 5):
            m = mpm.Matcher(P, sigma=95, map_kind=2, k=max(1, p["k"]),
                            q=min(p["q"], 4), sigma_r=16)
        ms.append(m)
    return ms


def triples(tid, pos, pid):
    return np.stack([tid.cpu().numpy().view(np.uint32), pos.cpu().numpy().view(np.uint32),
                     pid.cpu().numpy().view(np.uint32)], axis=1)


@pytest.mark.parametrize("generic", [False, True], ids=["compiled", "precompiled"])
def test_batch_matches_oracle_graph_and_plain(mpm, native, generic):
    """The kernel compiled for the batch's parameter sets and the precompiled
    one with run-time parameters."""
    texts, sets, sot = small_config4()
    want = expected(native, texts, sets, sot)
    assert want.shape[0] > 1000
    dev = [torch.from_numpy(t).cuda() for t in texts]
    ms = batch_matchers(mpm, sets)
    for graph in (True, False):
        b = mpm.Batch(ms, dev, sot, graph=graph, generic=generic)
        assert (b.stats["variants"] == 0) == generic
        for _ in range(2):  # replays must not see the previous run
            got = triples(*b.run())
            assert np.array_equal(got, want)
        st = b.stats
        assert st["z"] == want.shape[0] and st["bytes"] == sum(t.size for t in texts)
        # the scan kernel's own time, from the events around it (graph nodes
        # when replayed from the graph), lies inside the whole run's
        assert 0.0 < st["scan_ms"] <= st["ms"]
        b.close()


def test_batch_small_lanes_and_one_shot_call(mpm, native):
    texts, sets, sot = small_config4(ntexts=120, nsets=5, max_log2=14, seed=11)
    want = expected(native, texts, sets, sot)
    dev = [torch.from_numpy(t).cuda() for t in texts]
    ms = batch_matchers(mpm, sets)
    for generic in (False, True):
        b = mpm.Batch(ms, dev, sot, lane_bytes=40, generic=generic)
        assert np.array_equal(triples(*b.run()), want)
        b.close()
    # unaligned texts: the compiled kernel's lanes fall back to byte loads
    unal = [torch.cat([torch.zeros(1, dtype=torch.uint8, device="cuda"), t])[1:] for t in dev]
    b = mpm.Batch(ms, unal, sot)
    assert b.stats["variants"] > 0
    assert np.array_equal(triples(*b.run()), want)
    b.close()
    # the one-shot C call, host outputs
    L = mpm.lib()
    n = len(dev)
    hs = (ctypes.c_void_p * len(ms))(*[m._h for m in ms])
    tp = (ctypes.c_void_p * n)(*[t.data_ptr() for t in dev])
    ln = (ctypes.c_size_t * n)(*[t.numel() for t in dev])
    st = (ctypes.c_uint32 * n)(*[int(s) for s in sot])
    cap = want.shape[0] + 10
    out = np.zeros((3, cap), np.uint32)
    z = ctypes.c_size_t(cap)
    rc = L.mpm_search_batch(hs, len(ms), tp, ln, st, n, out[0].ctypes.data, out[1].ctypes.data,
                            out[2].ctypes.data, ctypes.byref(z))
    assert rc == 0 and z.value == want.shape[0]
    assert np.array_equal(out[:, :z.value].T, want)


def test_batch_grows_when_occurrences_outgrow_its_buffers(mpm, native):
    # runs of one symbol: an occurrence at almost every position
    texts = [np.full(60_000 + 1000 * i, 65, np.uint8) for i in range(3)]
    texts[1][::997] = 66
    sets = [np.full((2, 8), 65, np.uint8), np.frombuffer(b"ABABABAB", np.uint8).reshape(1, 8)]
    sot = np.array([0, 0, 1], np.uint32)
    want = expected(native, texts, sets, sot)
    assert want.shape[0] > (1 << 16)
    dev = [torch.from_numpy(t).cuda() for t in texts]
    ms = [mpm.Matcher(P, sigma=2) for P in sets]
    b = mpm.Batch(ms, dev, sot)
    assert np.array_equal(triples(*b.run()), want)
    assert np.array_equal(triples(*b.run()), want)


def test_config4_full_shape_learned_parameters_equal_oracle(mpm, native):
    """The benchmarked batch exactly as the benchmark builds it: 4096 texts of
    1 KiB - 4 MiB against 64 pattern sets (r up to 10^4), each set's
    parameters proposed by the committed cost model among mask tables that fit
    the batched kernel's shared memory; every (text, pos, pid) triple equals
    Aho-Corasick per text."""
    from concurrent.futures import ThreadPoolExecutor

    from paper_1405_5483_gb300 import _native
    from paper_1405_5483_gb300 import cost_model as CM
    b = W.config4()
    model = CM.Model.load()
    params = CM.learned_batch_params(b, model, _native.BATCH_SMEM_TABLE_BYTES)
    ms = [CM.batch_matcher(P, b.sigma, p) for P, p in zip(b.sets, params)]
    assert max(P.shape[0] for P in b.sets) > 5000 and max(t.size for t in b.texts) > 1 << 21
    # the texts in one buffer at 256-byte offsets, as the benchmark lays them out
    offs = np.zeros(len(b.texts) + 1, np.int64)
    for i, t in enumerate(b.texts):
        offs[i + 1] = (offs[i] + t.size + 255) & ~255
    flat = torch.zeros(int(offs[-1]), dtype=torch.uint8, device="cuda")
    dev = []
    for i, t in enumerate(b.texts):
        flat[int(offs[i]): int(offs[i]) + t.size] = torch.from_numpy(t).cuda()
        dev.append(flat[int(offs[i]): int(offs[i]) + t.size])
    B = mpm.Batch(ms, dev, b.set_of_text)
    assert B.stats["variants"] > 0
    got = triples(*B.run())
    B.close()

    acs = [native.AhoCorasick(P) for P in b.sets]

    def one(t):
        pos, pid = acs[b.set_of_text[t]].search(b.texts[t])
        return np.stack([np.full(pos.size, t, np.uint32), pos, pid], axis=1)

    with ThreadPoolExecutor(max_workers=16) as ex:
        parts = list(ex.map(one, range(len(b.texts))))
    for ac in acs:
        ac.close()
    want = np.concatenate(parts)
    assert want.shape[0] > 10_000
    assert got.shape == want.shape
    assert np.array_equal(got, want)
