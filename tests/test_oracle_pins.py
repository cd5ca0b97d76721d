"""Pins of the oracle to the paper and to mathematics (CPU only).

Each test ties a part of oracle/ to something other than itself: a value the
paper prints (tests/golden/), a closed form, a textbook special case, brute
force on tiny inputs, or an invariant.  A dropped term, a wrong shift count,
a transposed digit order or a wrong AOSO bit would fail at least one.
"""
import itertools
import json
import os
import random

import numpy as np
import pytest

from oracle import brute
from oracle import filter as F

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def _strs(qpattern):
    return ["".join(g) for g in qpattern]


# -------------------------------------------------- Section 2 worked examples

def test_superimposition_worked_example():
    g = _golden("section2_examples.json")
    P = [list(p) for p in g["patterns"]]
    cls = F.superimpose(P)
    assert [sorted(c) for c in cls] == [sorted(c) for c in g["superimposed_q1"]]
    # brute-force count of length-4 strings over the whole lowercase alphabet
    # that the superimposed pattern accepts
    letters = "abcdefghijklmnopqrstuvwxyz"
    accepted = sum(all(s[j] in cls[j] for j in range(4))
                   for s in itertools.product(letters, repeat=4))
    assert accepted == g["strings_accepted_by_filter"]


def test_overlapping_qgrams_worked_example():
    g = _golden("section2_examples.json")
    qp = F.overlapping_qgram_patterns([list(p) for p in g["patterns"]], 2)
    assert [_strs(x) for x in qp] == g["overlapping_q2_patterns"]
    sup = F.superimpose(qp)
    assert [sorted("".join(t) for t in c) for c in sup] == \
        [sorted(c) for c in g["overlapping_q2_superimposed"]]


def test_nonoverlapping_qgrams_worked_example():
    g = _golden("section2_examples.json")
    qp = F.nonoverlapping_qgram_patterns([list(p) for p in g["patterns"]], 2, shifts=False)
    sup = F.superimpose(qp)
    assert [sorted("".join(t) for t in c) for c in sup] == \
        [sorted(c) for c in g["nonoverlapping_q2_superimposed_without_shifts"]]


def test_nonoverlapping_all_q_shifts():
    # every shift s = 0..q-1, cut to L' = floor((m-q+1)/q) q-grams
    qp = F.nonoverlapping_qgram_patterns([list("abba"), list("bbac")], 2, shifts=True)
    assert [_strs(x) for x in qp] == [["ab"], ["bb"], ["bb"], ["ba"]]
    qp3 = F.nonoverlapping_qgram_patterns([list("abcdefgh")], 3, shifts=True)
    # L' = floor(6/3) = 2 for every shift
    assert [_strs(x) for x in qp3] == [["abc", "def"], ["bcd", "efg"], ["cde", "fgh"]]


# ---------------------------------------- Section 2 illustration, closed forms

def _mc_class_sizes(sigma, r, m, sets, rng):
    sizes = []
    for _ in range(sets):
        P = rng.integers(0, sigma, size=(r, m))
        sizes += [len(c) for c in F.superimpose([list(p) for p in P])]
    return np.array(sizes, dtype=float)


@pytest.mark.parametrize("row", [0, 1])
def test_class_size_and_match_probability_q1(row):
    g = _golden("section2_false_positive_rates.json")
    sigma = g["sigma"]
    ref = g["q1"][row]
    closed = F.expected_class_size(sigma, ref["r"])
    # the closed form reproduces the printed figures
    assert abs(closed - ref["expected_class_size"]) < 0.06
    assert abs(closed / sigma - ref["match_probability"]) < 0.006
    # and the oracle's superimposition reproduces the closed form
    sizes = _mc_class_sizes(sigma, ref["r"], 8, 600, np.random.default_rng(7 + row))
    se = sizes.std() / np.sqrt(sizes.size)
    assert abs(sizes.mean() - closed) < 4 * se + 1e-9


@pytest.mark.parametrize("row", [0, 1])
def test_match_probability_q2(row):
    g = _golden("section2_false_positive_rates.json")
    sigma = g["sigma"]
    ref = g["q2"][row]
    r = ref["r"]
    closed = 1.0 - (1.0 - 1.0 / sigma ** 2) ** r
    assert abs(closed - ref["match_probability"]) < 0.006
    # overlapping 2-grams of random patterns: one q-gram per pattern and position
    rng = np.random.default_rng(11 + row)
    fr = []
    for _ in range(300):
        P = rng.integers(0, sigma, size=(r, 6))
        sup = F.superimpose(F.overlapping_qgram_patterns([list(p) for p in P], 2))
        fr += [len(c) / sigma ** 2 for c in sup]
    fr = np.array(fr)
    assert abs(fr.mean() - closed) < 4 * fr.std() / np.sqrt(fr.size) + 1e-9


def test_shifted_classes_follow_section32_probability():
    # Section 3.2: with all q shifts superimposed a class holds q*r q-grams, so
    # a random q-gram falls in it with p = 1 - (1 - sigma^-q)^(q r).  Dropping a
    # shift (the garbled printed list has q-1) would give exponent (q-1) r.
    sigma, q, r, m = 16, 2, 16, 9
    rng = np.random.default_rng(3)
    fp = F.FilterParams(q, sigma, 1, F.map_lowbits(sigma, 0), "lsd")
    fr = []
    for _ in range(300):
        P = rng.integers(0, sigma, size=(r, m)).astype(np.uint8)
        fr += [len(c) / sigma ** q for c in F.pattern_classes(P, fp)]
    fr = np.array(fr)
    p_all = 1 - (1 - sigma ** -q) ** (q * r)
    p_missing = 1 - (1 - sigma ** -q) ** ((q - 1) * r)
    assert abs(fr.mean() - p_all) < 0.004
    assert abs(fr.mean() - p_missing) > 0.04


# ---------------------------------------------- Section 3.2 q-gram numbering

@pytest.mark.parametrize("order", ["lsd", "msd"])
@pytest.mark.parametrize("sigma_r,q", [(2, 5), (4, 3), (5, 2), (16, 2)])
def test_qgram_code_is_a_bijection(order, sigma_r, q):
    codes = sorted(F.qgram_code(s, sigma_r, order)
                   for s in itertools.product(range(sigma_r), repeat=q))
    assert codes == list(range(sigma_r ** q))


def test_qgram_code_digit_orders():
    # Section 3.2: S[1] carries weight sigma^0; the multiply trick of Section
    # 3.3 puts S[1] in the most significant digit.
    assert F.qgram_code([1, 0, 0], 4, "lsd") == 1
    assert F.qgram_code([1, 0, 0], 4, "msd") == 16
    assert F.qgram_code([3, 2, 1], 10, "lsd") == 123
    assert F.qgram_code([3, 2, 1], 10, "msd") == 321


# ------------------------------------------------ Section 3.3 multiply trick

def _word(s):
    return int.from_bytes(s.encode("ascii"), "little")


def test_multiply_trick_dna_example():
    mu = F.map_lowbits(4, shift=1)
    # A, C, G, T get four distinct 2-bit codes, lower case the same
    assert [int(mu[ord(c)]) for c in "ACGT"] == [0, 1, 3, 2]
    assert [int(mu[ord(c)]) for c in "acgt"] == [0, 1, 3, 2]
    assert F.multiply_trick(_word("ACGT")) == 0 * 64 + 1 * 16 + 3 * 4 + 2
    assert F.multiply_trick(_word("acgt")) == F.multiply_trick(_word("ACGT"))


def test_multiply_trick_equals_msd_code_for_every_masked_input():
    # after masking only the four 2-bit fields matter: check all 256 of them,
    # each with random bits in the positions the mask removes
    rng = random.Random(5)
    mu = F.map_lowbits(4, shift=1)
    for fields in itertools.product(range(4), repeat=4):
        for _ in range(16):
            bs = [(f << 1) | (rng.randrange(128) << 3) | rng.randrange(2) for f in fields]
            bs = [b & 0xFF for b in bs]
            x = int.from_bytes(bytes(bs), "little")
            want = F.qgram_code([int(mu[b]) for b in bs], 4, "msd")
            assert F.multiply_trick(x) == want


# ------------------------------------------------- Section 3.3 the mappings

def test_rank_map_hand_example():
    P = np.frombuffer(b"aaab" b"bbcd" b"eeee", np.uint8).reshape(3, 4)
    # counts: a3 b3 c1 d1 e4 -> order e, a, b, c, d (ties by byte value)
    mu = F.map_rank(P, 4)
    assert [int(mu[ord(c)]) for c in "eabcd"] == [0, 1, 2, 3, 3]
    assert int(mu[ord("z")]) == 3 and int(mu[0]) == 3
    mu2 = F.map_rank(P, 2)
    assert [int(mu2[ord(c)]) for c in "eabcd"] == [0, 1, 1, 1, 1]


def test_greedy_map_hand_example():
    P = np.frombuffer(b"aaaaaaab" b"bbbbbccd", np.uint8).reshape(2, 8)
    # counts a7 b6 c2 d1: a->0, b->1, c->1 (lighter), d->1 (7 vs 8 -> bin 0)
    mu = F.map_greedy(P, 2)
    assert [int(mu[ord(c)]) for c in "abcd"] == [0, 1, 1, 0]
    assert int(mu[ord("z")]) == 1


def test_greedy_map_is_near_equal_weight():
    # Section 3.3 asks for (approximately) equal bin weights; the greedy
    # heuristic must stay within the longest-processing-time bound of the
    # exhaustive optimum: max load <= (4/3 - 1/(3 s)) * OPT.
    rng = np.random.default_rng(1)
    for _ in range(60):
        nsym = int(rng.integers(3, 8))
        s = int(rng.choice([2, 4]))
        counts = rng.integers(1, 50, size=nsym)
        P = np.repeat(np.arange(nsym, dtype=np.uint8) + 65, counts)[None, :]
        mu = F.map_greedy(P, s)
        loads = np.zeros(s)
        for c, w in zip(range(nsym), counts):
            loads[mu[65 + c]] += w
        opt = min(max(np.bincount(a, weights=counts, minlength=s))
                  for a in itertools.product(range(s), repeat=nsym))
        assert loads.max() <= (4 / 3 - 1 / (3 * s)) * opt + 1e-9


# ---------------------------------------------- Sections 3.1, 3.2: the filter

def _rand_case(rng, sigma, n, r, m, planted):
    T = rng.integers(0, sigma, size=n).astype(np.uint8) + 97
    P = rng.integers(0, sigma, size=(r, m)).astype(np.uint8) + 97
    for i in range(min(planted, r)):
        if n >= m:
            o = int(rng.integers(0, n - m + 1))
            P[i] = T[o:o + m]
    return T, P


def test_aoso_is_textbook_shift_or_for_one_pattern():
    # r = 1, q = 1, k = 1 and an injective mapping: the superimposed pattern is
    # the pattern itself and the scan is plain Shift-Or (Section 1.1), an exact
    # matcher; its windows must be exactly the occurrences.
    rng = np.random.default_rng(2)
    for _ in range(300):
        m = int(rng.integers(1, 12))
        T, P = _rand_case(rng, int(rng.integers(1, 4)), int(rng.integers(0, 80)), 1, m, 1)
        fp = F.make_params(P, 1, 256, 1, "rank")
        cls = F.pattern_classes(P, fp)
        wins = F.aoso_scan(F.text_codes(T, fp), F.mask_table(cls, fp), fp, len(cls))
        occ = [i for i, _ in brute.occurrences(T.tobytes(), [P[0].tobytes()])]
        assert wins == occ


def _feasible(m, q):
    return (m - q + 1) // q >= 1


def test_aoso_scan_equals_candidate_definition_and_has_no_false_negatives():
    rng = np.random.default_rng(4)
    checked = 0
    while checked < 400:
        sigma = int(rng.integers(1, 5))
        m = int(rng.integers(2, 14))
        q = int(rng.integers(1, 4))
        if not _feasible(m, q):
            continue
        Lc = (m - q + 1) // q
        k = int(rng.integers(1, Lc + 1))
        kind = ["rank", "greedy", "lowbits"][int(rng.integers(0, 3))]
        sr = [2, 4, 8][int(rng.integers(0, 3))]
        order = ["lsd", "msd"][int(rng.integers(0, 2))]
        n = int(rng.integers(0, 90))
        r = int(rng.integers(1, 6))
        T, P = _rand_case(rng, sigma, n, r, m, int(rng.integers(0, r + 1)))
        fp = F.make_params(P, q, sr, k, kind, shift=0, order=order)
        cls = F.pattern_classes(P, fp)
        codes = F.text_codes(T, fp)
        wins = F.aoso_scan(codes, F.mask_table(cls, fp), fp, len(cls))
        assert wins == F.candidate_windows_by_definition(codes, cls, fp)
        occ = brute.occurrences(T.tobytes(), [p.tobytes() for p in P])
        wset = set(wins)
        for i, _ in occ:
            s = (-i) % q
            assert (i + s) // q in wset, "false negative"
        assert F.verify(T, P, wins, q) == occ
        assert F.search(T, P, fp) == occ
        checked += 1


def test_candidate_set_independent_of_digit_order_and_k1_is_superset():
    rng = np.random.default_rng(8)
    for _ in range(100):
        T, P = _rand_case(rng, 3, 120, 4, 10, 2)
        base = None
        for order in ("lsd", "msd"):
            fp = F.make_params(P, 2, 4, 2, "greedy", order=order)
            cls = F.pattern_classes(P, fp)
            w = F.aoso_scan(F.text_codes(T, fp), F.mask_table(cls, fp), fp, len(cls))
            base = w if base is None else base
            assert w == base


# --------------------------------------- the exact result, three ways agree

def test_brute_naive_aho_corasick_agree(oracle_native):
    rng = np.random.default_rng(9)
    for it in range(1500):
        sigma = int(rng.integers(1, 4))
        m = int(rng.integers(1, 7))
        n = int(rng.integers(0, 40))
        r = int(rng.integers(1, 6))
        T, P = _rand_case(rng, sigma, n, r, m, int(rng.integers(0, r + 1)))
        if it % 7 == 0 and r > 1:
            P[r - 1] = P[0]  # duplicate patterns are each reported
        want = brute.occurrences(T.tobytes(), [p.tobytes() for p in P])
        for pos, pid in (oracle_native.naive(T, P),
                         oracle_native.aho_corasick(T, P, threads=1),
                         oracle_native.aho_corasick(T, P, threads=3)):
            assert list(zip(pos.tolist(), pid.tolist())) == want


def test_aho_corasick_threaded_matches_single_thread_on_planted_text(oracle_native):
    rng = np.random.default_rng(10)
    T = rng.integers(0, 4, size=200_000).astype(np.uint8)
    P = rng.integers(0, 4, size=(300, 12)).astype(np.uint8)
    offs = rng.integers(0, T.size - 12, size=150)
    for i, o in enumerate(offs):
        P[i] = T[o:o + 12]
    ac = oracle_native.AhoCorasick(P)
    a = ac.search(T, threads=1)
    b = ac.search(T, threads=8)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    got = set(zip(a[0].tolist(), a[1].tolist()))
    for i, o in enumerate(offs):
        assert (int(o), i) in got  # planted occurrences are found
    pos, pid = oracle_native.naive(T[:20000], P)
    c = ac.search(T[:20000])
    assert np.array_equal(pos, c[0]) and np.array_equal(pid, c[1])


# --------------------------------------- Section 3.3, mapping whole q-grams

def test_qgram_hash_bins_are_an_invertible_map_at_full_width():
    # with as many bins as raw values the multiplicative map must lose
    # nothing: multiplication by an odd constant is invertible mod 2^32 and
    # mod 2^64, so every raw q-gram gets its own bin and the raw bytes come
    # back by multiplying with the inverse
    rng = random.Random(12)
    inv32 = pow(0x9E3779B1, -1, 1 << 32)
    inv64 = pow(0x9E3779B97F4A7C15, -1, 1 << 64)
    for q in (1, 2, 3, 4):
        for _ in range(200):
            raw = bytes(rng.randrange(256) for _ in range(q))
            h = F.qgram_hash(raw, 32)
            assert (h * inv32) % (1 << 32) == int.from_bytes(raw, "little")
    for q in (5, 8):
        for _ in range(200):
            raw = bytes(rng.randrange(256) for _ in range(q))
            h = F.qgram_hash(raw, 32)  # top 32 of 64 bits: check the full product instead
            full = (int.from_bytes(raw, "little") * 0x9E3779B97F4A7C15) % (1 << 64)
            assert full >> 32 == h and (full * inv64) % (1 << 64) == int.from_bytes(raw, "little")


def test_qgram_hash_spreads_bins_uniformly():
    # 20 000 distinct 4-grams over a 20-letter alphabet into 2^10 bins: the
    # bin counts must look uniform (chi-square within 5 sigma of its mean)
    rng = np.random.default_rng(3)
    letters = np.frombuffer(b"ACDEFGHIKLMNPQRSTVWY", np.uint8)
    grams = {bytes(letters[rng.integers(0, 20, 4)]) for _ in range(40000)}
    grams = list(grams)[:20000]
    counts = np.bincount([F.qgram_hash(g, 10) for g in grams], minlength=1024)
    e = len(grams) / 1024
    chi2 = ((counts - e) ** 2 / e).sum()
    assert abs(chi2 - 1023) < 5 * np.sqrt(2 * 1023)


def test_qhash_filter_equals_definition_and_search_is_exact():
    rng = np.random.default_rng(13)
    for _ in range(150):
        m = int(rng.integers(2, 20))
        q = int(rng.integers(1, 9))
        if (m - q + 1) // q < 1:
            continue
        Lc = (m - q + 1) // q
        k = int(rng.integers(1, min(Lc, 4) + 1))
        T, P = _rand_case(rng, int(rng.integers(1, 5)), int(rng.integers(0, 200)),
                          int(rng.integers(1, 6)), m, 2)
        fp = F.make_params(P, q, int(rng.choice([2, 16, 256, 4096])), k, "qhash")
        cls = F.pattern_classes(P, fp)
        codes = F.text_codes(T, fp)
        wins = F.aoso_scan(codes, F.mask_table(cls, fp), fp, len(cls))
        assert wins == F.candidate_windows_by_definition(codes, cls, fp)
        assert F.search(T, P, fp) == brute.occurrences(T.tobytes(), [p.tobytes() for p in P])


# ------------------------------------------------ overlapping q-grams (Section 2)

def _overlap_case(rng, sigma, n, r, m, planted):
    T = rng.integers(0, sigma, n).astype(np.uint8) + 97
    P = rng.integers(0, sigma, (r, m)).astype(np.uint8) + 97
    for i in range(min(planted, r)):
        o = int(rng.integers(0, n - m + 1))
        P[i] = T[o:o + m]
    return T, P


def test_overlapping_classes_follow_the_worked_example():
    # Section 2's overlapping 2-grams of {abba, bbac}: {ab, bb}, {bb, ba}, {ba, ac}
    g = _golden("section2_examples.json")
    P = np.array([list(p.encode()) for p in g["patterns"]], np.uint8)
    mu = np.zeros(256, np.uint8)
    for c in b"abc":
        mu[c] = c - 97
    fp = F.FilterParams(2, 4, 1, mu, overlap=True)
    classes = F.pattern_classes(P, fp)
    code = lambda s2: F.qgram_code([ord(c) - 97 for c in s2], 4, "msd")  # noqa: E731
    want = [set(code(x) for x in cls) for cls in g["overlapping_q2_superimposed"]]
    assert classes == want
    assert fp.lengths(4) == (3, 3, 3)


def test_overlap_with_q1_equals_the_nonoverlapping_filter():
    rng = np.random.default_rng(71)
    for _ in range(40):
        T, P = _overlap_case(rng, 4, 300, 5, int(rng.integers(2, 12)), 2)
        k = int(rng.integers(1, 4))
        if P.shape[1] // k < 1:
            continue
        a = F.make_params(P, 1, 4, k, "rank")
        b = F.make_params(P, 1, 4, k, "rank", overlap=True)
        ca, cb = F.pattern_classes(P, a), F.pattern_classes(P, b)
        assert ca == cb
        ta, tb = F.text_codes(T, a), F.text_codes(T, b)
        assert np.array_equal(ta, tb)
        assert F.aoso_scan(ta, F.mask_table(ca, a), a, len(ca)) == \
            F.aoso_scan(tb, F.mask_table(cb, b), b, len(cb))


def test_overlap_single_pattern_lossless_filter_is_exact():
    # one pattern, an injective map, k = 1: every position's class is one
    # q-gram, and the m - q + 1 overlapping q-grams cover the whole window,
    # so the candidates are exactly the occurrences
    rng = np.random.default_rng(72)
    for _ in range(60):
        m = int(rng.integers(2, 20))
        q = int(rng.integers(1, min(m, 4) + 1))
        T, P = _overlap_case(rng, 3, 400, 1, m, 1)
        fp = F.make_params(P, q, 4, 1, "rank", overlap=True)
        classes = F.pattern_classes(P, fp)
        windows = F.aoso_scan(F.text_codes(T, fp), F.mask_table(classes, fp), fp, len(classes))
        occ = [i for i in range(T.size - m + 1) if bytes(T[i:i + m]) == bytes(P[0])]
        assert windows == occ


def test_overlap_scan_equals_definition_and_search_equals_brute_force():
    rng = np.random.default_rng(73)
    for it in range(80):
        m = int(rng.integers(3, 24))
        q = int(rng.integers(1, min(m, 5) + 1))
        Lc = m - q + 1
        k = int(rng.integers(1, min(Lc, 6) + 1))
        sigma = int(rng.choice([2, 4, 8]))
        T, P = _overlap_case(rng, sigma, 500, int(rng.integers(1, 12)), m, 2)
        kind = ["rank", "greedy", "qhash"][it % 3]
        sr = 1 << 10 if kind == "qhash" else min(8, max(2, sigma // 2))
        fp = F.make_params(P, q, sr, k, kind, overlap=True)
        classes = F.pattern_classes(P, fp)
        codes = F.text_codes(T, fp)
        windows = F.aoso_scan(codes, F.mask_table(classes, fp), fp, len(classes))
        assert windows == F.candidate_windows_by_definition(codes, classes, fp)
        got = F.search(T, P, fp)
        assert got == sorted(brute.occurrences(T, P))
        # no false negatives: every occurrence is a candidate window
        assert {i for i, _ in got} <= set(windows)


def test_aho_corasick_variable_lengths_equals_brute_force():
    from oracle import native
    native.build()
    rng = random.Random(81)
    for _ in range(300):
        alpha = "ab" if rng.random() < 0.5 else "abcd"
        T = "".join(rng.choice(alpha) for _ in range(rng.randint(0, 60))).encode()
        P = ["".join(rng.choice(alpha) for _ in range(rng.randint(1, 7))).encode()
             for _ in range(rng.randint(1, 6))]
        if rng.random() < 0.3:
            P.append(P[0])   # a duplicate
        want = brute.occurrences(T, P)
        for threads in (1, 3):
            pos, pid = native.AhoCorasick(P).search(np.frombuffer(T, np.uint8), threads=threads)
            assert list(zip(pos.tolist(), pid.tolist())) == want


# ------------------------------------------- two words of Shift-Or state (Section 3.2)

def test_wider_filter_is_exact_for_long_single_patterns_and_tighter_than_64():
    rng = np.random.default_rng(91)
    for _ in range(25):
        m = int(rng.integers(70, 140))
        T, P = _overlap_case(rng, 2, 3000, 1, m, 1)
        for k in (1, 2):
            wide = F.make_params(P, 1, 2, k, "rank", max_positions=128)
            narrow = F.make_params(P, 1, 2, k, "rank")
            assert wide.lengths(m)[2] == k * (min(m, 128) // k)
            cw, cn = F.pattern_classes(P, wide), F.pattern_classes(P, narrow)
            # the first classes coincide; the wider filter adds positions
            assert cw[:len(cn)] == cn
            ww = F.aoso_scan(F.text_codes(T, wide), F.mask_table(cw, wide), wide, len(cw))
            wn = F.aoso_scan(F.text_codes(T, narrow), F.mask_table(cn, narrow), narrow, len(cn))
            assert ww == F.candidate_windows_by_definition(F.text_codes(T, wide), cw, wide)
            occ = [i for i in range(T.size - m + 1) if bytes(T[i:i + m]) == bytes(P[0])]
            if k == 1 and m <= 128:
                assert ww == occ   # one pattern, injective map, every position checked
            assert F.search(T, P, wide) == sorted(brute.occurrences(T, P))
