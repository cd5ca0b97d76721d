"""The MAG/SMAG filter restated step by step from the paper -- TEST INFRASTRUCTURE ONLY.

Only tests/, the smoke check and bench.py's CPU-baseline leg may import this.
It shares no code with the CUDA library; every step follows the paper's
order and notation, in plain Python/numpy, slow and obvious.

Steps and where they come from
  histogram / map_rank / map_greedy   Section 3.3 "Alphabet mapping": the
                                      pattern-set histogram; frequency-rank
                                      bins; (approximately) equal-weight bins
                                      by a simple greedy heuristic.
  map_lowbits, multiply_trick         Section 3.3, "Combined alphabet mapping
                                      and q-gram generation": the l low-order
                                      bits of each symbol, and the DNA
                                      multiply trick for a 4-gram.
  qgram_hash                          Section 3.3, "Alphabet mapping on the
                                      q-grams": whole q-grams mapped to sigma'
                                      bins, the mapping given by hashing.
  qgram_code                          Section 3.2 "Implementation": the
                                      numeric value of a q-gram by Horner's
                                      rule.
  overlapping_qgram_patterns          Section 2: P'_i[j] = P_i[j..j+q-1].
  nonoverlapping_qgram_patterns       Section 2: P'_i[j] = P_i[(j-1)q+1..jq]
                                      and all q shifts of each pattern.
  superimpose                         Section 2: P[i] = union_j P_j[i].
  mask_table                          Section 1.1 (Shift-Or: a bit 0 means
                                      "still matching") and Section 3.2
                                      (FAOSO: character classes only change
                                      the preprocessing of one table).
  aoso_scan                           Section 3.1 (k subpatterns
                                      P^j[i] = P[j + i k], every k-th text
                                      symbol read) with Section 3.2 (FAOSO
                                      over the superimposed non-overlapping
                                      q-gram pattern).
  candidate_windows_by_definition     the filter condition of Section 2
                                      ("T[i+j] in P[j] for all j") applied to
                                      the sampled subpattern of Section 3.1;
                                      a brute-force statement of what the
                                      scan must report.
  verify / search                     Section 3.2: verification against the
                                      r patterns in the original alphabet
                                      (Section 3.3).
  overlap=True                        Section 2's first filter, before MAG's
                                      non-overlapping factoring: the m-q+1
                                      overlapping q-grams of every pattern
                                      superimposed, the text's q-gram at
                                      every position, a window standing for
                                      its own start (no shifts).

Readings where the paper is silent or garbled (each is listed with its
reason in the design notes):
  * all q shifts s = 0..q-1 are superimposed (the printed shift list is
    garbled and lists q-1 of them; with fewer shifts occurrences are lost);
  * the shifted q-gram patterns are cut to the common length
    L' = floor((m - q + 1) / q), the length of the shortest shift;
  * the filter uses at most 64 q-gram positions (one 64-bit word), or 128
    with two words of state (Section 3.2's ceil((m/q)/w) words, w = 64);
  * AOSO subpattern j, element i sits at bit i*k + j, the sampled text
    q-grams are those with index h = k-1 (mod k), D starts all ones;
  * rank ties are broken by byte value; the greedy heuristic is
    longest-processing-time first, ties to the lowest bin; bytes absent
    from the patterns go to bin sigma'-1;
  * with overlapping q-grams the AOSO scan reads the text q-grams h = k-1
    (mod k) by byte position, the same recurrence over a longer sequence;
  * q-gram digit order: "lsd" is the formula of Section 3.2 (S[1] least
    significant); "msd" is the order the multiply trick of Section 3.3
    produces (S[1] most significant).  Both are bijections, so the filter's
    candidate set does not depend on the order.
"""
import math

import numpy as np


# ----------------------------------------------------------------- Section 3.3

def histogram(P):
    """Counts of each byte value over all pattern symbols (Section 3.3)."""
    P = np.asarray(P, dtype=np.uint8)
    return np.bincount(P.ravel(), minlength=256).astype(np.int64)


def _present_by_frequency(h):
    present = [c for c in range(256) if h[c] > 0]
    present.sort(key=lambda c: (-int(h[c]), c))
    return present


def map_rank(P, sigma_r):
    """Frequency-rank mapping (Section 3.3): code 0 to the most frequent
    pattern symbol, 1 to the next, ...; the symbols ranked sigma'-1 and below
    and the symbols that do not occur in the patterns all get sigma'-1."""
    h = histogram(P)
    mu = np.full(256, sigma_r - 1, dtype=np.uint8)
    for rank, c in enumerate(_present_by_frequency(h)):
        mu[c] = min(rank, sigma_r - 1)
    return mu


def map_greedy(P, sigma_r):
    """Equal-weight bins (Section 3.3), greedy: symbols by decreasing
    frequency, each into the currently lightest bin."""
    h = histogram(P)
    mu = np.full(256, sigma_r - 1, dtype=np.uint8)
    load = [0] * sigma_r
    for c in _present_by_frequency(h):
        b = min(range(sigma_r), key=lambda i: (load[i], i))
        mu[c] = b
        load[b] += int(h[c])
    return mu


def map_lowbits(sigma_r, shift=0):
    """Low-order-bit mapping (Section 3.3): keep l = log2(sigma') bits of each
    symbol, after a right shift (the DNA example shifts by one)."""
    assert sigma_r >= 2 and sigma_r & (sigma_r - 1) == 0
    return np.array([(c >> shift) & (sigma_r - 1) for c in range(256)], dtype=np.uint8)


def multiply_trick(x):
    """The 8-bit 4-gram of a 32-bit word of four ASCII DNA symbols
    (Section 3.3): mask the 2 bits after a right shift by one, then a single
    multiplication gathers the four 2-bit codes into the top byte."""
    return ((((x >> 1) & 0x03030303) * 0x40100401) & 0xFFFFFFFF) >> 24


def qgram_hash(raw, bits):
    """Mapping of a whole q-gram to one of 2^bits bins (Section 3.3, "Alphabet
    mapping on the q-grams": the q-grams are mapped to 0..sigma'-1 and the
    mapping is stored by hashing).  Here the bin is the multiplicative
    (Fibonacci) hash of the q raw bytes read as a little-endian integer:
    the top `bits` bits of raw * 0x9E3779B1 mod 2^32 for q <= 4, of
    raw * 0x9E3779B97F4A7C15 mod 2^64 for 5 <= q <= 8."""
    raw = bytes(raw)
    q = len(raw)
    assert 1 <= q <= 8 and 1 <= bits <= 32
    x = int.from_bytes(raw, "little")
    if q <= 4:
        return ((x * 0x9E3779B1) & 0xFFFFFFFF) >> (32 - bits)
    return ((x * 0x9E3779B97F4A7C15) & 0xFFFFFFFFFFFFFFFF) >> (64 - bits)


# ----------------------------------------------------------------- Section 3.2

def qgram_code(symbols, sigma_r, order="lsd"):
    """Numeric value of a q-gram S[1..q] by Horner's rule (Section 3.2).

    order="lsd": sum_i S[i] * sigma'^(i-1)  (the printed formula);
    order="msd": S[1] is the most significant digit (the multiply trick)."""
    code = 0
    seq = list(symbols)
    if order == "lsd":
        seq = seq[::-1]
    else:
        assert order == "msd"
    for s in seq:
        code = code * sigma_r + int(s)
    return code


# ------------------------------------------------------------------- Section 2

def overlapping_qgram_patterns(P, q):
    """P'_i[j] = P_i[j..j+q-1], j = 1..m-q+1, as tuples of q symbols."""
    return [[tuple(p[j:j + q]) for j in range(len(p) - q + 1)] for p in P]


def nonoverlapping_qgram_patterns(P, q, shifts=True, length=None):
    """Non-overlapping q-grams P'_i[j] = P_i[(j-1)q+1..jq] of every shift
    P_i[s..m), s = 0..q-1 (all q shifts; without `shifts`, only s = 0).

    Every shifted pattern is cut to `length` q-grams; the default is the
    common length L' = floor((m - q + 1) / q) of the shortest shift (with
    shifts) or floor(m / q) (without).  Returns a list over (pattern, shift)
    of lists of q-tuples."""
    out = []
    for p in P:
        m = len(p)
        svals = range(q) if shifts else [0]
        L = length
        if L is None:
            L = (m - q + 1) // q if shifts else m // q
        for s in svals:
            out.append([tuple(p[s + j * q: s + j * q + q]) for j in range(L)])
    return out


def superimpose(qpatterns):
    """Superimposed pattern: position j is the set of the j-th symbols of all
    patterns (Section 2)."""
    L = min(len(x) for x in qpatterns)
    return [set(x[j] for x in qpatterns) for j in range(L)]


# ------------------------------------------------------- the filter's tables

class FilterParams:
    """q, sigma' (power of two), k and the mapping of one filter instance.

    With mu, sigma' is the reduced symbol alphabet and a q-gram code has q
    digits; with qhash=True, sigma' is the number of q-gram bins and a
    q-gram's code is qgram_hash of its raw bytes."""

    def __init__(self, q, sigma_r, k, mu=None, order="msd", qhash=False, overlap=False,
                 max_positions=64):
        self.q, self.sigma_r, self.k = int(q), int(sigma_r), int(k)
        self.qhash = bool(qhash)
        self.overlap = bool(overlap)
        self.max_positions = int(max_positions)
        self.mu = None if mu is None else np.asarray(mu, dtype=np.uint8)
        self.order = order

    def lengths(self, m):
        """(L', m', m''): the q-gram pattern length (m - q + 1 overlapping
        q-grams, or the common length floor((m - q + 1) / q) of the q shifts'
        non-overlapping q-grams), the AOSO subpattern length and the number of
        filter positions k*m' (at most max_positions: 64 for one 64-bit word
        of Shift-Or state, 128 for two)."""
        Lc = (m - self.q + 1) if self.overlap else (m - self.q + 1) // self.q
        Lf = min(Lc, self.max_positions)
        mp = Lf // self.k
        return Lc, mp, self.k * mp


def _qgram_patterns(rows, fp, Lc):
    if fp.overlap:
        return overlapping_qgram_patterns(rows, fp.q)
    return nonoverlapping_qgram_patterns(rows, fp.q, shifts=True, length=Lc)


def pattern_classes(P, fp):
    """Cls[p] for the filter positions p < m'': the reduced-alphabet codes of
    the p-th q-gram of every pattern (every shift of it, for non-overlapping
    q-grams)."""
    P = np.asarray(P, dtype=np.uint8)
    m = P.shape[1]
    Lc, mp, mpp = fp.lengths(m)
    assert mp >= 1, "infeasible: need floor(min(L',64)/k) >= 1"
    if fp.qhash:
        qp = _qgram_patterns([list(row) for row in P], fp, Lc)
        classes = superimpose(qp)[:mpp]
        bits = log2i(fp.sigma_r)
        return [set(qgram_hash(g, bits) for g in cls) for cls in classes]
    reduced = [[int(fp.mu[c]) for c in row] for row in P]
    qp = _qgram_patterns(reduced, fp, Lc)
    classes = superimpose(qp)[:mpp]
    return [set(qgram_code(g, fp.sigma_r, fp.order) for g in cls) for cls in classes]


def mask_table(classes, fp):
    """Shift-Or table over the q-gram alphabet: bit p of B[c] is 0 iff c is
    in Cls[p]; bits >= len(classes) are 0 (they are never tested)."""
    size = fp.sigma_r if fp.qhash else fp.sigma_r ** fp.q
    full = (1 << len(classes)) - 1
    B = [full] * size
    for p, cls in enumerate(classes):
        for c in cls:
            B[c] &= ~(1 << p)
    # more than 64 positions: entries as Python integers (two words of state)
    return np.array(B, dtype=np.uint64 if len(classes) <= 64 else object)


def text_codes(T, fp):
    """t'(h) for h = 0..floor(n/q)-1: the codes of the text's non-overlapping
    q-grams (the text factored like the patterns, Section 2); with overlap,
    the code of T[h..h+q) for every h = 0..n-q."""
    T = np.asarray(T, dtype=np.uint8)
    if fp.overlap:
        nh = max(0, T.size - fp.q + 1)
        grams = [T[h:h + fp.q] for h in range(nh)]
        if fp.qhash:
            bits = log2i(fp.sigma_r)
            return np.array([qgram_hash(g.tobytes(), bits) for g in grams], dtype=np.int64)
        return np.array([qgram_code([int(fp.mu[c]) for c in g], fp.sigma_r, fp.order)
                         for g in grams], dtype=np.int64)
    nq = T.size // fp.q
    if fp.qhash:
        bits = log2i(fp.sigma_r)
        raw = T[: nq * fp.q].reshape(nq, fp.q)
        return np.array([qgram_hash(g.tobytes(), bits) for g in raw], dtype=np.int64)
    red = fp.mu[T[: nq * fp.q]].reshape(nq, fp.q).astype(np.int64)
    code = np.zeros(nq, dtype=np.int64)
    cols = range(fp.q) if fp.order == "msd" else range(fp.q - 1, -1, -1)
    for t in cols:
        code = code * fp.sigma_r + red[:, t]
    return code


# -------------------------------------------------------- Sections 3.1, 3.2

def aoso_scan(codes, B, fp, mpp):
    """FAOSO over the sampled text q-grams.

    Only q-grams h = k-1, 2k-1, ... are read; D <- (D << k) | B[t'(h)].  After
    reading h, a zero at bit (m'-1)k + j means subpattern j matched, i.e. a
    candidate window starting at q-gram h0 = h - (m'-1)k - j.  Returns the
    sorted list of window starts h0."""
    k = fp.k
    mp = mpp // k
    width_mask = (1 << mpp) - 1
    report = ((1 << k) - 1) << ((mp - 1) * k)
    D = width_mask
    out = []
    for h in range(k - 1, len(codes), k):
        D = ((D << k) | int(B[codes[h]])) & width_mask
        fired = ~D & report
        if fired:
            for j in range(k):
                if fired >> ((mp - 1) * k + j) & 1:
                    out.append(h - (mp - 1) * k - j)
    out.sort()
    return out


def candidate_windows_by_definition(codes, classes, fp):
    """The windows the AOSO filter must report, by brute force: window h0 is
    read by the one subpattern j with h0 + j = k-1 (mod k), and is a
    candidate iff t'(h0 + j + i k) is in Cls[j + i k] for every i < m'."""
    k = fp.k
    mpp = len(classes)
    mp = mpp // k
    nq = len(codes)
    out = []
    for h0 in range(nq):
        j = (k - 1 - h0) % k
        last = h0 + j + (mp - 1) * k
        if last >= nq:
            continue
        if all(int(codes[h0 + j + i * k]) in classes[j + i * k] for i in range(mp)):
            out.append(h0)
    return out


def verify(T, P, windows, q):
    """Exact check of each candidate window (Section 3.2, in the original
    alphabet): window h0 stands for the text starts i = h0*q - s, s < q."""
    T = bytes(np.asarray(T, dtype=np.uint8).tobytes())
    P = [bytes(np.asarray(p, dtype=np.uint8).tobytes()) for p in P]
    m = len(P[0])
    n = len(T)
    by_bytes = {}
    for pid, p in enumerate(P):
        by_bytes.setdefault(p, []).append(pid)
    out = []
    for h0 in windows:
        for s in range(q):
            i = h0 * q - s
            if 0 <= i <= n - m:
                for pid in by_bytes.get(T[i:i + m], ()):
                    out.append((i, pid))
    out.sort()
    return out


def make_params(P, q, sigma_r, k, map_kind, shift=0, order="msd", overlap=False,
                max_positions=64):
    """Convenience: the mapping of `map_kind` ("rank", "greedy", "lowbits",
    "qhash")."""
    if map_kind == "qhash":
        return FilterParams(q, sigma_r, k, None, order, qhash=True, overlap=overlap,
                            max_positions=max_positions)
    if map_kind == "rank":
        mu = map_rank(P, sigma_r)
    elif map_kind == "greedy":
        mu = map_greedy(P, sigma_r)
    elif map_kind == "lowbits":
        mu = map_lowbits(sigma_r, shift)
    else:
        raise ValueError(map_kind)
    return FilterParams(q, sigma_r, k, mu, order, overlap=overlap, max_positions=max_positions)


def search(T, P, fp):
    """The whole filter-then-verify search (MAG's result, without its speed)."""
    P = np.asarray(P, dtype=np.uint8)
    classes = pattern_classes(P, fp)
    B = mask_table(classes, fp)
    codes = text_codes(T, fp)
    windows = aoso_scan(codes, B, fp, len(classes))
    # a window of overlapping q-grams starts at its own text position
    return verify(T, P, windows, 1 if fp.overlap else fp.q)


def expected_class_size(sigma, r):
    """Expected number of distinct symbols among r uniform draws from sigma
    (the closed form behind the Section 2 illustration)."""
    return sigma * (1.0 - (1.0 - 1.0 / sigma) ** r)


def log2i(x):
    l = int(round(math.log2(x)))
    assert 1 << l == x
    return l
