"""Seeded synthetic inputs shaped like the paper's workloads.

This module only draws random texts and pattern sets; it holds none of the
search's arithmetic and is shared by the tests, the benchmark and the CPU
baseline.  The paper measures on the Pizza&Chili 200 MB ``dna``, ``english``
and ``proteins`` texts (Section 4); those files are not available here, so
these generators stand in for them with the same alphabet sizes and
comparable symbol statistics:

  dna       uniform i.i.d. over ``ACGT`` (sigma = 4)
  protein   i.i.d. over the 20 amino-acid letters, P(rank i) ~ i^-0.8
  english   i.i.d. over the 95 printable bytes 0x20..0x7E, P(rank i) ~ i^-1.0,
            ranks assigned by a seeded permutation

Pattern sets mix "planted" patterns (substrings of the text at uniform random
offsets, so each occurs at least once) with patterns drawn i.i.d. from the
text's symbol distribution.  Seeds: text 1000 + config, patterns 2000 + config.
"""
import math

import numpy as np

DNA = np.frombuffer(b"ACGT", np.uint8)
PROTEIN = np.frombuffer(b"ACDEFGHIKLMNPQRSTVWY", np.uint8)
PRINTABLE = np.arange(0x20, 0x7F, dtype=np.uint8)

_CHUNK = 1 << 24


class Source:
    """An i.i.d. symbol source: `symbols[i]` with probability `probs[i]`
    (drawn through a 2^16-slot inverse-CDF table, so each probability is
    realised to within 2^-16)."""

    def __init__(self, symbols, probs):
        self.symbols = np.asarray(symbols, dtype=np.uint8)
        p = np.asarray(probs, dtype=np.float64)
        self.probs = p / p.sum()
        self.cdf = np.cumsum(self.probs)
        self.cdf[-1] = 1.0
        u = (np.arange(1 << 16) + 0.5) / (1 << 16)
        idx = np.minimum(np.searchsorted(self.cdf, u), self.symbols.size - 1)
        self._slot = self.symbols[idx]

    @property
    def entropy_bits(self):
        p = self.probs[self.probs > 0]
        return float(-(p * np.log2(p)).sum())

    def draw(self, n, rng):
        out = np.empty(n, dtype=np.uint8)
        uniform = np.allclose(self.probs, self.probs[0])
        for a in range(0, n, _CHUNK):
            b = min(n, a + _CHUNK)
            if uniform:
                out[a:b] = self.symbols[rng.integers(0, self.symbols.size, size=b - a,
                                                     dtype=np.uint8)]
            else:
                out[a:b] = self._slot[rng.integers(0, 1 << 16, size=b - a, dtype=np.uint16)]
        return out


def dna_source():
    return Source(DNA, np.ones(4))


def zipf_source(symbols, s, perm_seed=None):
    symbols = np.asarray(symbols, dtype=np.uint8)
    if perm_seed is not None:
        symbols = np.random.default_rng(perm_seed).permutation(symbols)
    ranks = np.arange(1, symbols.size + 1, dtype=np.float64)
    return Source(symbols, ranks ** -float(s))


def protein_source():
    return zipf_source(PROTEIN, 0.8)


def english_source(perm_seed=4000):
    return zipf_source(PRINTABLE, 1.0, perm_seed=perm_seed)


def make_patterns(text, source, r, m, planted, rng):
    """r patterns of length m: the first `planted` are substrings of `text` at
    uniform random offsets, the rest are i.i.d. from `source`.  Returns
    (P uint8[r, m], offsets of the planted ones)."""
    n = int(text.size)
    planted = min(planted, r) if n >= m else 0
    P = np.empty((r, m), dtype=np.uint8)
    offs = rng.integers(0, n - m + 1, size=planted) if planted else np.zeros(0, np.int64)
    for i, o in enumerate(offs):
        P[i] = text[o:o + m]
    if r > planted:
        P[planted:] = source.draw((r - planted) * m, rng).reshape(r - planted, m)
    return P, offs


class Case:
    """One search problem: text T (uint8[n]) and patterns P (uint8[r, m], or
    a list of byte strings of different lengths)."""

    def __init__(self, name, T, P, sigma, planted_offsets, source):
        self.name, self.T, self.P, self.sigma = name, T, P, sigma
        self.planted_offsets = planted_offsets
        self.source = source

    @property
    def variable(self):
        return isinstance(self.P, list)

    @property
    def n(self):
        return int(self.T.size)

    @property
    def r(self):
        return len(self.P) if self.variable else int(self.P.shape[0])

    @property
    def m(self):
        """The pattern length (the shortest one for variable lengths)."""
        return min(len(p) for p in self.P) if self.variable else int(self.P.shape[1])

    def prefix_matrix(self):
        """uint8[r, m]: every pattern's first m bytes."""
        if not self.variable:
            return self.P
        m = self.m
        return np.stack([np.frombuffer(p[:m], np.uint8) for p in self.P])


def dna_case(n, r, m, planted, cfg=1, name=None):
    src = dna_source()
    T = src.draw(n, np.random.default_rng(1000 + cfg))
    P, offs = make_patterns(T, src, r, m, planted, np.random.default_rng(2000 + cfg))
    return Case(name or "dna n=%d r=%d m=%d" % (n, r, m), T, P, 4, offs, src)


def protein_case(n, r, m, planted, cfg=2, name=None):
    src = protein_source()
    T = src.draw(n, np.random.default_rng(1000 + cfg))
    P, offs = make_patterns(T, src, r, m, planted, np.random.default_rng(2000 + cfg))
    return Case(name or "protein n=%d r=%d m=%d" % (n, r, m), T, P, 20, offs, src)


def english_case(n, r, m, planted, cfg=4, name=None):
    src = english_source()
    T = src.draw(n, np.random.default_rng(1000 + cfg))
    P, offs = make_patterns(T, src, r, m, planted, np.random.default_rng(2000 + cfg))
    return Case(name or "english n=%d r=%d m=%d" % (n, r, m), T, P, 95, offs, src)


# ------------------------------------------------------------ the five configs

def config1():
    """DNA, n = 2^20, r = 100, m = 16, 50 planted + 50 random."""
    return dna_case(1 << 20, 100, 16, 50, cfg=1, name="dna-1MiB r=100 m=16")


def config1_scaled(n=1 << 30):
    """Config 1's distribution and pattern shape at a text larger than L2."""
    return dna_case(n, 100, 16, 50, cfg=1, name="dna-%dMiB r=100 m=16" % (n >> 20))


def config2(n=1 << 28):
    """Protein-like, n = 2^28, r = 1000, m = 32, half planted."""
    return protein_case(n, 1000, 32, 500, cfg=2, name="protein-%dMiB r=1000 m=32" % (n >> 20))


def config2_varlen(n=1 << 28, r=1000, lo=16, hi=64):
    """Config 2's text with patterns of different lengths: r patterns with
    lengths uniform over [lo, hi], half planted (text seed 1002, pattern
    seed 2102)."""
    src = protein_source()
    T = src.draw(n, np.random.default_rng(1000 + 2))
    rng = np.random.default_rng(2100 + 2)
    P, offs = [], []
    for i in range(r):
        L = int(rng.integers(lo, hi + 1))
        if i < r // 2:
            o = int(rng.integers(0, n - L + 1))
            P.append(T[o:o + L].tobytes())
            offs.append(o)
        else:
            P.append(src.draw(L, rng).tobytes())
    return Case("protein-%dMiB r=%d m=%d..%d" % (n >> 20, r, lo, hi), T, P, 20,
                np.array(offs, np.int64), src)


def config3(n=1 << 30, r=100_000, m=32):
    """Uniform DNA, n = 2^30, r = 100,000, m = 32, 10% planted (also r = 10^4
    with m = 16 and m = 64)."""
    return dna_case(n, r, m, r // 10, cfg=3,
                    name="dna-%dMiB r=%d m=%d" % (n >> 20, r, m))


class Batch:
    """Config 4: many texts of uneven length against many pattern sets.

    texts[t] is paired with pattern set set_of_text[t]."""

    def __init__(self, texts, sets, set_of_text, sigma=95):
        self.texts, self.sets, self.set_of_text = texts, sets, set_of_text
        self.sigma = sigma

    @property
    def total_bytes(self):
        return int(sum(t.size for t in self.texts))


def config4(ntexts=4096, nsets=64, min_log2=10, max_log2=22, cfg=4):
    """4096 texts with lengths log-uniform over [2^10, 2^22] bytes (95
    printable symbols, Zipf s = 1.0); 64 pattern sets with r log-uniform over
    [10, 10^4] and m uniform over {8, 16, 32, 64}; each text is paired with
    one set chosen uniformly; half of each set is planted from its texts."""
    src = english_source()
    rng_t = np.random.default_rng(1000 + cfg)
    rng_p = np.random.default_rng(2000 + cfg)
    lens = np.exp(rng_t.uniform(min_log2 * math.log(2), max_log2 * math.log(2),
                                size=ntexts)).astype(np.int64)
    texts = [src.draw(int(L), rng_t) for L in lens]
    set_of_text = rng_p.integers(0, nsets, size=ntexts).astype(np.uint32)
    sets = []
    for s in range(nsets):
        r = int(round(math.exp(rng_p.uniform(math.log(10), math.log(10_000)))))
        m = int(rng_p.choice([8, 16, 32, 64]))
        mine = np.flatnonzero(set_of_text == s)
        P = np.empty((r, m), dtype=np.uint8)
        planted = r // 2 if mine.size else 0
        for i in range(planted):
            t = texts[int(mine[rng_p.integers(0, mine.size)])]
            if t.size < m:
                P[i] = src.draw(m, rng_p)
                continue
            o = int(rng_p.integers(0, t.size - m + 1))
            P[i] = t[o:o + m]
        if r > planted:
            P[planted:] = src.draw((r - planted) * m, rng_p).reshape(r - planted, m)
        sets.append(P)
    return Batch(texts, sets, set_of_text)


def config5_set(index, cfg=5):
    """Pattern set `index` of the cost model's data, config-4-shaped: one text
    of n bytes, n log-uniform over [2^20, 2^23] (95 printable symbols, Zipf
    s = 1.0); r log-uniform over [10, 10^4]; m uniform over {8, 16, 32, 64};
    half of the patterns planted from the text.  Seeds (1000 + cfg, index)
    for the text and (2000 + cfg, index) for the patterns."""
    src = english_source()
    rng_t = np.random.default_rng([1000 + cfg, index])
    rng_p = np.random.default_rng([2000 + cfg, index])
    n = int(math.exp(rng_t.uniform(20 * math.log(2), 23 * math.log(2))))
    T = src.draw(n, rng_t)
    r = int(round(math.exp(rng_p.uniform(math.log(10), math.log(10_000)))))
    m = int(rng_p.choice([8, 16, 32, 64]))
    P, offs = make_patterns(T, src, r, m, r // 2, rng_p)
    return Case("set %d n=%d r=%d m=%d" % (index, n, r, m), T, P, 95, offs, src)


def random_case(rng, sigma, n, r, m, planted=0, base=97):
    """A small random case over `sigma` symbols starting at byte `base`."""
    T = (rng.integers(0, sigma, size=n) + base).astype(np.uint8)
    P = (rng.integers(0, sigma, size=(r, m)) + base).astype(np.uint8)
    if n >= m:
        for i in range(min(planted, r)):
            o = int(rng.integers(0, n - m + 1))
            P[i] = T[o:o + m]
    return T, P
