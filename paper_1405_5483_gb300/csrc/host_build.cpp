// Host half of mpm_build: alphabet mapping, automatic parameters, the
// superimposed Shift-Or mask table and the pattern table for verification.
//
// Sections of "Multiple pattern matching revisited" followed here:
//   Section 3.3  the mapping mu (frequency rank, equal-weight greedy bins,
//                low-order bits after a shift);
//   Section 2    non-overlapping q-grams of all q shifts of every pattern,
//                superimposed position by position;
//   Section 3.2  one Shift-Or table over the q-gram alphabet holds the
//                classes (FAOSO); q-gram numbering by Horner's rule, here
//                with the first symbol most significant (the order the
//                multiply trick of Section 3.3 produces);
//   Sections 3.1, 3.2  the choice of q and k (the paper picks q from
//                log_sigma(rm) and then k as large as the verification
//                probability allows; this file scores a small grid with an
//                estimate of that probability instead of a closed form).
#include <algorithm>
#include <functional>
#include <cmath>
#include <cstring>
#include <numeric>
#include <unordered_set>

#include "mpm_internal.h"

namespace mpm {

namespace {

int log2_exact(int x) {
    int l = 0;
    while ((1 << l) < x) l++;
    return l;
}

bool is_pow2(int x) { return x >= 1 && (x & (x - 1)) == 0; }

int pow2_ceil(int x) {
    int p = 1;
    while (p < x) p <<= 1;
    return p;
}

void histogram(const uint8_t* P, size_t r, size_t m, uint64_t h[256]) {
    std::fill(h, h + 256, 0ull);
    for (size_t i = 0; i < r * m; i++) h[P[i]]++;
}

// Pattern bytes that occur, by decreasing count, ties by byte value.
std::vector<int> by_frequency(const uint64_t h[256]) {
    std::vector<int> v;
    for (int c = 0; c < 256; c++)
        if (h[c]) v.push_back(c);
    std::stable_sort(v.begin(), v.end(), [&](int a, int b) { return h[a] > h[b]; });
    return v;
}

// Number of distinct reduced values among the occurring bytes under the
// low-bit map with this shift.
int lowbits_distinct(const uint64_t h[256], int sigma_r, int shift) {
    bool seen[256] = {false};
    int d = 0;
    for (int c = 0; c < 256; c++) {
        if (!h[c]) continue;
        int v = (c >> shift) & (sigma_r - 1);
        if (!seen[v]) { seen[v] = true; d++; }
    }
    return d;
}

int best_shift(const uint64_t h[256], int sigma_r) {
    int best = 0, bd = -1;
    for (int s = 0; s < 8; s++) {
        int d = lowbits_distinct(h, sigma_r, s);
        if (d > bd) { bd = d; best = s; }
    }
    return best;
}

uint32_t msd_code(const uint8_t* red, int q, int ell) {
    uint32_t c = 0;
    for (int u = 0; u < q; u++) c = (c << ell) | red[u];
    return c;
}

struct Lengths {
    int L, Lf, mprime, positions;
};

// L' = the q-gram pattern length: floor((m-q+1)/q) non-overlapping q-grams
// (common to the q shifts), or m-q+1 overlapping ones; the filter keeps at
// most maxpos of them (64 for each 64-bit word of Shift-Or state).
Lengths lengths(size_t m, int q, int k, bool overlap, int maxpos) {
    Lengths x;
    long L = overlap ? ((long)m - q + 1) : ((long)m - q + 1) / q;
    x.L = (int)std::max(0L, L);
    x.Lf = std::min(x.L, maxpos);
    x.mprime = k >= 1 ? x.Lf / k : 0;
    x.positions = k * x.mprime;
    return x;
}

// Bytes of a mask-table entry: the smallest word that holds the positions,
// above 64 positions ceil(positions / 64) words of 8 bytes (Section 3.2).
int entry_bytes_for(int positions) {
    if (positions <= 8) return 1;
    if (positions <= 16) return 2;
    if (positions <= 32) return 4;
    return 8 * ((positions + 63) / 64);
}

// Probability, under the pattern-set symbol frequencies mapped by mu, that a
// random text q-gram falls in the class of each filter position
// (the "p" of Section 3.2, measured on the actual classes).
// Position t's q-grams start at s + t * stride for s < shifts: q and q for
// non-overlapping q-grams of all shifts, 1 and 1 for overlapping ones.
std::vector<double> class_probabilities(const uint8_t* P, size_t r, size_t m, int q,
                                        int ell, const uint8_t mu[256],
                                        const uint64_t h[256], int npos, bool overlap) {
    const int shifts = overlap ? 1 : q, stride = overlap ? 1 : q;
    const int sr = 1 << ell;
    std::vector<double> ps(sr, 0.0);
    const double tot = (double)(r * m);
    for (int c = 0; c < 256; c++) ps[mu[c]] += (double)h[c] / tot;
    std::vector<double> pt(npos, 0.0);
    std::vector<uint8_t> red(m);
    std::vector<std::vector<uint32_t>> codes(npos);
    for (auto& v : codes) v.reserve(r * q);
    for (size_t i = 0; i < r; i++) {
        for (size_t j = 0; j < m; j++) red[j] = mu[P[i * m + j]];
        for (int s = 0; s < shifts; s++)
            for (int t = 0; t < npos; t++)
                codes[t].push_back(msd_code(&red[s + t * stride], q, ell));
    }
    for (int t = 0; t < npos; t++) {
        auto& v = codes[t];
        std::sort(v.begin(), v.end());
        v.erase(std::unique(v.begin(), v.end()), v.end());
        double acc = 0.0;
        for (uint32_t c : v) {
            double pr = 1.0;
            for (int u = 0; u < q; u++) pr *= ps[(c >> (ell * (q - 1 - u))) & (sr - 1)];
            acc += pr;
        }
        pt[t] = std::min(1.0, acc);
    }
    return pt;
}

uint64_t raw_qgram(const uint8_t* g, int q) {
    uint64_t x = 0;
    for (int u = 0; u < q; u++) x |= (uint64_t)g[u] << (8 * u);
    return x;
}

// The same probability for the q-gram hashing map: a text q-gram falls in
// class t when it is one of the pattern q-grams there, or when it is another
// q-gram that shares a bin with one of them.  GramStats holds what does not
// depend on the number of bins.
struct GramStats {
    std::vector<std::vector<uint64_t>> grams;  // distinct raw q-grams per position
    std::vector<double> ptrue;                 // their total probability
};

GramStats gram_stats(const uint8_t* P, size_t r, size_t m, int q, const uint64_t h[256],
                     int npos, bool overlap) {
    const int shifts = overlap ? 1 : q, stride = overlap ? 1 : q;
    double pb[256];
    const double tot = (double)(r * m);
    for (int c = 0; c < 256; c++) pb[c] = (double)h[c] / tot;
    GramStats g;
    g.grams.resize(npos);
    g.ptrue.assign(npos, 0.0);
    for (auto& v : g.grams) v.reserve(r * q);
    for (size_t i = 0; i < r; i++)
        for (int s = 0; s < shifts; s++)
            for (int t = 0; t < npos; t++)
                g.grams[t].push_back(raw_qgram(P + i * m + s + t * stride, q));
    for (int t = 0; t < npos; t++) {
        auto& v = g.grams[t];
        std::sort(v.begin(), v.end());
        v.erase(std::unique(v.begin(), v.end()), v.end());
        double acc = 0.0;
        for (uint64_t x : v) {
            double pr = 1.0;
            for (int u = 0; u < q; u++) pr *= pb[(x >> (8 * u)) & 0xFF];
            acc += pr;
        }
        g.ptrue[t] = std::min(1.0, acc);
    }
    return g;
}

std::vector<double> qhash_class_probabilities(const GramStats& g, int q, int bits) {
    const int npos = (int)g.grams.size();
    std::vector<double> pt(npos, 0.0);
    std::vector<uint32_t> bins;
    for (int t = 0; t < npos; t++) {
        bins.clear();
        for (uint64_t x : g.grams[t]) bins.push_back(qgram_bin(x, q, bits));
        std::sort(bins.begin(), bins.end());
        bins.erase(std::unique(bins.begin(), bins.end()), bins.end());
        const double pcoll = (double)bins.size() / (double)(1ull << bits);
        pt[t] = std::min(1.0, g.ptrue[t] + pcoll * (1.0 - g.ptrue[t]));
    }
    return pt;
}

// Expected candidate records per sampled q-gram for step k: subpattern j
// fires when all its m' q-grams fall in their classes.
double candidate_rate(const std::vector<double>& pt, int k, int mprime) {
    double rate = 0.0;
    for (int j = 0; j < k; j++) {
        double pj = 1.0;
        for (int i = 0; i < mprime; i++) pj *= pt[j + i * k];
        rate += pj;
    }
    return std::min(1.0, rate);
}

constexpr uint64_t kSmemTableBudget = 96 * 1024;
constexpr uint64_t kMaxTableBytes = 1ull << 30;
constexpr uint64_t kAutoTableBytes = 64ull << 20;

// Relative cost per text byte of one parameter choice (a planning
// heuristic; the autotuner replaces it with measurements).
double plan_cost(int kind, int q, int k, double rate, uint64_t table_bytes, bool overlap) {
    // bytes per sampled q-gram; a candidate record stands for q windows (one
    // per shift), or one with overlapping q-grams
    const double P = overlap ? (double)k : (double)q * k;
    const int shifts = overlap ? 1 : q;
    const double per_byte = kind == MPM_MAP_QHASH ? 0.5 : (kind == MPM_MAP_LOWBITS ? 1.5 : 3.5);
    double alu = per_byte + 10.0 / P;
    double scan = std::max(1.0, alu / 4.0);
    double verify = rate / P * shifts * 48.0;
    double table = table_bytes <= kSmemTableBudget ? 0.0
                   : (table_bytes <= (8ull << 20) ? 6.0 / P : 14.0 / P);
    return scan + verify + table;
}

}  // namespace

void make_mu(const uint8_t* P, size_t r, size_t m, int kind, int sigma_r, int shift,
             uint8_t mu[256]) {
    uint64_t h[256];
    histogram(P, r, m, h);
    if (kind == MPM_MAP_LOWBITS) {
        for (int c = 0; c < 256; c++) mu[c] = (uint8_t)((c >> shift) & (sigma_r - 1));
        return;
    }
    if (kind == MPM_MAP_QHASH) {  // whole q-grams are hashed; bytes pass as they are
        for (int c = 0; c < 256; c++) mu[c] = (uint8_t)c;
        return;
    }
    std::fill(mu, mu + 256, (uint8_t)(sigma_r - 1));
    std::vector<int> order = by_frequency(h);
    if (kind == MPM_MAP_RANK) {
        for (size_t rank = 0; rank < order.size(); rank++)
            mu[order[rank]] = (uint8_t)std::min<size_t>(rank, sigma_r - 1);
        return;
    }
    // MPM_MAP_GREEDY: longest-processing-time first into the lightest bin
    std::vector<uint64_t> load(sigma_r, 0);
    for (int c : order) {
        int b = 0;
        for (int i = 1; i < sigma_r; i++)
            if (load[i] < load[b]) b = i;
        mu[c] = (uint8_t)b;
        load[b] += h[c];
    }
}

int make_plan(const uint8_t* P, size_t r, size_t m, int sigma, const mpm_params* in,
              Plan* out, std::vector<Plan>* all) {
    if (!P || !out || r == 0 || m == 0 || sigma < 1 || sigma > 256) return MPM_EINVAL;
    if (r >= (1ull << 31) || m >= (1ull << 20) || r * m / m != r || r * m >= (1ull << 40))
        return MPM_EINVAL;
    mpm_params req;
    if (in) {
        req = *in;
    } else {
        std::memset(&req, 0, sizeof(req));
        req.map_shift = -1;
    }
    if (req.map_kind < 0 || req.map_kind > MPM_MAP_QHASH) return MPM_EINVAL;
    const bool want_qhash = req.map_kind == MPM_MAP_QHASH;
    if (req.q < 0 || req.q > (want_qhash ? 8 : 16)) return MPM_EINVAL;
    if (req.sigma_r != 0 && want_qhash &&
        (!is_pow2(req.sigma_r) || req.sigma_r < 2 || req.sigma_r > (1 << 24)))
        return MPM_EINVAL;
    if (req.sigma_r != 0 && !want_qhash &&
        (!is_pow2(req.sigma_r) || req.sigma_r < 2 || req.sigma_r > 256 ||
         req.sigma_r > std::max(2, pow2_ceil(sigma))))
        return MPM_EINVAL;
    if (req.k < 0 || req.k > kMaxK) return MPM_EINVAL;
    if (req.map_shift > 7) return MPM_EINVAL;
    if (req.table_place < 0 || req.table_place > MPM_TABLE_GLOBAL) return MPM_EINVAL;
    if (req.smag < 0 || req.smag > 1 || req.chunk < 0) return MPM_EINVAL;
    if (req.overlap < 0 || req.overlap > 1) return MPM_EINVAL;
    if (req.wide < 0 || req.wide > kMaxWords - 1) return MPM_EINVAL;
    const bool ov = req.overlap == 1;
    const int maxpos = (req.wide + 1) * kMaxPositions;
    if (req.kernel < MPM_KERNEL_AUTO || req.kernel > MPM_KERNEL_SPLIT) return MPM_EINVAL;

    uint64_t h[256];
    histogram(P, r, m, h);
    int distinct = 0;
    for (int c = 0; c < 256; c++) distinct += h[c] ? 1 : 0;

    std::vector<int> sigmas;
    if (req.sigma_r) {
        sigmas.push_back(req.sigma_r);
    } else {
        int top = std::min(256, pow2_ceil(std::max(2, distinct)));
        for (int s = 2; s <= top; s <<= 1) sigmas.push_back(s);
    }

    bool found = false;
    double best_cost = 0.0;
    Plan best;
    std::memset(&best, 0, sizeof(best));
    // scores every k for one (mapping, sigma', q) given the per-position
    // class probabilities pt
    auto consider = [&](int kind, int sr, int ell, int shift, int q, uint64_t entries,
                        const std::vector<double>& pt, const Lengths& L1) {
        std::vector<int> ks;
        if (req.k) {
            ks.push_back(req.k);
        } else {
            for (int k = 1; k <= std::min(L1.Lf, kMaxK); k++) ks.push_back(k);
        }
        for (int k : ks) {
            Lengths Lk = lengths(m, q, k, ov, maxpos);
            if (Lk.mprime < 1) continue;
            const int eb = entry_bytes_for(Lk.positions);
            // a table too large for shared memory, of filters of at most 4
            // positions, packs 8, 4 or 2 entries into a byte for the
            // specialised kernels, so that it stays in L2
            const bool pack = Lk.positions <= 4 && !req.smag && req.kernel != MPM_KERNEL_GENERIC &&
                              entries * (uint64_t)eb > kSmemTableBudget;
            const int ebits = pack ? (Lk.positions <= 1 ? 1 : Lk.positions <= 2 ? 2 : 4) : 8 * eb;
            const uint64_t tb = pack ? (entries * (uint64_t)ebits + 7) / 8 : entries * (uint64_t)eb;
            if (tb > kMaxTableBytes) continue;
            if (!(req.q && req.sigma_r && req.k) && tb > kAutoTableBytes) continue;
            double rate = candidate_rate(pt, k, Lk.mprime);
            double cost = plan_cost(kind, q, k, rate, tb, ov);
            Plan cand;
            std::memset(&cand, 0, sizeof(cand));
            cand.p = req;
            cand.p.q = q;
            cand.p.sigma_r = sr;
            cand.p.k = k;
            cand.p.map_kind = kind;
            cand.p.map_shift = kind == MPM_MAP_LOWBITS ? shift : 0;
            cand.ell = ell;
            cand.info.L = Lk.L;
            cand.info.mprime = Lk.mprime;
            cand.info.positions = Lk.positions;
            cand.info.entry_bytes = eb;
            cand.info.entry_bits = ebits;
            cand.info.entries = entries;
            cand.info.table_bytes = tb;
            cand.info.est_candidate_rate = rate;
            cand.r = r;
            cand.m = m;
            cand.sigma = sigma;
            if (all) {
                Plan c2 = cand;
                if (c2.p.table_place == MPM_TABLE_AUTO)
                    c2.p.table_place =
                        tb <= kSmemTableBudget ? MPM_TABLE_SMEM : MPM_TABLE_GLOBAL;
                if (!(c2.p.table_place == MPM_TABLE_SMEM && tb > kSmemTableBudget))
                    all->push_back(c2);
            }
            if (!found || cost < best_cost) {
                found = true;
                best_cost = cost;
                best = cand;
            }
        }
    };
    // q-gram hashing: whole q-grams into sigma' bins
    if (want_qhash || req.map_kind == MPM_MAP_AUTO) {
        std::vector<int> bins;
        if (req.sigma_r && want_qhash) {
            bins.push_back(req.sigma_r);
        } else if (!req.sigma_r) {
            for (int b = 10; b <= 16; b++) bins.push_back(1 << b);
        }
        // overlapping q-grams run in the generic kernel, which hashes q <= 5
        const int qmax = ov ? 5 : 8;
        std::vector<int> qs;
        if (req.q) {
            if (req.q <= qmax) qs.push_back(req.q);
        } else {
            for (int q = 2; q <= qmax; q++) qs.push_back(q);
        }
        for (int q : qs) {
            Lengths L1 = lengths(m, q, 1, ov, maxpos);
            if (L1.L < 1) continue;
            const GramStats g = gram_stats(P, r, m, q, h, L1.Lf, ov);
            for (int sr : bins) {
                const int bits = log2_exact(sr);
                std::vector<double> pt = qhash_class_probabilities(g, q, bits);
                consider(MPM_MAP_QHASH, sr, bits, 0, q, (uint64_t)sr, pt, L1);
            }
        }
    }
    if (want_qhash) sigmas.clear();
    for (int sr : sigmas) {
        const int ell = log2_exact(sr);
        // the mapping for this sigma'
        int kind = req.map_kind, shift = 0;
        if (kind == MPM_MAP_AUTO) {
            int bs = best_shift(h, sr);
            bool lossless = lowbits_distinct(h, sr, bs) == std::min(distinct, sr);
            kind = lossless ? MPM_MAP_LOWBITS : MPM_MAP_GREEDY;
            shift = lossless ? bs : 0;
        } else if (kind == MPM_MAP_LOWBITS) {
            shift = req.map_shift >= 0 ? req.map_shift : best_shift(h, sr);
        }
        uint8_t mu[256];
        make_mu(P, r, m, kind, sr, shift, mu);

        std::vector<int> qs;
        if (req.q) {
            qs.push_back(req.q);
        } else {
            // around the paper's q = log_sigma(r m), widened by one below and
            // three above (large sets: packed tables make longer q-grams
            // affordable)
            double q0 = std::log((double)r * (double)m) / std::log((double)sr);
            int lo = std::max(1, (int)std::floor(q0) - 1), hi = (int)std::ceil(q0) + 3;
            for (int q = lo; q <= hi && q <= 16; q++) qs.push_back(q);
        }
        for (int q : qs) {
            if (q * ell > 30) continue;
            Lengths L1 = lengths(m, q, 1, ov, maxpos);
            if (L1.L < 1) continue;
            const uint64_t entries = 1ull << (q * ell);
            // the smallest table this q can have: packed when it has at most
            // 4 positions
            const uint64_t least = L1.Lf <= 4 && !req.smag && req.kernel != MPM_KERNEL_GENERIC
                                       ? (entries * (L1.Lf <= 1 ? 1 : L1.Lf <= 2 ? 2 : 4) + 7) / 8
                                       : entries;
            if (!req.q && least > kAutoTableBytes && q * ell > 26) continue;
            std::vector<double> pt =
                class_probabilities(P, r, m, q, ell, mu, h, L1.Lf, ov);
            consider(kind, sr, ell, shift, q, entries, pt, L1);
        }
    }
    if (!found) return MPM_EINVAL;
    if (best.p.table_place == MPM_TABLE_AUTO)
        best.p.table_place =
            best.info.table_bytes <= kSmemTableBudget ? MPM_TABLE_SMEM : MPM_TABLE_GLOBAL;
    if (best.p.table_place == MPM_TABLE_SMEM && best.info.table_bytes > kSmemTableBudget)
        return MPM_EINVAL;
    best.r = r;
    best.m = m;
    best.sigma = sigma;
    *out = best;
    return MPM_OK;
}

int make_mask_table(const uint8_t* P, const Plan& plan, const uint8_t mu[256],
                    uint8_t* table) {
    const int q = plan.p.q, ell = plan.ell, eb = plan.info.entry_bytes;
    const int ebits = plan.info.entry_bits;
    // clears filter position t of entry c (packed: bit c * ebits + t)
    auto clear = [&](uint64_t c, int t) {
        if (ebits < 8) {
            const uint64_t bit = c * (uint64_t)ebits + (uint64_t)t;
            table[bit >> 3] &= (uint8_t)~(1u << (bit & 7));
        } else {
            table[c * (uint64_t)eb + (uint64_t)(t >> 3)] &= (uint8_t)~(1u << (t & 7));
        }
    };
    const int npos = plan.info.positions;
    const size_t r = plan.r, m = plan.m;
    // position t's q-grams: s + t * stride, s < shifts (see class_probabilities)
    const int shifts = plan.p.overlap ? 1 : q, stride = plan.p.overlap ? 1 : q;
    std::memset(table, 0xFF, plan.info.table_bytes);
    if (plan.p.map_kind == MPM_MAP_QHASH) {
        for (size_t i = 0; i < r; i++)
            for (int s = 0; s < shifts; s++)
                for (int t = 0; t < npos; t++) {
                    const uint32_t c =
                        qgram_bin(raw_qgram(P + i * m + s + t * stride, q), q, ell);
                    clear(c, t);
                }
        return MPM_OK;
    }
    std::vector<uint8_t> red(m);
    for (size_t i = 0; i < r; i++) {
        for (size_t j = 0; j < m; j++) red[j] = mu[P[i * m + j]];
        for (int s = 0; s < shifts; s++) {
            for (int t = 0; t < npos; t++) {
                uint32_t c = msd_code(&red[s + t * stride], q, ell);
                clear(c, t);
            }
        }
    }
    return MPM_OK;
}

namespace {

// The open-addressing table of pattern groups: rows with equal first kb
// bytes are contiguous in lexicographic order and form one group.
void build_slots(HostTables* out, size_t r, int kb, const std::function<const uint8_t*(size_t)>& row) {
    out->key_bytes = kb;
    auto key_of = [&](size_t i, uint64_t* lo, uint64_t* hi) {
        uint8_t buf[16] = {0};
        std::memcpy(buf, row(i), kb);
        std::memcpy(lo, buf, 8);
        std::memcpy(hi, buf + 8, 8);
    };
    std::vector<std::pair<size_t, size_t>> groups;
    for (size_t i = 0; i < r;) {
        size_t j = i + 1;
        while (j < r && std::memcmp(row(i), row(j), kb) == 0) j++;
        groups.push_back({i, j - i});
        i = j;
    }
    size_t nslots = 16;
    while (nslots < 2 * groups.size()) nslots <<= 1;
    out->slots.assign(nslots, Slot{0, 0, 0, 0});
    for (auto& g : groups) {
        uint64_t lo, hi;
        key_of(g.first, &lo, &hi);
        size_t s = key_hash(lo, hi) & (nslots - 1);
        while (out->slots[s].count) s = (s + 1) & (nslots - 1);
        out->slots[s] = Slot{lo, hi, (uint32_t)g.first, (uint32_t)g.second};
    }
}

}  // namespace

int make_verify_tables(const uint8_t* P, size_t r, size_t m, HostTables* out) {
    std::vector<uint32_t> idx(r);
    std::iota(idx.begin(), idx.end(), 0u);
    std::stable_sort(idx.begin(), idx.end(), [&](uint32_t a, uint32_t b) {
        return std::memcmp(P + (size_t)a * m, P + (size_t)b * m, m) < 0;
    });
    out->sorted_pat.resize(r * m);
    out->sorted_pid.resize(r);
    out->sorted_off.clear();
    for (size_t i = 0; i < r; i++) {
        std::memcpy(&out->sorted_pat[i * m], P + (size_t)idx[i] * m, m);
        out->sorted_pid[i] = idx[i];
    }
    const int kb = (int)std::min<size_t>(m, 16);
    build_slots(out, r, kb, [&](size_t i) { return &out->sorted_pat[i * m]; });
    return MPM_OK;
}

int make_verify_tables_var(const uint8_t* cat, const size_t* off, size_t r, size_t mmin,
                           HostTables* out) {
    std::vector<uint32_t> idx(r);
    std::iota(idx.begin(), idx.end(), 0u);
    auto less = [&](uint32_t a, uint32_t b) {
        const size_t la = off[a + 1] - off[a], lb = off[b + 1] - off[b];
        const int c = std::memcmp(cat + off[a], cat + off[b], std::min(la, lb));
        return c != 0 ? c < 0 : la < lb;
    };
    std::stable_sort(idx.begin(), idx.end(), less);
    out->sorted_pat.resize(off[r]);
    out->sorted_pid.resize(r);
    out->sorted_off.resize(r + 1);
    size_t at = 0;
    for (size_t i = 0; i < r; i++) {
        const size_t len = off[idx[i] + 1] - off[idx[i]];
        out->sorted_off[i] = (uint32_t)at;
        std::memcpy(&out->sorted_pat[at], cat + off[idx[i]], len);
        out->sorted_pid[i] = idx[i];
        at += len;
    }
    out->sorted_off[r] = (uint32_t)at;
    const int kb = (int)std::min<size_t>(mmin, 16);
    build_slots(out, r, kb, [&](size_t i) { return &out->sorted_pat[out->sorted_off[i]]; });
    return MPM_OK;
}

std::vector<uint32_t> key_bitmap(const HostTables& t, uint32_t max_bits) {
    uint64_t groups = 0;
    for (const auto& sl : t.slots) groups += sl.count ? 1 : 0;
    uint32_t bits = 1u << 10;
    while (bits < max_bits && bits < 64ull * groups) bits <<= 1;
    std::vector<uint32_t> bm(bits / 32, 0u);
    for (const auto& sl : t.slots) {
        if (!sl.count) continue;
        const uint32_t bit = key_bit(sl.lo, sl.hi, 64u - (uint32_t)__builtin_ctz(bits));
        bm[bit / 32] |= 1u << (bit % 32);
    }
    return bm;
}

}  // namespace mpm

// ------------------------------------------------------- host-only C ABI

extern "C" int mpm_plan(const uint8_t* P, size_t r, size_t m, int sigma,
                        const mpm_params* in, mpm_params* out, mpm_table_info* info) {
    if (!out) return mpm::set_error(MPM_EINVAL);
    mpm::Plan plan;
    int rc = mpm::make_plan(P, r, m, sigma, in, &plan);
    if (rc) return mpm::set_error(rc);
    *out = plan.p;
    if (info) *info = plan.info;
    return mpm::set_error(MPM_OK);
}

extern "C" int mpm_host_tables(const uint8_t* P, size_t r, size_t m, int sigma,
                               const mpm_params* params, uint8_t* mu, void* table,
                               size_t table_bytes) {
    mpm::Plan plan;
    int rc = mpm::make_plan(P, r, m, sigma, params, &plan);
    if (rc) return mpm::set_error(rc);
    uint8_t mu_l[256];
    mpm::make_mu(P, r, m, plan.p.map_kind, plan.p.sigma_r, plan.p.map_shift, mu_l);
    if (mu) std::memcpy(mu, mu_l, 256);
    if (table) {
        if (table_bytes < plan.info.table_bytes) return mpm::set_error(MPM_EINVAL);
        mpm::make_mask_table(P, plan, mu_l, (uint8_t*)table);
    }
    return mpm::set_error(MPM_OK);
}
