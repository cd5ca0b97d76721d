// Exact check of one text window against the pattern set (Section 3.2:
// verification, in the original alphabet of Section 3.3).  Shared by the
// verification kernel and the specialised scan that verifies by itself, so
// it has no includes (NVRTC takes it as text).
#pragma once

namespace mpm {

struct WindowCtx {
    const unsigned char* T;
    unsigned int n, m, key_bytes, slot_mask, occ_cap;
    const Slot* slots;
    const unsigned char* pat;     // patterns sorted by bytes, r * m
    const unsigned int* pid;      // pattern id of each sorted row
    const unsigned int* off;      // null: rows of m bytes; else row i is
                                  // pat[off[i] .. off[i+1]) (lengths >= m)
    unsigned long long* occ;      // tag | (pos << pos_shift) | pid
    unsigned int* occ_count;
    unsigned long long tag;       // 0 for one text; the text id's bits in a batch
    unsigned int pos_shift;       // 32 for one text; 20 in a batch
};

// The first key_bytes (<= 16) bytes of T[i..) as two little-endian words.
// Away from the end of the text: three (key of at most 8 bytes) or five
// independent aligned word loads and funnel shifts; near the end: byte loads.
__device__ __forceinline__ void window_key(const WindowCtx& c, unsigned int i,
                                           unsigned long long* lo, unsigned long long* hi) {
    const unsigned char* w = c.T + i;
    if ((unsigned long long)i + 20 <= c.n) {
        const unsigned long long a = reinterpret_cast<unsigned long long>(w);
        const unsigned int* b = reinterpret_cast<const unsigned int*>(a & ~3ull);
        const unsigned int sh = (unsigned int)(a & 3) * 8;
        const bool wide = c.key_bytes > 8;
        const unsigned int x0 = __ldg(b), x1 = __ldg(b + 1), x2 = __ldg(b + 2);
        const unsigned int x3 = wide ? __ldg(b + 3) : 0u, x4 = wide ? __ldg(b + 4) : 0u;
        unsigned long long l = (unsigned long long)__funnelshift_r(x0, x1, sh) |
                               ((unsigned long long)__funnelshift_r(x1, x2, sh) << 32);
        unsigned long long h = (unsigned long long)__funnelshift_r(x2, x3, sh) |
                               ((unsigned long long)__funnelshift_r(x3, x4, sh) << 32);
        const unsigned int kb = c.key_bytes;
        if (kb < 16) {
            if (kb <= 8) {
                h = 0;
                if (kb < 8) l &= (1ull << (8 * kb)) - 1;
            } else {
                h &= (1ull << (8 * (kb - 8))) - 1;
            }
        }
        *lo = l;
        *hi = h;
        return;
    }
    unsigned long long l = 0, h = 0;
    for (unsigned int u = 0; u < c.key_bytes; u++) {
        const unsigned long long x = __ldg(w + u);
        if (u < 8)
            l |= x << (8 * u);
        else
            h |= x << (8 * (u - 8));
    }
    *lo = l;
    *hi = h;
}

// Looks the window T[i..i+m), whose key is (lo, hi) and key hash h, up
// among the pattern groups and appends tag | (i << pos_shift) | pid for
// every pattern equal to the text there (for patterns of different lengths,
// each compared over its own length; m is then the shortest).
static __device__ __forceinline__ void probe_window(const WindowCtx& c, unsigned int i,
                                                    unsigned long long lo, unsigned long long hi,
                                                    unsigned long long h) {
    unsigned int slot = (unsigned int)h & c.slot_mask;
    for (unsigned int probes = 0; probes <= c.slot_mask; probes++) {
        const Slot sl = c.slots[slot];
        if (sl.count == 0) return;
        if (sl.lo == lo && sl.hi == hi) {
            const unsigned char* w = c.T + i;
            for (unsigned int row = sl.first; row < sl.first + sl.count; row++) {
                const unsigned char* p;
                unsigned int len;
                if (c.off) {  // patterns of different lengths: each its own
                    p = c.pat + c.off[row];
                    len = c.off[row + 1] - c.off[row];
                    if ((unsigned long long)i + len > c.n) continue;
                } else {
                    p = c.pat + (unsigned long long)row * c.m;
                    len = c.m;
                }
                unsigned int u = c.key_bytes;
                while (u < len && __ldg(w + u) == __ldg(p + u)) u++;
                if (u == len) {
                    const unsigned int idx = atomicAdd(c.occ_count, 1u);
                    if (idx < c.occ_cap)
                        c.occ[idx] = c.tag | ((unsigned long long)i << c.pos_shift) | c.pid[row];
                }
            }
            return;
        }
        slot = (slot + 1) & c.slot_mask;
    }
}

// The text starts first .. end (first <= end) of one candidate, in ascending
// order: the key of each start (the first key_bytes bytes of its window) is
// tested against the key bitmap `keys` (key_mask + 1 bits, the bit key_bit
// of every pattern group's key set), and only a set bit probes the groups.  The keys of all the starts lie in end - first + key_bytes
// bytes; when these fit the aligned 24 (keys of at most 8 bytes) or 32 bytes
// around them they are read with three or four independent 8-byte loads, so
// the walk waits for memory once, and each next key is that window shifted
// by a byte.  Otherwise the first key is read whole and each next one takes
// in the byte after it.  KW: 1 for keys of at most 8 bytes, 2 for longer
// keys, 0 to decide from key_bytes at run time.
template <int KW = 0>
static __device__ __forceinline__ void check_starts(const WindowCtx& c, unsigned int first,
                                                    unsigned int end, const unsigned int* keys,
                                                    unsigned int key_mask) {
    const unsigned int kb = c.key_bytes;  // 1 .. 16
    const bool narrow = KW == 1 || (KW == 0 && kb <= 8);
    const unsigned long long tb = reinterpret_cast<unsigned long long>(c.T);
    const unsigned long long ad = tb + first;
    const unsigned long long ab = ad & ~7ull;
    const unsigned int span = narrow ? 24u : 32u;
    const unsigned int kshift = 64u - (unsigned int)__popc(key_mask);
    if (end - first + kb + 7 <= span && ab >= tb && ab + span <= tb + c.n) {
        const unsigned long long* p = reinterpret_cast<const unsigned long long*>(ab);
        const unsigned long long x0 = __ldg(p), x1 = __ldg(p + 1), x2 = __ldg(p + 2);
        const unsigned long long x3 = narrow ? 0ull : __ldg(p + 3);
        // bytes first .. in a (lowest), b, d; (x << (63 - s)) << 1 is
        // x << (64 - s), and 0 for s = 0
        const unsigned int s8 = (unsigned int)(ad - ab) * 8;
        unsigned long long a = (x0 >> s8) | ((x1 << (63 - s8)) << 1);
        unsigned long long b = (x1 >> s8) | ((x2 << (63 - s8)) << 1);
        unsigned long long d = narrow ? 0ull : (x2 >> s8) | ((x3 << (63 - s8)) << 1);
        const unsigned long long lom = kb >= 8 ? ~0ull : (1ull << (8 * kb)) - 1;
        const unsigned long long him =
            kb <= 8 ? 0ull : (kb >= 16 ? ~0ull : (1ull << (8 * (kb - 8))) - 1);
        for (unsigned int i = first;; i++) {
            const unsigned long long lo = a & lom;
            const unsigned long long hi = narrow ? 0ull : b & him;
            const unsigned int bit = narrow ? key_bit(lo, 0ull, kshift) : key_bit(lo, hi, kshift);
            if ((keys[bit >> 5] >> (bit & 31)) & 1u) probe_window(c, i, lo, hi, key_hash(lo, hi));
            if (i >= end) break;
            a = (a >> 8) | (b << 56);
            if (narrow) {
                b >>= 8;
            } else {
                b = (b >> 8) | (d << 56);
                d >>= 8;
            }
        }
        return;
    }
    const unsigned int top = 8 * ((kb - 1) & 7);  // bit offset of a key's last byte
    unsigned int i = first;
    unsigned long long lo, hi;
    window_key(c, i, &lo, &hi);
    for (;;) {
        const unsigned int bit = key_bit(lo, hi, kshift);
        if ((keys[bit >> 5] >> (bit & 31)) & 1u) probe_window(c, i, lo, hi, key_hash(lo, hi));
        if (i >= end) break;
        // i + kb <= i + m - 1 < n: the byte after the key is in the text
        const unsigned long long nb = __ldg(c.T + i + kb);
        lo = (lo >> 8) | (hi << 56);
        hi >>= 8;
        if (kb <= 8)
            lo |= nb << top;
        else
            hi |= nb << top;
        i++;
    }
}

// The window T[i..i+m) checked against the pattern set.
static __device__ __noinline__ void check_window(const WindowCtx& c, unsigned int i) {
    unsigned long long lo, hi;
    window_key(c, i, &lo, &hi);
    probe_window(c, i, lo, hi, key_hash(lo, hi));
}

}  // namespace mpm
