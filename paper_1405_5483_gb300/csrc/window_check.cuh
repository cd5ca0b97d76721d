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

// The window T[i..i+m) checked against the pattern set.
static __device__ __noinline__ void check_window(const WindowCtx& c, unsigned int i) {
    unsigned long long lo, hi;
    window_key(c, i, &lo, &hi);
    probe_window(c, i, lo, hi, key_hash(lo, hi));
}

}  // namespace mpm
