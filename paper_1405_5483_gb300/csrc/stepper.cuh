// The generic per-thread stepper of the MAG scan: a 64-bit window of the
// last text bytes (or of their reduced symbols), the q-gram code of a
// sampled q-gram cut from it, and the Shift-Or state D (Sections 3.1, 3.2).
// Used by the generic single-text scan (scan.cu) and the batched scan
// (batch.cu), whose q, k and mapping are runtime values.
#pragma once

#include <cstdint>
#include <type_traits>

#include "device_common.cuh"
#include "multiword.h"

namespace mpm {

enum ScanMode : int {
    kLow2 = 0,    // low-bit map with 2 bits: the multiply trick of Section 3.3
    kLowG = 1,    // low-bit map, any width
    kLutRed = 2,  // byte map mu on every byte, reduced-symbol window
    kLutRaw = 3,  // raw-byte window, mu on the q bytes of sampled q-grams (q <= 5)
    kQHash = 4    // raw-byte window, whole q-gram hashed to a bin (q <= 5)
};

// Shift-Or state of more than one 64-bit word: Words<W> (multiword.h), the
// mask-table entries of the same width (8 W bytes), for filters of up to
// 64 W positions.
template <typename ET>
struct StateOf {  // the Shift-Or state type for table entries of type ET
    using type = typename std::conditional<sizeof(ET) == 8, uint64_t, uint32_t>::type;
};
template <int W>
struct StateOf<Words<W>> {
    using type = Words<W>;
};

template <int MODE, typename ET>
struct Stepper {
    using DT = typename StateOf<ET>::type;
    const ET* tab;
    const uint8_t* smu;
    int q, k, ell, shift, raw_base;
    uint32_t qmask, lowmask4;
    uint64_t W;
    DT D;

    __device__ __forceinline__ void push(uint32_t x) {
        if (MODE == kLow2) {
            uint32_t y = (x >> shift) & lowmask4;
            W = (W << 8) | ((y * 0x40100401u) >> 24);
        } else if (MODE == kLowG) {
            uint32_t y = (x >> shift) & lowmask4;
            uint32_t v = ((y & 0xFFu) << (3 * ell)) | (((y >> 8) & 0xFFu) << (2 * ell)) |
                         (((y >> 16) & 0xFFu) << ell) | (y >> 24);
            W = (W << (4 * ell)) | v;
        } else if (MODE == kLutRed) {
            uint32_t v = ((uint32_t)smu[x & 0xFFu] << (3 * ell)) |
                         ((uint32_t)smu[(x >> 8) & 0xFFu] << (2 * ell)) |
                         ((uint32_t)smu[(x >> 16) & 0xFFu] << ell) | (uint32_t)smu[x >> 24];
            W = (W << (4 * ell)) | v;
        } else {  // kLutRaw, kQHash: raw bytes, the newest word on top
            W = (W >> 32) | ((uint64_t)x << 32);
        }
    }

    // Code of the q-gram that ends e bytes before the end of the last word.
    __device__ __forceinline__ uint32_t code(int e) const {
        if (MODE == kQHash) {
            uint64_t raw = W >> (raw_base - 8 * e);
            if (q < 8) raw &= (1ull << (8 * q)) - 1;
            return qgram_bin(raw, q, ell);
        } else if (MODE == kLutRaw) {
            uint64_t raw = W >> (raw_base - 8 * e);
            uint32_t c = 0;
#pragma unroll
            for (int u = 0; u < 5; u++)
                if (u < q) c = (c << ell) | smu[(raw >> (8 * u)) & 0xFFu];
            return c;
        } else {
            return (uint32_t)(W >> (e * ell)) & qmask;
        }
    }

    __device__ __forceinline__ void init(const FilterDev& f, const ET* t, const uint8_t* mu_s) {
        tab = t;
        smu = mu_s;
        q = f.q;
        k = f.k;
        ell = f.ell;
        shift = f.shift;
        raw_base = 8 * (8 - f.q);
        qmask = (f.q * f.ell >= 32) ? 0xFFFFFFFFu : ((1u << (f.q * f.ell)) - 1u);
        // per byte: the ell bits above the shift, never bits of the next byte
        lowmask4 = (((1u << f.ell) - 1u) & (0xFFu >> f.shift)) * 0x01010101u;
        W = 0;
        D = ~(DT)0;
    }
};

// Little-endian word of T[at..at+4) (all four bytes inside the text); byte
// loads when the address is not 4-byte aligned.
__device__ __forceinline__ uint32_t load_word(const uint8_t* T, uint64_t at) {
    const uint8_t* p = T + at;
    if ((reinterpret_cast<uintptr_t>(p) & 3) == 0) return ldg_u32(p);
    return (uint32_t)p[0] | ((uint32_t)p[1] << 8) | ((uint32_t)p[2] << 16) | ((uint32_t)p[3] << 24);
}

template <typename DT>
__device__ __forceinline__ uint32_t fired_bits(DT D, int rsh, uint32_t kmask) {
    return ~bits_at(D, rsh) & kmask;
}

// Warm-up over the bytes [row_start - Wr, row_start): builds D from the
// sampled q-grams that precede the row (positions before the text are
// virtual and leave D's bits at one).  Uniform across lanes.
template <int MODE, typename ET>
__device__ __forceinline__ void warm_up(Stepper<MODE, ET>& st, const uint8_t* T, uint32_t n,
                                        uint32_t row_start, uint32_t Wr, uint32_t P, bool valid) {
    using DT = typename Stepper<MODE, ET>::DT;
    const int q = st.q, k = st.k;
    const int64_t a0 = (int64_t)row_start - (int64_t)Wr;
    const int tmax = (int)(((k - 1) * q + (int)Wr) / (int)P);
    int nxt = (int)P * (1 - tmax) + (int)Wr;
    int64_t hs = (int64_t)(row_start / (uint32_t)q) + (k - 1) - (int64_t)tmax * k;
    for (uint32_t w = 0; w < Wr / 4; w++) {
        const int64_t addr = a0 + 4 * (int64_t)w;
        uint32_t x = 0;
        if (valid && addr >= 0 && addr + 4 <= (int64_t)n) x = load_word(T, (uint64_t)addr);
        st.push(x);
        const int pos = 4 * (int)(w + 1);
        while (nxt <= pos) {
            const uint32_t c = st.code(pos - nxt);
            const DT b = (hs >= 0) ? (DT)st.tab[c] : ~(DT)0;
            st.D = (st.D << k) | b;
            nxt += (int)P;
            hs += k;
        }
    }
}

}  // namespace mpm
