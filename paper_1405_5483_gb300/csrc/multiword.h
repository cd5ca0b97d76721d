// Shift-Or state of W 64-bit words, and mask-table entries of the same
// width (Section 3.2: the scan costs ceil((m/q)/w) words of state, w = 64):
// filter bit b is bit b % 64 of word b / 64, an entry's bytes little-endian.
// Used for filters of more than 64 positions by the precompiled generic
// kernels and by the scan compiled at run time, so it has no includes.
#pragma once

namespace mpm {

template <int W>
struct Words {
    unsigned long long w[W];
    Words() = default;
    // the value v in the lowest word, zeros above
    __host__ __device__ Words(unsigned long long v) {
#pragma unroll
        for (int i = 0; i < W; i++) w[i] = i == 0 ? v : 0ull;
    }
    __host__ __device__ explicit operator unsigned int() const { return (unsigned int)w[0]; }
};

template <int W>
__device__ __forceinline__ Words<W> operator~(const Words<W>& a) {
    Words<W> r;
#pragma unroll
    for (int i = 0; i < W; i++) r.w[i] = ~a.w[i];
    return r;
}

template <int W>
__device__ __forceinline__ Words<W> operator|(const Words<W>& a, const Words<W>& b) {
    Words<W> r;
#pragma unroll
    for (int i = 0; i < W; i++) r.w[i] = a.w[i] | b.w[i];
    return r;
}

template <int W>
__device__ __forceinline__ Words<W> operator&(const Words<W>& a, const Words<W>& b) {
    Words<W> r;
#pragma unroll
    for (int i = 0; i < W; i++) r.w[i] = a.w[i] & b.w[i];
    return r;
}

template <int W>
__device__ __forceinline__ Words<W>& operator&=(Words<W>& a, const Words<W>& b) {
    a = a & b;
    return a;
}

// a << s for 0 <= s < 64 (the Shift-Or step shifts by k <= 32)
template <int W>
__device__ __forceinline__ Words<W> operator<<(const Words<W>& a, int s) {
    Words<W> r;
#pragma unroll
    for (int i = W - 1; i >= 0; i--) {
        const unsigned long long carry = (i > 0 && s > 0) ? a.w[i - 1] >> (64 - s) : 0ull;
        r.w[i] = (a.w[i] << s) | carry;
    }
    return r;
}

// The 32 bits of a starting at bit pos (0 <= pos < 64 W); bits above the
// top word read as zero.  The word index is selected without indexing the
// array at run time, so the state stays in registers.
template <int W>
__device__ __forceinline__ unsigned int bits_at(const Words<W>& a, int pos) {
    const int j = pos >> 6, b = pos & 63;
    unsigned long long lo = 0, hi = 0;
#pragma unroll
    for (int i = 0; i < W; i++) {
        if (i == j) lo = a.w[i];
        if (i == j + 1) hi = a.w[i];
    }
    const unsigned long long v = b ? ((lo >> b) | (hi << (64 - b))) : lo;
    return (unsigned int)v;
}

// The same for one 32- or 64-bit word of state (pos below its width).
template <typename T>
__device__ __forceinline__ unsigned int bits_at(T a, int pos) {
    return (unsigned int)(a >> pos);
}

}  // namespace mpm
