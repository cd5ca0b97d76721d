// The stage primitives of the specialised scan (Sections 3.1, 3.2): the
// filter's constants, the reduced symbols of a text word, the code of a
// sampled q-gram at a fixed offset, one mask-table lookup and the Shift-Or
// step over a stage of C bytes held in registers.  Compiled at run time
// (NVRTC) inside a namespace, with these macros defined:
//   MPM_Q, MPM_K      q-gram length and sampling step
//   MPM_MP            AOSO subpattern length m' (filter positions k*m')
//   MPM_ELL, MPM_SHIFT reduced symbol width log2(sigma') and, for the
//                     low-bit map, the right shift applied to each byte
//   MPM_MODE          0: low-bit map (Section 3.3, combined mapping and
//                     q-gram generation), 1: byte map mu through a table,
//                     2: whole q-grams hashed to 2^MPM_ELL bins (Section 3.3,
//                     alphabet mapping on the q-grams)
//   MPM_EB            bytes per mask-table entry (1, 2, 4, 8; 16, 24, 32 for
//                     2 - 4 words of Shift-Or state, multiword.h)
//   MPM_EBITS         bits per entry: 8 MPM_EB (default), or 1, 2, 4 for a
//                     packed table (entry c at bit c * MPM_EBITS, MPM_EB = 1)
//   MPM_SMEM          1: the table pointer may be read as is (shared memory,
//                     or a generic pointer); 0: global memory, read with an
//                     L2 policy
//   MPM_C             bytes of a stage: a multiple of 16 and of P
//   MPM_STAGES        1 (default); 0 when the stage functions are not used
//                     (a batch set whose sampling period has no stage of at
//                     most 256 bytes): the stage constants are then unchecked
//   MPM_OV            0: MAG's non-overlapping q-grams of all q shifts;
//                     1: the overlapping q-grams of Section 2 (the text's
//                     q-gram at every byte, every k-th read, a window at its
//                     own start)
// The single-text scan (scan_jit.cuh) includes it once; the batched kernel
// (batch_jit.cuh) once per parameter set of its batch, each in a namespace
// of its own.

constexpr int Q = MPM_Q, K = MPM_K, MP = MPM_MP, ELL = MPM_ELL, SHIFT = MPM_SHIFT;
constexpr bool OV = MPM_OV != 0;
constexpr int P = OV ? K : Q * K;  // text bytes per sampled q-gram
constexpr int VQ = OV ? 1 : Q;     // text starts a window stands for
constexpr int C = MPM_C;
constexpr int NS = C / P;
// overlapping q-grams: words before a stage that hold the first bytes of its
// samples, and the offset of the last byte of its first sample
constexpr int TW = OV ? (Q + 2) / 4 : 0;
constexpr int E0 = OV ? (K + Q - 2) % K : 0;
// bytes of the samples that precede a row
constexpr int WB = OV ? (MP - 1) * K + Q - 1 : (MP - 1) * P;
constexpr int WSTAGES = (WB + C - 1) / C;
constexpr int RSH = (MP - 1) * K;
constexpr u32 KMASK = K >= 32 ? 0xFFFFFFFFu : ((1u << K) - 1u);
constexpr u32 QMASK = Q * ELL >= 32 ? 0xFFFFFFFFu : ((1u << (Q * ELL)) - 1u);
constexpr u32 SYMMASK = ((1u << ELL) - 1u) & (0xFFu >> SHIFT);

#if MPM_EB == 1
typedef u8 ET;
#elif MPM_EB == 2
typedef u16 ET;
#elif MPM_EB == 4
typedef u32 ET;
#elif MPM_EB == 8
typedef u64 ET;
#else
typedef Words<MPM_EB / 8> ET;  // more than 64 positions: several words
#endif
#if MPM_EB > 8
typedef Words<MPM_EB / 8> DT;
#else
typedef Cond<(MPM_EB == 8), u64, u32>::T DT;
#endif
typedef Cond<(OV || NS * K > 32), u64, u32>::T FT;
// overlapping q-grams: samples per 64-bit word of report bits, and words
constexpr int SPW = 64 / K;
constexpr int FW = (NS + SPW - 1) / SPW;

#ifndef MPM_STAGES
#define MPM_STAGES 1
#endif
static_assert(!MPM_STAGES || (C % 16 == 0 && C % P == 0), "stage bytes");
static_assert(!MPM_STAGES || OV || NS * K <= 64, "fired mask");
static_assert(!OV || 4 * TW >= Q - 1, "tail words");

// Reduced symbols of the four bytes of a word, first byte most significant.
__device__ __forceinline__ u32 pack_word(u32 x) {
    if (ELL == 2) {
        const u32 y = (x >> SHIFT) & (SYMMASK * 0x01010101u);
        return (y * 0x40100401u) >> 24;  // the multiply trick of Section 3.3
    } else if (ELL == 1) {
        const u32 y = (x >> SHIFT) & (SYMMASK * 0x01010101u);
        return (y * 0x80402010u) >> 28;
    } else if (ELL == 4) {
        const u32 y = (x >> SHIFT) & (SYMMASK * 0x01010101u);
        const u32 z = __byte_perm(y, 0, 0x0123);
        const u32 t = (z & 0x000F000Fu) | ((z >> 4) & 0x00F000F0u);
        return (t & 0xFFu) | ((t >> 8) & 0xFF00u);
    } else {
        u32 v = 0;
#pragma unroll
        for (int j = 0; j < 4; j++) v = (v << ELL) | ((x >> (8 * j + SHIFT)) & SYMMASK);
        return v;
    }
}

// Code of the q-gram at byte offset o of the stage (o constant after
// unrolling), first symbol most significant.
__device__ __forceinline__ u32 code_at(const u32* w, const u32* rw, const u8* smu, int o) {
    if (MPM_MODE == 2) {
        // the q raw bytes at o, little-endian, from at most three words
        const int first = o >> 2, last = (o + Q - 1) >> 2, sh = 8 * (o & 3);
        u64 a = w[first];
        if (first + 1 <= last) a |= (u64)w[first + 1] << 32;
        u64 raw = a >> sh;
        if (first + 2 <= last) raw |= (u64)w[first + 2] << (64 - sh);
        if (Q < 8) raw &= (1ull << (8 * Q)) - 1;
        return qgram_bin(raw, Q, ELL);
    } else if (MPM_MODE == 0) {
        const int first = o >> 2, last = (o + Q - 1) >> 2;
        u64 acc = 0;
#pragma unroll
        for (int i = first; i <= last; i++) acc = (acc << (4 * ELL)) | rw[i];
        const int after = (last + 1) * 4 - (o + Q);
        return (u32)(acc >> (after * ELL)) & QMASK;
    } else {
        u32 c = 0;
#pragma unroll
        for (int t = 0; t < Q; t++) {
            const int p = o + t;
            const u32 b = (w[p >> 2] >> (8 * (p & 3))) & 0xFFu;
            c = (c << ELL) | smu[b];
        }
        return c;
    }
}

// Mask-table entry c: from shared memory, or from global memory with an
// evict_last L2 policy (pol), so that the streamed text, loaded with
// evict_first, does not push a table read at random out of L2.
#ifndef MPM_EBITS
#define MPM_EBITS (8 * MPM_EB)
#endif
__device__ __forceinline__ DT entry(const ET* tab, u32 c, u64 pol) {
#if MPM_EBITS < 8
    // packed: the entry's bits within its byte (q l <= 30, so c * bits < 2^32)
    const u32 bit = c * (u32)MPM_EBITS;
    const u8* t8 = reinterpret_cast<const u8*>(tab) + (bit >> 3);
#if MPM_SMEM
    (void)pol;
    const u32 byte = *t8;
#else
    const u32 byte = ldg_hint_u8(t8, pol);
#endif
    return (DT)((byte >> (bit & 7u)) & ((1u << MPM_EBITS) - 1u));
#elif MPM_SMEM || MPM_EB > 8
    (void)pol;
    return (DT)tab[c];
#elif MPM_EB == 1
    return (DT)ldg_hint_u8(reinterpret_cast<const u8*>(tab) + c, pol);
#elif MPM_EB == 2
    return (DT)ldg_hint_u16(reinterpret_cast<const u16*>(tab) + c, pol);
#elif MPM_EB == 4
    return (DT)ldg_hint_u32(reinterpret_cast<const u32*>(tab) + c, pol);
#else
    return (DT)ldg_hint_u64(reinterpret_cast<const u64*>(tab) + c, pol);
#endif
}

// One stage of C bytes: the NS sampled q-grams fold into D; with REPORT the
// report bits after each go into fm (k bits per sample).
template <bool REPORT>
__device__ __forceinline__ void run_stage(const u32* w, DT& D, FT& fm, const ET* tab,
                                          const u8* smu, u64 pol) {
    u32 rw[C / 4];
    if (MPM_MODE == 0) {
#pragma unroll
        for (int i = 0; i < C / 4; i++) rw[i] = pack_word(w[i]);
    }
#pragma unroll
    for (int u = 0; u < NS; u++) {
        const u32 c = code_at(w, rw, smu, u * P + (K - 1) * Q);
        D = (D << K) | entry(tab, c, pol);
        if (REPORT) fm |= ((FT)(~bits_at(D, RSH) & KMASK)) << (u * K);
    }
}

// Overlapping q-grams: the NS samples of a stage, the q-gram of sample u
// starting at byte TW*4 + E0 - (q-1) + u*k of x (the TW words before the
// stage, then its C/4 words; rx: their reduced symbols for the low-bit map).
// Every D is ANDed into acc, so a zero report bit of acc means that some
// sample of the stage fired.
__device__ __forceinline__ void run_stage_ov(const u32* x, const u32* rx, DT& D, DT& acc,
                                             const ET* tab, const u8* smu, u64 pol) {
#pragma unroll
    for (int u = 0; u < NS; u++) {
        const u32 c = code_at(x, rx, smu, TW * 4 + E0 - (Q - 1) + u * K);
        D = (D << K) | entry(tab, c, pol);
        acc &= D;
    }
}

// The same stage again from D0, with the report bits of sample u in word
// u / SPW of fm, bits (u % SPW) k ..; hs0 = h - (m'-1)k of sample 0 (h its
// start byte): a window h - (m'-1)k - j before the text start is dropped.
__device__ __forceinline__ void fired_stage_ov(const u32* x, const u32* rx, DT D, FT* fm,
                                               i64 hs0, const ET* tab, const u8* smu, u64 pol) {
#pragma unroll
    for (int w = 0; w < FW; w++) fm[w] = 0;
#pragma unroll
    for (int u = 0; u < NS; u++) {
        const u32 c = code_at(x, rx, smu, TW * 4 + E0 - (Q - 1) + u * K);
        D = (D << K) | entry(tab, c, pol);
        u32 f = ~bits_at(D, RSH) & KMASK;
        const i64 hs = hs0 + (i64)u * K;
        if (hs < K - 1) f &= hs < 0 ? 0u : ((1u << (u32)(hs + 1)) - 1u);
        fm[u / SPW] |= (FT)f << ((u % SPW) * K);
    }
}

// The q-gram code of text bytes [st, st + q) read with byte loads.
__device__ __forceinline__ u32 code_bytes(const u8* T, u32 st, const u8* smu) {
    if (MPM_MODE == 2) {
        u64 raw = 0;
#pragma unroll
        for (int t = 0; t < Q; t++) raw |= (u64)__ldg(T + st + t) << (8 * t);
        return qgram_bin(raw, Q, ELL);
    }
    u32 c = 0;
#pragma unroll
    for (int t = 0; t < Q; t++) {
        const u32 b = __ldg(T + st + t);
        const u32 s = (MPM_MODE == 0) ? ((b >> SHIFT) & SYMMASK) : (u32)smu[b];
        c = (c << ELL) | s;
    }
    return c;
}
