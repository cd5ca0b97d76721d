// Specialised MAG scan: the fused encode + average-optimal Shift-Or filter
// of Sections 3.1 and 3.2 with the filter's parameters compiled in.  This
// file is compiled at run time (NVRTC) once per parameter set, after
// scan_jit_args.h and ptx_common.cuh, with these macros defined:
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
//   MPM_SMEM          1: mask table copied to shared memory
//   MPM_TABLE_BYTES   mask-table bytes (padded to 16)
//   MPM_C             bytes of a row per stage: a multiple of 16 and of k*q
//   MPM_S, MPM_WARPS  stages per warp, warps per block
//   MPM_VERIFY        1: verify the candidates in the kernel and append
//                     occurrences; 0: append the candidate records
//   MPM_EMIT_CAP      records a warp buffers in shared memory
//   MPM_OV            0: MAG's non-overlapping q-grams of all q shifts;
//                     1: the overlapping q-grams of Section 2 (the text's
//                     q-gram at every byte, every k-th read, a window at its
//                     own start)
//
// Layout and flow.  Rows of Lst bytes (a multiple of C, starting on a
// multiple of k*q) are owned by threads; a warp streams its 32 rows through
// shared memory with 2-D TMA boxes of 32 rows x C bytes, MPM_S stages deep,
// on its own mbarriers.  Because C is a multiple of P = k*q, every stage
// holds exactly C/P sampled q-grams at the same byte offsets: the sampled
// q-gram u of a stage is bytes [u*P + (k-1)*q, (u+1)*P).  The per-stage loop
// is therefore straight-line code with constant offsets: cut the q-gram
// code, one table lookup, D <- (D << k) | B[code], and the k report bits of
// D go into a per-stage bit mask.  Only after the stage, if some lane of the
// warp has a bit set, are records (fired << 32) | h appended to the warp's
// buffer in shared memory.  A full buffer is flushed: either copied out with
// one atomicAdd, or (MPM_VERIFY) verified by the warp on the spot -- every
// window the records stand for is looked up in the pattern-group table and
// compared byte by byte (Section 3.2), while the text is still in L2.  The
// bytes after the last full row are scanned by the last lanes of the grid
// with plain loads while the other warps stream rows.
//
// Overlapping q-grams (MPM_OV).  The sampled q-grams start at the bytes
// h = k-1 (mod k), one every k bytes, so a stage of C bytes (a multiple of k)
// holds C/k of them at fixed offsets: those whose last byte lies in the
// stage, their first bytes possibly in the TW words before it, which a lane
// keeps in registers from its previous stage.  The hot loop only folds the
// lookups into D and ANDs every D into one word; only when a report bit of
// that word is zero for some lane (rare: this filter is chosen for its low
// candidate rate) does the warp run the stage again from the saved D to find
// which samples fired.

typedef unsigned char u8;
typedef unsigned short u16;
typedef unsigned int u32;
typedef unsigned long long u64;
typedef long long i64;

namespace mpm {

template <bool B, class X, class Y>
struct Cond {
    typedef X T;
};
template <class X, class Y>
struct Cond<false, X, Y> {
    typedef Y T;
};

constexpr int Q = MPM_Q, K = MPM_K, MP = MPM_MP, ELL = MPM_ELL, SHIFT = MPM_SHIFT;
constexpr bool OV = MPM_OV != 0;
constexpr int P = OV ? K : Q * K;  // text bytes per sampled q-gram
constexpr int VQ = OV ? 1 : Q;     // text starts a window stands for
constexpr int C = MPM_C;
constexpr int NS = C / P;
constexpr int S = MPM_S;
constexpr int WARPS = MPM_WARPS;
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
constexpr u32 SLOT = 32u * C;

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

enum { kCandCountJ = 0, kOccCountJ = 1, kErrorFlagJ = 2 };
constexpr u32 ECAP = MPM_EMIT_CAP;
static_assert(ECAP >= 64, "emit buffer");

static_assert(C % 16 == 0 && C % P == 0, "stage bytes");
static_assert(OV || NS * K <= 64, "fired mask");
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
__device__ __forceinline__ DT entry(const ET* tab, u32 c, u64 pol) {
#if MPM_SMEM || MPM_EB > 8
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

// The windows of one record (sampled q-gram h, report bits `fired`) at
// shift s: window h0 = h - (m'-1)k - j stands for the text start h0*q - s
// (overlapping q-grams: h is a byte, and the window starts at h0).
__device__ __forceinline__ WindowCtx window_ctx(const JitScanArgs& A) {
    WindowCtx c;
    c.T = A.T;
    c.n = A.n;
    c.m = A.m;
    c.key_bytes = A.key_bytes;
    c.slot_mask = A.slot_mask;
    c.occ_cap = A.occ_cap;
    c.slots = reinterpret_cast<const Slot*>(A.slots);
    c.pat = A.pat;
    c.pid = A.pid;
    c.off = A.pat_off;
    c.occ = A.occ;
    c.occ_count = &A.counters[kOccCountJ];
    c.tag = 0;
    c.pos_shift = 32;
    return c;
}

__device__ __forceinline__ void verify_record(const JitScanArgs& A, u32 h, u32 fired, int s) {
    const WindowCtx c = window_ctx(A);
    while (fired) {
        const int j = __ffs((int)fired) - 1;
        fired &= fired - 1;
        const i64 i = ((i64)h - RSH - j) * VQ - s;
        if (i < 0 || i + (i64)A.m > (i64)A.n) continue;
        check_window(c, (u32)i);
    }
}

// A warp's buffer of candidate records in shared memory (count warp-uniform).
struct Emitter {
    u64* buf;
    u32 n;
};

__device__ __forceinline__ void flush(Emitter& E, const JitScanArgs& A) {
    if (E.n == 0) return;
    __syncwarp();
    const int lane = threadIdx.x & 31;
#if MPM_VERIFY
    if (lane == 0) atomicAdd(&A.counters[kCandCountJ], E.n);
    const u32 items = E.n * (u32)VQ;
    for (u32 t = lane; t < items; t += 32) {
        const u64 rec = E.buf[t / VQ];
        verify_record(A, (u32)rec, (u32)(rec >> 32), (int)(t % VQ));
    }
#else
    u32 base = 0;
    if (lane == 0) base = atomicAdd(&A.counters[kCandCountJ], E.n);
    base = __shfl_sync(0xFFFFFFFFu, base, 0);
    for (u32 i = lane; i < E.n; i += 32)
        if (base + i < A.cap) A.cand[base + i] = E.buf[i];
#endif
    __syncwarp();
    E.n = 0;
}

// Buffers the records of one stage: for every lane, every sample u with
// report bits, ((bits) << 32) | (h1 + u*k), h1 the stage's first sample.
__device__ __forceinline__ void emit_stage(FT fm, u32 h1, Emitter& E, const JitScanArgs& A) {
    while (true) {
        const bool has = fm != 0;
        const u32 bal = __ballot_sync(0xFFFFFFFFu, has);
        if (bal == 0) break;
        if (E.n + 32 > ECAP) flush(E, A);
        if (has) {
            const int bit = (sizeof(FT) == 8) ? (__ffsll((long long)fm) - 1) : (__ffs((int)fm) - 1);
            const int u = bit / K;
            const u32 fired = (u32)(fm >> (u * K)) & KMASK;
            fm &= ~((FT)KMASK << (u * K));
            const u32 h = h1 + (u32)(u * K);
            E.buf[E.n + __popc(bal & lanemask_lt())] = ((u64)fired << 32) | h;
        }
        E.n += __popc(bal);
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

struct __align__(64) TmapParam {
    u64 v[16];
};

extern "C" __global__ void __launch_bounds__(MPM_WARPS * 32, 1)
    mpm_scan_jit(const JitScanArgs A, const __grid_constant__ TmapParam tmap) {
    extern __shared__ __align__(128) u8 smem[];
    // shared layout: [mask table?][mu, 256][mbarriers][emit buffers]
    //                [stages, 128-aligned]
    constexpr u32 TAB = MPM_SMEM ? MPM_TABLE_BYTES : 0u;
    constexpr u32 EMIT_OFF = TAB + 256u + 8u * WARPS * S;
    constexpr u32 STAGE_OFF = (EMIT_OFF + 8u * WARPS * ECAP + 127u) / 128u * 128u;
    u8* s_tab = smem;
    u8* s_mu = smem + TAB;
    u64* s_bar = reinterpret_cast<u64*>(s_mu + 256);
    u8* s_stage = smem + STAGE_OFF;

    if (TAB) {
        for (u32 i = threadIdx.x; i < TAB / 16; i += blockDim.x)
            reinterpret_cast<uint4*>(s_tab)[i] = reinterpret_cast<const uint4*>(A.table)[i];
    }
    for (u32 i = threadIdx.x; i < 256; i += blockDim.x) s_mu[i] = A.mu[i];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    u64* bars = s_bar + warp * S;
    u8* stage = s_stage + (u64)warp * S * SLOT;
    Emitter E;
    E.buf = reinterpret_cast<u64*>(smem + EMIT_OFF) + warp * ECAP;
    E.n = 0;
    if (lane == 0) {
        for (int i = 0; i < S; i++) mbar_init(smem_addr(&bars[i]), 1);
        mbar_fence_init();
    }
    __syncthreads();
    const ET* tab = MPM_SMEM ? reinterpret_cast<const ET*>(s_tab)
                             : reinterpret_cast<const ET*>(A.table);
    // a table in global memory is kept in L2 ahead of the text stream
    const u64 tpol = MPM_SMEM ? 0ull : l2_policy_evict_last();
    const u64 spol = MPM_SMEM ? 0ull : l2_policy_evict_first();
    const u32 gw = blockIdx.x * WARPS + warp;
    const u32 GW = gridDim.x * WARPS;

    // ------------------------------------------------ rows through TMA
    const u32 nst = A.Lst / C;
    const u32 RW = A.row_warps;
    const u32 my_rg = (gw < RW && A.RG > gw) ? (A.RG - gw + RW - 1) / RW : 0;
    const u32 total = my_rg * nst;
    if (total > 0) {
        if (lane == 0) {
            for (u32 i = 0; i < (u32)S && i < total; i++) {
                const u32 bar = smem_addr(&bars[i]);
                // the test hook expects 16 bytes more than the copy brings:
                // the phase never completes and the bounded wait gives up
                mbar_arrive_expect_tx(bar, SLOT + ((A.inject & 1u) && gw == 0 && i == 0 ? 16u : 0u));
                if (MPM_SMEM)
                    tma_load_2d(smem_addr(stage + i * SLOT), &tmap, (int)((i % nst) * C),
                                (int)((gw + (i / nst) * RW) * 32), bar);
                else
                    tma_load_2d_hint(smem_addr(stage + i * SLOT), &tmap, (int)((i % nst) * C),
                                     (int)((gw + (i / nst) * RW) * 32), bar, spol);
            }
        }
        __syncwarp();
        u32 it = 0;
        for (u32 r = 0; r < my_rg; r++) {
            const u32 rg = gw + r * RW;
            const u32 row = rg * 32 + lane;
            const bool valid = row < A.R;
            const u32 row_start = row * A.Lst;
            DT D = ~(DT)0;
#if MPM_OV
            // x: the TW words before the stage, then the stage's C/4 words;
            // rx: their reduced symbols (low-bit map).  Row 0 starts from
            // zero words: the samples that would start before the text only
            // reach windows before it, which fired_stage_ov drops.
            u32 x[TW + C / 4], rx[TW + C / 4];
#pragma unroll
            for (int i = 0; i < TW; i++) x[i] = rx[i] = 0u;
            if (WB > 0 && valid && row_start > 0) {
                // the samples before the row: whole stages ending at row_start
                // (the first stage's own first samples may read zero words:
                // they come more than m'-1 samples before the row)
                const u8* wp = A.T + row_start - (u32)(WSTAGES * C);
#pragma unroll 1
                for (int ws = 0; ws < WSTAGES; ws++) {
#pragma unroll
                    for (int i = 0; i < C / 16; i++) {
                        const uint4 v = ldg_v4(wp + ws * C + 16 * i);
                        x[TW + 4 * i] = v.x;
                        x[TW + 4 * i + 1] = v.y;
                        x[TW + 4 * i + 2] = v.z;
                        x[TW + 4 * i + 3] = v.w;
                    }
                    if (MPM_MODE == 0) {
#pragma unroll
                        for (int i = TW; i < TW + C / 4; i++) rx[i] = pack_word(x[i]);
                    }
                    DT acc = ~(DT)0;
                    run_stage_ov(x, rx, D, acc, tab, s_mu, tpol);
#pragma unroll
                    for (int i = 0; i < TW; i++) {
                        x[i] = x[C / 4 + i];
                        rx[i] = rx[C / 4 + i];
                    }
                }
            }
#else
            FT fm = 0;
            if (WB > 0 && valid && row_start > 0) {
                // the samples before the row: whole stages ending at row_start
                const u8* wp = A.T + row_start - (u32)(WSTAGES * C);
#pragma unroll 1
                for (int ws = 0; ws < WSTAGES; ws++) {
                    u32 w[C / 4];
#pragma unroll
                    for (int i = 0; i < C / 16; i++) {
                        const uint4 v = ldg_v4(wp + ws * C + 16 * i);
                        w[4 * i] = v.x;
                        w[4 * i + 1] = v.y;
                        w[4 * i + 2] = v.z;
                        w[4 * i + 3] = v.w;
                    }
                    run_stage<false>(w, D, fm, tab, s_mu, tpol);
                }
            }
            const u32 h_row = row_start / (u32)Q;
#endif
            for (u32 st = 0; st < nst; st++, it++) {
                const u32 slot = it % S;
                const bool ok = mbar_wait_bounded(smem_addr(&bars[slot]), (it / S) & 1u);
                if (!__all_sync(0xFFFFFFFFu, ok)) {
                    if (lane == 0) {
                        atomicExch(&A.counters[kErrorFlagJ], 5u /* MPM_ETIMEOUT */);
                        const u32 issued = min(total, it + (u32)S);
                        for (u32 j = it; j < issued; j++)
                            mbar_wait_bounded(smem_addr(&bars[j % S]), (j / S) & 1u);
                    }
                    __syncwarp();
                    return;
                }
                const u32 base = smem_addr(stage + slot * SLOT + lane * C);
#if MPM_OV
#pragma unroll
                for (int i = 0; i < C / 16; i++) {
                    const uint4 v = lds128(base + 16 * i);
                    x[TW + 4 * i] = v.x;
                    x[TW + 4 * i + 1] = v.y;
                    x[TW + 4 * i + 2] = v.z;
                    x[TW + 4 * i + 3] = v.w;
                }
                if (MPM_MODE == 0) {
#pragma unroll
                    for (int i = TW; i < TW + C / 4; i++) rx[i] = pack_word(x[i]);
                }
                const DT D0 = D;
                DT acc = ~(DT)0;
                run_stage_ov(x, rx, D, acc, tab, s_mu, tpol);
#else
                u32 w[C / 4];
#pragma unroll
                for (int i = 0; i < C / 16; i++) {
                    const uint4 v = lds128(base + 16 * i);
                    w[4 * i] = v.x;
                    w[4 * i + 1] = v.y;
                    w[4 * i + 2] = v.z;
                    w[4 * i + 3] = v.w;
                }
                fm = 0;
                run_stage<true>(w, D, fm, tab, s_mu, tpol);
#endif
                // the slot's words are consumed: refill it
                __syncwarp();
                if (lane == 0 && it + S < total) {
                    const u32 j = it + S;
                    const u32 bar = smem_addr(&bars[slot]);
                    mbar_arrive_expect_tx(bar, SLOT);
                    if (MPM_SMEM)
                        tma_load_2d(smem_addr(stage + slot * SLOT), &tmap, (int)((j % nst) * C),
                                    (int)((gw + (j / nst) * RW) * 32), bar);
                    else
                        tma_load_2d_hint(smem_addr(stage + slot * SLOT), &tmap,
                                         (int)((j % nst) * C), (int)((gw + (j / nst) * RW) * 32),
                                         bar, spol);
                }
#if MPM_OV
                const bool any = valid && ((~bits_at(acc, RSH) & KMASK) != 0u);
                if (__any_sync(0xFFFFFFFFu, any)) {
                    // some lane fired: which samples, from the saved D
                    const i64 h1 = (i64)row_start + (i64)st * C + (E0 - (Q - 1));
                    FT fmw[FW];
                    fired_stage_ov(x, rx, D0, fmw, h1 - RSH, tab, s_mu, tpol);
#pragma unroll
                    for (int w = 0; w < FW; w++) {
                        const FT f = valid ? fmw[w] : (FT)0;
                        if (__any_sync(0xFFFFFFFFu, f != 0))
                            emit_stage(f, (u32)(h1 + (i64)w * SPW * K), E, A);
                    }
                }
#pragma unroll
                for (int i = 0; i < TW; i++) {
                    x[i] = x[C / 4 + i];
                    rx[i] = rx[C / 4 + i];
                }
#else
                if (!valid) fm = 0;
                if (__any_sync(0xFFFFFFFFu, fm != 0))
                    emit_stage(fm, h_row + st * (u32)(C / Q) + (u32)(K - 1), E, A);
#endif
            }
        }
        flush(E, A);
    }

    // ------------------------------------- bytes after the rows, plain loads
    const u32 GL = GW * 32;
    const u32 rev = GL - 1 - (gw * 32 + lane);
    for (u32 s = rev; s < A.nstreams; s += GL) {
        const u32 a = A.pa + s * A.Ls;
        const u32 b = min(A.n, a + A.Ls);
        DT D = ~(DT)0;
#if MPM_OV
        // the samples whose last byte lies in [a, b): starts from a - (q-1),
        // at h = k-1 (mod k); the m'-1 samples before them warm D up, and
        // samples starting before the text do not exist (D stays all ones)
        i64 h = (i64)a - (Q - 1);
        h += (((i64)(K - 1) - h) % K + K) % K;
        for (int t = MP - 1; t >= 1; t--) {
            const i64 hw = h - (i64)t * K;
            if (hw < 0) continue;
            D = (D << K) | entry(tab, code_bytes(A.T, (u32)hw, s_mu), tpol);
        }
        for (; h + Q <= (i64)b; h += K) {
            if (h < 0) continue;
            D = (D << K) | entry(tab, code_bytes(A.T, (u32)h, s_mu), tpol);
            const u32 fired = ~bits_at(D, RSH) & KMASK;
            if (fired) {
                // rare: handled by the lane alone
                const u32 idx = atomicAdd(&A.counters[kCandCountJ], 1u);
#if MPM_VERIFY
                (void)idx;
                verify_record(A, (u32)h, fired, 0);
#else
                if (idx < A.cap) A.cand[idx] = ((u64)fired << 32) | (u32)h;
#endif
            }
        }
#else
        // the m'-1 samples that end at a, a-P, ...; those starting before
        // the text are virtual and leave D at all ones
        for (int j = MP - 2; j >= 0; j--) {
            const i64 e = (i64)a - (i64)j * P;
            if (e - Q < 0) continue;
            D = (D << K) | entry(tab, code_bytes(A.T, (u32)(e - Q), s_mu), tpol);
        }
        for (u32 e = a + P; e <= b; e += P) {
            const u32 st = e - Q;
            D = (D << K) | entry(tab, code_bytes(A.T, st, s_mu), tpol);
            const u32 fired = ~bits_at(D, RSH) & KMASK;
            if (fired) {
                // rare: handled by the lane alone
                const u32 idx = atomicAdd(&A.counters[kCandCountJ], 1u);
#if MPM_VERIFY
                (void)idx;
                for (int sh = 0; sh < Q; sh++) verify_record(A, st / (u32)Q, fired, sh);
#else
                if (idx < A.cap) A.cand[idx] = ((u64)fired << 32) | (st / (u32)Q);
#endif
            }
        }
#endif
    }
}

}  // namespace mpm
