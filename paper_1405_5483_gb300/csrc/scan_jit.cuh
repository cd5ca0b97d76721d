// Specialised MAG scan: the fused encode + average-optimal Shift-Or filter
// of Sections 3.1 and 3.2 with the filter's parameters compiled in.  This
// file is compiled at run time (NVRTC) once per parameter set, after
// scan_jit_args.h, ptx_common.cuh and the stage primitives of
// scan_stage.cuh (whose macros it takes too), with these macros defined:
//   MPM_S, MPM_WARPS  stages per warp, warps per block
//   MPM_TABLE_BYTES   mask-table bytes (padded to 16) copied to shared memory
//   MPM_VERIFY        1: verify the candidates in the kernel and append
//                     occurrences; 0: append the candidate records
//   MPM_EMIT_CAP      records a warp buffers in shared memory
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

namespace mpm {

constexpr int S = MPM_S;
constexpr int WARPS = MPM_WARPS;
constexpr u32 SLOT = 32u * C;

enum { kCandCountJ = 0, kOccCountJ = 1, kErrorFlagJ = 2 };
constexpr u32 ECAP = MPM_EMIT_CAP;
static_assert(ECAP >= 64, "emit buffer");

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
