// One lane's range of one text in the batched search, for the parameter set
// whose stage primitives (scan_stage.cuh) precede this text in the same
// namespace: the MAG filter of Sections 3.1 and 3.2 with q, k, m', the
// mapping and the entry width compiled in, and the exact check of the
// windows it nominates (Section 3.2).  Compiled at run time (NVRTC) once per
// parameter set of a batch, inside that set's namespace.
//
// The lane's range [a, b) starts on a multiple of C from the text start, so
// every stage of C bytes holds the same C/P sampled q-grams at the same
// offsets, as in the single-text scan; the warp's lanes step through their
// stages together, each stage read with C/16 vector loads, and queue the
// fired samples in shared memory, verifying them 32 at a time.

// The warp verifies its queued fired samples, one record per lane: record
// (h << 32) | fired stands, for each fired bit j, for the window of q-grams
// h0 = h - (m'-1)k - j, i.e. the text starts h0 q - s, s = q-1 .. 0, walked
// in ascending order (check_starts: the keys of all of them read at once); a
// key whose hash misses the set's bitmap has no pattern group to probe.
// Texts of a batch are shorter than 2^24 bytes, so 32-bit arithmetic holds
// every start.  KW: the key width class (1: at most 8 bytes, 2: more).
template <int KW>
__device__ __forceinline__ void flush_records(const u64* queue, int count, const u32* keys,
                                              u32 key_mask, const WindowCtx& wc) {
    const int last = (int)wc.n - (int)wc.m;  // the last start of a whole window
    for (int r = (int)(threadIdx.x & 31); r < count; r += 32) {
        const u64 rec = queue[r];
        const int h = (int)(rec >> 32);
        u32 fired = (u32)rec;
        while (fired) {
            const int j = __ffs((int)fired) - 1;
            fired &= fired - 1;
            const int h0 = h - RSH - j;
            const int first = max(h0 * VQ - (VQ - 1), 0);
            const int end = min(h0 * VQ, last);
            if (first > end) continue;
            check_starts<KW>(wc, (u32)first, (u32)end, keys, key_mask);
        }
    }
}

__device__ __forceinline__ void flush_queue(const u64* queue, int count, const u32* keys,
                                            u32 key_mask, const WindowCtx& wc) {
    if (wc.key_bytes <= 8)
        flush_records<1>(queue, count, keys, key_mask, wc);
    else
        flush_records<2>(queue, count, keys, key_mask, wc);
}

// Queues the fired samples of one stage (for every lane, every sample u
// with report bits: (h1 + u k) << 32 | bits), verifying whenever 32 or more
// are queued.  Warp-collective.
__device__ __forceinline__ void queue_stage(FT fm, u32 h1, u64* queue, int& qcount, u32& ncand,
                                            const u32* keys, u32 key_mask, const WindowCtx& wc) {
    for (;;) {
        const bool has = fm != 0;
        const u32 bal = __ballot_sync(0xFFFFFFFFu, has);
        if (bal == 0) break;
        if (has) {
            const int bit = (sizeof(FT) == 8) ? (__ffsll((long long)fm) - 1) : (__ffs((int)fm) - 1);
            const int u = bit / K;
            const u32 fired = (u32)(fm >> (u * K)) & KMASK;
            fm &= ~((FT)KMASK << (u * K));
            queue[qcount + __popc(bal & lanemask_lt())] = ((u64)(h1 + (u32)(u * K)) << 32) | fired;
            ncand++;
        }
        qcount += __popc(bal);
        if (qcount >= 32) {
            __syncwarp();
            flush_queue(queue, qcount, keys, key_mask, wc);
            qcount = 0;
            __syncwarp();
        }
    }
}

// Where this parameter set's mask table is read: shared memory (the
// kernel's copy of a table of at most kBatchSmemTable bytes; the caller
// passes the shared-memory copy itself, so that the lookups compile to
// shared-memory loads, not generic ones), else global memory through L2.
constexpr bool kTableInSmem = MPM_SMEM != 0;

// All 32 lanes of a warp call this together for one tile; lane range
// [a, b), live = a < b.  tab: the set's mask table (in shared memory when
// kTableInSmem, else in global memory), smu: its byte map in shared memory.
__device__ __forceinline__ void batch_lane(const ET* tab, const u8* smu, const u32* keys,
                                           u32 key_mask, const u8* T, u32 n, u32 a, u32 b,
                                           bool live, const WindowCtx& wc, u64* queue,
                                           u32& ncand) {
    (void)n;
    // a table in global memory is kept in L2 ahead of the text stream
    const u64 tpol = kTableInSmem ? 0ull : l2_policy_evict_last();
    DT D = ~(DT)0;
    // the m'-1 samples that end at a, a - P, ...; those that would start
    // before the text do not exist and leave D at all ones
    if (live) {
        for (int j = MP - 2; j >= 0; j--) {
            const i64 e = (i64)a - (i64)j * P;
            if (e - Q < 0) continue;
            D = (D << K) | entry(tab, code_bytes(T, (u32)(e - Q), smu), tpol);
        }
    }
    const bool vec = (reinterpret_cast<unsigned long long>(T) & 15) == 0;
    const u32 nst = (MPM_STAGES && live && vec) ? (b - a) / (u32)C : 0u;
    int qcount = 0;
#if MPM_STAGES
    // the lane's stages stream into L2 kPrefetch stages ahead of its loads
    constexpr u32 kPrefetch = MPM_BATCH_PREFETCH;
    if (kPrefetch > 0 && nst > 0)
        prefetch_l2_bulk(T + a, (nst < kPrefetch ? nst : kPrefetch) * (u32)C);
    u32 nmax = nst;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) nmax = max(nmax, __shfl_xor_sync(0xFFFFFFFFu, nmax, o));
    const u32 h_a = a / (u32)Q + (u32)(K - 1);  // q-gram index of the first sample
#pragma unroll 1
    for (u32 st = 0; st < nmax; st++) {
        const bool act = st < nst;
        if (kPrefetch > 0 && st + kPrefetch < nst)
            prefetch_l2_bulk(T + a + (st + kPrefetch) * (u32)C, (u32)C);
        u32 w[C / 4];
        if (act) {
            const uint4* p = reinterpret_cast<const uint4*>(T + a + st * (u32)C);
#pragma unroll
            for (int i = 0; i < C / 16; i++) {
                const uint4 v = __ldg(p + i);
                w[4 * i] = v.x;
                w[4 * i + 1] = v.y;
                w[4 * i + 2] = v.z;
                w[4 * i + 3] = v.w;
            }
        } else {
#pragma unroll
            for (int i = 0; i < C / 4; i++) w[i] = 0u;
        }
        // a lane past its own stages steps with the warp but keeps its state
        // for the rest of its range
        const DT keep = D;
        FT fm = 0;
        run_stage<true>(w, D, fm, tab, smu, tpol);
        if (!act) {
            D = keep;
            fm = 0;
        }
        if (__any_sync(0xFFFFFFFFu, fm != 0))
            queue_stage(fm, h_a + st * (u32)(C / Q), queue, qcount, ncand, keys, key_mask, wc);
    }
#endif
    // the rest of the range, sample by sample with byte loads
    const u32 e0 = a + nst * (u32)C;
    const u32 nrest = live ? (b - e0) / (u32)P : 0u;
    u32 rmax = nrest;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) rmax = max(rmax, __shfl_xor_sync(0xFFFFFFFFu, rmax, o));
    const u32 below = lanemask_lt();
#pragma unroll 1
    for (u32 t = 0; t < rmax; t++) {
        u32 fired = 0, hq = 0;
        if (t < nrest) {
            const u32 st = e0 + (t + 1) * (u32)P - (u32)Q;
            D = (D << K) | entry(tab, code_bytes(T, st, smu), tpol);
            fired = ~bits_at(D, RSH) & KMASK;
            hq = st / (u32)Q;
        }
        const u32 bal = __ballot_sync(0xFFFFFFFFu, fired != 0);
        if (bal) {
            if (fired) {
                queue[qcount + __popc(bal & below)] = ((u64)hq << 32) | fired;
                ncand++;
            }
            qcount += __popc(bal);
            if (qcount >= 32) {
                __syncwarp();
                flush_queue(queue, qcount, keys, key_mask, wc);
                qcount = 0;
                __syncwarp();
            }
        }
    }
    if (qcount) {
        __syncwarp();
        flush_queue(queue, qcount, keys, key_mask, wc);
        __syncwarp();
    }
}
