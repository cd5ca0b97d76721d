// The batched search compiled at run time for one batch: the persistent
// work loop of the precompiled batched kernel (batch.cu), with every pattern
// set's scan taken from its parameter set's namespace (bv0, bv1, ...: the
// stage primitives of scan_stage.cuh and the lane scan of batch_lane.cuh
// compiled with that set's q, k, m', mapping and entry width), chosen per
// work unit by the set's variant index.  The source that precedes this text
// defines MPM_BATCH_CASES as CASE(0) CASE(1) ... for the batch's parameter
// sets.
//
// Persistent blocks of MPM_BATCH_WARPS warps pop work units (consecutive
// tiles of one set) from a device counter, copy the set's mask table (when
// it fits) and key bitmap into shared memory, and their warps pop the unit's
// tiles from a shared counter; each warp scans a tile's 32 lane ranges.

#ifndef MPM_BATCH_WARPS
#define MPM_BATCH_WARPS 16
#endif

namespace mpm {

extern "C" __global__ void __launch_bounds__(MPM_BATCH_WARPS * 32, 1)
    mpm_batch_jit(const BatchJitArgs A) {
    extern __shared__ __align__(16) u8 smem[];
    u8* s_mu = smem;
    u8* s_tab = smem + 256;
    u32* s_keys = reinterpret_cast<u32*>(smem + 256 + kBatchSmemTable);
    __shared__ u32 s_unit, s_next;
    __shared__ u64 s_queue[MPM_BATCH_WARPS][kWarpQueue];
    const int lane = threadIdx.x & 31;
    u32 ncand = 0;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) {
            s_unit = atomicAdd(&A.counters[kQueue], 1u);
            s_next = 0;
        }
        __syncthreads();
        const u32 ui = s_unit;
        if (ui >= A.nunits) break;
        const BatchUnit U = A.units[ui];
        const BatchSet S = A.sets[U.set];
        const bool in_smem = S.table_bytes <= kBatchSmemTable;
        for (u32 i = threadIdx.x; i < 256; i += blockDim.x) s_mu[i] = S.mu[i];
        if (in_smem)
            for (u32 i = threadIdx.x; i < S.table_bytes / 16; i += blockDim.x)
                reinterpret_cast<uint4*>(s_tab)[i] = reinterpret_cast<const uint4*>(S.table)[i];
        for (u32 i = threadIdx.x; i < S.key_bits / 128; i += blockDim.x)
            reinterpret_cast<uint4*>(s_keys)[i] = reinterpret_cast<const uint4*>(S.keys)[i];
        const u32 kmask = S.key_bits - 1;
        __syncthreads();
        for (;;) {
            u32 t = 0;
            if (lane == 0) t = atomicAdd(&s_next, 1u);
            t = __shfl_sync(0xFFFFFFFFu, t, 0) + U.tile_begin;
            if (t >= U.tile_end) break;
            const BatchTile tl = A.tiles[t];
            const BatchText tx = A.texts[tl.text];
            WindowCtx wc;
            wc.T = tx.T;
            wc.n = tx.n;
            wc.m = S.m;
            wc.key_bytes = S.key_bytes;
            wc.slot_mask = S.slot_mask;
            wc.occ_cap = A.occ_cap;
            wc.slots = S.slots;
            wc.pat = S.pat;
            wc.pid = S.pid;
            wc.off = S.pat_off;
            wc.occ = A.occ;
            wc.occ_count = &A.counters[kBOcc];
            wc.tag = (unsigned long long)tl.text << kTextShift;
            wc.pos_shift = kPidBits;
            const u32 a = tl.start + (u32)lane * tl.sub;
            const u32 b = min(tl.start + tl.len, a + tl.sub);
            const bool live = a < b;
            u64* queue = s_queue[threadIdx.x >> 5];
            switch (S.variant) {
#define CASE(i)                                                                               \
    case i:                                                                                   \
        bv##i::batch_lane(bv##i::kTableInSmem ? reinterpret_cast<const bv##i::ET*>(s_tab)       \
                                              : reinterpret_cast<const bv##i::ET*>(S.table),   \
                          s_mu, s_keys, kmask, tx.T, tx.n, a, b, live, wc, queue, ncand);      \
        break;
                MPM_BATCH_CASES
#undef CASE
                default:
                    break;
            }
        }
    }
    // one atomic per warp for the candidate count
    for (int o = 16; o > 0; o >>= 1) ncand += __shfl_xor_sync(0xFFFFFFFFu, ncand, o);
    if (lane == 0 && ncand) atomicAdd(&A.counters[kBCand], ncand);
}

}  // namespace mpm
