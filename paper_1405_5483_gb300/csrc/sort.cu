// K4: deterministic order of the occurrence list.  The paper fixes no output
// order; verification appends occurrences through atomics in an order that
// varies from run to run, so the keys (pos << 32) | pid are sorted.
//
// Up to 4096 keys counted on the device: a grid-wide rank sort -- the keys
// are unique, so each one goes to the slot given by the number of smaller
// keys -- which needs no host read-back of the count.
// Up to 8192 keys with the count known on the host: one block, bitonic sort
// in shared memory.
// More: least-significant-digit radix sort, 8-bit digits, only over the
// digit positions that can be non-zero (pid bits and position bits).  Each
// pass is a per-block digit histogram, one exclusive scan over
// (digit, block), and a stable scatter in which each warp ranks its keys
// with __match_any_sync, warps and blocks in key order.
#include <algorithm>
#include <vector>

#include "device_common.cuh"
#include "kernels.h"

namespace mpm {

namespace {

constexpr int kSmallSort = (int)kSortSmallMax;
constexpr int kRadixThreads = 256;
constexpr int kRadixWarps = kRadixThreads / 32;
constexpr int kRadixTile = 4096;  // keys per block
constexpr int kWarpTile = kRadixTile / kRadixWarps;

__global__ void __launch_bounds__(1024)
    sort_small_kernel(const uint64_t* keys, uint32_t z, uint32_t npow2, uint32_t* out_pos,
                      uint32_t* out_pid) {
    extern __shared__ uint64_t sk[];
    for (uint32_t i = threadIdx.x; i < npow2; i += blockDim.x) sk[i] = i < z ? keys[i] : ~0ull;
    __syncthreads();
    for (uint32_t size = 2; size <= npow2; size <<= 1) {
        for (uint32_t stride = size >> 1; stride > 0; stride >>= 1) {
            for (uint32_t i = threadIdx.x; i < npow2; i += blockDim.x) {
                const uint32_t j = i ^ stride;
                if (j > i) {
                    const bool up = (i & size) == 0;
                    const uint64_t a = sk[i], b = sk[j];
                    if ((a > b) == up) {
                        sk[i] = b;
                        sk[j] = a;
                    }
                }
            }
            __syncthreads();
        }
    }
    for (uint32_t i = threadIdx.x; i < z; i += blockDim.x) {
        out_pos[i] = (uint32_t)(sk[i] >> 32);
        out_pid[i] = (uint32_t)sk[i];
    }
}

__global__ void __launch_bounds__(kRadixThreads)
    radix_hist_kernel(const uint64_t* keys, uint32_t z, int shift, uint32_t* hist,
                      uint32_t nblocks) {
    __shared__ uint32_t h[256];
    for (int i = threadIdx.x; i < 256; i += blockDim.x) h[i] = 0;
    __syncthreads();
    const uint32_t a = blockIdx.x * kRadixTile;
    const uint32_t b = min(z, a + kRadixTile);
    for (uint32_t i = a + threadIdx.x; i < b; i += blockDim.x)
        atomicAdd(&h[(keys[i] >> shift) & 0xFF], 1u);
    __syncthreads();
    for (int d = threadIdx.x; d < 256; d += blockDim.x) hist[(size_t)d * nblocks + blockIdx.x] = h[d];
}

// Exclusive prefix sum over hist[0 .. len) in place, one block.
__global__ void __launch_bounds__(1024) radix_scan_kernel(uint32_t* hist, uint32_t len) {
    __shared__ uint32_t warp_sums[32];
    __shared__ uint32_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (uint32_t base = 0; base < len; base += blockDim.x) {
        const uint32_t i = base + threadIdx.x;
        const uint32_t v = i < len ? hist[i] : 0;
        uint32_t x = v;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) warp_sums[warp] = x;
        __syncthreads();
        if (warp == 0) {
            const int nw = blockDim.x / 32;
            uint32_t s = lane < nw ? warp_sums[lane] : 0;
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, s, o);
                if (lane >= o) s += y;
            }
            if (lane < nw) warp_sums[lane] = s;  // inclusive over warps
        }
        __syncthreads();
        const uint32_t before = (warp > 0 ? warp_sums[warp - 1] : 0) + carry;
        if (i < len) hist[i] = before + x - v;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry = before + x;
        __syncthreads();
    }
}

__global__ void __launch_bounds__(kRadixThreads)
    radix_scatter_kernel(const uint64_t* in, uint64_t* out, uint32_t z, int shift,
                         const uint32_t* offs, uint32_t nblocks) {
    __shared__ uint32_t cnt[kRadixWarps][256];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < kRadixWarps * 256; i += blockDim.x) (&cnt[0][0])[i] = 0;
    __syncthreads();
    const uint32_t a = blockIdx.x * kRadixTile + warp * kWarpTile;
    const uint32_t b = min(z, a + kWarpTile);
    // per-warp digit counts
    for (uint32_t c = a; c < b; c += 32) {
        const uint32_t i = c + lane;
        const bool live = i < b;
        const uint32_t d = live ? (uint32_t)((in[i] >> shift) & 0xFF) : 256u + lane;
        const uint32_t peers = __match_any_sync(0xFFFFFFFFu, d);
        if (live && lane == __ffs(peers) - 1) cnt[warp][d] += __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    // starting offset of each (warp, digit)
    for (int d = threadIdx.x; d < 256; d += blockDim.x) {
        uint32_t run = offs[(size_t)d * nblocks + blockIdx.x];
        for (int w = 0; w < kRadixWarps; w++) {
            const uint32_t c = cnt[w][d];
            cnt[w][d] = run;
            run += c;
        }
    }
    __syncthreads();
    for (uint32_t c = a; c < b; c += 32) {
        const uint32_t i = c + lane;
        const bool live = i < b;
        const uint64_t key = live ? in[i] : 0;
        const uint32_t d = live ? (uint32_t)((key >> shift) & 0xFF) : 256u + lane;
        const uint32_t peers = __match_any_sync(0xFFFFFFFFu, d);
        if (live) {
            const uint32_t rank = __popc(peers & lanemask_lt());
            out[cnt[warp][d] + rank] = key;
        }
        __syncwarp();
        if (live && lane == __ffs(peers) - 1) cnt[warp][d] += __popc(peers);
        __syncwarp();
    }
}

constexpr int kRankThreads = 256;
constexpr int kRankTile = 2048;

// counters: the search's counter block (occurrences at kOccCount).  With a
// snapshot, every block counts itself in (kDoneCount) after reading the
// occurrence count, and the last one copies the counters to the snapshot
// (mapped host memory) and zeroes them for the next search.
__global__ void __launch_bounds__(kRankThreads)
    rank_sort_kernel(const uint64_t* keys, uint32_t* counters, uint32_t out_cap,
                     uint32_t* out_pos, uint32_t* out_pid, uint32_t* snapshot,
                     uint32_t cand_cap, uint32_t occ_cap) {
    __shared__ uint64_t tile[kRankTile];
    __shared__ uint32_t s_z;
    if (threadIdx.x == 0) s_z = *(volatile uint32_t*)&counters[kOccCount];
    __syncthreads();
    const uint32_t z = s_z;
    if (snapshot && threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(&counters[kDoneCount], 1u) == gridDim.x - 1) {
            __threadfence();
            volatile uint32_t* c = counters;
            const uint32_t cand = c[kCandCount], occ = c[kOccCount], err = c[kErrorFlag];
            snapshot[kCandCount] = cand;
            snapshot[kOccCount] = occ;
            snapshot[kErrorFlag] = err;
            // 1: the outputs hold every occurrence, sorted
            snapshot[kDoneCount] = (err == 0 && occ <= out_cap && occ <= kRankSortMax &&
                                    occ <= occ_cap && cand <= cand_cap) ? 1u : 0u;
            // the snapshot is read after the stream completes, which makes
            // these writes visible (also in mapped host memory): no fence
            for (int i = 0; i < kNumCounters; i++) c[i] = 0;
        }
    }
    if (z > kRankSortMax || z > out_cap) return;
    if (blockIdx.x * blockDim.x >= z) return;
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    const bool mine = i < z;
    const uint64_t key = mine ? keys[i] : 0;
    uint32_t rank = 0;
    for (uint32_t t0 = 0; t0 < z; t0 += kRankTile) {
        const uint32_t len = min((uint32_t)kRankTile, z - t0);
        __syncthreads();
        for (uint32_t j = threadIdx.x; j < len; j += blockDim.x) tile[j] = keys[t0 + j];
        __syncthreads();
        if (mine) {
#pragma unroll 8
            for (uint32_t j = 0; j < len; j++) rank += tile[j] < key ? 1u : 0u;
        }
    }
    if (mine) {
        out_pos[rank] = (uint32_t)(key >> 32);
        out_pid[rank] = (uint32_t)key;
    }
}

__global__ void split_kernel(const uint64_t* keys, uint32_t z, uint32_t* out_pos,
                             uint32_t* out_pid) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < z; i += gridDim.x * blockDim.x) {
        const uint64_t k = keys[i];
        out_pos[i] = (uint32_t)(k >> 32);
        out_pid[i] = (uint32_t)k;
    }
}

// ---- radix sort with the count on the device (fixed grids: graph-capturable)

constexpr int kDevTile = 4096;

__device__ __forceinline__ uint32_t dev_tiles(const uint32_t* count, uint32_t cap) {
    const uint32_t z = min(*count, cap);
    return (z + kDevTile - 1) / kDevTile;
}

__global__ void __launch_bounds__(kRadixThreads)
    dev_hist_kernel(const uint64_t* keys, const uint32_t* count, uint32_t cap, int shift,
                    uint32_t* hist, uint32_t ntmax, uint32_t skip) {
    __shared__ uint32_t h[256];
    if (*count <= skip) return;
    const uint32_t z = min(*count, cap);
    const uint32_t nt = dev_tiles(count, cap);
    for (uint32_t t = blockIdx.x; t < nt; t += gridDim.x) {
        for (int i = threadIdx.x; i < 256; i += blockDim.x) h[i] = 0;
        __syncthreads();
        const uint32_t a = t * kDevTile, b = min(z, a + kDevTile);
        for (uint32_t i = a + threadIdx.x; i < b; i += blockDim.x)
            atomicAdd(&h[(keys[i] >> shift) & 0xFF], 1u);
        __syncthreads();
        for (int d = threadIdx.x; d < 256; d += blockDim.x) hist[(size_t)d * ntmax + t] = h[d];
        __syncthreads();
    }
}

// Exclusive prefix sum, in (digit, tile) order, over the tiles in use.
__global__ void __launch_bounds__(1024)
    dev_scan_kernel(uint32_t* hist, const uint32_t* count, uint32_t cap, uint32_t ntmax,
                    uint32_t skip) {
    __shared__ uint32_t warp_sums[32];
    __shared__ uint32_t carry;
    if (*count <= skip) return;
    const uint32_t nt = dev_tiles(count, cap);
    const uint32_t len = 256 * nt;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (uint32_t base = 0; base < len; base += blockDim.x) {
        const uint32_t f = base + threadIdx.x;
        const size_t at = f < len ? (size_t)(f / nt) * ntmax + (f % nt) : 0;
        const uint32_t v = f < len ? hist[at] : 0;
        uint32_t x = v;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) warp_sums[warp] = x;
        __syncthreads();
        if (warp == 0) {
            const int nw = blockDim.x / 32;
            uint32_t sum = lane < nw ? warp_sums[lane] : 0;
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, sum, o);
                if (lane >= o) sum += y;
            }
            if (lane < nw) warp_sums[lane] = sum;
        }
        __syncthreads();
        const uint32_t before = (warp > 0 ? warp_sums[warp - 1] : 0) + carry;
        if (f < len) hist[at] = before + x - v;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry = before + x;
        __syncthreads();
    }
}

__global__ void __launch_bounds__(kRadixThreads)
    dev_scatter_kernel(const uint64_t* in, uint64_t* out, const uint32_t* count, uint32_t cap,
                       int shift, const uint32_t* offs, uint32_t ntmax, uint32_t skip) {
    __shared__ uint32_t cnt[kRadixWarps][256];
    if (*count <= skip) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t z = min(*count, cap);
    const uint32_t nt = dev_tiles(count, cap);
    constexpr uint32_t kWarpSpan = kDevTile / kRadixWarps;
    for (uint32_t t = blockIdx.x; t < nt; t += gridDim.x) {
        for (int i = threadIdx.x; i < kRadixWarps * 256; i += blockDim.x) (&cnt[0][0])[i] = 0;
        __syncthreads();
        const uint32_t a = t * kDevTile + warp * kWarpSpan;
        const uint32_t b = min(z, a + kWarpSpan);
        for (uint32_t c = a; c < b; c += 32) {
            const uint32_t i = c + lane;
            const bool live = i < b;
            const uint32_t d = live ? (uint32_t)((in[i] >> shift) & 0xFF) : 256u + lane;
            const uint32_t peers = __match_any_sync(0xFFFFFFFFu, d);
            if (live && lane == __ffs(peers) - 1) cnt[warp][d] += __popc(peers);
            __syncwarp();
        }
        __syncthreads();
        for (int d = threadIdx.x; d < 256; d += blockDim.x) {
            uint32_t run = offs[(size_t)d * ntmax + t];
            for (int w = 0; w < kRadixWarps; w++) {
                const uint32_t c = cnt[w][d];
                cnt[w][d] = run;
                run += c;
            }
        }
        __syncthreads();
        for (uint32_t c = a; c < b; c += 32) {
            const uint32_t i = c + lane;
            const bool live = i < b;
            const uint64_t key = live ? in[i] : 0;
            const uint32_t d = live ? (uint32_t)((key >> shift) & 0xFF) : 256u + lane;
            const uint32_t peers = __match_any_sync(0xFFFFFFFFu, d);
            if (live) out[cnt[warp][d] + __popc(peers & lanemask_lt())] = key;
            __syncwarp();
            if (live && lane == __ffs(peers) - 1) cnt[warp][d] += __popc(peers);
            __syncwarp();
        }
        __syncthreads();
    }
}

// The end of a pipelined search whose keys were radix-sorted on the device
// (more than `from` occurrences): the sorted keys split into the outputs,
// and, as in rank_sort_kernel, the counters copied to the snapshot with the
// completeness word and zeroed for the next search by the last block.
__global__ void __launch_bounds__(256)
    close_sorted_kernel(const uint64_t* sorted, uint32_t* counters, uint32_t out_cap,
                        uint32_t* out_pos, uint32_t* out_pid, uint32_t* snapshot,
                        uint32_t cand_cap, uint32_t occ_cap, uint32_t from) {
    __shared__ uint32_t s_z;
    if (threadIdx.x == 0) s_z = *(volatile uint32_t*)&counters[kOccCount];
    __syncthreads();
    const uint32_t z = s_z;
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(&counters[kDoneCount], 1u) == gridDim.x - 1) {
            __threadfence();
            volatile uint32_t* c = counters;
            const uint32_t cand = c[kCandCount], occ = c[kOccCount], err = c[kErrorFlag];
            snapshot[kCandCount] = cand;
            snapshot[kOccCount] = occ;
            snapshot[kErrorFlag] = err;
            snapshot[kDoneCount] =
                (err == 0 && occ <= out_cap && occ <= occ_cap && cand <= cand_cap) ? 1u : 0u;
            for (int i = 0; i < kNumCounters; i++) c[i] = 0;
        }
    }
    if (z <= from || z > out_cap || z > occ_cap) return;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < z; i += gridDim.x * blockDim.x) {
        const uint64_t k = sorted[i];
        out_pos[i] = (uint32_t)(k >> 32);
        out_pid[i] = (uint32_t)k;
    }
}

// The whole close of a pipelined search with more than `from` occurrences
// in one block: an LSD radix sort of the keys over the digits at `sh`
// (ping-pong between keys and tmp in global memory; warp w owns the w-th
// contiguous chunk of the keys, so ranks by (warp, lane) are stable), the
// split into the outputs, and the counters copied to the snapshot and
// zeroed.  One launch whatever the count, so a search with few occurrences
// pays one kernel that returns at once.
constexpr int kBlockSortThreads = 256;
constexpr int kBlockSortWarps = kBlockSortThreads / 32;

struct DigitShifts {
    int v[8];
    int n;
};

__global__ void __launch_bounds__(kBlockSortThreads)
    block_sort_close_kernel(uint64_t* keys, uint64_t* tmp, uint32_t* counters, uint32_t out_cap,
                            uint32_t* out_pos, uint32_t* out_pid, uint32_t* snapshot,
                            uint32_t cand_cap, uint32_t occ_cap, DigitShifts sh, uint32_t from) {
    static_assert(kBlockSortThreads == 256, "one thread per digit");
    __shared__ uint32_t cnt[kBlockSortWarps][256];
    __shared__ uint32_t s_tot[256];
    __shared__ uint32_t s_c[3];
    if (threadIdx.x == 0) {
        volatile uint32_t* c = counters;
        s_c[0] = c[kCandCount];
        s_c[1] = c[kOccCount];
        s_c[2] = c[kErrorFlag];
    }
    __syncthreads();
    const uint32_t cand = s_c[0], z = s_c[1], err = s_c[2];
    const bool complete = err == 0 && z <= out_cap && z <= occ_cap && cand <= cand_cap;
    if (threadIdx.x == 0) {
        snapshot[kCandCount] = cand;
        snapshot[kOccCount] = z;
        snapshot[kErrorFlag] = err;
        snapshot[kDoneCount] = complete ? 1u : 0u;
        for (int i = 0; i < kNumCounters; i++) counters[i] = 0;
    }
    if (!complete || z <= from) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t span = ((z + kBlockSortWarps - 1) / kBlockSortWarps + 31) & ~31u;
    const uint32_t a = min(z, (uint32_t)warp * span), b = min(z, a + span);
    uint64_t* src = keys;
    uint64_t* dst = tmp;
    for (int p = 0; p < sh.n; p++) {
        const int shift = sh.v[p];
        for (int i = threadIdx.x; i < kBlockSortWarps * 256; i += blockDim.x) (&cnt[0][0])[i] = 0;
        __syncthreads();
        for (uint32_t c = a; c < b; c += 32) {
            const uint32_t i = c + lane;
            const bool live = i < b;
            const uint32_t d = live ? (uint32_t)((src[i] >> shift) & 0xFF) : 256u + lane;
            const uint32_t peers = __match_any_sync(0xFFFFFFFFu, d);
            if (live && lane == __ffs(peers) - 1) cnt[warp][d] += __popc(peers);
            __syncwarp();
        }
        __syncthreads();
        // start of every (digit, warp): the digits before it, then the
        // earlier warps' keys of the same digit (thread d takes digit d)
        {
            const int d = threadIdx.x;
            uint32_t tot = 0;
            for (int w = 0; w < kBlockSortWarps; w++) tot += cnt[w][d];
            s_tot[d] = tot;
            __syncthreads();
            for (int o = 1; o < 256; o <<= 1) {  // inclusive scan of the totals
                const uint32_t v = d >= o ? s_tot[d - o] : 0u;
                __syncthreads();
                s_tot[d] += v;
                __syncthreads();
            }
            uint32_t run = s_tot[d] - tot;
            for (int w = 0; w < kBlockSortWarps; w++) {
                const uint32_t c = cnt[w][d];
                cnt[w][d] = run;
                run += c;
            }
        }
        __syncthreads();
        for (uint32_t c = a; c < b; c += 32) {
            const uint32_t i = c + lane;
            const bool live = i < b;
            const uint64_t key = live ? src[i] : 0;
            const uint32_t d = live ? (uint32_t)((key >> shift) & 0xFF) : 256u + lane;
            const uint32_t peers = __match_any_sync(0xFFFFFFFFu, d);
            if (live) dst[cnt[warp][d] + __popc(peers & lanemask_lt())] = key;
            __syncwarp();
            if (live && lane == __ffs(peers) - 1) cnt[warp][d] += __popc(peers);
            __syncwarp();
        }
        __syncthreads();
        uint64_t* t = src;
        src = dst;
        dst = t;
    }
    for (uint32_t i = threadIdx.x; i < z; i += blockDim.x) {
        const uint64_t k = src[i];
        out_pos[i] = (uint32_t)(k >> 32);
        out_pid[i] = (uint32_t)k;
    }
}

}  // namespace

int launch_block_sort_close(uint64_t* keys, uint64_t* tmp, uint32_t* counters, uint32_t out_cap,
                            uint32_t* out_pos, uint32_t* out_pid, uint32_t* snapshot,
                            uint32_t cand_cap, uint32_t occ_cap, const int* shifts, int nshifts,
                            uint32_t from, cudaStream_t s) {
    if (nshifts < 0 || nshifts > 8) return -1;
    DigitShifts sh{};
    for (int i = 0; i < nshifts; i++) sh.v[i] = shifts[i];
    sh.n = nshifts;
    block_sort_close_kernel<<<1, kBlockSortThreads, 0, s>>>(keys, tmp, counters, out_cap, out_pos,
                                                            out_pid, snapshot, cand_cap, occ_cap,
                                                            sh, from);
    return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

int launch_close_sorted(const uint64_t* sorted, uint32_t* counters, uint32_t out_cap,
                        uint32_t* out_pos, uint32_t* out_pid, uint32_t* snapshot,
                        uint32_t cand_cap, uint32_t occ_cap, uint32_t from, int num_sms,
                        cudaStream_t s) {
    close_sorted_kernel<<<num_sms, 256, 0, s>>>(sorted, counters, out_cap, out_pos, out_pid,
                                                 snapshot, cand_cap, occ_cap, from);
    return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

size_t sort_dev_hist_entries(uint32_t cap) {
    return 256 * (size_t)((cap + kDevTile - 1) / kDevTile + 1);
}

int launch_sort_dev(uint64_t* keys, uint64_t* tmp, uint32_t* hist, uint32_t cap,
                    const uint32_t* count, const int* shifts, int nshifts, int num_sms,
                    uint64_t** sorted, cudaStream_t s, uint32_t skip) {
    const uint32_t ntmax = (cap + kDevTile - 1) / kDevTile + 1;
    const uint32_t grid = std::min<uint32_t>(ntmax, (uint32_t)num_sms * 4);
    uint64_t* src = keys;
    uint64_t* dst = tmp;
    int launches = 0;
    for (int p = 0; p < nshifts; p++) {
        dev_hist_kernel<<<grid, kRadixThreads, 0, s>>>(src, count, cap, shifts[p], hist, ntmax,
                                                       skip);
        dev_scan_kernel<<<1, 1024, 0, s>>>(hist, count, cap, ntmax, skip);
        dev_scatter_kernel<<<grid, kRadixThreads, 0, s>>>(src, dst, count, cap, shifts[p], hist,
                                                          ntmax, skip);
        launches += 3;
        uint64_t* t = src;
        src = dst;
        dst = t;
    }
    *sorted = src;
    return cudaPeekAtLastError() == cudaSuccess ? launches : -1;
}

int launch_rank_sort(const uint64_t* keys, uint32_t* counters, uint32_t out_cap,
                     uint32_t* out_pos, uint32_t* out_pid, uint32_t* snapshot, uint32_t cand_cap,
                     uint32_t occ_cap, cudaStream_t s) {
    const uint32_t blocks = (kRankSortMax + kRankThreads - 1) / kRankThreads;
    rank_sort_kernel<<<blocks, kRankThreads, 0, s>>>(keys, counters, out_cap, out_pos, out_pid,
                                                     snapshot, cand_cap, occ_cap);
    return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

size_t sort_hist_entries(uint32_t z) {
    const size_t nblocks = (z + kRadixTile - 1) / kRadixTile;
    return 256 * (nblocks ? nblocks : 1);
}

int launch_sort_output(uint64_t* d_keys, uint64_t* d_tmp, uint32_t* d_hist, size_t hist_cap,
                       uint32_t z, uint32_t key_bits, uint32_t* out_pos, uint32_t* out_pid,
                       cudaStream_t s) {
    if (z == 0) return 0;
    if (z <= (uint32_t)kSmallSort) {
        uint32_t p2 = 1;
        while (p2 < z) p2 <<= 1;
        const size_t smem = (size_t)p2 * 8;
        cudaFuncSetAttribute(sort_small_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(kSmallSort * 8));
        sort_small_kernel<<<1, 1024, smem, s>>>(d_keys, z, p2, out_pos, out_pid);
        return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
    }
    const uint32_t nblocks = (z + kRadixTile - 1) / kRadixTile;
    if (sort_hist_entries(z) > hist_cap) return -1;
    // digit positions that can hold non-zero bits: the low word carries the
    // pattern id (< 2^pid_bits), the high word the position
    const uint32_t pid_bits = key_bits & 0xFFFF, pos_bits = key_bits >> 16;
    std::vector<int> shifts;
    for (uint32_t b = 0; b < pid_bits; b += 8) shifts.push_back((int)b);
    for (uint32_t b = 0; b < pos_bits; b += 8) shifts.push_back(32 + (int)b);
    int launches = 0;
    uint64_t* src = d_keys;
    uint64_t* dst = d_tmp;
    for (int sh : shifts) {
        radix_hist_kernel<<<nblocks, kRadixThreads, 0, s>>>(src, z, sh, d_hist, nblocks);
        radix_scan_kernel<<<1, 1024, 0, s>>>(d_hist, 256 * nblocks);
        radix_scatter_kernel<<<nblocks, kRadixThreads, 0, s>>>(src, dst, z, sh, d_hist, nblocks);
        launches += 3;
        uint64_t* t = src;
        src = dst;
        dst = t;
    }
    split_kernel<<<(z + 255) / 256 < 4096 ? (z + 255) / 256 : 4096, 256, 0, s>>>(src, z, out_pos,
                                                                                 out_pid);
    launches++;
    return cudaPeekAtLastError() == cudaSuccess ? launches : -1;
}

}  // namespace mpm
