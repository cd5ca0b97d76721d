// K3: exact verification of the candidate windows (Section 3.2: the filter
// only nominates windows; each is checked against the r patterns in the
// original alphabet, Section 3.3).
//
// A candidate record (fired << 32) | h stands, for every set bit j of fired,
// for the window of q-grams starting at h0 = h - (m'-1)k - j, i.e. for the
// text starts i = h0*q - s, s = 0..q-1 (each start has exactly one (h0, s)).
// One thread takes one record and walks its q starts in ascending order
// (check_starts: the keys, the first min(m, 16) bytes of each window, read
// together from the aligned 32 bytes around them when they fit).  A key whose
// hash hits a clear bit of the key bitmap (copied into shared memory by
// every block: random bit tests there cost a few bank conflicts, where in L1
// each lane's test is a cache line of its own) has no pattern group; the others
// are looked up in the open-addressing table of pattern groups, the patterns
// of a matching group compared byte by byte beyond the key, and every equal
// pattern id appended as (i << 32) | pid.
#include "device_common.cuh"
#include "kernels.h"
#include "window_check.cuh"

namespace mpm {

namespace {

constexpr int kVerifyThreads = 1024;

__global__ void __launch_bounds__(kVerifyThreads, 2) verify_kernel(const VerifyArgs A) {
    extern __shared__ __align__(16) uint32_t s_keys[];
    if (A.n < A.m) return;
    // the key bitmap: (key_mask + 1) / 8 bytes, a multiple of 128
    for (uint32_t w = threadIdx.x; w < (A.key_mask + 1) / 128; w += blockDim.x)
        reinterpret_cast<uint4*>(s_keys)[w] = __ldg(reinterpret_cast<const uint4*>(A.keys) + w);
    __syncthreads();
    const uint32_t count = min(A.counters[kCandCount], A.cand_cap);
    const int64_t lead = (int64_t)(A.mprime - 1) * A.k;
    const int64_t q = A.q;
    const int64_t last = (int64_t)(A.n - A.m);  // the last start of a whole window
    const uint32_t kb = (uint32_t)A.key_bytes;   // 1 .. 16
    WindowCtx wc;
    wc.T = A.T;
    wc.n = A.n;
    wc.m = A.m;
    wc.key_bytes = kb;
    wc.slot_mask = A.slot_mask;
    wc.occ_cap = A.occ_cap;
    wc.slots = A.slots;
    wc.pat = A.pat;
    wc.pid = A.pid;
    wc.off = A.pat_off;
    wc.occ = reinterpret_cast<unsigned long long*>(A.occ);
    wc.occ_count = &A.counters[kOccCount];
    wc.tag = 0;
    wc.pos_shift = 32;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t c = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; c < count; c += stride) {
        const uint64_t rec = A.cand[c];
        const int64_t h = (int64_t)(uint32_t)rec;
        uint32_t fired = (uint32_t)(rec >> 32);
        while (fired) {
            const int j = __ffs(fired) - 1;
            fired &= fired - 1;
            const int64_t h0 = h - lead - j;
            const int64_t first = max(h0 * q - (q - 1), (int64_t)0);
            const int64_t end = min(h0 * q, last);
            if (first > end) continue;
            if (kb <= 8)
                check_starts<1>(wc, (uint32_t)first, (uint32_t)end, s_keys, A.key_mask);
            else
                check_starts<2>(wc, (uint32_t)first, (uint32_t)end, s_keys, A.key_mask);
        }
    }
}

}  // namespace

int launch_verify(const VerifyArgs& a, int num_sms, cudaStream_t s) {
    const uint32_t bits = a.key_mask + 1;
    if (!a.keys || bits < 1024 || bits > kVerifyKeyBitsMax || (bits & (bits - 1))) return -1;
    // above the default 48 KiB of dynamic shared memory (set on the current
    // device, at every such launch)
    if (bits / 8 > 48 * 1024 &&
        cudaFuncSetAttribute(verify_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(bits / 8)) != cudaSuccess)
        return -1;
    verify_kernel<<<num_sms * 2, kVerifyThreads, bits / 8, s>>>(a);
    return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

}  // namespace mpm
