// K3: exact verification of the candidate windows (Section 3.2: the filter
// only nominates windows; each is checked against the r patterns in the
// original alphabet, Section 3.3).
//
// A candidate record (fired << 32) | h stands, for every set bit j of fired,
// for the window of q-grams starting at h0 = h - (m'-1)k - j, i.e. for the
// text starts i = h0*q - s, s = 0..q-1 (each start has exactly one (h0, s)).
// One thread takes one (record, s) pair.  A start i is looked up by the key
// of its first min(m, 16) bytes in an open-addressing table of pattern
// groups; the patterns of a matching group are compared byte by byte beyond
// the key and every equal pattern id is appended as (i << 32) | pid.
#include "device_common.cuh"
#include "kernels.h"

namespace mpm {

namespace {

__device__ __forceinline__ void emit_occ(const VerifyArgs& A, uint32_t i, uint32_t pid) {
    const uint32_t idx = atomicAdd(&A.counters[kOccCount], 1u);
    if (idx < A.occ_cap) A.occ[idx] = ((uint64_t)i << 32) | pid;
}

__device__ void check_window(const VerifyArgs& A, uint32_t i) {
    const uint8_t* w = A.T + i;
    uint64_t lo = 0, hi = 0;
    for (int u = 0; u < A.key_bytes; u++) {
        const uint64_t b = w[u];
        if (u < 8)
            lo |= b << (8 * u);
        else
            hi |= b << (8 * (u - 8));
    }
    uint32_t slot = (uint32_t)key_hash(lo, hi) & A.slot_mask;
    for (uint32_t probes = 0; probes <= A.slot_mask; probes++) {
        const Slot sl = A.slots[slot];
        if (sl.count == 0) return;
        if (sl.lo == lo && sl.hi == hi) {
            for (uint32_t row = sl.first; row < sl.first + sl.count; row++) {
                const uint8_t* p = A.pat + (size_t)row * A.m;
                uint32_t u = (uint32_t)A.key_bytes;
                while (u < A.m && w[u] == p[u]) u++;
                if (u == A.m) emit_occ(A, i, A.pid[row]);
            }
            return;
        }
        slot = (slot + 1) & A.slot_mask;
    }
}

__global__ void __launch_bounds__(256) verify_kernel(const VerifyArgs A) {
    const uint32_t count = min(A.counters[kCandCount], A.cand_cap);
    const uint64_t total = (uint64_t)count * A.q;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    const int64_t lead = (int64_t)(A.mprime - 1) * A.k;
    for (uint64_t idx = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += stride) {
        const uint32_t c = (uint32_t)(idx / A.q);
        const int s = (int)(idx % A.q);
        const uint64_t rec = A.cand[c];
        const int64_t h = (int64_t)(uint32_t)rec;
        uint32_t fired = (uint32_t)(rec >> 32);
        while (fired) {
            const int j = __ffs(fired) - 1;
            fired &= fired - 1;
            const int64_t h0 = h - lead - j;
            const int64_t i = h0 * A.q - s;
            if (i < 0 || i + (int64_t)A.m > (int64_t)A.n) continue;
            check_window(A, (uint32_t)i);
        }
    }
}

}  // namespace

int launch_verify(const VerifyArgs& a, int num_sms, cudaStream_t s) {
    verify_kernel<<<num_sms * 8, 256, 0, s>>>(a);
    return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

}  // namespace mpm
