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
#include "window_check.cuh"

namespace mpm {

namespace {

__global__ void __launch_bounds__(256) verify_kernel(const VerifyArgs A) {
    const uint32_t count = min(A.counters[kCandCount], A.cand_cap);
    const uint64_t total = (uint64_t)count * A.q;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    const int64_t lead = (int64_t)(A.mprime - 1) * A.k;
    WindowCtx wc;
    wc.T = A.T;
    wc.n = A.n;
    wc.m = A.m;
    wc.key_bytes = (unsigned int)A.key_bytes;
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
            check_window(wc, (uint32_t)i);
        }
    }
}

}  // namespace

int launch_verify(const VerifyArgs& a, int num_sms, cudaStream_t s) {
    verify_kernel<<<num_sms * 8, 256, 0, s>>>(a);
    return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

}  // namespace mpm
