// K1: SMAG's separate encoding pass (Section 3.2): the code of every
// non-overlapping text q-gram, h = 0 .. floor(n/q) - 1, with the byte map mu
// of Section 3.3 applied to each symbol and the first symbol most
// significant (or, with the q-gram hashing map, the bin of its raw bytes).  A block stages 1024 q-grams' worth of text (1024 * q bytes)
// in shared memory with 16-byte vector loads, then each thread encodes four
// q-grams and the codes are written coalesced.
#include "device_common.cuh"
#include "kernels.h"

namespace mpm {

namespace {

constexpr int kEncThreads = 256;
constexpr int kEncPerThread = 4;
constexpr int kEncTile = kEncThreads * kEncPerThread;  // q-grams per block

__global__ void __launch_bounds__(kEncThreads)
    encode_kernel(const uint8_t* T, uint32_t n, const FilterDev f, uint32_t* codes, uint32_t nq) {
    extern __shared__ __align__(16) uint8_t smem[];
    uint8_t* s_mu = smem;
    uint8_t* s_txt = smem + 256;
    for (int i = threadIdx.x; i < 256; i += blockDim.x) s_mu[i] = f.mu[i];
    const int q = f.q, ell = f.ell;
    const uint64_t tile0 = (uint64_t)blockIdx.x * kEncTile;
    const uint64_t b0 = tile0 * q;
    const uint64_t b1 = min((uint64_t)nq * q, b0 + (uint64_t)kEncTile * q);
    const uint32_t bytes = (uint32_t)(b1 - b0);
    const bool vec = ((reinterpret_cast<uintptr_t>(T + b0) & 15) == 0);
    if (vec) {
        const uint32_t nv = bytes / 16;
        for (uint32_t i = threadIdx.x; i < nv; i += blockDim.x)
            reinterpret_cast<uint4*>(s_txt)[i] = __ldg(reinterpret_cast<const uint4*>(T + b0) + i);
        for (uint32_t i = nv * 16 + threadIdx.x; i < bytes; i += blockDim.x) s_txt[i] = T[b0 + i];
    } else {
        for (uint32_t i = threadIdx.x; i < bytes; i += blockDim.x) s_txt[i] = T[b0 + i];
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < kEncPerThread; u++) {
        const uint32_t local = threadIdx.x + u * kEncThreads;
        const uint64_t h = tile0 + local;
        if (h >= nq) break;
        const uint8_t* g = s_txt + (size_t)local * q;
        uint32_t c = 0;
        if (f.map_kind == MPM_MAP_QHASH) {
            uint64_t raw = 0;
            for (int t = 0; t < q; t++) raw |= (uint64_t)g[t] << (8 * t);
            c = qgram_bin(raw, q, ell);
        } else {
            for (int t = 0; t < q; t++) c = (c << ell) | s_mu[g[t]];
        }
        codes[h] = c;
    }
}

}  // namespace

int launch_encode(const uint8_t* T, uint32_t n, const FilterDev& f, uint32_t* codes,
                  cudaStream_t s) {
    const uint32_t nq = n / (uint32_t)f.q;
    if (nq == 0) return 0;
    const uint32_t blocks = (nq + kEncTile - 1) / kEncTile;
    const size_t smem = 256 + (size_t)kEncTile * f.q;
    if (smem > 48 * 1024)
        cudaFuncSetAttribute(encode_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    encode_kernel<<<blocks, kEncThreads, smem, s>>>(T, n, f, codes, nq);
    return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

}  // namespace mpm
