// K2: the MAG scan -- alphabet reduction and q-gram encoding fused with the
// average-optimal Shift-Or filter (Sections 3.1, 3.2) and candidate
// compaction.
//
// Data layout.  The text bulk is cut into R rows of Lst bytes (Lst a multiple
// of 48, of 16 and of P = k*q, so every row starts on a sampled-period
// boundary).  Each thread owns one row and runs the Shift-Or recurrence
// D <- (D << k) | B[t'(h)] over the sampled q-grams h = k-1 (mod k) of its
// row, after warming up on the (m'-1) sampled q-grams that precede the row.
// A warp's 32 rows are streamed through shared memory by 2-D TMA boxes of
// 32 rows x 48 bytes, four stages deep, each warp with its own mbarriers, so
// no block-wide synchronisation is needed.  48-byte rows make the three
// 16-byte shared loads of a quarter warp hit eight distinct bank groups.
// Bytes after the last full row go through the same recurrence with plain
// loads (scan_plain).
//
// Per 4-byte word the thread pushes the bytes into a 64-bit window: reduced
// symbols (low-bit map, or the byte map mu applied to every byte) or raw
// bytes (mu applied only to the q bytes of each sampled q-gram).  A sampled
// q-gram whose last byte lies in the word is cut from the window, looked up
// in the mask table (shared memory when it fits) and folded into D.  All
// rows share the same phase, so the "does a sampled q-gram end here" branch
// is warp-uniform.  When a report bit (m'-1)k + j of D is zero, the warp
// ballots, one lane reserves space with one atomicAdd and every firing lane
// writes the record (fired_mask << 32) | h.
#include <algorithm>
#include <cstdio>
#include <type_traits>

#include <cudaTypedefs.h>

#include "device_common.cuh"
#include "kernels.h"
#include "stepper.cuh"

namespace mpm {

// Appends one record per firing lane among `active` lanes.
__device__ __forceinline__ void emit(uint32_t active, uint32_t fired, uint32_t h, uint64_t* cand,
                                     uint32_t cap, uint32_t* counters) {
    uint32_t bal = __ballot_sync(active, fired != 0);
    if (bal == 0) return;
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(bal) - 1;
    uint32_t base = 0;
    if (lane == leader) base = atomicAdd(&counters[kCandCount], (uint32_t)__popc(bal));
    base = __shfl_sync(active, base, leader);
    if (fired) {
        uint32_t idx = base + __popc(bal & lanemask_lt());
        if (idx < cap) cand[idx] = ((uint64_t)fired << 32) | h;
    }
}

// ------------------------------------------------------------ TMA row path

template <int MODE, typename ET>
__global__ void __launch_bounds__(kScanWarps * 32, 2)
    scan_tma_kernel(const ScanArgs A, const __grid_constant__ CUtensorMap tmap) {
    using DT = typename Stepper<MODE, ET>::DT;
    constexpr uint32_t C = kScanRowBytes;
    constexpr uint32_t SLOT = 32 * C;
    constexpr int S = kScanStages;
    extern __shared__ __align__(128) uint8_t smem[];

    // shared layout: [table?][mu 256][barriers][stages]
    const uint32_t tab_bytes = A.f.smem_table ? A.f.table_bytes : 0u;
    uint8_t* s_tab = smem;
    uint8_t* s_mu = smem + tab_bytes;
    uint64_t* s_bar = reinterpret_cast<uint64_t*>(s_mu + 256);
    uint8_t* s_stage = reinterpret_cast<uint8_t*>(
        (reinterpret_cast<uintptr_t>(s_bar + kScanWarps * S) + 127) & ~uintptr_t(127));

    for (uint32_t i = threadIdx.x; i < tab_bytes / 16; i += blockDim.x)
        reinterpret_cast<uint4*>(s_tab)[i] = reinterpret_cast<const uint4*>(A.f.table)[i];
    for (uint32_t i = threadIdx.x; i < 256; i += blockDim.x) s_mu[i] = A.f.mu[i];

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    uint64_t* bars = s_bar + warp * S;
    uint8_t* stage = s_stage + (size_t)warp * S * SLOT;
    if (lane == 0) {
        for (int i = 0; i < S; i++) mbar_init(smem_addr(&bars[i]), 1);
        mbar_fence_init();
    }
    __syncthreads();

    const ET* tab = A.f.smem_table ? reinterpret_cast<const ET*>(s_tab)
                                   : reinterpret_cast<const ET*>(A.f.table);
    const uint32_t gw = blockIdx.x * kScanWarps + warp;
    const uint32_t GW = gridDim.x * kScanWarps;
    const uint32_t nst = A.Lst / C;
    const uint32_t my_rg = (A.RG > gw) ? (A.RG - gw + GW - 1) / GW : 0;
    const uint32_t total = my_rg * nst;
    const int rsh = (A.f.mprime - 1) * A.f.k;
    const uint32_t kmask = (A.f.k >= 32) ? 0xFFFFFFFFu : ((1u << A.f.k) - 1u);

    auto issue = [&](uint32_t i) {
        const uint32_t slot = i % S;
        const uint32_t rg = gw + (i / nst) * GW;
        const uint32_t st = i % nst;
        const uint32_t bar = smem_addr(&bars[slot]);
        mbar_arrive_expect_tx(bar, SLOT);
        tma_load_2d(smem_addr(stage + slot * SLOT), &tmap, (int32_t)(st * C), (int32_t)(rg * 32),
                    bar);
    };
    if (lane == 0)
        for (uint32_t i = 0; i < (uint32_t)S && i < total; i++) issue(i);
    __syncwarp();

    Stepper<MODE, ET> sp;
    uint32_t it = 0;
    for (uint32_t r = 0; r < my_rg; r++) {
        const uint32_t rg = gw + r * GW;
        const uint32_t row = rg * 32 + lane;
        const bool valid = row < A.R;
        const uint32_t row_start = row * A.Lst;
        sp.init(A.f, tab, s_mu);
        warm_up(sp, A.T, A.n, row_start, A.warm_bytes, A.P, valid);
        uint32_t hq = row_start / (uint32_t)A.f.q + (uint32_t)(A.f.k - 1);
        int pos = 0, nxt = (int)A.P;
        for (uint32_t st = 0; st < nst; st++, it++) {
            const uint32_t slot = it % S;
            const bool ok = mbar_wait_bounded(smem_addr(&bars[slot]), (it / S) & 1u);
            if (!__all_sync(0xFFFFFFFFu, ok)) {
                // give up: flag it, let the copies already issued land, leave
                if (lane == 0) {
                    atomicExch(&A.counters[kErrorFlag], (uint32_t)MPM_ETIMEOUT);
                    const uint32_t issued = min(total, it + (uint32_t)S);
                    for (uint32_t j = it; j < issued; j++)
                        mbar_wait_bounded(smem_addr(&bars[j % S]), (j / S) & 1u);
                }
                __syncwarp();
                return;
            }
            const uint32_t base = smem_addr(stage + slot * SLOT + lane * C);
            uint32_t wv[12];
            {
                uint4 v0 = lds128(base), v1 = lds128(base + 16), v2 = lds128(base + 32);
                wv[0] = v0.x; wv[1] = v0.y; wv[2] = v0.z; wv[3] = v0.w;
                wv[4] = v1.x; wv[5] = v1.y; wv[6] = v1.z; wv[7] = v1.w;
                wv[8] = v2.x; wv[9] = v2.y; wv[10] = v2.z; wv[11] = v2.w;
            }
#pragma unroll
            for (int w = 0; w < 12; w++) {
                sp.push(wv[w]);
                pos += 4;
                while (nxt <= pos) {
                    const uint32_t c = sp.code(pos - nxt);
                    sp.D = (sp.D << sp.k) | (DT)tab[c];
                    const uint32_t fired = valid ? fired_bits(sp.D, rsh, kmask) : 0u;
                    emit(0xFFFFFFFFu, fired, hq, A.cand, A.cap, A.counters);
                    nxt += (int)A.P;
                    hq += (uint32_t)sp.k;
                }
            }
            // every lane has consumed the slot (its words fed the recurrence
            // above), so the slot can be refilled
            __syncwarp();
            if (lane == 0 && it + S < total) issue(it + S);
            pos -= 48;
            nxt -= 48;
        }
    }
}

// --------------------------------------------------------- plain-load path

template <int MODE, typename ET>
__global__ void __launch_bounds__(256) scan_plain_kernel(const ScanArgs A) {
    using DT = typename Stepper<MODE, ET>::DT;
    __shared__ uint8_t s_mu[256];
    for (uint32_t i = threadIdx.x; i < 256; i += blockDim.x) s_mu[i] = A.f.mu[i];
    __syncthreads();
    const ET* tab = reinterpret_cast<const ET*>(A.f.table);
    const int rsh = (A.f.mprime - 1) * A.f.k;
    const uint32_t kmask = (A.f.k >= 32) ? 0xFFFFFFFFu : ((1u << A.f.k) - 1u);
    const uint32_t stride = gridDim.x * blockDim.x;
    // every lane of a warp runs the same number of outer iterations
    const uint32_t first = blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t warp_first = first & ~31u;
    for (uint32_t s0 = warp_first; s0 < A.nstreams; s0 += stride) {
        const uint32_t s = s0 + (threadIdx.x & 31);
        const bool live = s < A.nstreams;
        const uint32_t a = A.pa + (live ? s : 0) * A.Ls;
        const uint32_t b = live ? min(A.n, a + A.Ls) : a;
        Stepper<MODE, ET> sp;
        sp.init(A.f, tab, s_mu);
        warm_up(sp, A.T, A.n, a, A.warm_bytes, A.P, live);
        uint32_t hq = a / (uint32_t)A.f.q + (uint32_t)(A.f.k - 1);
        int pos = 0, nxt = (int)A.P;
        const uint32_t len = b - a;
        const uint32_t words = (len + 3) / 4;
        for (uint32_t w = 0; w < words; w++) {
            const uint32_t at = a + 4 * w;
            uint32_t x;
            if (at + 4 <= A.n) {
                x = load_word(A.T, at);
            } else {
                x = 0;
                for (uint32_t u = 0; u < 4 && at + u < A.n; u++) x |= (uint32_t)A.T[at + u] << (8 * u);
            }
            sp.push(x);
            pos += 4;
            while (nxt <= pos && a + (uint32_t)nxt <= b) {
                const uint32_t c = sp.code(pos - nxt);
                sp.D = (sp.D << sp.k) | (DT)tab[c];
                const uint32_t fired = fired_bits(sp.D, rsh, kmask);
                emit(__activemask(), fired, hq, A.cand, A.cap, A.counters);
                nxt += (int)A.P;
                hq += (uint32_t)sp.k;
            }
            if (nxt <= pos) break;  // the next sampled q-gram would pass b
        }
    }
}

// ------------------------------------------ overlapping q-grams (Section 2)

// The text's q-gram T[h..h+q) at every byte position h; the sampled ones are
// h = k-1 (mod k), and D <- (D << k) | B[code].  Stream s owns the sampled
// positions in [a, b), a = s Ls (Ls a multiple of lcm(k, 4)); it starts at
// the earliest of the m'-1 sampled positions before its first one (positions
// below 0 are skipped: they would leave D's bits at one), and emits records
// (fired << 32) | h only for its own positions.  Verification reads a
// record's windows as the starts h - (m'-1) k - j themselves.
template <int MODE, typename ET>
__global__ void __launch_bounds__(256) scan_overlap_kernel(const ScanArgs A) {
    using DT = typename Stepper<MODE, ET>::DT;
    __shared__ uint8_t s_mu[256];
    for (uint32_t i = threadIdx.x; i < 256; i += blockDim.x) s_mu[i] = A.f.mu[i];
    __syncthreads();
    const ET* tab = reinterpret_cast<const ET*>(A.f.table);
    const int k = A.f.k, q = A.f.q;
    const int rsh = (A.f.mprime - 1) * k;
    const uint32_t kmask = (k >= 32) ? 0xFFFFFFFFu : ((1u << k) - 1u);
    const uint32_t nh = A.n >= (uint32_t)q ? A.n - (uint32_t)q + 1 : 0;  // q-gram positions
    const uint32_t stride = gridDim.x * blockDim.x;
    const uint32_t warp_first = (blockIdx.x * blockDim.x + threadIdx.x) & ~31u;
    for (uint32_t s0 = warp_first; s0 < A.nstreams; s0 += stride) {
        const uint32_t s = s0 + (threadIdx.x & 31);
        const bool live = s < A.nstreams;
        const uint32_t a = live ? s * A.Ls : 0;
        const uint32_t b = live ? min(nh, a + A.Ls) : 0;
        Stepper<MODE, ET> sp;
        sp.init(A.f, tab, s_mu);
        int64_t h = (int64_t)a + (k - 1) - (int64_t)(A.f.mprime - 1) * k;
        if (h < 0) h += (-h + k - 1) / k * k;
        uint32_t at = (uint32_t)h & ~3u;  // next byte to push
        while ((uint64_t)h < (uint64_t)b) {
            const uint32_t end = (uint32_t)h + (uint32_t)q;  // <= n
            while (at < end) {
                uint32_t x;
                if (at + 4 <= A.n) {
                    x = load_word(A.T, at);
                } else {
                    x = 0;
                    for (uint32_t u = 0; u < 4 && at + u < A.n; u++)
                        x |= (uint32_t)A.T[at + u] << (8 * u);
                }
                sp.push(x);
                at += 4;
            }
            const uint32_t c = sp.code((int)(at - end));
            sp.D = (sp.D << k) | (DT)tab[c];
            if ((uint64_t)h >= a)
                emit(__activemask(), fired_bits(sp.D, rsh, kmask), (uint32_t)h, A.cand, A.cap,
                     A.counters);
            h += k;
        }
    }
}

// ------------------------------------------------------ SMAG: scan of codes

template <typename ET>
__global__ void __launch_bounds__(256)
    scan_codes_kernel(const uint32_t* codes, uint32_t nq, const FilterDev f, uint64_t* cand,
                      uint32_t cap, uint32_t* counters, uint32_t per_stream, uint32_t nstreams) {
    using DT = typename std::conditional<sizeof(ET) == 8, uint64_t, uint32_t>::type;
    const ET* tab = reinterpret_cast<const ET*>(f.table);
    const int k = f.k;
    const int rsh = (f.mprime - 1) * k;
    const uint32_t kmask = (k >= 32) ? 0xFFFFFFFFu : ((1u << k) - 1u);
    const uint32_t nsamp = nq / (uint32_t)k;  // sampled q-grams t -> h = t k + k - 1
    const uint32_t stride = gridDim.x * blockDim.x;
    const uint32_t first = (blockIdx.x * blockDim.x + threadIdx.x) & ~31u;
    for (uint32_t s0 = first; s0 < nstreams; s0 += stride) {
        const uint32_t s = s0 + (threadIdx.x & 31);
        const uint32_t t0 = min(nsamp, s * per_stream);
        const uint32_t t1 = (s < nstreams) ? min(nsamp, t0 + per_stream) : t0;
        DT D = ~(DT)0;
        const uint32_t w0 = t0 >= (uint32_t)(f.mprime - 1) ? t0 - (f.mprime - 1) : 0;
        for (uint32_t t = w0; t < t0; t++) D = (D << k) | (DT)tab[codes[t * k + k - 1]];
        for (uint32_t t = t0; t < t1; t++) {
            const uint32_t h = t * k + k - 1;
            D = (D << k) | (DT)tab[codes[h]];
            emit(__activemask(), fired_bits(D, rsh, kmask), h, cand, cap, counters);
        }
    }
}

// ----------------------------------------------------------------- launch

namespace {

PFN_cuTensorMapEncodeTiled_v12000 get_encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000,
                                             cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

uint32_t gcd_u(uint32_t a, uint32_t b) {
    while (b) {
        uint32_t t = a % b;
        a = b;
        b = t;
    }
    return a;
}

uint32_t lcm_u(uint32_t a, uint32_t b) { return a / gcd_u(a, b) * b; }

int scan_mode(const FilterDev& f) {
    if (f.map_kind == MPM_MAP_QHASH) return kQHash;
    if (f.map_kind == MPM_MAP_LOWBITS) return f.ell == 2 ? kLow2 : kLowG;
    return f.q <= 5 ? kLutRaw : kLutRed;
}

size_t tma_smem_bytes(const FilterDev& f) {
    size_t b = (f.smem_table ? f.table_bytes : 0) + 256 + 8 * kScanWarps * kScanStages;
    b = (b + 127) & ~size_t(127);
    return b + (size_t)kScanWarps * kScanStages * 32 * kScanRowBytes + 128;
}

template <int MODE, typename ET>
int launch_typed(const ScanArgs& A0, int num_sms, int chunk, cudaStream_t s) {
    ScanArgs A = A0;
    int launches = 0;
    const uint32_t n = A.n;
    const uint32_t L0 = lcm_u(lcm_u(kScanRowBytes, A.P), 16);
    const uint32_t L4 = lcm_u(A.P, 4);
    const bool aligned = (reinterpret_cast<uintptr_t>(A.T) & 15) == 0;
    auto encode = get_encode_fn();

    // row length: about one row group per resident warp
    const size_t smem = tma_smem_bytes(A.f);
    int per_sm = 1;
    {
        auto kfn = scan_tma_kernel<MODE, ET>;
        cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kfn, kScanWarps * 32, smem);
        if (per_sm < 1) per_sm = 1;
    }
    const uint64_t warps_total = (uint64_t)num_sms * per_sm * kScanWarps;
    uint64_t Lst = chunk > 0 ? (uint64_t)chunk : (uint64_t)n / (32 * warps_total);
    Lst = std::max<uint64_t>(L0 * 4, (Lst + L0 - 1) / L0 * L0);
    uint64_t R = (aligned && encode) ? n / Lst : 0;
    if (R < 32) R = 0;  // below one row group the plain path is as good
    A.Lst = (uint32_t)Lst;
    A.R = (uint32_t)R;
    A.RG = (uint32_t)((R + 31) / 32);
    if (R > 0) {
        CUtensorMap tmap;
        cuuint64_t dims[2] = {Lst, R};
        cuuint64_t strides[1] = {Lst};
        cuuint32_t box[2] = {kScanRowBytes, 32};
        cuuint32_t estr[2] = {1, 1};
        CUresult cr = encode(&tmap, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, const_cast<uint8_t*>(A.T),
                             dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                             CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (cr != CUDA_SUCCESS) return -1;
        const uint64_t blocks =
            std::min<uint64_t>((A.RG + kScanWarps - 1) / kScanWarps, (uint64_t)num_sms * per_sm);
        scan_tma_kernel<MODE, ET><<<(unsigned)blocks, kScanWarps * 32, smem, s>>>(A, tmap);
        launches++;
    }
    A.pa = (uint32_t)(R * Lst);
    if (A.pa < n) {
        const uint32_t rest = n - A.pa;
        uint32_t Ls = chunk > 0 ? (uint32_t)chunk : rest / (uint32_t)(num_sms * 256);
        Ls = std::max(L4 * std::max(1u, 64u / L4), (Ls + L4 - 1) / L4 * L4);
        A.Ls = Ls;
        A.nstreams = (rest + Ls - 1) / Ls;
        const uint32_t threads = 256;
        const uint32_t blocks =
            std::min<uint32_t>((A.nstreams + threads - 1) / threads, (uint32_t)num_sms * 8);
        scan_plain_kernel<MODE, ET><<<blocks, threads, 0, s>>>(A);
        launches++;
    }
    if (cudaPeekAtLastError() != cudaSuccess) return -1;
    return launches;
}

template <int MODE, typename ET>
int launch_overlap(const ScanArgs& A0, int num_sms, int chunk, cudaStream_t s) {
    ScanArgs A = A0;
    const uint32_t nh = A.n >= (uint32_t)A.f.q ? A.n - (uint32_t)A.f.q + 1 : 0;
    if (nh == 0) return 0;
    const uint32_t L4 = lcm_u((uint32_t)A.f.k, 4);
    uint32_t Ls = chunk > 0 ? (uint32_t)chunk : nh / (uint32_t)(num_sms * 256);
    Ls = std::max(L4 * std::max(1u, 64u / L4), (Ls + L4 - 1) / L4 * L4);
    A.Ls = Ls;
    A.nstreams = (nh + Ls - 1) / Ls;
    const uint32_t threads = 256;
    const uint32_t blocks =
        std::min<uint32_t>((A.nstreams + threads - 1) / threads, (uint32_t)num_sms * 8);
    scan_overlap_kernel<MODE, ET><<<blocks, threads, 0, s>>>(A);
    return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

template <int MODE>
int launch_mode(const ScanArgs& A, int num_sms, int chunk, cudaStream_t s) {
    if (A.f.overlap) {
        switch (A.f.entry_bytes) {
            case 1: return launch_overlap<MODE, uint8_t>(A, num_sms, chunk, s);
            case 2: return launch_overlap<MODE, uint16_t>(A, num_sms, chunk, s);
            case 4: return launch_overlap<MODE, uint32_t>(A, num_sms, chunk, s);
            case 8: return launch_overlap<MODE, uint64_t>(A, num_sms, chunk, s);
            case 16: return launch_overlap<MODE, Words<2>>(A, num_sms, chunk, s);
            case 24: return launch_overlap<MODE, Words<3>>(A, num_sms, chunk, s);
            default: return launch_overlap<MODE, Words<4>>(A, num_sms, chunk, s);
        }
    }
    switch (A.f.entry_bytes) {
        case 1: return launch_typed<MODE, uint8_t>(A, num_sms, chunk, s);
        case 2: return launch_typed<MODE, uint16_t>(A, num_sms, chunk, s);
        case 4: return launch_typed<MODE, uint32_t>(A, num_sms, chunk, s);
        case 8: return launch_typed<MODE, uint64_t>(A, num_sms, chunk, s);
        case 16: return launch_typed<MODE, Words<2>>(A, num_sms, chunk, s);
        case 24: return launch_typed<MODE, Words<3>>(A, num_sms, chunk, s);
        default: return launch_typed<MODE, Words<4>>(A, num_sms, chunk, s);
    }
}

}  // namespace

int launch_scan(const ScanArgs& A, int num_sms, int chunk, cudaStream_t s) {
    if (A.n == 0) return 0;
    // packed tables are read by the specialised kernels only
    if (A.f.entry_bits > 0 && A.f.entry_bits < 8) return -2;
    // the generic kernel's raw window holds q-grams of at most 5 bytes
    if (A.f.map_kind == MPM_MAP_QHASH && A.f.q > 5) return -2;
    switch (scan_mode(A.f)) {
        case kQHash: return launch_mode<kQHash>(A, num_sms, chunk, s);
        case kLow2: return launch_mode<kLow2>(A, num_sms, chunk, s);
        case kLowG: return launch_mode<kLowG>(A, num_sms, chunk, s);
        case kLutRed: return launch_mode<kLutRed>(A, num_sms, chunk, s);
        default: return launch_mode<kLutRaw>(A, num_sms, chunk, s);
    }
}

int launch_scan_codes(const uint32_t* codes, uint32_t nq, const FilterDev& f, uint64_t* cand,
                      uint32_t cap, uint32_t* counters, cudaStream_t s) {
    if (f.entry_bytes > 8) return -2;  // several words of state: the MAG scans only
    if (f.entry_bits > 0 && f.entry_bits < 8) return -2;  // packed: specialised kernels only
    const uint32_t nsamp = nq / (uint32_t)f.k;
    if (nsamp == 0) return 0;
    const uint32_t per = std::max<uint32_t>(64, nsamp / (1u << 18));
    const uint32_t nstreams = (nsamp + per - 1) / per;
    const uint32_t blocks = std::min<uint32_t>((nstreams + 255) / 256, 4096);
    switch (f.entry_bytes) {
        case 1:
            scan_codes_kernel<uint8_t><<<blocks, 256, 0, s>>>(codes, nq, f, cand, cap, counters, per, nstreams);
            break;
        case 2:
            scan_codes_kernel<uint16_t><<<blocks, 256, 0, s>>>(codes, nq, f, cand, cap, counters, per, nstreams);
            break;
        case 4:
            scan_codes_kernel<uint32_t><<<blocks, 256, 0, s>>>(codes, nq, f, cand, cap, counters, per, nstreams);
            break;
        default:
            scan_codes_kernel<uint64_t><<<blocks, 256, 0, s>>>(codes, nq, f, cand, cap, counters, per, nstreams);
            break;
    }
    return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

}  // namespace mpm
