// Batched search: many texts of uneven length, each against one of many
// pattern sets, in one persistent launch (the MAG filter of Sections 3.1 and
// 3.2 with each set's own q, k and mapping as runtime values).
//
// Work list.  Every text is cut into tiles of at most 32 lanes x L bytes,
// each lane's range a multiple of lcm(k*q, 32) from the text start (its
// set's sampling period, and whole 32-byte sectors).  Consecutive tiles of one
// pattern set form work units of about equal estimated cost (scan plus
// verification), handed out most expensive first.
// Persistent blocks of 32 warps pop units from a device counter; a block
// loads the unit's mask table into shared memory (at its own entry width,
// when it fits) and its warps pop the unit's tiles from a shared counter.
// Each lane runs the Shift-Or recurrence over its range (after warming up
// on the m'-1 sampled q-grams before it), reading 32 bytes at a time; the
// warp queues its fired steps in shared memory and verifies them 32 at a time
// against the set's key bitmap and pattern groups, appending
// (text << 44) | (pos << 20) | pid.  A radix sort driven by the
// device count orders the keys; the whole run -- counter reset, scan, sort,
// split into (text, pos, pid) and the count read-back -- is captured once
// into a CUDA graph and replayed by every run.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <string>
#include <new>
#include <numeric>
#include <vector>

#include "handle.h"
#include "stepper.cuh"
#include "window_check.cuh"
#include "batch_args.h"

namespace mpm {

namespace {

constexpr uint32_t kBatchThreads = 1024;
static_assert(kBatchSmemTable == MPM_BATCH_SMEM_TABLE_BYTES, "batch table bound");
constexpr uint32_t kBatchSmem = 256 + kBatchSmemTable + kBatchKeyBits / 8;

static __device__ __noinline__ void batch_probe(const WindowCtx& wc, uint32_t i,
                                                unsigned long long lo, unsigned long long hi,
                                                unsigned long long h) {
    probe_window(wc, i, lo, hi, h);
}

// A window whose key hash misses the set's bitmap (shared memory) matches no
// pattern; the others are looked up among the pattern groups.
__device__ __forceinline__ void batch_check(const WindowCtx& wc, const uint32_t* keys,
                                            uint32_t key_mask, uint32_t i) {
    unsigned long long lo, hi;
    window_key(wc, i, &lo, &hi);
    const uint32_t bit = key_bit(lo, hi, 64u - (uint32_t)__popc(key_mask));
    if (!((keys[bit >> 5] >> (bit & 31)) & 1u)) return;
    batch_probe(wc, i, lo, hi, key_hash(lo, hi));
}

// The warp verifies its queued fired steps, one record per lane at a time:
// record (hq << 32) | fired bits stands for the windows
// (hq - (m'-1)k - j) q - s, j a fired bit, s = 0 .. q-1 (Section 3.2).
__device__ __forceinline__ void flush_queue(const uint64_t* queue, int count, const BatchSet& S,
                                            const uint32_t* keys, uint32_t key_mask,
                                            const WindowCtx& wc, int rsh) {
    for (int r = (int)(threadIdx.x & 31); r < count; r += 32) {
        const uint64_t rec = queue[r];
        const int64_t hq = (int64_t)(rec >> 32);
        uint32_t fired = (uint32_t)rec;
        while (fired) {
            const int j = __ffs((int)fired) - 1;
            fired &= fired - 1;
            for (int sh = 0; sh < S.q; sh++) {
                const int64_t i = (hq - rsh - j) * S.q - sh;
                if (i < 0 || i + (int64_t)S.m > (int64_t)wc.n) continue;
                batch_check(wc, keys, key_mask, (uint32_t)i);
            }
        }
    }
}

// All 32 lanes of a warp call this together for one tile; lane range
// [a, b) (live = a < b).  Lane ranges are multiples of the sampling period
// from the text start, so every lane's steps fall at the same offsets and the
// step loop is uniform across the warp; fired steps go to the warp's queue
// (ballot + prefix count) and are verified 32 at a time.
template <int MODE, typename ET>
__device__ void batch_lane(const BatchSet& S, const ET* tab, const uint8_t* smu,
                           const uint32_t* keys, uint32_t key_mask, const BatchText& tx,
                           uint32_t a, uint32_t b, bool live, const WindowCtx& wc,
                           uint64_t* queue, uint32_t& ncand) {
    using DT = typename Stepper<MODE, ET>::DT;
    FilterDev f{};
    f.q = S.q;
    f.k = S.k;
    f.ell = S.ell;
    f.shift = S.shift;
    f.map_kind = S.map_kind;
    Stepper<MODE, ET> sp;
    sp.init(f, tab, smu);
    const uint32_t P = (uint32_t)(S.k * S.q);
    const uint32_t Wr = (((uint32_t)(S.mprime - 1) * P) + 3) & ~3u;
    warm_up(sp, tx.T, tx.n, a, Wr, P, live);
    const int rsh = (S.mprime - 1) * S.k;
    const uint32_t kmask = S.k >= 32 ? 0xFFFFFFFFu : ((1u << S.k) - 1u);
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t below = (1u << lane) - 1u;
    uint32_t hq = a / (uint32_t)S.q + (uint32_t)(S.k - 1);
    int pos = 0, nxt = (int)P;
    const uint32_t words = live ? (b - a + 3) / 4 : 0;
    uint32_t wmax = words;
    for (int o = 16; o > 0; o >>= 1) wmax = max(wmax, __shfl_xor_sync(0xFFFFFFFFu, wmax, o));
    // a is a multiple of 32 from the text start: whole 32-byte sectors, read
    // as two 16-byte loads that stay in L1 between them
    const bool vec = (reinterpret_cast<uintptr_t>(tx.T) & 15) == 0;
    int qcount = 0;  // the same in every lane
    for (uint32_t w0 = 0; w0 < wmax; w0 += 8) {
        const uint32_t at0 = a + 4 * w0;
        // the lane's sector four blocks ahead (inside the text: at0 + 160 <= b + 3),
        // into L2 while this one is scanned
        if (w0 + 40 <= words)
            asm volatile("prefetch.global.L2 [%0];" ::"l"(tx.T + at0 + 128));
        const bool whole = vec && w0 + 8 <= words && at0 + 32 <= tx.n;
        uint4 lo4 = make_uint4(0, 0, 0, 0), hi4 = make_uint4(0, 0, 0, 0);
        if (whole) {
            lo4 = __ldg(reinterpret_cast<const uint4*>(tx.T + at0));
            hi4 = __ldg(reinterpret_cast<const uint4*>(tx.T + at0 + 16));
        }
        // one copy of the step loop (the instruction caches are shared by
        // the kernel's mapping and entry-width instantiations)
#pragma unroll 1
        for (int u = 0; u < 8; u++) {
            if (w0 + u >= wmax) break;
            uint32_t x = 0;
            if (whole) {
                const uint4 v = u < 4 ? lo4 : hi4;
                const int t = u & 3;
                x = t == 0 ? v.x : t == 1 ? v.y : t == 2 ? v.z : v.w;
            } else if (w0 + u < words) {
                const uint32_t at = at0 + 4 * u;
                if (at + 4 <= tx.n) {
                    x = load_word(tx.T, at);
                } else {
                    for (uint32_t v = 0; v < 4 && at + v < tx.n; v++)
                        x |= (uint32_t)tx.T[at + v] << (8 * v);
                }
            }
            sp.push(x);
            pos += 4;
            while (nxt <= pos) {
                const uint32_t c = sp.code(pos - nxt);
                sp.D = (sp.D << S.k) | (DT)tab[c];
                const bool act = live && a + (uint32_t)nxt <= b;
                const uint32_t fired = act ? ((uint32_t)(~sp.D >> rsh) & kmask) : 0u;
                const uint32_t bal = __ballot_sync(0xFFFFFFFFu, fired != 0);
                if (bal) {
                    if (fired) {
                        queue[qcount + __popc(bal & below)] = ((uint64_t)hq << 32) | fired;
                        ncand++;
                    }
                    qcount += __popc(bal);
                    if (qcount >= 32) {
                        __syncwarp();
                        flush_queue(queue, qcount, S, keys, key_mask, wc, rsh);
                        qcount = 0;
                        __syncwarp();
                    }
                }
                nxt += (int)P;
                hq += (uint32_t)S.k;
            }
        }
    }
    if (qcount) {
        __syncwarp();
        flush_queue(queue, qcount, S, keys, key_mask, wc, rsh);
        __syncwarp();
    }
}

template <int MODE>
__device__ __forceinline__ void batch_lane_eb(const BatchSet& S, const void* tab,
                                              const uint8_t* smu, const uint32_t* keys,
                                              uint32_t key_mask, const BatchText& tx,
                                              uint32_t a, uint32_t b, bool live,
                                              const WindowCtx& wc, uint64_t* queue,
                                              uint32_t& ncand) {
    switch (S.entry_bytes) {
        case 1:
            batch_lane<MODE>(S, (const uint8_t*)tab, smu, keys, key_mask, tx, a, b, live, wc,
                             queue, ncand);
            break;
        case 2:
            batch_lane<MODE>(S, (const uint16_t*)tab, smu, keys, key_mask, tx, a, b, live, wc,
                             queue, ncand);
            break;
        default:
            batch_lane<MODE>(S, (const uint32_t*)tab, smu, keys, key_mask, tx, a, b, live, wc,
                             queue, ncand);
            break;
    }
}

__global__ void __launch_bounds__(kBatchThreads, 1)
    batch_scan_kernel(const BatchSet* sets, const BatchText* texts, const BatchTile* tiles,
                      const BatchUnit* units, uint32_t nunits, uint64_t* occ, uint32_t occ_cap,
                      uint32_t* counters) {
    extern __shared__ __align__(16) uint8_t smem[];
    uint8_t* s_mu = smem;
    uint8_t* s_tab = smem + 256;
    uint32_t* s_keys = reinterpret_cast<uint32_t*>(smem + 256 + kBatchSmemTable);
    __shared__ uint32_t s_unit, s_next;
    __shared__ uint64_t s_queue[kBatchThreads / 32][kWarpQueue];
    const int lane = threadIdx.x & 31;
    uint32_t ncand = 0;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) {
            s_unit = atomicAdd(&counters[kQueue], 1u);
            s_next = 0;
        }
        __syncthreads();
        const uint32_t ui = s_unit;
        if (ui >= nunits) break;
        const BatchUnit U = units[ui];
        const BatchSet S = sets[U.set];
        const bool in_smem = S.table_bytes <= kBatchSmemTable;
        for (uint32_t i = threadIdx.x; i < 256; i += blockDim.x) s_mu[i] = S.mu[i];
        if (in_smem)
            for (uint32_t i = threadIdx.x; i < S.table_bytes / 16; i += blockDim.x)
                reinterpret_cast<uint4*>(s_tab)[i] = reinterpret_cast<const uint4*>(S.table)[i];
        for (uint32_t i = threadIdx.x; i < S.key_bits / 128; i += blockDim.x)
            reinterpret_cast<uint4*>(s_keys)[i] = reinterpret_cast<const uint4*>(S.keys)[i];
        const uint32_t kmask = S.key_bits - 1;
        __syncthreads();
        const void* tab = in_smem ? (const void*)s_tab : S.table;
        for (;;) {
            uint32_t t = 0;
            if (lane == 0) t = atomicAdd(&s_next, 1u);
            t = __shfl_sync(0xFFFFFFFFu, t, 0) + U.tile_begin;
            if (t >= U.tile_end) break;
            const BatchTile tl = tiles[t];
            const BatchText tx = texts[tl.text];
            WindowCtx wc;
            wc.T = tx.T;
            wc.n = tx.n;
            wc.m = S.m;
            wc.key_bytes = S.key_bytes;
            wc.slot_mask = S.slot_mask;
            wc.occ_cap = occ_cap;
            wc.slots = S.slots;
            wc.pat = S.pat;
            wc.pid = S.pid;
            wc.off = S.pat_off;
            wc.occ = reinterpret_cast<unsigned long long*>(occ);
            wc.occ_count = &counters[kBOcc];
            wc.tag = (unsigned long long)tl.text << kTextShift;
            wc.pos_shift = kPidBits;
            const uint32_t a = tl.start + (uint32_t)lane * tl.sub;
            const uint32_t b = min(tl.start + tl.len, a + tl.sub);
            const bool live = a < b;
            uint64_t* queue = s_queue[threadIdx.x >> 5];
            switch (S.mode) {
                case kLow2: batch_lane_eb<kLow2>(S, tab, s_mu, s_keys, kmask, tx, a, b, live, wc, queue, ncand); break;
                case kLowG: batch_lane_eb<kLowG>(S, tab, s_mu, s_keys, kmask, tx, a, b, live, wc, queue, ncand); break;
                case kLutRed: batch_lane_eb<kLutRed>(S, tab, s_mu, s_keys, kmask, tx, a, b, live, wc, queue, ncand); break;
                case kLutRaw: batch_lane_eb<kLutRaw>(S, tab, s_mu, s_keys, kmask, tx, a, b, live, wc, queue, ncand); break;
                default: batch_lane_eb<kQHash>(S, tab, s_mu, s_keys, kmask, tx, a, b, live, wc, queue, ncand); break;
            }
        }
    }
    // one atomic per warp for the candidate count
    for (int o = 16; o > 0; o >>= 1) ncand += __shfl_xor_sync(0xFFFFFFFFu, ncand, o);
    if (lane == 0 && ncand) atomicAdd(&counters[kBCand], ncand);
}

__global__ void batch_split_kernel(const uint64_t* keys, const uint32_t* count, uint32_t cap,
                                   uint32_t* out) {
    const uint32_t z = min(*count, cap);
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < z; i += gridDim.x * blockDim.x) {
        const uint64_t k = keys[i];
        out[i] = (uint32_t)(k >> kTextShift);
        out[cap + i] = (uint32_t)(k >> kPidBits) & ((1u << kPosBits) - 1);
        out[2 * (size_t)cap + i] = (uint32_t)k & ((1u << kPidBits) - 1);
    }
}

int mode_of(const mpm_handle* h) {
    const auto& p = h->plan.p;
    if (p.map_kind == MPM_MAP_QHASH) return kQHash;
    if (p.map_kind == MPM_MAP_LOWBITS) return h->plan.ell == 2 ? kLow2 : kLowG;
    return p.q <= 5 ? kLutRaw : kLutRed;
}

bool on_device(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

// The batched kernel's specialisation of one pattern set's plan.
BatchVariant batch_variant_of(const Plan& plan) {
    BatchVariant v{};
    v.q = plan.p.q;
    v.k = plan.p.k;
    v.mp = plan.info.mprime;
    v.ell = plan.ell;
    v.mode = plan.p.map_kind == MPM_MAP_LOWBITS ? 0 : (plan.p.map_kind == MPM_MAP_QHASH ? 2 : 1);
    v.shift = v.mode == 0 ? plan.p.map_shift : 0;
    v.eb = plan.info.entry_bytes;
    v.C = jit_stage_bytes((uint32_t)(v.q * v.k), v.k, false);
    v.stages = v.C > 0 ? 1 : 0;
    v.ebits = plan.info.entry_bits;
    // the kernel copies a table of at most kBatchSmemTable bytes (padded to
    // 16) into shared memory; the variant then reads it there with
    // shared-memory loads, else from global memory kept in L2
    v.smem = ((plan.info.table_bytes + 15) & ~uint64_t(15)) <= kBatchSmemTable ? 1 : 0;
    if (!v.stages) v.C = (uint32_t)(v.q * v.k);  // sample by sample: lanes of whole periods
    return v;
}

// Index of v in vs, appended when new.
int batch_variant_index(std::vector<BatchVariant>& vs, const BatchVariant& v) {
    size_t idx = 0;
    while (idx < vs.size() && std::memcmp(&vs[idx], &v, sizeof(v)) != 0) idx++;
    if (idx == vs.size()) vs.push_back(v);
    return (int)idx;
}

}  // namespace mpm

struct mpm_batch {
    int device = 0, num_sms = 0;
    cudaStream_t stream = nullptr;
    mpm::BatchSet* d_sets = nullptr;
    mpm::BatchText* d_texts = nullptr;
    mpm::BatchTile* d_tiles = nullptr;
    mpm::BatchUnit* d_units = nullptr;
    uint32_t* d_keys = nullptr;  // the sets' key bitmaps, one after another
    uint32_t ntiles = 0, ntexts = 0, nunits = 0;
    uint64_t* d_occ = nullptr;
    uint64_t* d_tmp = nullptr;
    uint32_t* d_hist = nullptr;
    uint32_t* d_out = nullptr;
    uint32_t cap = 0;
    uint32_t* d_counters = nullptr;
    uint32_t* h_counters = nullptr;
    int shifts[8] = {0};
    int nshifts = 0;
    uint64_t* sorted = nullptr;
    bool use_graph = true;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};  // run start/end, scan start/end
    bool scan_events = true;  // ev[2..3] bracket the scan kernel (inside the graph too)
    const mpm::BatchJit* jit = nullptr;  // the kernel compiled for this batch, or null
    uint64_t bytes = 0;
    mpm_batch_stats stats{};
};

namespace {

using mpm::set_error;

void drop_graph(mpm_batch* b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
}

void drop_buffers(mpm_batch* b) {
    cudaFree(b->d_occ);
    cudaFree(b->d_tmp);
    cudaFree(b->d_hist);
    cudaFree(b->d_out);
    b->d_occ = b->d_tmp = nullptr;
    b->d_hist = b->d_out = nullptr;
    b->cap = 0;
}

void release_batch(mpm_batch* b) {
    if (!b) return;
    if (b->stream) cudaStreamSynchronize(b->stream);
    drop_graph(b);
    drop_buffers(b);
    cudaFree(b->d_sets);
    cudaFree(b->d_texts);
    cudaFree(b->d_tiles);
    cudaFree(b->d_units);
    cudaFree(b->d_keys);
    cudaFree(b->d_counters);
    if (b->h_counters) cudaFreeHost(b->h_counters);
    for (auto& e : b->ev)
        if (e) cudaEventDestroy(e);
    if (b->stream) cudaStreamDestroy(b->stream);
    cudaGetLastError();
    delete b;
}

int alloc_buffers(mpm_batch* b, uint32_t cap) {
    drop_buffers(b);
    if (cudaMalloc(&b->d_occ, (size_t)cap * 8) != cudaSuccess ||
        cudaMalloc(&b->d_tmp, (size_t)cap * 8) != cudaSuccess ||
        cudaMalloc(&b->d_hist, mpm::sort_dev_hist_entries(cap) * 4) != cudaSuccess ||
        cudaMalloc(&b->d_out, (size_t)cap * 12) != cudaSuccess) {
        cudaGetLastError();
        drop_buffers(b);
        return MPM_ENOMEM;
    }
    b->cap = cap;
    return MPM_OK;
}

// An event record that is also kept when the stream is being captured (as
// an event-record node of the graph, so that replays time the scan too).
bool record_event(cudaEvent_t e, cudaStream_t s, bool capturing) {
    return (capturing ? cudaEventRecordWithFlags(e, s, cudaEventRecordExternal)
                      : cudaEventRecord(e, s)) == cudaSuccess;
}

// Counter reset, scan, sort, split and count read-back on the batch stream.
int enqueue_batch(mpm_batch* b, bool capturing = false) {
    cudaStream_t s = b->stream;
    if (cudaMemsetAsync(b->d_counters, 0, 16, s) != cudaSuccess) return MPM_ECUDA;
    if (b->scan_events && !record_event(b->ev[2], s, capturing)) return MPM_ECUDA;
    if (b->jit) {
        mpm::BatchJitArgs a{};
        a.sets = b->d_sets;
        a.texts = b->d_texts;
        a.tiles = b->d_tiles;
        a.units = b->d_units;
        a.occ = reinterpret_cast<unsigned long long*>(b->d_occ);
        a.counters = b->d_counters;
        a.nunits = b->nunits;
        a.occ_cap = b->cap;
        if (mpm::launch_batch_jit(b->jit, a, b->num_sms, s) < 0) return MPM_ECUDA;
    } else {
        mpm::batch_scan_kernel<<<b->num_sms, mpm::kBatchThreads, mpm::kBatchSmem, s>>>(
            b->d_sets, b->d_texts, b->d_tiles, b->d_units, b->nunits, b->d_occ, b->cap,
            b->d_counters);
    }
    if (b->scan_events && !record_event(b->ev[3], s, capturing)) return MPM_ECUDA;
    int l = mpm::launch_sort_dev(b->d_occ, b->d_tmp, b->d_hist, b->cap, b->d_counters + mpm::kBOcc,
                                 b->shifts, b->nshifts, b->num_sms, &b->sorted, s);
    if (l < 0) return MPM_ECUDA;
    mpm::batch_split_kernel<<<b->num_sms * 4, 256, 0, s>>>(b->sorted, b->d_counters + mpm::kBOcc,
                                                           b->cap, b->d_out);
    if (cudaMemcpyAsync(b->h_counters, b->d_counters, 16, cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return MPM_ECUDA;
    b->stats.launches = (uint32_t)(2 + l);
    return cudaPeekAtLastError() == cudaSuccess ? MPM_OK : MPM_ECUDA;
}

int capture_once(mpm_batch* b) {
    if (cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
        return MPM_ECUDA;
    int rc = enqueue_batch(b, true);
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(b->stream, &g);
    if (rc || e != cudaSuccess || !g) {
        cudaGetLastError();
        if (g) cudaGraphDestroy(g);
        return rc ? rc : MPM_ECUDA;
    }
    b->graph = g;
    return MPM_OK;
}

int capture(mpm_batch* b) {
    drop_graph(b);
    if (!b->use_graph) return MPM_OK;
    int rc = capture_once(b);
    if (rc == MPM_ECUDA && b->scan_events) {
        // a graph without the scan's event-record nodes: runs are still
        // timed as a whole, the scan alone is not
        b->scan_events = false;
        rc = capture_once(b);
    }
    if (rc) return rc;
    if (cudaGraphInstantiate(&b->exec, b->graph, 0) != cudaSuccess) {
        cudaGetLastError();
        drop_graph(b);
        return MPM_ECUDA;
    }
    return MPM_OK;
}

int bits_for(uint64_t v) {
    int x = 0;
    while (x < 64 && (v >> x)) x++;
    return x;
}

}  // namespace

extern "C" {

mpm_batch* mpm_batch_create(mpm_handle* const* sets, int nsets, const uint8_t* const* texts,
                            const size_t* lens, const uint32_t* set_of_text, int ntexts,
                            const mpm_batch_opts* opts) {
    if (!sets || nsets <= 0 || !texts || !lens || !set_of_text || ntexts <= 0 ||
        ntexts >= (1 << 20)) {
        set_error(MPM_EINVAL);
        return nullptr;
    }
    mpm_batch_opts o{};
    if (opts) o = *opts;
    int device = -1;
    for (int i = 0; i < nsets; i++) {
        const mpm_handle* h = sets[i];
        if (!h) {
            set_error(MPM_EINVAL);
            return nullptr;
        }
        if (device < 0) device = h->device;
        if (h->device != device || h->plan.info.positions > 32 || h->plan.r > (1u << mpm::kPidBits)) {
            set_error(MPM_ENOTSUP);
            return nullptr;
        }
        if ((h->plan.p.map_kind == MPM_MAP_QHASH && h->plan.p.q > 5) || h->plan.p.overlap) {
            set_error(MPM_ENOTSUP);
            return nullptr;
        }
    }
    for (int t = 0; t < ntexts; t++)
        if (set_of_text[t] >= (uint32_t)nsets || lens[t] >= (1u << mpm::kPosBits) ||
            (lens[t] > 0 && !texts[t])) {
            set_error(MPM_EINVAL);
            return nullptr;
        }
    if (cudaSetDevice(device) != cudaSuccess) {
        cudaGetLastError();
        set_error(MPM_ECUDA);
        return nullptr;
    }
    for (int t = 0; t < ntexts; t++)
        if (lens[t] > 0 && !mpm::on_device(texts[t])) {
            set_error(MPM_EINVAL);
            return nullptr;
        }
    mpm_batch* b = new (std::nothrow) mpm_batch();
    if (!b) {
        set_error(MPM_ENOMEM);
        return nullptr;
    }
    b->device = device;
    b->use_graph = !o.no_graph;
    b->ntexts = (uint32_t)ntexts;
    bool ok = cudaDeviceGetAttribute(&b->num_sms, cudaDevAttrMultiProcessorCount, device) ==
                  cudaSuccess &&
              cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) == cudaSuccess &&
              cudaEventCreate(&b->ev[0]) == cudaSuccess && cudaEventCreate(&b->ev[1]) == cudaSuccess &&
              cudaEventCreate(&b->ev[2]) == cudaSuccess && cudaEventCreate(&b->ev[3]) == cudaSuccess &&
              cudaMalloc(&b->d_counters, 16) == cudaSuccess &&
              cudaMallocHost(&b->h_counters, 16) == cudaSuccess;
    // per-set descriptors pointing at the handles' device tables
    std::vector<mpm::BatchSet> hs(nsets);
    for (int i = 0; ok && i < nsets; i++) {
        const mpm_handle* h = sets[i];
        mpm::BatchSet S{};
        S.table = h->d_table;
        S.table_bytes = h->table_bytes_padded;
        S.entry_bytes = h->plan.info.entry_bytes;
        S.mu = h->d_mu;
        S.slots = h->d_slots;
        S.pat = h->d_pat;
        S.pid = h->d_pid;
        S.pat_off = h->d_pat_off;
        S.slot_mask = (uint32_t)h->host.slots.size() - 1;
        S.key_bytes = (uint32_t)h->host.key_bytes;
        // key bitmap: 64 bits per pattern group, 2^10 .. 2^19 bits
        uint32_t groups = 0;
        for (const auto& sl : h->host.slots) groups += sl.count ? 1 : 0;
        uint32_t bits = 1u << 10;
        while (bits < mpm::kBatchKeyBits && bits < 64ull * groups) bits <<= 1;
        S.key_bits = bits;
        S.m = (uint32_t)h->plan.m;
        S.q = h->plan.p.q;
        S.k = h->plan.p.k;
        S.mprime = h->plan.info.mprime;
        S.ell = h->plan.ell;
        S.shift = h->plan.p.map_shift;
        S.map_kind = h->plan.p.map_kind;
        S.mode = mpm::mode_of(h);
        hs[i] = S;
    }
    // the kernel compiled for this batch: one specialisation per distinct
    // parameter set (q, k, m', sigma', shift, mapping, entry width)
    if (ok && !o.generic) {
        std::vector<mpm::BatchVariant> vs;
        for (int i = 0; i < nsets; i++) {
            const mpm::BatchVariant v = mpm::batch_variant_of(sets[i]->plan);
            hs[i].variant = mpm::batch_variant_index(vs, v);
            hs[i].stage = v.C;
        }
        int err = MPM_OK;
        std::string log;
        b->jit = mpm::jit_batch_kernel(vs, device, &err, &log);
        if (!b->jit) {
            if (!log.empty()) std::fprintf(stderr, "mpm: batched kernel compilation failed:\n%s\n", log.c_str());
            for (auto& S : hs) S.variant = 0, S.stage = 0;
        }
        b->stats.variants = b->jit ? (uint32_t)vs.size() : 0u;
    }
    // packed mask tables are read by the compiled kernel only
    for (int i = 0; ok && !b->jit && i < nsets; i++)
        if (sets[i]->plan.info.entry_bits < 8) {
            release_batch(b);
            set_error(MPM_ENOTSUP);
            return nullptr;
        }
    // the key bitmaps, one after another (each a multiple of 16 bytes)
    if (ok) {
        size_t words = 0;
        for (const auto& S : hs) words += S.key_bits / 32;
        std::vector<uint32_t> bm(words, 0u);
        size_t at = 0;
        for (int i = 0; i < nsets; i++) {
            const uint32_t mask = hs[i].key_bits - 1;
            for (const auto& sl : sets[i]->host.slots) {
                if (!sl.count) continue;
                const uint32_t bit = mpm::key_bit(sl.lo, sl.hi, 64u - (uint32_t)__builtin_ctz(mask + 1));
                bm[at + bit / 32] |= 1u << (bit % 32);
            }
            at += hs[i].key_bits / 32;
        }
        ok = cudaMalloc(&b->d_keys, words * 4) == cudaSuccess &&
             cudaMemcpy(b->d_keys, bm.data(), words * 4, cudaMemcpyHostToDevice) == cudaSuccess;
        at = 0;
        for (auto& S : hs) {
            S.keys = b->d_keys + at;
            at += S.key_bits / 32;
        }
    }
    // texts and tiles, grouped by set: per lane a multiple of lcm(period, 32)
    std::vector<mpm::BatchText> ht(ntexts);
    std::vector<uint32_t> order(ntexts);
    std::iota(order.begin(), order.end(), 0u);
    std::stable_sort(order.begin(), order.end(), [&](uint32_t x, uint32_t y) {
        if (set_of_text[x] != set_of_text[y]) return set_of_text[x] < set_of_text[y];
        return lens[x] > lens[y];
    });
    std::vector<mpm::BatchTile> tiles;
    std::vector<mpm::BatchUnit> units;
    const uint32_t lane_bytes = o.lane_bytes > 0 ? (uint32_t)o.lane_bytes : 512;
    const uint64_t unit_bytes = (uint64_t)(o.unit_kib > 0 ? o.unit_kib : 2048) << 10;
    uint32_t max_r = 1;
    for (int i = 0; i < nsets; i++) max_r = std::max<uint32_t>(max_r, (uint32_t)sets[i]->plan.r);
    for (int t = 0; t < ntexts; t++) {
        ht[t] = mpm::BatchText{texts[t], (uint32_t)lens[t], set_of_text[t]};
        b->bytes += lens[t];
    }
    // Work units: consecutive tiles of one set whose estimated cost reaches
    // unit_bytes.  A byte costs 1 to scan plus 10 per window it sends to
    // verification (rate * q * max(1, k * rate) / (k * q) windows per byte),
    // so verification-heavy sets get short units and short lanes; units are
    // handed out most expensive first.
    std::vector<double> unit_cost;
    for (size_t oi = 0; oi < order.size(); oi++) {
        const uint32_t t = order[oi];
        const uint32_t set = set_of_text[t];
        const mpm::BatchSet& S = hs[set];
        const uint32_t P = (uint32_t)(S.k * S.q);
        // lane shares: whole stages of the compiled kernel, or whole sectors
        // and sampling periods, lcm(P, 32), for the precompiled one
        uint32_t G = P;
        if (b->jit) {
            G = S.stage;
        } else {
            while (G % 32) G += P;
        }
        const uint32_t n = (uint32_t)lens[t];
        if (n < S.m) continue;
        const double rate = std::min(1.0, std::max(0.0, sets[set]->plan.info.est_candidate_rate));
        const double w = 1.0 + 10.0 * rate * S.q * std::max(1.0, S.k * rate) / P;
        // at least 64 tiles per unit, lanes no shorter than 2m
        const double set_unit = (double)unit_bytes / w;
        uint32_t L = (uint32_t)std::min<double>(lane_bytes, set_unit / (64.0 * 32.0));
        L = std::max<uint32_t>(L, std::min<uint32_t>(lane_bytes, 2 * S.m));
        L = std::max<uint32_t>(G, (L + G - 1) / G * G);
        for (uint32_t start = 0; start < n; start += 32 * L) {
            const uint32_t len = std::min<uint32_t>(32 * L, n - start);
            uint32_t sub = (len + 31) / 32;
            sub = std::max<uint32_t>(G, (sub + G - 1) / G * G);
            if (units.empty() || units.back().set != set || unit_cost.back() >= (double)unit_bytes) {
                units.push_back(mpm::BatchUnit{set, (uint32_t)tiles.size(), (uint32_t)tiles.size(), 0});
                unit_cost.push_back(0.0);
            }
            tiles.push_back(mpm::BatchTile{t, start, len, sub});
            units.back().tile_end = (uint32_t)tiles.size();
            unit_cost.back() += w * len;
        }
    }
    {
        std::vector<uint32_t> by_cost(units.size());
        std::iota(by_cost.begin(), by_cost.end(), 0u);
        std::stable_sort(by_cost.begin(), by_cost.end(),
                         [&](uint32_t x, uint32_t y) { return unit_cost[x] > unit_cost[y]; });
        std::vector<mpm::BatchUnit> sorted;
        for (uint32_t i : by_cost) sorted.push_back(units[i]);
        units.swap(sorted);
    }
    b->ntiles = (uint32_t)tiles.size();
    b->nunits = (uint32_t)units.size();
    ok = ok && cudaMalloc(&b->d_sets, sizeof(mpm::BatchSet) * nsets) == cudaSuccess &&
         cudaMalloc(&b->d_texts, sizeof(mpm::BatchText) * ntexts) == cudaSuccess &&
         cudaMalloc(&b->d_tiles, sizeof(mpm::BatchTile) * std::max<size_t>(1, tiles.size())) ==
             cudaSuccess &&
         cudaMalloc(&b->d_units, sizeof(mpm::BatchUnit) * std::max<size_t>(1, units.size())) ==
             cudaSuccess &&
         cudaFuncSetAttribute(mpm::batch_scan_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              mpm::kBatchSmem) == cudaSuccess;
    ok = ok &&
         cudaMemcpy(b->d_sets, hs.data(), sizeof(mpm::BatchSet) * nsets, cudaMemcpyHostToDevice) ==
             cudaSuccess &&
         cudaMemcpy(b->d_texts, ht.data(), sizeof(mpm::BatchText) * ntexts,
                    cudaMemcpyHostToDevice) == cudaSuccess &&
         (tiles.empty() || cudaMemcpy(b->d_tiles, tiles.data(), sizeof(mpm::BatchTile) * tiles.size(),
                                      cudaMemcpyHostToDevice) == cudaSuccess) &&
         (units.empty() || cudaMemcpy(b->d_units, units.data(), sizeof(mpm::BatchUnit) * units.size(),
                                      cudaMemcpyHostToDevice) == cudaSuccess);
    // digit positions of the keys that can be non-zero
    const int pid_bits = bits_for(max_r - 1 ? max_r - 1 : 1);
    const int text_bits = bits_for((uint64_t)ntexts - 1 ? (uint64_t)ntexts - 1 : 1);
    const int top = mpm::kTextShift + text_bits;  // highest key bit + 1
    for (int sh = 0; sh < top && b->nshifts < 8; sh += 8) {
        // skip digits that only cover the unused high bits of the pattern id
        if (sh >= pid_bits && sh + 8 <= mpm::kPidBits) continue;
        b->shifts[b->nshifts++] = sh;
    }
    ok = ok && cudaStreamSynchronize(b->stream) == cudaSuccess &&
         alloc_buffers(b, 1u << 16) == MPM_OK && capture(b) == MPM_OK;
    if (!ok) {
        cudaGetLastError();
        release_batch(b);
        set_error(MPM_ECUDA);
        return nullptr;
    }
    b->stats.tiles = b->ntiles;
    b->stats.bytes = b->bytes;
    set_error(MPM_OK);
    return b;
}

int mpm_batch_run(mpm_batch* b, uint32_t* out_tid, uint32_t* out_pos, uint32_t* out_pid,
                  size_t* z) {
    if (!b || !z) return set_error(MPM_EINVAL);
    if (*z > 0 && (!out_tid || !out_pos || !out_pid)) return set_error(MPM_EINVAL);
    if (cudaSetDevice(b->device) != cudaSuccess) {
        cudaGetLastError();
        return set_error(MPM_ECUDA);
    }
    const size_t out_capacity = *z;
    for (int attempt = 0;; attempt++) {
        cudaEventRecord(b->ev[0], b->stream);
        int rc = b->exec ? (cudaGraphLaunch(b->exec, b->stream) == cudaSuccess ? MPM_OK : MPM_ECUDA)
                         : enqueue_batch(b);
        if (rc) return set_error(rc);
        cudaEventRecord(b->ev[1], b->stream);
        if (cudaStreamSynchronize(b->stream) != cudaSuccess) {
            cudaGetLastError();
            return set_error(MPM_ECUDA);
        }
        if (b->h_counters[mpm::kBError]) return set_error((int)b->h_counters[mpm::kBError]);
        const uint32_t zz = b->h_counters[mpm::kBOcc];
        if (zz > b->cap) {
            // more occurrences than the buffers hold: grow, re-capture, run again
            if (attempt > 3 || alloc_buffers(b, zz + zz / 4 + 1024) != MPM_OK ||
                capture(b) != MPM_OK)
                return set_error(MPM_ENOMEM);
            continue;
        }
        float ms = 0.f, scan_ms = 0.f;
        cudaEventElapsedTime(&ms, b->ev[0], b->ev[1]);
        if (!b->scan_events || cudaEventElapsedTime(&scan_ms, b->ev[2], b->ev[3]) != cudaSuccess)
            scan_ms = 0.f;
        cudaGetLastError();
        b->stats.ms = ms;
        b->stats.scan_ms = scan_ms;
        b->stats.candidates = b->h_counters[mpm::kBCand];
        b->stats.z = zz;
        *z = zz;
        if (zz > out_capacity) return set_error(MPM_ECAPACITY);
        if (zz == 0) return set_error(MPM_OK);
        const bool dev = mpm::on_device(out_tid) && mpm::on_device(out_pos) && mpm::on_device(out_pid);
        const cudaMemcpyKind kind = dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
        if (cudaMemcpyAsync(out_tid, b->d_out, (size_t)zz * 4, kind, b->stream) != cudaSuccess ||
            cudaMemcpyAsync(out_pos, b->d_out + b->cap, (size_t)zz * 4, kind, b->stream) !=
                cudaSuccess ||
            cudaMemcpyAsync(out_pid, b->d_out + 2 * (size_t)b->cap, (size_t)zz * 4, kind,
                            b->stream) != cudaSuccess ||
            cudaStreamSynchronize(b->stream) != cudaSuccess) {
            cudaGetLastError();
            return set_error(MPM_ECUDA);
        }
        return set_error(MPM_OK);
    }
}

int mpm_batch_jit_compile(const uint8_t* const* P, const size_t* r, const size_t* m,
                          const int* sigma, const mpm_params* params, int nsets, char* log,
                          size_t log_bytes) {
    if (!P || !r || !m || !sigma || nsets <= 0) return set_error(MPM_EINVAL);
    std::vector<mpm::BatchVariant> vs;
    for (int i = 0; i < nsets; i++) {
        mpm::Plan plan;
        const int rc = mpm::make_plan(P[i], r[i], m[i], sigma[i], params ? &params[i] : nullptr,
                                      &plan);
        if (rc) return set_error(rc);
        if (plan.info.positions > 32 || plan.p.overlap ||
            (plan.p.map_kind == MPM_MAP_QHASH && plan.p.q > 5))
            return set_error(MPM_ENOTSUP);
        mpm::batch_variant_index(vs, mpm::batch_variant_of(plan));
    }
    std::string text;
    const int rc = mpm::jit_batch_compile_only(vs, &text);
    if (log && log_bytes) {
        const size_t c = std::min(log_bytes - 1, text.size());
        std::memcpy(log, text.data(), c);
        log[c] = 0;
    }
    return set_error(rc);
}

int mpm_batch_get_stats(const mpm_batch* b, mpm_batch_stats* out) {
    if (!b || !out) return set_error(MPM_EINVAL);
    *out = b->stats;
    return set_error(MPM_OK);
}

void mpm_batch_free(mpm_batch* b) { release_batch(b); }

int mpm_search_batch(mpm_handle* const* sets, int nsets, const uint8_t* const* texts,
                     const size_t* lens, const uint32_t* set_of_text, int ntexts,
                     uint32_t* out_tid, uint32_t* out_pos, uint32_t* out_pid, size_t* z) {
    mpm_batch_opts o{};
    o.no_graph = 1;  // a single run gains nothing from a graph
    mpm_batch* b = mpm_batch_create(sets, nsets, texts, lens, set_of_text, ntexts, &o);
    if (!b) return mpm_last_error();
    const int rc = mpm_batch_run(b, out_tid, out_pos, out_pid, z);
    mpm_batch_free(b);
    return set_error(rc);
}

}  // extern "C"
