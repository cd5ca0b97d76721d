// Batched search: many texts of uneven length, each against one of many
// pattern sets, in one persistent launch (the MAG filter of Sections 3.1 and
// 3.2 with each set's own q, k and mapping as runtime values).
//
// Work list.  Every text is cut into tiles of at most 32 lanes x L bytes,
// each lane's range a multiple of its set's sampling period k*q from the
// text start; tiles are listed longest text first.  Warps of a persistent
// grid pop tiles from a device counter; each lane runs the Shift-Or
// recurrence over its range (after warming up on the m'-1 sampled q-grams
// before it), verifies its candidates on the spot against its set's pattern
// groups, and appends (text << 44) | (pos << 20) | pid.  A radix sort driven
// by the device count orders the keys; the whole run -- counter reset, scan,
// sort, split into (text, pos, pid) and the count read-back -- is captured
// once into a CUDA graph and replayed by every run.
#include <algorithm>
#include <cstring>
#include <new>
#include <numeric>
#include <vector>

#include "handle.h"
#include "stepper.cuh"
#include "window_check.cuh"

namespace mpm {

namespace {

struct BatchSet {
    const uint32_t* table;  // mask table widened to 32-bit entries
    const uint8_t* mu;
    const Slot* slots;
    const uint8_t* pat;
    const uint32_t* pid;
    uint32_t slot_mask, key_bytes, m, pad;
    int q, k, mprime, ell, shift, mode, map_kind, pad2;
};

struct BatchText {
    const uint8_t* T;
    uint32_t n, set;
};

struct BatchTile {
    uint32_t text, start, len, sub;
};

enum BatchCounter : int { kQueue = 0, kBOcc = 1, kBError = 2, kBCand = 3 };

constexpr int kPosBits = 24;   // text positions < 2^24 in a batch
constexpr int kPidBits = 20;   // pattern ids < 2^20 per set
constexpr int kTextShift = kPosBits + kPidBits;  // 44

__global__ void widen_kernel(const uint8_t* src, int eb, uint32_t entries, uint32_t* dst) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < entries;
         i += gridDim.x * blockDim.x) {
        uint32_t v = 0;
        for (int b = 0; b < eb && b < 4; b++) v |= (uint32_t)src[(size_t)i * eb + b] << (8 * b);
        dst[i] = v;
    }
}

template <int MODE>
__device__ void batch_lane(const BatchSet& S, const BatchText& tx, uint32_t a, uint32_t b,
                           const WindowCtx& wc, uint32_t* counters) {
    FilterDev f{};
    f.q = S.q;
    f.k = S.k;
    f.ell = S.ell;
    f.shift = S.shift;
    f.map_kind = S.map_kind;
    Stepper<MODE, uint32_t> sp;
    sp.init(f, S.table, S.mu);
    const uint32_t P = (uint32_t)(S.k * S.q);
    const uint32_t Wr = (((uint32_t)(S.mprime - 1) * P) + 3) & ~3u;
    warm_up(sp, tx.T, tx.n, a, Wr, P, true);
    const int rsh = (S.mprime - 1) * S.k;
    const uint32_t kmask = S.k >= 32 ? 0xFFFFFFFFu : ((1u << S.k) - 1u);
    uint32_t hq = a / (uint32_t)S.q + (uint32_t)(S.k - 1);
    int pos = 0, nxt = (int)P;
    const uint32_t words = (b - a + 3) / 4;
    for (uint32_t w = 0; w < words; w++) {
        const uint32_t at = a + 4 * w;
        uint32_t x;
        if (at + 4 <= tx.n) {
            x = load_word(tx.T, at);
        } else {
            x = 0;
            for (uint32_t u = 0; u < 4 && at + u < tx.n; u++) x |= (uint32_t)tx.T[at + u] << (8 * u);
        }
        sp.push(x);
        pos += 4;
        while (nxt <= pos && a + (uint32_t)nxt <= b) {
            const uint32_t c = sp.code(pos - nxt);
            sp.D = (sp.D << S.k) | sp.tab[c];
            uint32_t fired = (uint32_t)(~sp.D >> rsh) & kmask;
            if (fired) {
                atomicAdd(&counters[kBCand], 1u);
                while (fired) {
                    const int j = __ffs((int)fired) - 1;
                    fired &= fired - 1;
                    for (int s = 0; s < S.q; s++) {
                        const int64_t i = ((int64_t)hq - rsh - j) * S.q - s;
                        if (i < 0 || i + (int64_t)S.m > (int64_t)tx.n) continue;
                        check_window(wc, (uint32_t)i);
                    }
                }
            }
            nxt += (int)P;
            hq += (uint32_t)S.k;
        }
        if (nxt <= pos) break;
    }
}

__global__ void __launch_bounds__(256)
    batch_scan_kernel(const BatchSet* sets, const BatchText* texts, const BatchTile* tiles,
                      uint32_t ntiles, uint64_t* occ, uint32_t occ_cap, uint32_t* counters) {
    const int lane = threadIdx.x & 31;
    for (;;) {
        uint32_t t = 0;
        if (lane == 0) t = atomicAdd(&counters[kQueue], 1u);
        t = __shfl_sync(0xFFFFFFFFu, t, 0);
        if (t >= ntiles) break;
        const BatchTile tl = tiles[t];
        const BatchText tx = texts[tl.text];
        const BatchSet S = sets[tx.set];
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
        wc.occ = reinterpret_cast<unsigned long long*>(occ);
        wc.occ_count = &counters[kBOcc];
        wc.tag = (unsigned long long)tl.text << kTextShift;
        wc.pos_shift = kPidBits;
        const uint32_t a = tl.start + (uint32_t)lane * tl.sub;
        const uint32_t b = min(tl.start + tl.len, a + tl.sub);
        if (a >= b) continue;
        switch (S.mode) {
            case kLow2: batch_lane<kLow2>(S, tx, a, b, wc, counters); break;
            case kLowG: batch_lane<kLowG>(S, tx, a, b, wc, counters); break;
            case kLutRed: batch_lane<kLutRed>(S, tx, a, b, wc, counters); break;
            case kLutRaw: batch_lane<kLutRaw>(S, tx, a, b, wc, counters); break;
            default: batch_lane<kQHash>(S, tx, a, b, wc, counters); break;
        }
    }
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

}  // namespace mpm

struct mpm_batch {
    int device = 0, num_sms = 0;
    cudaStream_t stream = nullptr;
    mpm::BatchSet* d_sets = nullptr;
    mpm::BatchText* d_texts = nullptr;
    mpm::BatchTile* d_tiles = nullptr;
    uint32_t ntiles = 0, ntexts = 0;
    std::vector<uint32_t*> tables;
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
    cudaEvent_t ev[2] = {nullptr, nullptr};
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
    for (auto* t : b->tables) cudaFree(t);
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

// Counter reset, scan, sort, split and count read-back on the batch stream.
int enqueue_batch(mpm_batch* b) {
    cudaStream_t s = b->stream;
    if (cudaMemsetAsync(b->d_counters, 0, 16, s) != cudaSuccess) return MPM_ECUDA;
    mpm::batch_scan_kernel<<<b->num_sms * 8, 256, 0, s>>>(b->d_sets, b->d_texts, b->d_tiles,
                                                          b->ntiles, b->d_occ, b->cap,
                                                          b->d_counters);
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

int capture(mpm_batch* b) {
    drop_graph(b);
    if (!b->use_graph) return MPM_OK;
    if (cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
        return MPM_ECUDA;
    int rc = enqueue_batch(b);
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(b->stream, &g);
    if (rc || e != cudaSuccess || !g) {
        cudaGetLastError();
        if (g) cudaGraphDestroy(g);
        return rc ? rc : MPM_ECUDA;
    }
    b->graph = g;
    if (cudaGraphInstantiate(&b->exec, g, 0) != cudaSuccess) {
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
        if (h->plan.p.map_kind == MPM_MAP_QHASH && h->plan.p.q > 5) {
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
              cudaMalloc(&b->d_counters, 16) == cudaSuccess &&
              cudaMallocHost(&b->h_counters, 16) == cudaSuccess;
    // per-set descriptors with tables widened to 32-bit entries
    std::vector<mpm::BatchSet> hs(nsets);
    for (int i = 0; ok && i < nsets; i++) {
        const mpm_handle* h = sets[i];
        const uint32_t entries = (uint32_t)h->plan.info.entries;
        uint32_t* wide = nullptr;
        ok = cudaMalloc(&wide, (size_t)entries * 4) == cudaSuccess;
        if (!ok) break;
        b->tables.push_back(wide);
        mpm::widen_kernel<<<std::min<uint32_t>((entries + 255) / 256, 4096), 256, 0, b->stream>>>(
            static_cast<const uint8_t*>(h->d_table), h->plan.info.entry_bytes, entries, wide);
        mpm::BatchSet S{};
        S.table = wide;
        S.mu = h->d_mu;
        S.slots = h->d_slots;
        S.pat = h->d_pat;
        S.pid = h->d_pid;
        S.slot_mask = (uint32_t)h->host.slots.size() - 1;
        S.key_bytes = (uint32_t)h->host.key_bytes;
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
    // texts and tiles: per lane a multiple of the set's period, longest first
    std::vector<mpm::BatchText> ht(ntexts);
    std::vector<uint32_t> order(ntexts);
    std::iota(order.begin(), order.end(), 0u);
    std::stable_sort(order.begin(), order.end(),
                     [&](uint32_t x, uint32_t y) { return lens[x] > lens[y]; });
    std::vector<mpm::BatchTile> tiles;
    const uint32_t lane_bytes = o.lane_bytes > 0 ? (uint32_t)o.lane_bytes : 1024;
    uint32_t max_r = 1;
    for (int i = 0; i < nsets; i++) max_r = std::max<uint32_t>(max_r, (uint32_t)sets[i]->plan.r);
    for (int t = 0; t < ntexts; t++) {
        ht[t] = mpm::BatchText{texts[t], (uint32_t)lens[t], set_of_text[t]};
        b->bytes += lens[t];
    }
    for (uint32_t t : order) {
        const mpm::BatchSet& S = hs[set_of_text[t]];
        const uint32_t P = (uint32_t)(S.k * S.q);
        const uint32_t n = (uint32_t)lens[t];
        if (n < S.m) continue;
        const uint32_t L = std::max<uint32_t>(P, (lane_bytes + P - 1) / P * P);
        for (uint32_t start = 0; start < n; start += 32 * L) {
            const uint32_t len = std::min<uint32_t>(32 * L, n - start);
            uint32_t sub = (len + 31) / 32;
            sub = std::max<uint32_t>(P, (sub + P - 1) / P * P);
            tiles.push_back(mpm::BatchTile{t, start, len, sub});
        }
    }
    b->ntiles = (uint32_t)tiles.size();
    ok = ok && cudaMalloc(&b->d_sets, sizeof(mpm::BatchSet) * nsets) == cudaSuccess &&
         cudaMalloc(&b->d_texts, sizeof(mpm::BatchText) * ntexts) == cudaSuccess &&
         cudaMalloc(&b->d_tiles, sizeof(mpm::BatchTile) * std::max<size_t>(1, tiles.size())) ==
             cudaSuccess;
    ok = ok &&
         cudaMemcpy(b->d_sets, hs.data(), sizeof(mpm::BatchSet) * nsets, cudaMemcpyHostToDevice) ==
             cudaSuccess &&
         cudaMemcpy(b->d_texts, ht.data(), sizeof(mpm::BatchText) * ntexts,
                    cudaMemcpyHostToDevice) == cudaSuccess &&
         (tiles.empty() || cudaMemcpy(b->d_tiles, tiles.data(), sizeof(mpm::BatchTile) * tiles.size(),
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
        float ms = 0.f;
        cudaEventElapsedTime(&ms, b->ev[0], b->ev[1]);
        b->stats.ms = ms;
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
