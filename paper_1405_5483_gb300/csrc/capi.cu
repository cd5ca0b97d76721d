// C ABI: handle life cycle and the orchestration of one search.
//
// mpm_search enqueues, on the handle's stream: the counter reset, the MAG
// scan (or SMAG encode + scan), the verification kernel and a 16-byte
// read-back of the counters; it waits for that read-back, grows an internal
// buffer and re-runs if one overflowed, then enqueues the sort that writes
// the caller's outputs.
#include <algorithm>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>

#include "handle.h"

namespace mpm {

static thread_local int t_last_error = MPM_OK;

int set_error(int code) {
    t_last_error = code;
    return code;
}

}  // namespace mpm

namespace {

using mpm::set_error;

template <typename T>
int grow(T** p, size_t* cap, size_t want) {
    if (*cap >= want && *p) return MPM_OK;
    if (*p) cudaFree(*p);
    *p = nullptr;
    *cap = 0;
    size_t n = std::max<size_t>(want, 16);
    if (cudaMalloc(reinterpret_cast<void**>(p), n * sizeof(T)) != cudaSuccess) {
        cudaGetLastError();
        return MPM_ENOMEM;
    }
    *cap = n;
    return MPM_OK;
}

bool is_device_ptr(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

mpm::FilterDev filter_dev(const mpm_handle* h) {
    mpm::FilterDev f;
    f.table = h->d_table;
    f.table_bytes = h->table_bytes_padded;
    f.entry_bytes = h->plan.info.entry_bytes;
    f.entry_bits = h->plan.info.entry_bits;
    f.smem_table = h->plan.p.table_place == MPM_TABLE_SMEM;
    f.mu = h->d_mu;
    f.map_kind = h->plan.p.map_kind;
    f.q = h->plan.p.q;
    f.k = h->plan.p.k;
    f.ell = h->plan.ell;
    f.shift = h->plan.p.map_shift;
    f.mprime = h->plan.info.mprime;
    f.positions = h->plan.info.positions;
    f.overlap = h->plan.p.overlap;
    return f;
}

void release(mpm_handle* h) {
    if (!h) return;
    if (h->stream) cudaStreamSynchronize(h->stream);
    else cudaDeviceSynchronize();
    cudaFree(h->d_mu);
    cudaFree(h->d_table);
    cudaFree(h->d_slots);
    cudaFree(h->d_pat);
    cudaFree(h->d_pat_off);
    cudaFree(h->d_pid);
    cudaFree(h->d_keys);
    cudaFree(h->d_cand);
    cudaFree(h->d_occ);
    cudaFree(h->d_occ_tmp);
    cudaFree(h->d_hist);
    cudaFree(h->d_counters);
    if (h->h_counters) cudaFreeHost(h->h_counters);
    if (h->h_snap) cudaFreeHost(h->h_snap);
    if (h->side) {
        cudaStreamSynchronize(h->side);
        cudaStreamDestroy(h->side);
    }
    for (int b = 0; b < 2; b++) {
        if (h->scan_done[b]) cudaEventDestroy(h->scan_done[b]);
        if (h->sort_done[b]) cudaEventDestroy(h->sort_done[b]);
    }
    cudaFree(h->d_cand1);
    cudaFree(h->d_occ1);
    cudaFree(h->d_occ1_tmp);
    cudaFree(h->d_ahist[0]);
    cudaFree(h->d_ahist[1]);
    cudaFree(h->d_counters1);
    for (auto& trio : h->ring)
        for (auto& e : trio)
            if (e) cudaEventDestroy(e);
    cudaFree(h->d_text);
    cudaFree(h->d_codes);
    cudaFree(h->d_out);
    for (auto& e : h->ev)
        if (e) cudaEventDestroy(e);
    cudaGetLastError();
    delete h;
}

int bits_for(uint64_t v) {
    int b = 0;
    while (b < 64 && (v >> b)) b++;
    return b;
}

mpm::ScanArgs scan_args(const mpm_handle* h, const uint8_t* dT, uint32_t n, uint64_t* cand,
                        uint32_t cap, uint32_t* counters) {
    mpm::ScanArgs a{};
    a.T = dT;
    a.n = n;
    a.f = filter_dev(h);
    // bytes per sampled q-gram: k q non-overlapping, k overlapping
    a.P = (uint32_t)(a.f.overlap ? a.f.k : a.f.k * a.f.q);
    const uint32_t wb = (uint32_t)(a.f.mprime - 1) * a.P;
    a.warm_bytes = (wb + 3) & ~3u;
    a.cand = cand;
    a.cap = cap;
    a.counters = counters;
    return a;
}

mpm::VerifyArgs verify_args(const mpm_handle* h, const uint8_t* dT, uint32_t n,
                            const uint64_t* cand, uint32_t cand_cap, uint64_t* occ,
                            uint32_t occ_cap, uint32_t* counters) {
    mpm::VerifyArgs v{};
    v.T = dT;
    v.n = n;
    v.m = (uint32_t)h->plan.m;
    // a record's window h0 stands for the starts h0 q - s, s < q; an
    // overlapping q-gram window for its own start h0 (one shift, factor 1)
    v.q = h->plan.p.overlap ? 1 : h->plan.p.q;
    v.k = h->plan.p.k;
    v.mprime = h->plan.info.mprime;
    v.cand = cand;
    v.cand_cap = cand_cap;
    v.slots = h->d_slots;
    v.slot_mask = (uint32_t)h->host.slots.size() - 1;
    v.pat = h->d_pat;
    v.pid = h->d_pid;
    v.pat_off = h->d_pat_off;
    v.key_bytes = h->host.key_bytes;
    v.keys = h->d_keys;
    v.key_mask = h->key_bits - 1;
    v.occ = occ;
    v.occ_cap = occ_cap;
    v.counters = counters;
    return v;
}

// True when mpm_search runs the specialised scan that verifies by itself.
bool fused_search(const mpm_handle* h) { return h->jit && !h->plan.p.smag; }

// Enqueues, without synchronising: the counter reset, the scan and the
// verification of text dT (device).  Occurrence keys go to occ, candidate
// records (generic and SMAG paths only) to cand.
int enqueue_filter(mpm_handle* h, const uint8_t* dT, uint32_t n, uint64_t* cand,
                   uint32_t cand_cap, uint64_t* occ, uint32_t occ_cap, uint32_t* counters,
                   int* launches, bool reset = true, cudaEvent_t* events = nullptr) {
    // events: three events recorded before the scan, between scan and
    // verification and after verification; the handle's when timing is on
    cudaEvent_t* ev = events ? events : (h->timing ? h->ev : nullptr);
    cudaStream_t s = h->stream;
    const mpm::FilterDev f = filter_dev(h);
    if (reset &&
        cudaMemsetAsync(counters, 0, mpm::kNumCounters * sizeof(uint32_t), s) != cudaSuccess)
        return MPM_ECUDA;
    const mpm::VerifyArgs v = verify_args(h, dT, n, cand, cand_cap, occ, occ_cap, counters);
    if (ev) cudaEventRecord(ev[0], s);
    int l;
    if (h->plan.p.smag) {
        const size_t nq = n / (uint32_t)f.q;
        if (grow(&h->d_codes, &h->codes_cap, nq)) return MPM_ENOMEM;
        l = mpm::launch_encode(dT, n, f, h->d_codes, s);
        if (l < 0) return MPM_ECUDA;
        *launches += l;
        l = mpm::launch_scan_codes(h->d_codes, (uint32_t)nq, f, cand, cand_cap, counters, s);
    } else if (fused_search(h)) {
        l = mpm::launch_scan_jit(scan_args(h, dT, n, cand, cand_cap, counters), &v, h->jit,
                                 h->num_sms, h->plan.p.chunk, s);
        if (l < 0) return MPM_ECUDA;
        *launches += l;
        if (ev) {
            cudaEventRecord(ev[1], s);
            cudaEventRecord(ev[2], s);
        }
        return MPM_OK;
    } else if (h->jit_cand) {
        // split: the specialised scan writes candidates, verification follows
        l = mpm::launch_scan_jit(scan_args(h, dT, n, cand, cand_cap, counters), nullptr,
                                 h->jit_cand, h->num_sms, h->plan.p.chunk, s);
    } else {
        l = mpm::launch_scan(scan_args(h, dT, n, cand, cand_cap, counters), h->num_sms,
                             h->plan.p.chunk, s);
    }
    if (l == -2) return MPM_ENOTSUP;
    if (l < 0) return MPM_ECUDA;
    *launches += l;
    if (ev) cudaEventRecord(ev[1], s);
    if (mpm::launch_verify(v, h->num_sms, s) < 0) return MPM_ECUDA;
    *launches += 1;
    if (ev) cudaEventRecord(ev[2], s);
    return MPM_OK;
}

// The one synchronisation of a search: the counters come back to the host.
int read_counters(mpm_handle* h, const uint32_t* counters) {
    cudaStream_t s = h->stream;
    if (cudaMemcpyAsync(h->h_counters, counters, mpm::kNumCounters * sizeof(uint32_t),
                        cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return MPM_ECUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return MPM_ECUDA;
    if (h->h_counters[mpm::kErrorFlag]) return (int)h->h_counters[mpm::kErrorFlag];
    if (h->timing) {
        float a = 0.f, b = 0.f;
        cudaEventElapsedTime(&a, h->ev[0], h->ev[1]);
        cudaEventElapsedTime(&b, h->ev[1], h->ev[2]);
        h->stats.ms_scan += a;
        h->stats.ms_verify += b;
    }
    return MPM_OK;
}

// The device address of a status block: device memory as is, mapped host
// memory through its device alias; null for anything else.
uint32_t* device_address(uint32_t* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged)
        return p;
    if (a.type == cudaMemoryTypeHost && a.devicePointer) return static_cast<uint32_t*>(a.devicePointer);
    return nullptr;
}

// Folds the device times of recorded pipelined searches into the
// statistics; wait = true waits for those still in flight.
int harvest_timing(mpm_handle* h, bool wait) {
    for (int i = 0; i < mpm_handle::kRing; i++) {
        if (!h->ring_used[i]) continue;
        cudaError_t e = cudaEventQuery(h->ring[i][2]);
        if (e == cudaErrorNotReady) {
            if (!wait) continue;
            e = cudaEventSynchronize(h->ring[i][2]);
        }
        if (e != cudaSuccess) {
            cudaGetLastError();
            return MPM_ECUDA;
        }
        float a = 0.f, b = 0.f;
        cudaEventElapsedTime(&a, h->ring[i][0], h->ring[i][1]);
        cudaEventElapsedTime(&b, h->ring[i][1], h->ring[i][2]);
        h->stats.ms_scan += a;
        h->stats.ms_verify += b;
        h->ring_used[i] = 0;
    }
    return MPM_OK;
}

// The next event triple of the ring; its earlier recording (long finished in
// a steady pipeline) is folded into the statistics first.
int next_timing_slot(mpm_handle* h, cudaEvent_t** ev) {
    const int i = h->ring_next;
    if (!h->ring[i][0]) {
        for (auto& e : h->ring[i])
            if (cudaEventCreate(&e) != cudaSuccess) {
                cudaGetLastError();
                return MPM_ECUDA;
            }
    }
    if (h->ring_used[i]) {
        if (cudaEventSynchronize(h->ring[i][2]) != cudaSuccess) {
            cudaGetLastError();
            return MPM_ECUDA;
        }
        float a = 0.f, b = 0.f;
        cudaEventElapsedTime(&a, h->ring[i][0], h->ring[i][1]);
        cudaEventElapsedTime(&b, h->ring[i][1], h->ring[i][2]);
        h->stats.ms_scan += a;
        h->stats.ms_verify += b;
    }
    h->ring_used[i] = 1;
    h->ring_next = (i + 1) % mpm_handle::kRing;
    *ev = h->ring[i];
    return MPM_OK;
}

// Orders everything enqueued on the handle's stream from now on after the
// closing sorts of pipelined searches still running on the side stream.
int join_sorts(mpm_handle* h) {
    for (int b = 0; b < 2; b++) {
        if (!h->sort_pending[b]) continue;
        if (cudaStreamWaitEvent(h->stream, h->sort_done[b], 0) != cudaSuccess) {
            cudaGetLastError();
            return MPM_ECUDA;
        }
        h->sort_pending[b] = false;
    }
    return MPM_OK;
}

// The end of a search closed by the rank sort kernel: wait for the stream and
// take the counters from the mapped snapshot.
int finish_counters(mpm_handle* h) {
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) return MPM_ECUDA;
    for (int i = 0; i < mpm::kNumCounters; i++)
        h->h_counters[i] = reinterpret_cast<volatile uint32_t*>(h->h_snap)[i];
    if (h->h_counters[mpm::kErrorFlag]) return (int)h->h_counters[mpm::kErrorFlag];
    if (h->timing) {
        float a = 0.f, b = 0.f;
        cudaEventElapsedTime(&a, h->ev[0], h->ev[1]);
        cudaEventElapsedTime(&b, h->ev[1], h->ev[2]);
        h->stats.ms_scan += a;
        h->stats.ms_verify += b;
    }
    return MPM_OK;
}

int prepare(mpm_handle* h) {
    cudaError_t e = cudaSetDevice(h->device);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return MPM_ECUDA;
    }
    return MPM_OK;
}

}  // namespace

extern "C" {

int mpm_last_error(void) { return mpm::t_last_error; }

const char* mpm_strerror(int code) {
    switch (code) {
        case MPM_OK: return "ok";
        case MPM_EINVAL: return "invalid argument or infeasible parameter";
        case MPM_ENOMEM: return "out of memory";
        case MPM_ECUDA: return "CUDA error (no device, launch or copy failure)";
        case MPM_ECAPACITY: return "output capacity too small";
        case MPM_ETIMEOUT: return "bounded device wait timed out";
        case MPM_ENOTSUP: return "unsupported combination";
        case MPM_ESCRATCH:
            return "the search needs more scratch than the fixed buffer of "
                   "mpm_search_noalloc holds; use mpm_search";
        default: return "unknown error";
    }
}

// P: r x m (the filter's patterns).  full/off (may be null): the patterns
// themselves when they differ in length, pattern p = full[off[p] .. off[p+1]),
// P holding their first m bytes.
static mpm_handle* build_handle(const uint8_t* P, size_t r, size_t m, int sigma,
                                const mpm_params* params, const uint8_t* full, const size_t* off) {
    mpm_handle* h = new (std::nothrow) mpm_handle();
    if (!h) {
        set_error(MPM_ENOMEM);
        return nullptr;
    }
    int rc = mpm::make_plan(P, r, m, sigma, params, &h->plan);
    if (rc) {
        delete h;
        set_error(rc);
        return nullptr;
    }
    if (h->plan.info.entry_bits < 8) {
        // a packed table is read by the specialised kernels only: without
        // them (no NVRTC, or a compilation error) the table is built
        // unpacked, in global memory
        const mpm::Plan packed = h->plan;
        h->table_bytes_padded = (uint32_t)((packed.info.table_bytes + 15) & ~uint64_t(15));
        int dev = 0, err = MPM_OK;
        std::string log;
        const bool jit_ok = cudaGetDevice(&dev) == cudaSuccess &&
                            mpm::jit_scan_kernel(filter_dev(h), packed.p.kernel != MPM_KERNEL_SPLIT,
                                                 dev, &err, &log) != nullptr;
        if (!jit_ok) {
            cudaGetLastError();
            h->plan.info.entry_bits = 8 * h->plan.info.entry_bytes;
            h->plan.info.table_bytes = h->plan.info.entries * (uint64_t)h->plan.info.entry_bytes;
            h->plan.p.table_place = MPM_TABLE_GLOBAL;
        }
    }
    if (h->plan.p.smag && (h->plan.p.overlap || h->plan.info.entry_bytes > 8)) {
        // SMAG encodes the text's non-overlapping q-grams and scans them with
        // one word of state
        delete h;
        set_error(MPM_ENOTSUP);
        return nullptr;
    }
    // host tables
    try {
        mpm::make_mu(P, r, m, h->plan.p.map_kind, h->plan.p.sigma_r, h->plan.p.map_shift,
                     h->host.mu);
        h->table_bytes_padded = (uint32_t)((h->plan.info.table_bytes + 15) & ~uint64_t(15));
        h->host.table.assign(h->table_bytes_padded, 0xFF);
        mpm::make_mask_table(P, h->plan, h->host.mu, h->host.table.data());
        if (full)
            mpm::make_verify_tables_var(full, off, r, m, &h->host);
        else
            mpm::make_verify_tables(P, r, m, &h->host);
    } catch (const std::bad_alloc&) {
        delete h;
        set_error(MPM_ENOMEM);
        return nullptr;
    }
    if (cudaGetDevice(&h->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device) !=
            cudaSuccess) {
        cudaGetLastError();
        delete h;
        set_error(MPM_ECUDA);
        return nullptr;
    }
    std::vector<uint32_t> keys;
    try {
        keys = mpm::key_bitmap(h->host, mpm::kVerifyKeyBitsMax);
    } catch (const std::bad_alloc&) {
        delete h;
        set_error(MPM_ENOMEM);
        return nullptr;
    }
    h->key_bits = (uint32_t)keys.size() * 32;
    bool ok = cudaMalloc(&h->d_mu, 256) == cudaSuccess &&
              cudaMalloc(&h->d_keys, keys.size() * 4) == cudaSuccess &&
              cudaMalloc(&h->d_table, h->table_bytes_padded) == cudaSuccess &&
              cudaMalloc(&h->d_slots, h->host.slots.size() * sizeof(mpm::Slot)) == cudaSuccess &&
              cudaMalloc(&h->d_pat, h->host.sorted_pat.size()) == cudaSuccess &&
              cudaMalloc(&h->d_pid, h->host.sorted_pid.size() * 4) == cudaSuccess &&
              (h->host.sorted_off.empty() ||
               cudaMalloc(&h->d_pat_off, h->host.sorted_off.size() * 4) == cudaSuccess) &&
              cudaMalloc(&h->d_counters, mpm::kNumCounters * 4) == cudaSuccess &&
              cudaMemset(h->d_counters, 0, mpm::kNumCounters * 4) == cudaSuccess &&
              cudaMallocHost(&h->h_counters, mpm::kNumCounters * 4) == cudaSuccess &&
              cudaHostAlloc(&h->h_snap, mpm::kNumCounters * 4, cudaHostAllocMapped) == cudaSuccess &&
              cudaHostGetDevicePointer(&h->d_snap, h->h_snap, 0) == cudaSuccess;
    ok = ok && cudaMemcpy(h->d_mu, h->host.mu, 256, cudaMemcpyHostToDevice) == cudaSuccess &&
         cudaMemcpy(h->d_keys, keys.data(), keys.size() * 4, cudaMemcpyHostToDevice) ==
             cudaSuccess &&
         cudaMemcpy(h->d_table, h->host.table.data(), h->table_bytes_padded,
                    cudaMemcpyHostToDevice) == cudaSuccess &&
         cudaMemcpy(h->d_slots, h->host.slots.data(), h->host.slots.size() * sizeof(mpm::Slot),
                    cudaMemcpyHostToDevice) == cudaSuccess &&
         cudaMemcpy(h->d_pat, h->host.sorted_pat.data(), h->host.sorted_pat.size(),
                    cudaMemcpyHostToDevice) == cudaSuccess &&
         cudaMemcpy(h->d_pid, h->host.sorted_pid.data(), h->host.sorted_pid.size() * 4,
                    cudaMemcpyHostToDevice) == cudaSuccess &&
         (h->host.sorted_off.empty() ||
          cudaMemcpy(h->d_pat_off, h->host.sorted_off.data(), h->host.sorted_off.size() * 4,
                     cudaMemcpyHostToDevice) == cudaSuccess);
    if (!ok) {
        cudaGetLastError();
        release(h);
        set_error(MPM_ECUDA);
        return nullptr;
    }
    h->host.table.clear();
    h->host.table.shrink_to_fit();
    if (!h->plan.p.smag && h->plan.p.kernel != MPM_KERNEL_GENERIC) {
        int err = MPM_OK;
        std::string log;
        const bool split = h->plan.p.kernel == MPM_KERNEL_SPLIT;
        if (split) {
            h->jit_cand = mpm::jit_scan_kernel(filter_dev(h), false, h->device, &err, &log);
            h->jit_cand_tried = true;
        } else {
            h->jit = mpm::jit_scan_kernel(filter_dev(h), true, h->device, &err, &log);
        }
        if (!h->jit && !h->jit_cand && (h->plan.p.kernel == MPM_KERNEL_SPECIALISED || split)) {
            if (!log.empty()) std::fprintf(stderr, "mpm: specialised scan failed:\n%s\n", log.c_str());
            release(h);
            set_error(err ? err : MPM_ENOTSUP);
            return nullptr;
        }
    }
    set_error(MPM_OK);
    return h;
}

mpm_handle* mpm_build(const uint8_t* P, size_t r, size_t m, int sigma, const mpm_params* params) {
    return build_handle(P, r, m, sigma, params, nullptr, nullptr);
}

mpm_handle* mpm_build_var(const uint8_t* P, const size_t* off, size_t r, int sigma,
                          const mpm_params* params) {
    if (!P || !off || r == 0 || off[0] != 0) {
        set_error(MPM_EINVAL);
        return nullptr;
    }
    size_t mmin = SIZE_MAX, mmax = 0;
    for (size_t p = 0; p < r; p++) {
        if (off[p + 1] <= off[p]) {  // every pattern at least one byte
            set_error(MPM_EINVAL);
            return nullptr;
        }
        mmin = std::min(mmin, off[p + 1] - off[p]);
        mmax = std::max(mmax, off[p + 1] - off[p]);
    }
    if (off[r] >= (1ull << 32)) {
        set_error(MPM_EINVAL);
        return nullptr;
    }
    // the filter runs on the first mmin bytes of every pattern
    std::vector<uint8_t> prefix;
    try {
        prefix.resize(r * mmin);
    } catch (const std::bad_alloc&) {
        set_error(MPM_ENOMEM);
        return nullptr;
    }
    for (size_t p = 0; p < r; p++) std::memcpy(&prefix[p * mmin], P + off[p], mmin);
    if (mmin == mmax) return build_handle(prefix.data(), r, mmin, sigma, params, nullptr, nullptr);
    return build_handle(prefix.data(), r, mmin, sigma, params, P, off);
}

void mpm_free(mpm_handle* h) { release(h); }

int mpm_set_stream(mpm_handle* h, void* stream) {
    if (!h) return set_error(MPM_EINVAL);
    h->stream = reinterpret_cast<cudaStream_t>(stream);
    // the new stream comes after the closing sorts still in flight
    return set_error(join_sorts(h));
}

int mpm_get_params(const mpm_handle* h, mpm_params* out, mpm_table_info* info) {
    if (!h || !out) return set_error(MPM_EINVAL);
    *out = h->plan.p;
    if (info) *info = h->plan.info;
    return set_error(MPM_OK);
}

int mpm_set_timing(mpm_handle* h, int on) {
    if (!h) return set_error(MPM_EINVAL);
    if (on && !h->ev[0]) {
        for (auto& e : h->ev)
            if (cudaEventCreate(&e) != cudaSuccess) {
                cudaGetLastError();
                return set_error(MPM_ECUDA);
            }
    }
    h->timing = on ? 1 : 0;
    return set_error(MPM_OK);
}

int mpm_get_stats(const mpm_handle* h, mpm_stats* out) {
    if (!h || !out) return set_error(MPM_EINVAL);
    *out = h->stats;
    return set_error(MPM_OK);
}

int mpm_search(mpm_handle* h, const uint8_t* T, size_t n, uint32_t* out_pos, uint32_t* out_pid,
               size_t* z) {
    if (!h || !z || (n > 0 && !T) || n >= (1ull << 32)) return set_error(MPM_EINVAL);
    if (*z > 0 && (!out_pos || !out_pid)) return set_error(MPM_EINVAL);
    int rc = prepare(h);
    if (rc) return set_error(rc);
    const size_t out_capacity = *z;
    rc = join_sorts(h);  // set 0's buffers may still be read by a pipelined sort
    if (rc) return set_error(rc);
    rc = harvest_timing(h, true);  // pipelined searches still timed belong to before
    if (rc) return set_error(rc);
    h->stats = mpm_stats{};
    h->stats.n = n;
    h->stats.specialised = (h->jit || h->jit_cand) && !h->plan.p.smag ? 1u : 0u;
    const uint32_t q = (uint32_t)h->plan.p.q, k = (uint32_t)h->plan.p.k;
    h->stats.sampled = (n / q) / k;
    int launches = 0;
    if (n < h->plan.m) {
        *z = 0;
        return set_error(MPM_OK);
    }
    cudaStream_t s = h->stream;
    // the text on the device
    const uint8_t* dT = T;
    if (!is_device_ptr(T)) {
        if (grow(&h->d_text, &h->text_cap, n)) return set_error(MPM_ENOMEM);
        if (cudaMemcpyAsync(h->d_text, T, n, cudaMemcpyHostToDevice, s) != cudaSuccess)
            return set_error(MPM_ECUDA);
        dT = h->d_text;
    }
    // first-call capacities: a candidate rate of 1/64 per byte (unused by the
    // specialised scan, which verifies its candidates itself), 64K occurrences
    if (!fused_search(h) &&
        grow(&h->d_cand, &h->cand_cap, std::max<size_t>(1 << 16, n / 64 + 1024)))
        return set_error(MPM_ENOMEM);
    if (!h->d_occ || h->occ_cap < (1u << 16)) {
        size_t c = 0;
        if (grow(&h->d_occ, &h->occ_cap, 1 << 16) || grow(&h->d_occ_tmp, &c, 1 << 16))
            return set_error(MPM_ENOMEM);
    }
    // where the rank sort writes: the caller's device outputs, or staging
    const bool dev_out =
        out_capacity == 0 || (is_device_ptr(out_pos) && is_device_ptr(out_pid));
    const uint32_t rank_cap = (uint32_t)std::min<size_t>(out_capacity, mpm::kRankSortMax);
    uint32_t* op = out_pos;
    uint32_t* oi = out_pid;
    if (!dev_out) {
        if (grow(&h->d_out, &h->out_cap, 2 * (size_t)rank_cap)) return set_error(MPM_ENOMEM);
        op = h->d_out;
        oi = h->d_out + rank_cap;
    }
    for (int attempt = 0;; attempt++) {
        // the counters are zero unless an earlier call left them otherwise;
        // the rank sort kernel closes the search and zeroes them again
        const bool reset = h->counters_dirty;
        h->counters_dirty = true;
        rc = enqueue_filter(h, dT, (uint32_t)n, h->d_cand, (uint32_t)h->cand_cap, h->d_occ,
                            (uint32_t)h->occ_cap, h->d_counters, &launches, reset);
        if (rc) return set_error(rc);
        if (mpm::launch_rank_sort(h->d_occ, h->d_counters, rank_cap, op, oi, h->d_snap,
                                  fused_search(h) ? 0xFFFFFFFFu : (uint32_t)h->cand_cap,
                                  (uint32_t)h->occ_cap, s) < 0)
            return set_error(MPM_ECUDA);
        launches++;
        rc = finish_counters(h);
        if (rc) return set_error(rc);
        h->counters_dirty = false;
        const uint32_t nc = h->h_counters[mpm::kCandCount];
        const uint32_t nz = h->h_counters[mpm::kOccCount];
        bool again = false;
        if (!fused_search(h) && nc > h->cand_cap) {
            if (grow(&h->d_cand, &h->cand_cap, (size_t)nc + nc / 4 + 1024))
                return set_error(MPM_ENOMEM);
            again = true;
        }
        if (nz > h->occ_cap) {
            size_t want = (size_t)nz + nz / 4 + 1024, c2 = 0;
            cudaFree(h->d_occ_tmp);
            h->d_occ_tmp = nullptr;
            if (grow(&h->d_occ, &h->occ_cap, want) || grow(&h->d_occ_tmp, &c2, want))
                return set_error(MPM_ENOMEM);
            again = true;
        }
        if (!again) break;
        h->stats.retries++;
        if (attempt > 4) return set_error(MPM_ENOMEM);
    }
    const uint32_t zz = h->h_counters[mpm::kOccCount];
    h->stats.candidates = h->h_counters[mpm::kCandCount];
    h->stats.z = zz;
    *z = zz;
    if (zz > out_capacity) {
        h->stats.launches = launches;
        return set_error(MPM_ECAPACITY);
    }
    if (zz > mpm::kRankSortMax) {
        // too many for the rank sort: sort now that the count is known
        if (!dev_out) {
            if (grow(&h->d_out, &h->out_cap, 2 * (size_t)zz)) return set_error(MPM_ENOMEM);
            op = h->d_out;
            oi = h->d_out + zz;
        }
        if (grow(&h->d_hist, &h->hist_cap, mpm::sort_hist_entries(zz))) return set_error(MPM_ENOMEM);
        const uint32_t key_bits =
            ((uint32_t)bits_for(n) << 16) | (uint32_t)bits_for(h->plan.r > 1 ? h->plan.r - 1 : 1);
        int l = mpm::launch_sort_output(h->d_occ, h->d_occ_tmp, h->d_hist, h->hist_cap, zz,
                                        key_bits, op, oi, s);
        if (l < 0) return set_error(MPM_ECUDA);
        launches += l;
    }
    if (!dev_out && zz > 0) {
        if (cudaMemcpyAsync(out_pos, op, (size_t)zz * 4, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaMemcpyAsync(out_pid, oi, (size_t)zz * 4, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return set_error(MPM_ECUDA);
    }
    h->stats.launches = launches;
    return set_error(MPM_OK);
}

int mpm_search_async(mpm_handle* h, const uint8_t* T, size_t n, uint32_t* out_pos,
                     uint32_t* out_pid, size_t cap, uint32_t* status) {
    if (!h || !status || (n > 0 && !T) || n >= (1ull << 32)) return set_error(MPM_EINVAL);
    if (cap > 0 && (!out_pos || !out_pid)) return set_error(MPM_EINVAL);
    int rc = prepare(h);
    if (rc) return set_error(rc);
    if ((n > 0 && !is_device_ptr(T)) ||
        (cap > 0 && (!is_device_ptr(out_pos) || !is_device_ptr(out_pid))))
        return set_error(MPM_EINVAL);
    uint32_t* dstatus = device_address(status);
    if (!dstatus) return set_error(MPM_EINVAL);
    cudaStream_t s = h->stream;
    // the side stream, its events and buffer set 1 on first use
    if (!h->side) {
        if (cudaStreamCreateWithFlags(&h->side, cudaStreamNonBlocking) != cudaSuccess ||
            cudaMalloc(&h->d_counters1, mpm::kNumCounters * 4) != cudaSuccess ||
            cudaMemset(h->d_counters1, 0, mpm::kNumCounters * 4) != cudaSuccess) {
            cudaGetLastError();
            return set_error(MPM_ECUDA);
        }
        for (int b = 0; b < 2; b++)
            if (cudaEventCreateWithFlags(&h->scan_done[b], cudaEventDisableTiming) != cudaSuccess ||
                cudaEventCreateWithFlags(&h->sort_done[b], cudaEventDisableTiming) != cudaSuccess) {
                cudaGetLastError();
                return set_error(MPM_ECUDA);
            }
    }
    // buffers as mpm_search sizes them on its first call, the same in both
    // sets (allocation waits for the device only when a buffer grows)
    if (!fused_search(h) &&
        (grow(&h->d_cand, &h->cand_cap, std::max<size_t>(1 << 16, n / 64 + 1024)) ||
         grow(&h->d_cand1, &h->cand1_cap, h->cand_cap)))
        return set_error(MPM_ENOMEM);
    if (!h->d_occ || h->occ_cap < (1u << 16)) {
        size_t c = 0;
        if (grow(&h->d_occ, &h->occ_cap, 1 << 16) || grow(&h->d_occ_tmp, &c, 1 << 16))
            return set_error(MPM_ENOMEM);
    }
    if (grow(&h->d_occ1, &h->occ1_cap, h->occ_cap)) return set_error(MPM_ENOMEM);
    const int b = h->async_set;
    uint64_t* cand = b ? h->d_cand1 : h->d_cand;
    const size_t cand_cap = b ? h->cand1_cap : h->cand_cap;
    uint64_t* occ = b ? h->d_occ1 : h->d_occ;
    const size_t occ_cap = b ? h->occ1_cap : h->occ_cap;
    uint32_t* counters = b ? h->d_counters1 : h->d_counters;
    bool& dirty = b ? h->counters1_dirty : h->counters_dirty;

    const uint32_t q = (uint32_t)h->plan.p.q, k = (uint32_t)h->plan.p.k;
    h->stats.n += n;
    h->stats.sampled += (n / q) / k;
    h->stats.specialised = (h->jit || h->jit_cand) && !h->plan.p.smag ? 1u : 0u;
    cudaEvent_t* ev = nullptr;
    if (h->timing) {
        rc = next_timing_slot(h, &ev);
        if (rc) return set_error(rc);
    }
    // the set's previous sort must have read its keys and zeroed its counters
    if (h->sort_pending[b] && cudaStreamWaitEvent(s, h->sort_done[b], 0) != cudaSuccess) {
        cudaGetLastError();
        return set_error(MPM_ECUDA);
    }
    const bool reset = dirty;
    dirty = true;
    int launches = 0;
    if (n >= h->plan.m) {
        rc = enqueue_filter(h, T, (uint32_t)n, cand, (uint32_t)cand_cap, occ, (uint32_t)occ_cap,
                            counters, &launches, reset, ev);
        if (rc) return set_error(rc);
    } else {
        if (reset && cudaMemsetAsync(counters, 0, mpm::kNumCounters * 4, s) != cudaSuccess)
            return set_error(MPM_ECUDA);
        if (ev) {
            for (int i = 0; i < 3; i++) cudaEventRecord(ev[i], s);
        }
    }
    // the closing sort on the side stream, after this scan: the rank sort
    // up to kRankSortMax occurrences; with room for more in the outputs, a
    // radix sort after it that reads the count on the device and returns at
    // once when the rank sort had them all -- one block for outputs of up to
    // kBlockSortCap, else the multi-block passes and the closing kernel
    const uint32_t rank_cap = (uint32_t)std::min<size_t>(cap, mpm::kRankSortMax);
    const bool radix = cap > mpm::kRankSortMax;
    const bool one_block = cap <= mpm::kBlockSortCap;
    const uint32_t cand_lim = fused_search(h) ? 0xFFFFFFFFu : (uint32_t)cand_cap;
    uint64_t* tmp = nullptr;
    const uint32_t sort_cap = (uint32_t)std::min<size_t>(cap, occ_cap);
    if (radix) {
        if (b == 0) {
            tmp = h->d_occ_tmp;  // grown with d_occ
        } else {
            if (grow(&h->d_occ1_tmp, &h->occ1_tmp_cap, occ_cap)) return set_error(MPM_ENOMEM);
            tmp = h->d_occ1_tmp;
        }
        if (!one_block &&
            grow(&h->d_ahist[b], &h->ahist_cap[b], mpm::sort_dev_hist_entries(sort_cap)))
            return set_error(MPM_ENOMEM);
    }
    if (cudaEventRecord(h->scan_done[b], s) != cudaSuccess ||
        cudaStreamWaitEvent(h->side, h->scan_done[b], 0) != cudaSuccess ||
        mpm::launch_rank_sort(occ, counters, rank_cap, out_pos, out_pid,
                              radix ? nullptr : dstatus, cand_lim, (uint32_t)occ_cap,
                              h->side) < 0) {
        cudaGetLastError();
        return set_error(MPM_ECUDA);
    }
    launches++;
    if (radix) {
        // digits of the key (pos << 32) | pid that can be non-zero
        int shifts[8], ns = 0;
        const int pid_bits = bits_for(h->plan.r > 1 ? h->plan.r - 1 : 1);
        const int pos_bits = bits_for(n);
        for (int v = 0; v < pid_bits; v += 8) shifts[ns++] = v;
        for (int v = 0; v < pos_bits; v += 8) shifts[ns++] = 32 + v;
        int l;
        if (one_block) {
            l = mpm::launch_block_sort_close(occ, tmp, counters, (uint32_t)cap, out_pos, out_pid,
                                             dstatus, cand_lim, (uint32_t)occ_cap, shifts, ns,
                                             mpm::kRankSortMax, h->side);
        } else {
            uint64_t* sorted = nullptr;
            l = mpm::launch_sort_dev(occ, tmp, h->d_ahist[b], sort_cap, counters + mpm::kOccCount,
                                     shifts, ns, h->num_sms, &sorted, h->side,
                                     mpm::kRankSortMax);
            if (l >= 0)
                l = mpm::launch_close_sorted(sorted, counters, (uint32_t)cap, out_pos, out_pid,
                                             dstatus, cand_lim, (uint32_t)occ_cap,
                                             mpm::kRankSortMax, h->num_sms, h->side) < 0
                        ? -1
                        : l + 1;
        }
        if (l < 0) {
            cudaGetLastError();
            return set_error(MPM_ECUDA);
        }
        launches += l;
    }
    if (cudaEventRecord(h->sort_done[b], h->side) != cudaSuccess) {
        cudaGetLastError();
        return set_error(MPM_ECUDA);
    }
    h->sort_pending[b] = true;
    h->stats.launches += (uint32_t)launches;
    dirty = false;
    h->async_set = b ^ 1;
    return set_error(MPM_OK);
}

int mpm_join(mpm_handle* h) {
    if (!h) return set_error(MPM_EINVAL);
    int rc = prepare(h);
    if (rc) return set_error(rc);
    return set_error(join_sorts(h));
}

int mpm_sync(mpm_handle* h) {
    if (!h) return set_error(MPM_EINVAL);
    int rc = prepare(h);
    if (rc) return set_error(rc);
    rc = join_sorts(h);
    if (rc) return set_error(rc);
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) {
        cudaGetLastError();
        return set_error(MPM_ECUDA);
    }
    return set_error(harvest_timing(h, true));
}

int mpm_reset_stats(mpm_handle* h) {
    if (!h) return set_error(MPM_EINVAL);
    int rc = harvest_timing(h, true);
    h->stats = mpm_stats{};
    return set_error(rc);
}

int mpm_jit_compile(const uint8_t* P, size_t r, size_t m, int sigma, const mpm_params* params,
                    char* log, size_t log_bytes) {
    mpm::Plan plan;
    int rc = mpm::make_plan(P, r, m, sigma, params, &plan);
    if (rc) return set_error(rc);
    mpm::FilterDev f{};
    f.table_bytes = (uint32_t)((plan.info.table_bytes + 15) & ~uint64_t(15));
    f.entry_bytes = plan.info.entry_bytes;
    f.entry_bits = plan.info.entry_bits;
    f.smem_table = plan.p.table_place == MPM_TABLE_SMEM;
    f.map_kind = plan.p.map_kind;
    f.q = plan.p.q;
    f.k = plan.p.k;
    f.ell = plan.ell;
    f.shift = plan.p.map_shift;
    f.mprime = plan.info.mprime;
    f.positions = plan.info.positions;
    f.overlap = plan.p.overlap;
    // both variants: the one mpm_search runs and the candidate one of mpm_scan
    std::string text;
    rc = mpm::jit_compile_only(f, true, &text);
    if (rc == MPM_OK) rc = mpm::jit_compile_only(f, false, &text);
    if (log && log_bytes) {
        const size_t c = std::min(log_bytes - 1, text.size());
        std::memcpy(log, text.data(), c);
        log[c] = 0;
    }
    return set_error(rc);
}

int mpm_encode(mpm_handle* h, const uint8_t* T, size_t n, uint32_t* codes) {
    if (!h || (n > 0 && (!T || !codes)) || n >= (1ull << 32)) return set_error(MPM_EINVAL);
    int rc = prepare(h);
    if (rc) return set_error(rc);
    const mpm::FilterDev f = filter_dev(h);
    int l = mpm::launch_encode(T, (uint32_t)n, f, codes, h->stream);
    if (l < 0) return set_error(MPM_ECUDA);
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) return set_error(MPM_ECUDA);
    return set_error(MPM_OK);
}

int mpm_scan(mpm_handle* h, const uint8_t* T, size_t n, uint64_t* cand, size_t* count) {
    if (!h || !count || (n > 0 && !T) || n >= (1ull << 32)) return set_error(MPM_EINVAL);
    if (*count > 0 && !cand) return set_error(MPM_EINVAL);
    int rc = prepare(h);
    if (rc) return set_error(rc);
    rc = join_sorts(h);  // set 0's counters may still be closed by a pipelined sort
    if (rc) return set_error(rc);
    cudaStream_t s = h->stream;
    const mpm::FilterDev f = filter_dev(h);
    if (!h->plan.p.smag && !h->jit_cand_tried && h->plan.p.kernel != MPM_KERNEL_GENERIC) {
        h->jit_cand_tried = true;
        int err = MPM_OK;
        std::string log;
        h->jit_cand = mpm::jit_scan_kernel(f, false, h->device, &err, &log);
        if (!h->jit_cand && h->plan.p.kernel == MPM_KERNEL_SPECIALISED)
            return set_error(err ? err : MPM_ENOTSUP);
    }
    h->counters_dirty = true;  // this call leaves its counts behind
    if (cudaMemsetAsync(h->d_counters, 0, mpm::kNumCounters * 4, s) != cudaSuccess)
        return set_error(MPM_ECUDA);
    int l = 0;
    if (h->plan.p.smag) {
        const size_t nq = n / (uint32_t)f.q;
        if (grow(&h->d_codes, &h->codes_cap, nq)) return set_error(MPM_ENOMEM);
        if (mpm::launch_encode(T, (uint32_t)n, f, h->d_codes, s) < 0) return set_error(MPM_ECUDA);
        l = mpm::launch_scan_codes(h->d_codes, (uint32_t)nq, f, cand, (uint32_t)*count,
                                   h->d_counters, s);
    } else {
        const mpm::ScanArgs a = scan_args(h, T, (uint32_t)n, cand, (uint32_t)*count, h->d_counters);
        l = h->jit_cand ? mpm::launch_scan_jit(a, nullptr, h->jit_cand, h->num_sms,
                                               h->plan.p.chunk, s)
                        : mpm::launch_scan(a, h->num_sms, h->plan.p.chunk, s);
    }
    if (l == -2) return set_error(MPM_ENOTSUP);
    if (l < 0) return set_error(MPM_ECUDA);
    if (cudaMemcpyAsync(h->h_counters, h->d_counters, mpm::kNumCounters * 4,
                        cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return set_error(MPM_ECUDA);
    if (h->h_counters[mpm::kErrorFlag]) return set_error((int)h->h_counters[mpm::kErrorFlag]);
    const size_t cap = *count;
    *count = h->h_counters[mpm::kCandCount];
    h->stats = mpm_stats{};
    h->stats.n = n;
    h->stats.candidates = *count;
    h->stats.specialised = h->jit_cand && !h->plan.p.smag ? 1u : 0u;
    return set_error(*count > cap ? MPM_ECAPACITY : MPM_OK);
}

}  // extern "C"

// ---------------------------------------------------------------------------
// mpm_search_noalloc: the same filter, verification and sort as mpm_search,
// with every scratch buffer carved out of one file-scope device array, so
// that the call itself allocates no device memory.
//
// Layout of the array: [counters, 256 B][candidate records][occurrence keys].
// The occurrence limit keeps the sort on its one-block path, which needs no
// further scratch.

namespace {

constexpr size_t kNaCounterBytes = 256;
constexpr size_t kNaMaxCand = MPM_NOALLOC_MAX_CANDIDATES;
constexpr size_t kNaMaxOcc = MPM_NOALLOC_MAX_OCCURRENCES;
constexpr size_t kNaBytes = MPM_NOALLOC_SCRATCH_BYTES;
static_assert(kNaBytes == kNaCounterBytes + 8 * (kNaMaxCand + kNaMaxOcc), "scratch layout");
// more occurrences than this would need the radix sort's temporary buffers
static_assert(kNaMaxOcc <= mpm::kSortSmallMax, "occurrence limit within the one-block sort");

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNaBytes];

// The array's address on each device, looked up once per device.  In host
// code g_noalloc_scratch names a host-side stand-in, never the device memory.
constexpr int kNaMaxDevices = 128;
std::mutex g_na_mutex;
void* g_na_base[kNaMaxDevices] = {};

int noalloc_base(int device, unsigned char** out) {
    if (device < 0 || device >= kNaMaxDevices) return MPM_ECUDA;
    std::lock_guard<std::mutex> lock(g_na_mutex);
    if (!g_na_base[device]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return MPM_ECUDA;
        }
        g_na_base[device] = p;
    }
    *out = static_cast<unsigned char*>(g_na_base[device]);
    return MPM_OK;
}

}  // namespace

extern "C" int mpm_search_noalloc(mpm_handle* h, const uint8_t* T, size_t n, uint32_t* out_pos,
                                  uint32_t* out_pid, size_t* z) {
    if (!h || !z || (n > 0 && !T) || n >= (1ull << 32)) return set_error(MPM_EINVAL);
    if (*z > 0 && (!out_pos || !out_pid)) return set_error(MPM_EINVAL);
    if (h->plan.p.smag) return set_error(MPM_ENOTSUP);
    int rc = prepare(h);
    if (rc) return set_error(rc);
    if (n > 0 && !is_device_ptr(T)) return set_error(MPM_EINVAL);
    if (*z > 0 && (!is_device_ptr(out_pos) || !is_device_ptr(out_pid)))
        return set_error(MPM_EINVAL);
    unsigned char* base = nullptr;
    rc = noalloc_base(h->device, &base);
    if (rc) return set_error(rc);
    uint32_t* counters = reinterpret_cast<uint32_t*>(base);
    uint64_t* cand = reinterpret_cast<uint64_t*>(base + kNaCounterBytes);
    uint64_t* occ = cand + kNaMaxCand;

    const size_t out_capacity = *z;
    // as in mpm_search: closing sorts of pipelined searches still running on
    // the side stream may write the same outputs, so later work waits for
    // them; their pending timings belong to the statistics reset below
    rc = join_sorts(h);
    if (rc) return set_error(rc);
    rc = harvest_timing(h, true);
    if (rc) return set_error(rc);
    h->stats = mpm_stats{};
    h->stats.n = n;
    h->stats.sampled = (n / (uint32_t)h->plan.p.q) / (uint32_t)h->plan.p.k;
    h->stats.specialised = (h->jit || h->jit_cand) && !h->plan.p.smag ? 1u : 0u;
    if (n < h->plan.m) {
        *z = 0;
        return set_error(MPM_OK);
    }
    cudaStream_t s = h->stream;
    int launches = 0;
    // the counters block is wider than the counters the kernels use; clear it
    if (cudaMemsetAsync(counters, 0, kNaCounterBytes, s) != cudaSuccess)
        return set_error(MPM_ECUDA);
    rc = enqueue_filter(h, T, (uint32_t)n, cand, (uint32_t)kNaMaxCand, occ, (uint32_t)kNaMaxOcc,
                        counters, &launches);
    if (rc) return set_error(rc);
    const uint32_t rank_cap = (uint32_t)std::min<size_t>(out_capacity, mpm::kRankSortMax);
    if (rank_cap > 0) {
        if (mpm::launch_rank_sort(occ, counters, rank_cap, out_pos, out_pid, nullptr, 0u, 0u,
                                  s) < 0)
            return set_error(MPM_ECUDA);
        launches++;
    }
    rc = read_counters(h, counters);
    if (rc) return set_error(rc);
    const uint32_t nc = h->h_counters[mpm::kCandCount];
    const uint32_t zz = h->h_counters[mpm::kOccCount];
    h->stats.candidates = nc;
    h->stats.launches = (uint32_t)launches;
    if (!fused_search(h) && nc > kNaMaxCand) {
        *z = 0;
        return set_error(MPM_ESCRATCH);
    }
    *z = zz;
    h->stats.z = zz;
    if (zz > kNaMaxOcc) return set_error(MPM_ESCRATCH);
    if (zz > out_capacity) return set_error(MPM_ECAPACITY);
    if (zz > mpm::kRankSortMax) {
        const uint32_t key_bits =
            ((uint32_t)bits_for(n) << 16) | (uint32_t)bits_for(h->plan.r > 1 ? h->plan.r - 1 : 1);
        // at most kNaMaxOcc keys: the one-block sort, no temporary buffers
        int l = mpm::launch_sort_output(occ, nullptr, nullptr, 0, zz, key_bits, out_pos, out_pid, s);
        if (l < 0) return set_error(MPM_ECUDA);
        h->stats.launches += (uint32_t)l;
    }
    return set_error(MPM_OK);
}
