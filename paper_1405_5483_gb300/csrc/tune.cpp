// Exhaustive autotuner over the filter parameters (sigma', mapping, q, k;
// the mappings are equal-weight bins, low-order bits and q-gram hashing)
// and the scan kernel variant: plan every feasible set on the host, drop the
// sets whose estimated candidate rate is hopeless, compile the remaining
// specialisations in parallel, then build and time each set on a sample
// text and keep the fastest.  The paper chooses q from log_sigma(rm) and k
// by a closed form (Section 3.2); here the choice is measured.
#include <algorithm>
#include <chrono>
#include <cstring>
#include <thread>
#include <vector>

#include <cuda_runtime.h>

#include "kernels.h"
#include "mpm_internal.h"

namespace {

using mpm::set_error;

mpm::FilterDev filter_of(const mpm::Plan& plan) {
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
    return f;
}

bool on_device(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

struct Candidate {
    mpm_params p;
    mpm::Plan plan;
    double key;  // estimated candidate records per text byte
};

// largest mask table of the cost model's grid, and of the tuner's own sets
// (a packed table of 32 MiB for r = 100 000 DNA patterns is among the best)
constexpr uint64_t kModelMaxTable = 16ull << 20;
constexpr uint64_t kTuneMaxTable = 64ull << 20;

}  // namespace

namespace {

// The cost model's parameter grid: q in 2..6 with sigma' in {2, 4, 8, 16}
// (the mapping the planner picks for that sigma'), and q in 2..5 with q-gram
// hashing into 2^12, 2^14 or 2^16 bins; every feasible k <= 8.
void model_grid(const uint8_t* P, size_t r, size_t m, int sigma, int max_positions,
                std::vector<mpm::Plan>* plans) {
    const int maxpos = max_positions > 0 ? max_positions : 64;
    auto add = [&](int kind, int sr, int q) {
        mpm_params p{};
        p.q = q;
        p.sigma_r = sr;
        p.map_kind = kind;
        p.map_shift = -1;
        mpm::Plan best_k;
        std::vector<mpm::Plan> all;
        if (mpm::make_plan(P, r, m, sigma, &p, &best_k, &all) != MPM_OK) return;
        for (const auto& pl : all) {
            if (pl.p.k > 8 || pl.info.positions > maxpos || pl.info.table_bytes > kModelMaxTable)
                continue;
            plans->push_back(pl);
        }
    };
    for (int q = 2; q <= 6; q++)
        for (int sr = 2; sr <= 16; sr <<= 1) add(MPM_MAP_AUTO, sr, q);
    for (int q = 2; q <= 5; q++)
        for (int bits = 12; bits <= 16; bits += 2) add(MPM_MAP_QHASH, 1 << bits, q);
}

}  // namespace

extern "C" int mpm_autotune(const uint8_t* P, size_t r, size_t m, int sigma, const uint8_t* T,
                            size_t n, const mpm_tune_opts* opts, mpm_params* best,
                            mpm_tune_entry* entries, size_t cap, size_t* count) {
    if (!P || !best || !count || r == 0 || m == 0 || (n > 0 && !T) || n >= (1ull << 32))
        return set_error(MPM_EINVAL);
    mpm_tune_opts o{};
    if (opts) o = *opts;
    const int max_q = o.max_q > 0 ? std::min(o.max_q, 16) : 8;
    const int max_k = o.max_k > 0 ? std::min(o.max_k, mpm::kMaxK) : 8;
    const int reps = o.reps > 0 ? o.reps : 3;
    const int kernels = o.kernels > 0 ? o.kernels : 1;
    const size_t max_sets = o.max_sets > 0 ? (size_t)o.max_sets : 64;
    const double max_rate = o.max_rate > 0 ? o.max_rate : 0.05;
    const int max_positions = o.max_positions > 0 ? o.max_positions : 64;
    const uint64_t max_table =
        o.max_table_kib > 0 ? std::min<uint64_t>((uint64_t)o.max_table_kib << 10, kTuneMaxTable)
                            : kTuneMaxTable;

    // the pattern alphabet bounds sigma'
    bool seen[256] = {false};
    int distinct = 0;
    for (size_t i = 0; i < r * m; i++)
        if (!seen[P[i]]) {
            seen[P[i]] = true;
            distinct++;
        }
    const int sigma_eff = std::min(256, std::max(sigma, distinct));
    int top = 2;
    while (top < distinct && top < 256) top <<= 1;

    std::vector<Candidate> cands;
    std::vector<Candidate> above_rate;  // timed only when no set passes max_rate
    if (o.grid < 0 || o.grid > 1) return set_error(MPM_EINVAL);
    if (o.overlap < 0 || o.overlap > 2) return set_error(MPM_EINVAL);
    if (o.batch_generic < 0 || o.batch_generic > 1) return set_error(MPM_EINVAL);
    if (o.grid == 1) {
        // exactly the cost model's grid (max_q, max_k, max_sets and max_rate unused)
        std::vector<mpm::Plan> plans;
        model_grid(P, r, m, sigma_eff, max_positions, &plans);
        for (const auto& pl : plans) {
            if (pl.info.table_bytes > max_table) continue;
            Candidate c;
            c.plan = pl;
            c.p = pl.p;
            c.key = 0.0;
            cands.push_back(c);
        }
    }
    // the overlapping-q-gram family (Section 2) is ranked apart: its sets
    // send far fewer windows to verification per byte but read k bytes per
    // sampled q-gram instead of k q, so one ranking would starve the other
    std::vector<Candidate> cands_ov, above_ov;
    const bool want_nov = o.grid == 1 || o.overlap != 2;
    const bool want_ov = o.grid == 0 && o.overlap != 0;
    // one planning pass per (mapping, sigma', q) scores every k at once
    auto add_all_k = [&](int kind, int sr, int q) {
        for (int ov = 0; ov <= 1; ov++) {
            if (!(ov ? want_ov : want_nov)) continue;
            mpm_params p{};
            p.q = q;
            p.sigma_r = sr;
            p.map_kind = kind;
            p.map_shift = -1;
            p.overlap = ov;
            mpm::Plan best_k;
            std::vector<mpm::Plan> all;
            if (mpm::make_plan(P, r, m, sigma_eff, &p, &best_k, &all) != MPM_OK) continue;
            for (const auto& pl : all) {
                if (pl.p.k > max_k) continue;
                if (pl.info.table_bytes > max_table) continue;
                if (pl.info.positions > max_positions) continue;
                Candidate c;
                c.plan = pl;
                c.p = pl.p;
                // candidate windows per text byte
                c.key = pl.info.est_candidate_rate / (double)(ov ? pl.p.k : pl.p.q * pl.p.k);
                const bool above = pl.info.est_candidate_rate > max_rate;
                (ov ? (above ? above_ov : cands_ov) : (above ? above_rate : cands)).push_back(c);
            }
        }
    };
    for (int sr = 2; o.grid == 0 && sr <= top; sr <<= 1) {
        // low-order bits only where they keep the pattern symbols apart
        std::vector<int> kinds = {MPM_MAP_GREEDY};
        {
            mpm_params a{};
            a.sigma_r = sr;
            a.map_shift = -1;
            mpm::Plan pa;
            if (mpm::make_plan(P, r, m, sigma_eff, &a, &pa) == MPM_OK &&
                pa.p.map_kind == MPM_MAP_LOWBITS)
                kinds.push_back(MPM_MAP_LOWBITS);
        }
        for (int kind : kinds)
            for (int q = 1; q <= max_q; q++) add_all_k(kind, sr, q);
    }
    // q-gram hashing: whole q-grams into 2^10 .. 2^16 bins
    for (int bits = 10; o.grid == 0 && bits <= 16; bits++)
        for (int q = 1; q <= std::min(max_q, 8); q++) add_all_k(MPM_MAP_QHASH, 1 << bits, q);
    // each family: its sets under max_rate by windows per byte, or, when
    // every set sends more windows to verification than max_rate (large
    // pattern sets), its lowest-rate ones
    auto rank = [](std::vector<Candidate>& in, std::vector<Candidate>& above) {
        if (in.empty()) {
            std::stable_sort(above.begin(), above.end(),
                             [](const Candidate& a, const Candidate& b) {
                                 return a.plan.info.est_candidate_rate <
                                        b.plan.info.est_candidate_rate;
                             });
            in.swap(above);
        } else {
            std::stable_sort(in.begin(), in.end(),
                             [](const Candidate& a, const Candidate& b) { return a.key < b.key; });
        }
    };
    if (o.grid == 0) {
        rank(cands, above_rate);
        rank(cands_ov, above_ov);
        // half of max_sets for each family present; one family's unused
        // share goes to the other
        size_t n_ov = std::min(cands_ov.size(), cands.empty() ? max_sets : max_sets / 2);
        size_t n_nov = std::min(cands.size(), max_sets - n_ov);
        n_ov = std::min(cands_ov.size(), max_sets - n_nov);
        cands.resize(n_nov);
        cands.insert(cands.end(), cands_ov.begin(), cands_ov.begin() + n_ov);
    }
    if (o.grid == 0 && want_nov) {
        // the planner's own choice (mpm_build with automatic parameters) is
        // always timed too, whatever its q or table size, unless the caller
        // bounded the table
        mpm::Plan pa;
        if (mpm::make_plan(P, r, m, sigma_eff, nullptr, &pa) == MPM_OK &&
            pa.info.positions <= max_positions &&
            (o.max_table_kib <= 0 || pa.info.table_bytes <= max_table)) {
            bool dup = false;
            for (const auto& c : cands)
                dup = dup || (c.p.q == pa.p.q && c.p.sigma_r == pa.p.sigma_r && c.p.k == pa.p.k &&
                              c.p.map_kind == pa.p.map_kind && c.p.map_shift == pa.p.map_shift &&
                              c.p.overlap == pa.p.overlap);
            if (!dup) {
                Candidate c;
                c.plan = pa;
                c.p = pa.p;
                c.key = 0.0;
                cands.insert(cands.begin(), c);
            }
        }
    }
    if (cands.empty()) return set_error(MPM_EINVAL);

    // compile every specialisation up front, in parallel
    const int threads = (int)std::max(1u, std::thread::hardware_concurrency());
    std::vector<mpm::FilterDev> fs;
    for (const auto& c : cands) fs.push_back(filter_of(c.plan));
    if (kernels & 1) mpm::jit_precompile(fs, true, threads);
    if (kernels & 2) mpm::jit_precompile(fs, false, threads);
    if ((kernels & 8) && !o.batch_generic) {
        // the batched kernel of every set the batch takes, as mpm_batch_create
        // compiles it for a batch of that one set
        std::vector<mpm::BatchVariant> vs;
        for (const auto& c : cands)
            if (c.plan.info.positions <= 32 && !c.plan.p.overlap &&
                !(c.plan.p.map_kind == MPM_MAP_QHASH && c.plan.p.q > 5))
                vs.push_back(mpm::batch_variant_of(c.plan));
        mpm::jit_batch_precompile(vs, threads);
    }

    // the sample on the device, and output buffers
    const uint8_t* dT = T;
    uint8_t* own_text = nullptr;
    if (n > 0 && !on_device(T)) {
        if (cudaMalloc(&own_text, n) != cudaSuccess ||
            cudaMemcpy(own_text, T, n, cudaMemcpyHostToDevice) != cudaSuccess) {
            cudaGetLastError();
            cudaFree(own_text);
            return set_error(MPM_ENOMEM);
        }
        dT = own_text;
    }
    size_t out_cap = 1 << 16;
    uint32_t* d_out = nullptr;
    if (cudaMalloc(&d_out, 3 * out_cap * sizeof(uint32_t)) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(own_text);
        return set_error(MPM_ENOMEM);
    }

    // batched timing: at least 128 MiB scanned per run (at most 256 copies)
    const size_t copies =
        n == 0 ? 1 : std::min<size_t>(256, std::max<size_t>(1, ((128ull << 20) + n - 1) / n));
    size_t timed = 0;
    bool have_best = false;
    double best_ms = 0.0;
    // bit 3 times the batched kernel (one text, the sample) with the generic
    // parameters the batch runs; the others time mpm_search
    const int modes[4] = {MPM_KERNEL_SPECIALISED, MPM_KERNEL_SPLIT, MPM_KERNEL_GENERIC,
                          MPM_KERNEL_GENERIC};
    for (const auto& c : cands) {
        for (int bit = 0; bit < 4; bit++) {
            if (!(kernels & (1 << bit))) continue;
            mpm_tune_entry e{};
            e.params = c.p;
            e.params.kernel = modes[bit];
            e.info = c.plan.info;
            mpm_handle* h = nullptr;
            mpm_batch* batch = nullptr;
            if (bit == 3 && c.plan.info.positions > 32) {
                e.status = MPM_ENOTSUP;
            } else {
                h = mpm_build(P, r, m, sigma_eff, &e.params);
                if (!h) e.status = mpm_last_error();
            }
            if (h && bit == 3) {
                // the sample repeated until the batch keeps the whole GPU busy
                const std::vector<const uint8_t*> texts(copies, dT);
                const std::vector<size_t> lens(copies, n);
                const std::vector<uint32_t> sot(copies, 0u);
                mpm_batch_opts bo{};
                bo.generic = o.batch_generic;
                batch = mpm_batch_create(&h, 1, texts.data(), lens.data(), sot.data(),
                                         (int)copies, &bo);
                if (!batch) e.status = mpm_last_error();
            }
            if (h && e.status == MPM_OK) {
                std::vector<double> ms;
                for (int it = 0; it <= reps && e.status == MPM_OK; it++) {
                    size_t z = out_cap;
                    const auto t0 = std::chrono::steady_clock::now();
                    int rc = batch ? mpm_batch_run(batch, d_out, d_out + out_cap,
                                                   d_out + 2 * out_cap, &z)
                                   : mpm_search(h, dT, n, d_out, d_out + out_cap, &z);
                    const auto t1 = std::chrono::steady_clock::now();
                    if (rc == MPM_ECAPACITY) {
                        cudaFree(d_out);
                        out_cap = z + 1024;
                        if (cudaMalloc(&d_out, 3 * out_cap * sizeof(uint32_t)) != cudaSuccess) {
                            cudaGetLastError();
                            d_out = nullptr;
                            e.status = MPM_ENOMEM;
                            break;
                        }
                        it--;
                        continue;
                    }
                    if (rc) {
                        e.status = rc;
                        break;
                    }
                    if (it > 0) {  // the first search warms up
                        if (batch) {
                            // device time of the run (events around the graph), per copy
                            mpm_batch_stats bs;
                            mpm_batch_get_stats(batch, &bs);
                            ms.push_back((double)bs.ms / (double)copies);
                        } else {
                            ms.push_back(std::chrono::duration<double, std::milli>(t1 - t0).count());
                        }
                    }
                }
                if (e.status == MPM_OK && !ms.empty()) {
                    std::sort(ms.begin(), ms.end());
                    e.ms = ms[ms.size() / 2];
                    if (batch) {
                        mpm_batch_stats bs;
                        mpm_batch_get_stats(batch, &bs);
                        e.candidates = bs.candidates;
                        e.z = bs.z;
                    } else {
                        mpm_stats st;
                        mpm_get_stats(h, &st);
                        e.candidates = st.candidates;
                        e.z = st.z;
                    }
                    if (!have_best || e.ms < best_ms) {
                        have_best = true;
                        best_ms = e.ms;
                        *best = e.params;
                    }
                }
            }
            mpm_batch_free(batch);
            mpm_free(h);
            if (entries && timed < cap) entries[timed] = e;
            timed++;
            if (!d_out) break;
        }
        if (!d_out) break;
    }
    cudaFree(d_out);
    cudaFree(own_text);
    *count = timed;
    return set_error(have_best ? MPM_OK : MPM_EINVAL);
}


extern "C" int mpm_model_grid(const uint8_t* P, size_t r, size_t m, int sigma, int max_positions,
                              mpm_params* out, mpm_table_info* info, size_t cap, size_t* count) {
    if (!P || !count || r == 0 || m == 0 || sigma < 1 || sigma > 256 || (cap > 0 && !out))
        return set_error(MPM_EINVAL);
    std::vector<mpm::Plan> plans;
    model_grid(P, r, m, sigma, max_positions, &plans);
    for (size_t i = 0; i < plans.size() && i < cap; i++) {
        out[i] = plans[i].p;
        if (info) info[i] = plans[i].info;
    }
    *count = plans.size();
    return set_error(MPM_OK);
}
