// The state behind an mpm_handle: the resolved plan, the host copies that
// stay, the device tables, the scratch buffers and the compiled kernels.
// Shared by the C ABI (capi.cu), the batched search (batch.cu) and the tuner.
#pragma once

#include "kernels.h"

struct mpm_handle {
    mpm::Plan plan;
    mpm::HostTables host;
    int device = 0;
    int num_sms = 0;
    cudaStream_t stream = nullptr;

    uint8_t* d_mu = nullptr;
    void* d_table = nullptr;
    uint32_t table_bytes_padded = 0;
    mpm::Slot* d_slots = nullptr;
    uint8_t* d_pat = nullptr;
    uint32_t* d_pat_off = nullptr;  // row starts when the patterns differ in length
    uint32_t* d_pid = nullptr;
    uint32_t* d_keys = nullptr;     // key bitmap of the pattern groups
    uint32_t key_bits = 0;

    // scratch, grown on demand
    uint64_t* d_cand = nullptr;
    size_t cand_cap = 0;
    uint64_t* d_occ = nullptr;
    uint64_t* d_occ_tmp = nullptr;
    size_t occ_cap = 0;
    uint32_t* d_hist = nullptr;
    size_t hist_cap = 0;
    uint32_t* d_counters = nullptr;
    uint32_t* h_counters = nullptr;  // pinned
    uint32_t* h_snap = nullptr;      // mapped pinned: counters at the end of a search
    uint32_t* d_snap = nullptr;      // its device address
    bool counters_dirty = false;     // d_counters not known to be zero
    uint8_t* d_text = nullptr;       // staging for host text
    size_t text_cap = 0;
    uint32_t* d_codes = nullptr;     // SMAG codes
    size_t codes_cap = 0;
    uint32_t* d_out = nullptr;       // staging for host outputs (pos | pid)
    size_t out_cap = 0;

    mpm_stats stats{};
    const mpm::JitKernel* jit = nullptr;       // specialised scan that verifies
    const mpm::JitKernel* jit_cand = nullptr;  // specialised scan, candidates only
    bool jit_cand_tried = false;
    int timing = 0;
    cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
    // Pipelined searches alternate between two buffer sets (set 0 is
    // d_cand, d_occ and d_counters above).  A search's scan runs on `stream`;
    // its closing sort runs on `side` once the scan is done, so that it
    // overlaps the next search's scan; a search waits for the sort that last
    // used its set.
    cudaStream_t side = nullptr;
    cudaEvent_t scan_done[2] = {nullptr, nullptr};
    cudaEvent_t sort_done[2] = {nullptr, nullptr};
    bool sort_pending[2] = {false, false};
    uint64_t* d_cand1 = nullptr;
    size_t cand1_cap = 0;
    uint64_t* d_occ1 = nullptr;
    size_t occ1_cap = 0;
    // the device-count radix sort that closes pipelined searches with more
    // than kRankSortMax outputs: key buffers for set 1 and a histogram each
    uint64_t* d_occ1_tmp = nullptr;
    size_t occ1_tmp_cap = 0;
    uint32_t* d_ahist[2] = {nullptr, nullptr};
    size_t ahist_cap[2] = {0, 0};
    uint32_t* d_counters1 = nullptr;
    bool counters1_dirty = false;
    int async_set = 0;
    // event triples of pipelined searches (mpm_search_async), reused in turn
    static constexpr int kRing = 64;
    cudaEvent_t ring[kRing][3] = {};
    int ring_used[kRing] = {};
    int ring_next = 0;
};

