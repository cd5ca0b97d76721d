// Launch interfaces of the search kernels (host side).
#pragma once

#include <cstdint>
#include <string>
#include <vector>
#include <cuda.h>
#include <cuda_runtime.h>

#include "mpm_internal.h"

namespace mpm {

// Indices into the per-search counter block in device memory.
enum Counter : int {
    kCandCount = 0,   // candidate records produced by the scan
    kOccCount = 1,    // occurrences produced by verification
    kErrorFlag = 2,   // MPM_ETIMEOUT when a bounded wait gave up
    kDoneCount = 3,   // blocks of the closing kernel that have read the counts
    kNumCounters = 4
};

// Filter description shared by the scan, encode and verify kernels.
struct FilterDev {
    const void* table;        // mask table, global memory
    uint32_t table_bytes;     // padded to a multiple of 16
    int entry_bytes;          // 1, 2, 4, 8; 16, 24, 32 (2 - 4 words of state)
    int entry_bits;           // 8 * entry_bytes, or 1, 2, 4: packed (specialised kernels only)
    int smem_table;           // copy the table into shared memory
    const uint8_t* mu;        // 256-entry byte -> reduced symbol map
    int map_kind, q, k, ell, shift, mprime, positions;
    int overlap;              // 1: overlapping q-grams (generic kernel only)
};

// The scan's view of one text.
struct ScanArgs {
    const uint8_t* T;
    uint32_t n;
    FilterDev f;
    uint32_t P;           // k * q, bytes per sampled q-gram period
    // rows handled through TMA: R rows of Lst bytes, in groups of 32
    uint32_t Lst, R, RG, warm_bytes;
    // bytes [pa, n) handled with plain loads, in streams of Ls bytes
    uint32_t pa, Ls, nstreams;
    uint64_t* cand;
    uint32_t cap;
    uint32_t* counters;
};

// Largest key bitmap the verification kernel keeps in shared memory (64 KiB).
constexpr uint32_t kVerifyKeyBitsMax = 1u << 19;

struct VerifyArgs {
    const uint8_t* T;
    uint32_t n, m;
    int q, k, mprime;
    const uint64_t* cand;
    uint32_t cand_cap;
    const Slot* slots;
    uint32_t slot_mask;
    const uint8_t* pat;   // sorted patterns, r * m (or concatenated, see pat_off)
    const uint32_t* pid;  // pattern id of each sorted row
    const uint32_t* pat_off;  // row starts when the patterns differ in length, else null
    int key_bytes;
    const uint32_t* keys;     // key bitmap of the pattern groups (key_mask + 1 bits,
    uint32_t key_mask;        // a power of two in 2^10 .. kVerifyKeyBitsMax)
    uint64_t* occ;        // (pos << 32) | pid
    uint32_t occ_cap;
    uint32_t* counters;
};

// Text bytes per row and per stage of the TMA scan.
constexpr uint32_t kScanRowBytes = 48;
constexpr int kScanWarps = 8;
constexpr int kScanStages = 4;

// Launches the MAG scan (fused encode + AOSO Shift-Or + compaction) over
// T[0..n).  Chooses the TMA row path for the 16-byte aligned bulk and plain
// loads for the rest.  Returns the number of kernels launched, or -1.
int launch_scan(const ScanArgs& base, int num_sms, int chunk, cudaStream_t s);

// SMAG: K1 encodes all q-grams, then the scan reads the codes.
int launch_encode(const uint8_t* T, uint32_t n, const FilterDev& f, uint32_t* codes,
                  cudaStream_t s);
int launch_scan_codes(const uint32_t* codes, uint32_t nq, const FilterDev& f, uint64_t* cand,
                      uint32_t cap, uint32_t* counters, cudaStream_t s);

int launch_verify(const VerifyArgs& a, int num_sms, cudaStream_t s);

// The scan specialised at run time for one filter (jit.cpp).
struct JitKernel;
// Compiles (NVRTC) and loads the specialised scan for this filter on the
// current device, cached per process; nullptr with *err = MPM_ENOTSUP when
// the filter is outside the specialised kernel or NVRTC is missing.
// verify: the variant that verifies candidates itself and appends
// occurrences (mpm_search); otherwise it appends candidate records.
const JitKernel* jit_scan_kernel(const FilterDev& f, bool verify, int device, int* err,
                                std::string* log);
// Compiles the specialisations of these filters that are not compiled yet,
// on `threads` host threads, and keeps the cubins for jit_scan_kernel.
void jit_precompile(const std::vector<FilterDev>& fs, bool verify, int threads);
// Host-only: compiles the specialisation without loading it.
int jit_compile_only(const FilterDev& f, bool verify, std::string* log);
bool jit_verifies(const JitKernel* k);
// v: where the verifying variant finds the patterns and puts occurrences.
int launch_scan_jit(const ScanArgs& a, const VerifyArgs* v, const JitKernel* k, int num_sms,
                    int chunk, cudaStream_t s);

// Stage bytes C of the specialised scans for P text bytes per sampled q-gram
// (0 when lcm(P, 16) > 256).
uint32_t jit_stage_bytes(uint32_t P, int k, bool overlap);

// One parameter set of a batch, as the batched kernel compiled at run time
// specialises it: q, k, m', log2 sigma', low-bit shift, mapping (0 low bits,
// 1 byte map, 2 q-gram hashing), entry bytes, stage bytes C and whether the
// lanes scan whole stages (else, when no stage of at most 256 bytes fits the
// sampling period, sample by sample; C is then the period).
struct BatchVariant {
    int q, k, mp, ell, shift, mode, eb;
    uint32_t C;
    int stages;
    int ebits;  // bits per mask-table entry (below 8: packed)
    int smem;   // 1: the table fits the kernel's shared-memory copy
};
struct BatchJit;
struct BatchJitArgs;
struct Plan;
// The specialisation of one pattern set's plan, and its index among vs
// (appended when new).
BatchVariant batch_variant_of(const Plan& plan);
int batch_variant_index(std::vector<BatchVariant>& vs, const BatchVariant& v);
// Compiles (NVRTC) the batched kernel of each single parameter set in vs that
// is not compiled yet, on `threads` host threads, into the process cache.
void jit_batch_precompile(const std::vector<BatchVariant>& vs, int threads);
// Compiles (NVRTC, cached per process) and loads the batched kernel for these
// parameter sets on the current device; nullptr with *err set when NVRTC or
// the driver entry points are missing or the compilation fails.
const BatchJit* jit_batch_kernel(const std::vector<BatchVariant>& vs, int device, int* err,
                                 std::string* log);
// Host-only: compiles it without loading.
int jit_batch_compile_only(const std::vector<BatchVariant>& vs, std::string* log);
// One persistent block per SM; returns 1 or -1.
int launch_batch_jit(const BatchJit* k, const BatchJitArgs& a, int num_sms, cudaStream_t s);

// Sorts the device-counted occurrence keys (counters[kOccCount], in keys)
// into out_pos/out_pid without the host knowing the count: one grid-wide
// rank sort, valid while the count is at most kRankSortMax and at most
// out_cap; otherwise it writes nothing and leaves the outputs to
// launch_sort_output.  With a snapshot (device address of device or mapped
// host memory), it also closes the search: the counters (candidates,
// occurrences, error) are copied there, with a fourth word that is 1 when
// the outputs hold every occurrence (no error, count <= out_cap, <= the rank
// sort's limit, <= occ_cap, candidates <= cand_cap), and are zeroed for the
// next search, so no reset or copy-back is enqueued.
constexpr uint32_t kRankSortMax = 4096;

// LSD radix sort of keys[0 .. min(*count, cap)) over the 8-bit digits at
// `shifts`, with the count read on the device and fixed grids, so that it
// can be captured in a CUDA graph.  tmp holds cap keys, hist
// sort_dev_hist_entries(cap) entries; *sorted receives keys or tmp,
// whichever holds the result.  Every kernel returns at once when
// *count <= skip (the rank sort has those).
size_t sort_dev_hist_entries(uint32_t cap);
int launch_sort_dev(uint64_t* keys, uint64_t* tmp, uint32_t* hist, uint32_t cap,
                    const uint32_t* count, const int* shifts, int nshifts, int num_sms,
                    uint64_t** sorted, cudaStream_t s, uint32_t skip = 0);
// Closes a pipelined search in one block (one launch): when from < count <=
// min(out_cap, occ_cap) (and no error or candidate overflow), the keys are
// radix-sorted over the digits at `shifts` (tmp holds as many keys) and split
// into out_pos/out_pid; always, the counters go to the snapshot with the
// completeness word and are zeroed.  For outputs of up to kBlockSortCap.
constexpr uint32_t kBlockSortCap = 1u << 20;
int launch_block_sort_close(uint64_t* keys, uint64_t* tmp, uint32_t* counters, uint32_t out_cap,
                            uint32_t* out_pos, uint32_t* out_pid, uint32_t* snapshot,
                            uint32_t cand_cap, uint32_t occ_cap, const int* shifts, int nshifts,
                            uint32_t from, cudaStream_t s);
// Closes a pipelined search after launch_sort_dev: when from < count <=
// min(out_cap, occ_cap) the sorted keys are split into out_pos/out_pid;
// always, the counters go to the snapshot (the fourth word 1 when the
// outputs hold every occurrence) and are zeroed.
int launch_close_sorted(const uint64_t* sorted, uint32_t* counters, uint32_t out_cap,
                        uint32_t* out_pos, uint32_t* out_pid, uint32_t* snapshot,
                        uint32_t cand_cap, uint32_t occ_cap, uint32_t from, int num_sms,
                        cudaStream_t s);
int launch_rank_sort(const uint64_t* keys, uint32_t* counters, uint32_t out_cap,
                     uint32_t* out_pos, uint32_t* out_pid, uint32_t* snapshot, uint32_t cand_cap,
                     uint32_t occ_cap, cudaStream_t s);

// Sorts z keys (in d_keys, device count unknown to the kernels: z is passed)
// and writes out_pos/out_pid.  tmp must hold z keys; returns launches or -1.
// Up to kSortSmallMax keys the sort runs in one block's shared memory and
// touches neither tmp nor hist (both may then be null).
constexpr uint32_t kSortSmallMax = 8192;
int launch_sort_output(uint64_t* d_keys, uint64_t* d_tmp, uint32_t* d_hist, size_t hist_cap,
                       uint32_t z, uint32_t key_bits, uint32_t* out_pos, uint32_t* out_pid,
                       cudaStream_t s);
size_t sort_hist_entries(uint32_t z);

}  // namespace mpm
