// Internal declarations shared by the host builder, the C ABI and the kernels.
#pragma once

#include <cstddef>
#include <cstdint>
#include <vector>

#include "keyhash.h"
#include "mpm.h"

#if defined(__CUDACC__)
#define MPM_HD __host__ __device__ __forceinline__
#else
#define MPM_HD inline
#endif

namespace mpm {

// Records the error code for mpm_last_error() and returns it.
int set_error(int code);

// Largest k (the sampling step) and filter width accepted by the kernels.
constexpr int kMaxK = 32;
constexpr int kMaxPositions = 64;  // per 64-bit word of Shift-Or state
constexpr int kMaxWords = 4;       // words of state: wide = 0 .. kMaxWords - 1

static_assert(sizeof(Slot) == 24, "slot layout");

// Parameters after automatic choices, plus what follows from them.
struct Plan {
    mpm_params p;
    mpm_table_info info;
    int ell;        // log2(sigma_r)
    size_t r, m;
    int sigma;
};

// Everything mpm_build uploads.
struct HostTables {
    uint8_t mu[256];
    std::vector<uint8_t> table;      // info.entries * info.entry_bytes
    std::vector<Slot> slots;         // power of two
    std::vector<uint8_t> sorted_pat; // r * m, patterns in lexicographic order
    std::vector<uint32_t> sorted_pid;
    std::vector<uint32_t> sorted_off; // patterns of different lengths: row starts (r + 1)
    int key_bytes;                   // min(m, 16)
};

// all (may be null) receives every plan scored, one per feasible k, when
// q, sigma' and the mapping are fixed and k is left to choose.
int make_plan(const uint8_t* P, size_t r, size_t m, int sigma, const mpm_params* in,
              Plan* out, std::vector<Plan>* all = nullptr);
void make_mu(const uint8_t* P, size_t r, size_t m, int kind, int sigma_r, int shift,
             uint8_t mu[256]);
int make_mask_table(const uint8_t* P, const Plan& plan, const uint8_t mu[256],
                    uint8_t* table);
int make_verify_tables(const uint8_t* P, size_t r, size_t m, HostTables* out);
// Patterns of different lengths: pattern p is cat[off[p] .. off[p+1]), the
// shortest mmin bytes long; keys are their first min(mmin, 16) bytes.
int make_verify_tables_var(const uint8_t* cat, const size_t* off, size_t r, size_t mmin,
                           HostTables* out);
// Bitmap of the pattern groups' key hashes (bit key_hash & (bits - 1)): 64
// bits per group, a power of two between 2^10 and max_bits.  A window whose
// key hash hits a clear bit has no pattern group to probe.
std::vector<uint32_t> key_bitmap(const HostTables& t, uint32_t max_bits);

}  // namespace mpm
