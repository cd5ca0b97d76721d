// Internal declarations shared by the host builder, the C ABI and the kernels.
#pragma once

#include <cstddef>
#include <cstdint>
#include <vector>

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
constexpr int kMaxPositions = 64;

// Verification key of a window or pattern: its first min(m, 16) bytes,
// zero padded, as two little-endian 64-bit words, hashed to a slot.
MPM_HD uint64_t key_hash(uint64_t lo, uint64_t hi) {
    uint64_t h = lo * 0x9E3779B97F4A7C15ull;
    h ^= hi * 0xC2B2AE3D27D4EB4Full;
    h ^= (lo ^ hi) >> 29;
    h *= 0x165667B19E3779F9ull;
    h ^= h >> 32;
    return h;
}

// One slot of the open-addressing table of pattern groups: all patterns
// whose key is (lo, hi) occupy rows [first, first + count) of the sorted
// pattern array.  count == 0 marks an empty slot.
struct Slot {
    uint64_t lo, hi;
    uint32_t first, count;
};
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
    int key_bytes;                   // min(m, 16)
};

int make_plan(const uint8_t* P, size_t r, size_t m, int sigma, const mpm_params* in,
              Plan* out);
void make_mu(const uint8_t* P, size_t r, size_t m, int kind, int sigma_r, int shift,
             uint8_t mu[256]);
int make_mask_table(const uint8_t* P, const Plan& plan, const uint8_t mu[256],
                    uint8_t* table);
int make_verify_tables(const uint8_t* P, size_t r, size_t m, HostTables* out);

}  // namespace mpm
