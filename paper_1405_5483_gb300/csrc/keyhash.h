// Verification key of a window or pattern: its first min(m, 16) bytes, zero
// padded, as two little-endian 64-bit words, hashed to a slot of the
// open-addressing table of pattern groups.  Shared by the host builder and
// every kernel that verifies (including the one compiled at run time), so it
// has no includes.
#pragma once

namespace mpm {

#if defined(__CUDACC__) || defined(__CUDACC_RTC__)
__host__ __device__
#endif
inline unsigned long long key_hash(unsigned long long lo, unsigned long long hi) {
    unsigned long long h = lo * 0x9E3779B97F4A7C15ull;
    h ^= hi * 0xC2B2AE3D27D4EB4Full;
    h ^= (lo ^ hi) >> 29;
    h *= 0x165667B19E3779F9ull;
    h ^= h >> 32;
    return h;
}

// Bit of a key in a key bitmap of 2^(64 - shift) bits: the top bits of one
// multiplicative (Fibonacci) hash of the key.  The bitmap only filters keys
// before the slot probe, which hashes with key_hash, so this hash is the
// cheaper one: for a key of at most 8 bytes (hi = 0) one 64-bit multiply.
#if defined(__CUDACC__) || defined(__CUDACC_RTC__)
__host__ __device__
#endif
inline unsigned int key_bit(unsigned long long lo, unsigned long long hi, unsigned int shift) {
    return (unsigned int)(((lo ^ (hi * 0xC2B2AE3D27D4EB4Full)) * 0x9E3779B97F4A7C15ull) >> shift);
}

// Bin of a whole q-gram for the q-gram hashing map (MPM_MAP_QHASH): raw is
// its q (<= 8) bytes read little-endian; the bin is the top `bits` bits of a
// multiplicative hash, 32-bit for q <= 4 and 64-bit above.
#if defined(__CUDACC__) || defined(__CUDACC_RTC__)
__host__ __device__ __forceinline__
#else
inline
#endif
unsigned int qgram_bin(unsigned long long raw, int q, int bits) {
    if (q <= 4) return ((unsigned int)raw * 0x9E3779B1u) >> (32 - bits);
    return (unsigned int)((raw * 0x9E3779B97F4A7C15ull) >> (64 - bits));
}

// One slot: the patterns whose key is (lo, hi) occupy rows
// [first, first + count) of the sorted pattern array; count == 0 is empty.
struct Slot {
    unsigned long long lo, hi;
    unsigned int first, count;
};

}  // namespace mpm
