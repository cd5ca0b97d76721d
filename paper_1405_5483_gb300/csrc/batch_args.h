// Work description of the batched search, shared by the host (batch.cu),
// the precompiled batched kernel and the one compiled at run time for a
// batch (batch_jit.cuh), so it uses only types both sides define.
#pragma once

namespace mpm {

// One pattern set: its handle's device tables and filter parameters.
struct BatchSet {
    const void* table;              // mask table (entry_bytes per entry), global memory
    const unsigned char* mu;
    const Slot* slots;
    const unsigned char* pat;
    const unsigned int* pid;
    const unsigned int* pat_off;    // row starts when the set's patterns differ in length
    const unsigned int* keys;       // bitmap of key hashes (key_bits bits), or null
    unsigned int slot_mask, key_bytes, m, table_bytes;  // table_bytes padded to 16
    int q, k, mprime, ell, shift, mode, map_kind, entry_bytes;
    unsigned int key_bits;
    int variant;                    // the batch's compiled parameter set (run-time kernel)
    unsigned int stage;             // its stage bytes C (lane shares are multiples of it)
    unsigned int pad;
};

struct BatchText {
    const unsigned char* T;
    unsigned int n, set;
};

// A tile: 32 lanes, lane i scans [start + i sub, min(start + len, start + (i + 1) sub)).
struct BatchTile {
    unsigned int text, start, len, sub;
};

// Consecutive tiles of one set, taken by one block.
struct BatchUnit {
    unsigned int set, tile_begin, tile_end, pad;
};

enum BatchCounter : int { kQueue = 0, kBOcc = 1, kBError = 2, kBCand = 3 };

constexpr int kPosBits = 24;                     // text positions < 2^24 in a batch
constexpr int kPidBits = 20;                     // pattern ids < 2^20 per set
constexpr int kTextShift = kPosBits + kPidBits;  // occurrence key (text << 44) | (pos << 20) | pid
constexpr int kWarpQueue = 64;                   // fired steps a warp holds before verifying them
constexpr unsigned int kBatchSmemTable = 128u << 10;  // larger tables stay in L2
constexpr unsigned int kBatchKeyBits = 1u << 19;      // key bitmap of a set, at most

// Arguments of the batched kernel compiled at run time.
struct BatchJitArgs {
    const BatchSet* sets;
    const BatchText* texts;
    const BatchTile* tiles;
    const BatchUnit* units;
    unsigned long long* occ;
    unsigned int* counters;
    unsigned int nunits, occ_cap;
};

}  // namespace mpm
