// Argument block of the specialised scan kernel (scan_jit.cuh).  Included by
// the host launcher and, as text, by the kernel source compiled at run time,
// so it uses only fixed-width integer types that both sides define.
#pragma once

namespace mpm {

struct JitScanArgs {
    const unsigned char* T;       // text (device)
    const void* table;            // mask table (device)
    const unsigned char* mu;      // byte -> reduced symbol (device, 256)
    unsigned long long* cand;     // candidate records (candidate variant)
    unsigned int* counters;       // kCandCount, kOccCount, kErrorFlag
    unsigned int n;               // text bytes
    unsigned int cap;             // capacity of cand
    unsigned int Lst;             // bytes per TMA row
    unsigned int R;               // rows [0, R * Lst) read through TMA
    unsigned int RG;              // row groups of 32 rows
    unsigned int row_warps;       // warps 0 .. row_warps-1 take row groups
    unsigned int pa;              // bytes [pa, n) are read with plain loads
    unsigned int Ls;              // ... in sub-streams of Ls bytes
    unsigned int nstreams;        // number of sub-streams
    unsigned int m;               // pattern length
    // verification (the fused variant): pattern groups and outputs
    const void* slots;            // open-addressing table of pattern groups
    const unsigned char* pat;     // patterns sorted by bytes, r * m
    const unsigned int* pid;      // pattern id of each sorted row
    const unsigned int* pat_off;  // row starts for patterns of different lengths, or null
    unsigned long long* occ;      // occurrences (pos << 32) | pid
    unsigned int slot_mask;
    unsigned int key_bytes;       // min(m, 16)
    unsigned int occ_cap;
    unsigned int inject;          // test hook: 1 = warp 0 over-arms its first stage's
                                  // barrier, so its bounded wait runs out (MPM_ETIMEOUT)
};

}  // namespace mpm
