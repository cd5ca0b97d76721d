/*
 * mpm.h -- exact multiple pattern matching on GB300 (MAG / SMAG).
 *
 * C ABI of the library built from paper_1405_5483_gb300/csrc.  It implements
 * the text scan of Susik, Grabowski and Fredriksson, "Multiple pattern
 * matching revisited": alphabet reduction, non-overlapping q-grams of all q
 * shifts of every pattern superimposed into one Shift-Or mask table, the
 * average-optimal Shift-Or scan that reads only every k-th text q-gram,
 * candidate compaction, exact verification and a deterministic order.
 *
 * Problem (Section 1): text T[0..n), patterns P_0..P_{r-1}, all of length m,
 * bytes as symbols; report every (i, p) with T[i..i+m) == P_p.
 *
 * Conventions shared by every entry point
 *   - Return value: MPM_OK (0) or a positive MPM_E* code; the same code is
 *     kept per thread for mpm_last_error().  Functions returning a pointer
 *     return NULL on error.
 *   - Device pointers are CUDA global memory of the current device.  Work is
 *     enqueued on the handle's stream (mpm_set_stream), default stream 0.
 *   - Occurrence lists are sorted by position, then pattern id; pattern ids
 *     are 0-based row indices of P; identical patterns are each reported.
 *   - Positions and q-gram indices are 32-bit: n < 2^32.
 *   - Nothing here falls back to the CPU: without a usable GPU the calls
 *     that launch kernels return MPM_ECUDA.
 */
#ifndef MPM_H
#define MPM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------ error codes */
#define MPM_OK         0
#define MPM_EINVAL     1  /* bad argument or infeasible explicit parameter   */
#define MPM_ENOMEM     2  /* host or device allocation failed                */
#define MPM_ECUDA      3  /* a CUDA call failed (no device, launch error ...) */
#define MPM_ECAPACITY  4  /* output capacity too small; *z = required count  */
#define MPM_ETIMEOUT   5  /* a bounded device wait gave up; results invalid  */
#define MPM_ENOTSUP    6  /* parameter combination the library does not run  */
#define MPM_ESCRATCH   7  /* mpm_search_noalloc: its fixed scratch is too small */

/* ----------------------------------------------------- parameter choices */
#define MPM_MAP_AUTO     0
#define MPM_MAP_RANK     1  /* frequency-rank bins (Section 3.3)                 */
#define MPM_MAP_GREEDY   2  /* equal-weight bins, greedy (Section 3.3)           */
#define MPM_MAP_LOWBITS  3  /* low-order bits after a right shift (Section 3.3)  */
#define MPM_MAP_QHASH    4  /* whole q-grams hashed to sigma_r bins (Section 3.3,
                               "alphabet mapping on the q-grams")               */

#define MPM_TABLE_AUTO   0
#define MPM_TABLE_SMEM   1  /* mask table copied to shared memory per block  */
#define MPM_TABLE_GLOBAL 2  /* mask table read from global memory (L2)       */

/*
 * Filter parameters (Sections 3.2, 3.3).  Zero in q, sigma_r, k, map_kind,
 * table_place or chunk means "choose automatically"; map_shift < 0 means
 * "choose automatically" (0 is a valid shift).
 *   q        q-gram length, 1..16 (1..8 with MPM_MAP_QHASH), with
 *            q*log2(sigma_r) <= 30 (symbol maps) and
 *            L' = floor((m - q + 1) / q) >= 1.
 *   sigma_r  reduced alphabet size sigma', a power of two in 2..256; with
 *            MPM_MAP_QHASH the number of q-gram bins, a power of two in
 *            2..2^24, a q-gram's bin being the top log2(sigma_r) bits of
 *            raw * 0x9E3779B1 mod 2^32 (q <= 4) or raw * 0x9E3779B97F4A7C15
 *            mod 2^64 (q <= 8), raw = its q bytes read little-endian.
 *   k        AOSO sampling step: every k-th text q-gram is read; 1..32 and
 *            k <= min(L', 64).
 *   map_kind MPM_MAP_*.
 *   map_shift right shift applied to a byte before its low log2(sigma_r)
 *            bits are kept (MPM_MAP_LOWBITS only), 0..7.
 *   table_place MPM_TABLE_*.
 *   smag     0: MAG, q-gram codes computed on the fly inside the scan;
 *            1: SMAG, the whole text is encoded first (Section 3.2).
 *   chunk    text bytes one scan thread handles before it moves on, or 0.
 *   kernel   MPM_KERNEL_*: the scan kernel compiled at build time for
 *            these parameters (NVRTC, sm_103a), or the precompiled generic
 *            one; AUTO takes the specialised kernel when it compiles.  The
 *            specialised kernel needs lcm(P, 16) <= 256, P = k*q text bytes
 *            per sampled q-gram (k with overlap = 1; an explicit request
 *            outside that fails with MPM_ENOTSUP); the generic one
 *            hashes q-grams of at most 5 bytes (MPM_ENOTSUP from the search
 *            otherwise).
 *   overlap  0: MAG's non-overlapping q-grams of all q shifts; 1: the
 *            overlapping q-grams of Section 2 (P_i[j..j+q-1], j < m-q+1, no
 *            shifts; the text's q-gram at every byte, every k-th one read),
 *            L' = m - q + 1.  Runs in the specialised kernels and the
 *            generic one; SMAG and mpm_batch answer MPM_ENOTSUP.
 *   wide     0: at most 64 filter positions (one 64-bit word of Shift-Or
 *            state); w = 1, 2, 3: at most 64 (w + 1) positions, the state
 *            then ceil(positions / 64) words (Section 3.2's ceil((m/q)/w)
 *            words, w = 64) and mask table entries of 8 bytes per word above
 *            64 positions.  Runs in the specialised kernels and the generic
 *            one; SMAG answers MPM_ENOTSUP above 64 positions.
 */
#define MPM_KERNEL_AUTO        0
#define MPM_KERNEL_GENERIC     1
#define MPM_KERNEL_SPECIALISED 2  /* specialised scan that verifies its candidates  */
#define MPM_KERNEL_SPLIT       3  /* specialised scan, then the verification kernel */

typedef struct {
    int q;
    int sigma_r;
    int k;
    int map_kind;
    int map_shift;
    int table_place;
    int smag;
    int chunk;
    int kernel;
    int overlap;
    int wide;
} mpm_params;

/* Sizes that follow from resolved parameters and m (Sections 3.1, 3.2). */
typedef struct {
    int L;             /* common q-gram length of the q shifted patterns, L'  */
    int mprime;        /* AOSO subpattern length m' = floor(min(L',cap)/k)    */
    int positions;     /* filter positions m'' = k * m' (<= 64 (wide + 1))      */
    int entry_bytes;   /* bytes per mask-table entry: 1, 2, 4, 8, 16, 24, 32  */
    uint64_t entries;  /* sigma_r^q                                           */
    uint64_t table_bytes;
    double est_candidate_rate; /* expected candidate windows (fired subpatterns)
                                  per sampled q-gram in i.i.d. text with the
                                  pattern set's symbol frequencies, at most 1  */
    int entry_bits;    /* bits per mask-table entry: 8 * entry_bytes, or 1, 2 or 4
                          when a table of filters of at most 4 positions, too
                          large for shared memory, packs several entries into a
                          byte (entry c at bit c * entry_bits, lowest first; the
                          specialised kernels only)                             */
} mpm_table_info;

/* Counters of the last mpm_search / mpm_scan on a handle. */
typedef struct {
    uint64_t n;            /* text bytes                                      */
    uint64_t sampled;      /* sampled q-grams read by the scan                */
    uint64_t candidates;   /* candidate records (sampled q-grams that fired)  */
    uint64_t z;            /* occurrences found                               */
    uint32_t launches;     /* kernels launched by the call                    */
    uint32_t retries;      /* re-runs after growing an internal buffer        */
    float ms_scan;         /* device time of the scan kernels (timing on)     */
    float ms_verify;       /* device time of the verification kernel          */
    uint32_t specialised;  /* 1 if the scan ran the specialised kernel        */
    uint32_t reserved;
} mpm_stats;

typedef struct mpm_handle mpm_handle;

/* ------------------------------------------------------------ core calls */

/*
 * Builds the filter for r patterns of length m (row-major, r*m bytes of host
 * memory at P; copied, the caller keeps ownership).  sigma is the declared
 * alphabet size (1..256; used to choose parameters and to validate
 * sigma_r <= the smallest power of two >= max(2, sigma) when sigma_r is
 * given).  params may be NULL (all
 * automatic).  Host work (Sections 2, 3.2, 3.3): pattern histogram, mapping
 * mu, the q shifts of every pattern cut into non-overlapping q-grams, their
 * superimposition into the mask table, and a hash of the patterns for
 * verification; then one upload to the device, which the handle owns.
 * Returns NULL on error (mpm_last_error(): MPM_EINVAL, MPM_ENOMEM, MPM_ECUDA).
 */
mpm_handle *mpm_build(const uint8_t *P, size_t r, size_t m, int sigma,
                      const mpm_params *params);

/*
 * Patterns of different lengths (the problem of Section 1 with a length per
 * pattern): pattern p is P[off[p] .. off[p+1]) (off has r + 1 entries,
 * off[0] = 0, every pattern at least one byte, off[r] < 2^32).  The filter is
 * built from the first m_min bytes of every pattern, m_min the shortest
 * length (params as for mpm_build with m = m_min); every candidate window is
 * verified against each pattern's full length, so an occurrence (pos, pid)
 * is reported exactly when T[pos .. pos + len_pid) = P_pid.  P and off are
 * host arrays, copied.  NULL on error (mpm_last_error: MPM_EINVAL for bad
 * offsets, else as mpm_build).
 */
mpm_handle *mpm_build_var(const uint8_t *P, const size_t *off, size_t r, int sigma,
                          const mpm_params *params);

/*
 * Finds all occurrences in T[0..n).  T may be device or host memory (host
 * text is copied to a device buffer the handle owns).  out_pos / out_pid
 * receive the sorted occurrence list and may be device or host memory; *z is
 * in: their capacity (entries), out: the number of occurrences.  When that
 * number exceeds the capacity the call returns MPM_ECAPACITY, sets *z to the
 * required count and the outputs hold nothing valid.  Blocks the calling
 * host thread until the occurrence count is known (one 16-byte read-back);
 * device outputs are complete when the handle's stream is.  Steps (Sections
 * 3.1, 3.2): one fused encode+scan kernel (or SMAG encode then scan), one
 * verification kernel, one sort.  Concurrent calls on the same handle race.
 */
int mpm_search(mpm_handle *h, const uint8_t *T, size_t n, uint32_t *out_pos,
               uint32_t *out_pid, size_t *z);

/* Releases the handle and all its device memory (after synchronizing its
 * stream).  NULL is ignored. */
void mpm_free(mpm_handle *h);

/* Last error code set on the calling thread. */
int mpm_last_error(void);

/* Static description of an error code. */
const char *mpm_strerror(int code);

/* Sets the CUDA stream (a cudaStream_t, e.g. PyTorch's current stream) on
 * which the handle enqueues all later work.  NULL selects stream 0. */
int mpm_set_stream(mpm_handle *h, void *stream);

/* The parameters the handle resolved (no zeros / negatives left) and the
 * sizes that follow from them; info may be NULL. */
int mpm_get_params(const mpm_handle *h, mpm_params *out, mpm_table_info *info);

/* Counters of the last search or scan on this handle (for pipelined
 * searches: the sums since mpm_reset_stats, complete after mpm_sync). */
int mpm_get_stats(const mpm_handle *h, mpm_stats *out);

/* on != 0: mpm_search records CUDA events around its scan and verification
 * launches on the handle's stream and reports their device times in
 * mpm_stats (read after the search's own count read-back, so no extra
 * synchronisation).  Off by default. */
int mpm_set_timing(mpm_handle *h, int on);

/*
 * Pipelined search: enqueues the whole search of T[0..n) (scan, verification
 * and the sort of the occurrences) on the handle's stream and returns
 * without waiting, so successive searches keep the GPU busy.  The sort is a
 * rank sort for up to 4096 occurrences; when cap is above 4096 a radix sort
 * that reads the count on the device follows it for larger counts (one
 * more kernel, in one block, for cap up to 2^20; above that, a multi-block
 * sort of about 3 kernels per byte of key; it returns at once when the
 * count is at most 4096).  T, out_pos and
 * out_pid (cap entries each) are device pointers; status points to 4
 * uint32 in device memory or in mapped host memory (cudaHostAlloc with
 * cudaHostAllocMapped).  When the stream reaches the end of the call:
 * status[0] = candidate records, status[1] = z, status[2] = 0 or the error
 * of the device work (MPM_ETIMEOUT), status[3] = 1 when out_pos/out_pid hold
 * all z occurrences sorted by (pos, pid); status[3] = 0 when they could not
 * (z > cap, an internal buffer too small, or an error): then run
 * mpm_search for this text, which grows what it needs.  Successive calls
 * alternate between two internal buffer sets: the scan runs on the handle's
 * stream and the closing sort on an internal stream after it, overlapping the
 * next call's scan, so the outputs and status of a call are complete on the
 * handle's stream only after mpm_join (or mpm_sync, or any synchronous call).
 * Outputs of a call are overwritten by later calls that use the same arrays.
 * Host-side argument errors return MPM_EINVAL; nothing is enqueued then.
 * With timing on, each call's scan and verification times are added to the
 * statistics.
 */
int mpm_search_async(mpm_handle *h, const uint8_t *T, size_t n, uint32_t *out_pos,
                     uint32_t *out_pid, size_t cap, uint32_t *status);
/* Orders all later work on the handle's stream after the pipelined searches
 * enqueued so far (their outputs and status included), without waiting on
 * the host. */
int mpm_join(mpm_handle *h);
/* mpm_join, then waits until the handle's stream is idle and completes the
 * statistics of pipelined searches. */
int mpm_sync(mpm_handle *h);
/* Clears the statistics (waiting for timed pipelined searches in flight). */
int mpm_reset_stats(mpm_handle *h);

/* ---------------------------------------------- host-only planning calls */

/*
 * Resolves automatic parameters exactly as mpm_build would, without any GPU
 * work.  P, r, m, sigma and in are as for mpm_build; out receives the
 * resolved parameters and info (may be NULL) the derived sizes.
 */
int mpm_plan(const uint8_t *P, size_t r, size_t m, int sigma, const mpm_params *in,
             mpm_params *out, mpm_table_info *info);

/*
 * Builds, on the host only, the tables mpm_build would upload: mu[256] (the
 * byte -> reduced symbol map, Section 3.3; the identity with MPM_MAP_QHASH)
 * and the Shift-Or mask table (Sections 2, 3.2): entry c (q-gram code, first
 * symbol most significant, c = sum_t mu(S[t]) * sigma_r^(q-1-t); with
 * MPM_MAP_QHASH the q-gram's bin), entry_bytes little-endian bytes,
 * bit p (p < positions) is 0 iff some pattern, at some shift s < q, has code
 * c as its p-th non-overlapping q-gram; bits >= positions are 1.  table
 * (host memory) must hold table_bytes bytes (mpm_plan); mu or table may be
 * NULL to skip them.
 */
int mpm_host_tables(const uint8_t *P, size_t r, size_t m, int sigma,
                    const mpm_params *params, uint8_t *mu, void *table,
                    size_t table_bytes);

/*
 * Host-only check that the specialised scan kernels for these parameters
 * (the variant mpm_search runs, which verifies its candidates itself, and
 * the candidate variant of mpm_scan) compile (NVRTC, sm_103a), without
 * loading them on a device.  Returns
 * MPM_OK, MPM_ENOTSUP (parameters outside the specialised kernel, or NVRTC
 * missing) or MPM_ECUDA (compile error; the compiler log is copied to log,
 * log_bytes bytes at most, when log is not NULL).
 */
int mpm_jit_compile(const uint8_t *P, size_t r, size_t m, int sigma, const mpm_params *params,
                    char *log, size_t log_bytes);

/* ----------------------------------------------- single steps of a search */

/*
 * SMAG encode (Section 3.2): codes[h] = code of text q-gram h (bytes
 * T[hq..hq+q), mu applied, first symbol most significant) for
 * h < floor(n/q).  T and codes are device pointers; codes holds
 * floor(n/q) uint32 entries.
 */
int mpm_encode(mpm_handle *h, const uint8_t *T, size_t n, uint32_t *codes);

/*
 * The filter alone (Sections 3.1, 3.2): the AOSO Shift-Or scan of the
 * sampled q-grams h = k-1 (mod k) of T (device), with candidate compaction.
 * Each record is ((uint64)fired << 32) | h where h is the sampled q-gram
 * index and bit j of fired says subpattern j matched, i.e. the window of
 * q-grams starting at h - (m'-1)k - j is a candidate.  Records come in no
 * particular order.  *count is in: capacity of cand (device, entries), out:
 * number of records (MPM_ECAPACITY if it exceeds the capacity).
 */
int mpm_scan(mpm_handle *h, const uint8_t *T, size_t n, uint64_t *cand,
             size_t *count);

/* ----------------------------------------------------- batched search */

/*
 * Many texts, each searched against one of many built pattern sets, in one
 * persistent kernel launch (not in the paper; its filter per set is the one
 * of Sections 3.1 and 3.2 with that set's own q, k and mapping).  Texts are
 * device memory, shorter than 2^24 bytes each, fewer than 2^20 of them;
 * each set must have at most 32 filter positions, at most 2^20 patterns and,
 * with MPM_MAP_QHASH, q <= 5 (MPM_ENOTSUP otherwise); all sets on one
 * device.  The handles and texts must outlive the batch.  Occurrences are
 * reported as (text index, position, pattern id), sorted in that order.
 *
 * Mask tables of at most MPM_BATCH_SMEM_TABLE_BYTES are read from shared
 * memory by the batched kernel, larger ones from L2 (where, next to the text
 * stream of a large batch, they are often evicted).
 *
 * mpm_batch_create cuts every text into tiles of up to 32 lanes x lane_bytes
 * (each lane's share a multiple of lcm(k*q, 4) for its set), groups the
 * tiles of each set into work units, builds per-set device descriptors
 * (pointing at the handles' tables) and, unless
 * opts->no_graph, captures one run -- counter reset, the persistent scan
 * with in-kernel verification, a radix sort driven by the device-side
 * count, the split into three arrays and the 16-byte count read-back -- into
 * a CUDA graph on its own stream.  mpm_batch_run replays it (growing its
 * buffers and re-capturing when the occurrences outgrow them), waits, and
 * copies the result into out_tid/out_pos/out_pid (device or host): *z is in:
 * their capacity, out: the number of occurrences (MPM_ECAPACITY when it
 * exceeds the capacity).  mpm_search_batch does create, run and free once.
 */
typedef struct mpm_batch mpm_batch;

#define MPM_BATCH_SMEM_TABLE_BYTES (128u << 10)

typedef struct {
    int lane_bytes;  /* text bytes per lane of a tile; 0 = 512 */
    int no_graph;    /* 1: launch the kernels on every run instead of a graph */
    int unit_kib;    /* estimated cost of a work unit, in KiB of scanned text
                        (verification counted as extra bytes); 0 = 2048 */
    int generic;     /* 0: the kernel compiled (NVRTC, sm_103a) at create time
                        for the batch's parameter sets, the precompiled one when
                        that is not possible; 1: the precompiled kernel, whose
                        q, k and mapping are run-time values */
} mpm_batch_opts;

typedef struct {
    uint64_t bytes;       /* text bytes in the batch                        */
    uint64_t candidates;  /* candidate records of the last run              */
    uint64_t z;           /* occurrences of the last run                    */
    uint32_t tiles;       /* tiles in the work list                         */
    uint32_t launches;    /* kernels per run                                */
    float ms;             /* device time of the last run (events on the
                             batch stream around the graph launch)           */
    float scan_ms;        /* device time of the last run's scan kernel alone
                             (event records on either side of it, kept as
                             nodes of the graph); 0 when unavailable          */
    uint32_t variants;    /* parameter sets the batch's compiled kernel
                             specialises; 0: the precompiled kernel runs      */
    uint32_t pad;
} mpm_batch_stats;

mpm_batch *mpm_batch_create(mpm_handle *const *sets, int nsets, const uint8_t *const *texts,
                            const size_t *lens, const uint32_t *set_of_text, int ntexts,
                            const mpm_batch_opts *opts);
int mpm_batch_run(mpm_batch *b, uint32_t *out_tid, uint32_t *out_pos, uint32_t *out_pid,
                  size_t *z);
int mpm_batch_get_stats(const mpm_batch *b, mpm_batch_stats *out);
/* Host-only: compiles (NVRTC, sm_103a) the batched kernel that
 * mpm_batch_create would compile for nsets pattern sets -- set i being the
 * r[i] x m[i] patterns P[i] over sigma[i] symbols with parameters params[i]
 * (params may be NULL: automatic) -- without loading it; the compiler's
 * messages go to log (log_bytes, may be NULL).  MPM_ENOTSUP for a set the
 * batched form does not take (more than 32 positions, overlapping q-grams,
 * hashed q-grams of more than 5 bytes) or when NVRTC is missing. */
int mpm_batch_jit_compile(const uint8_t *const *P, const size_t *r, const size_t *m,
                          const int *sigma, const mpm_params *params, int nsets, char *log,
                          size_t log_bytes);
void mpm_batch_free(mpm_batch *b);
int mpm_search_batch(mpm_handle *const *sets, int nsets, const uint8_t *const *texts,
                     const size_t *lens, const uint32_t *set_of_text, int ntexts,
                     uint32_t *out_tid, uint32_t *out_pos, uint32_t *out_pid, size_t *z);

/* --------------------------------------------------------- autotuning */

typedef struct {
    int max_q;           /* largest q tried; 0 = 8                                  */
    int max_k;           /* largest k tried; 0 = 8                                  */
    int reps;            /* timed searches per parameter set (median); 0 = 3       */
    int kernels;         /* bit 0 specialised, bit 1 split, bit 2 generic (timed
                            through mpm_search), bit 3 the batched kernel (one
                            mpm_batch over copies of the sample, at least 128 MiB
                            and at most 256 copies, sets of <= 32 positions);
                            0 = 1                                                  */
    int max_sets;        /* at most this many sets are timed, lowest estimated
                            candidate rate first; 0 = 64                            */
    double max_rate;     /* sets whose estimated candidate records per sampled
                            q-gram exceed this are not timed, unless no set stays
                            under it (then the lowest-rate sets are); 0 = 0.05      */
    int max_positions;   /* only sets with at most this many filter positions
                            (32 for mpm_batch); 0 = 64                              */
    int grid;            /* 0: the tuner's grid above; 1: every point of the cost
                            model's grid (mpm_model_grid)                          */
    int max_table_kib;   /* only sets whose mask table has at most this many KiB;
                            0 = 16384                                               */
    int overlap;         /* 0: MAG's non-overlapping q-grams only; 1: those and
                            the overlapping q-grams of Section 2, each family
                            ranked on its own and given half of max_sets; 2: the
                            overlapping ones only (tuner grid only)                */
    int batch_generic;   /* bit 3 times: 0 the batched kernel compiled for the set
                            (compiled for every timed set first, in parallel); 1 the
                            precompiled one (run-time q, k and mapping)           */
} mpm_tune_opts;

typedef struct {
    mpm_params params;   /* resolved parameters of the set                         */
    mpm_table_info info;
    double ms;           /* median time of one search of the sample: wall time of
                            mpm_search, or device time of the batched run divided
                            by the number of copies                               */
    uint64_t candidates; /* candidate records of that search                        */
    uint64_t z;          /* occurrences                                             */
    int status;          /* MPM_OK, or why the set could not be built or run       */
} mpm_tune_entry;

/*
 * Exhaustive autotuner (not in the paper, which fixes q from log_sigma(rm)
 * and k by a closed form, Section 3.2): every feasible combination of
 * mapping and sigma' (equal-weight greedy bins and, where they keep the
 * pattern symbols distinct, low-order bits, for sigma' up to the pattern
 * alphabet; q-gram hashing into 2^10 .. 2^16 bins), q <= max_q and
 * k <= max_k is planned, with non-overlapping and/or overlapping q-grams as
 * opts->overlap asks; sets whose estimated
 * candidate rate exceeds max_rate are dropped (when that would drop every
 * set, the max_sets sets of lowest rate are kept), the rest (at most max_sets,
 * plus the planner's automatic choice, which is always timed unless
 * max_table_kib excludes its table)
 * are built and timed on the sample T[0..n) (device or host memory) with
 * each kernel selected in opts->kernels.  *best receives the fastest set;
 * entries (may be NULL) receive up to cap timed sets in the order they were
 * timed and *count the number of sets timed.  opts may be NULL.  Returns
 * MPM_EINVAL for bad arguments or when no set can be run.
 */
int mpm_autotune(const uint8_t *P, size_t r, size_t m, int sigma, const uint8_t *T, size_t n,
                 const mpm_tune_opts *opts, mpm_params *best, mpm_tune_entry *entries,
                 size_t cap, size_t *count);

/* ------------------------------------------------------ learned cost model */

/*
 * A small MLP predicts the batched scan's time for one pattern set and one
 * parameter set, so that parameters can be proposed without timing them
 * (not in the paper, which fixes q from log_sigma(rm) and k by a closed
 * form, Section 3.2).  Inputs x = [sigma, entropy of the text in bits per
 * symbol, log2 m, log10 r, log2 n, q, log2 sigma', k], standardised with a
 * per-input mean and standard deviation held by the model; 8 -> 64 -> 64 -> 1
 * with ReLU hidden units, FP32; the output is the standardised natural log of
 * the time in ms, mapped back with the model's output mean and deviation.
 * Parameters: one flat FP32 vector of MPM_MODEL_PARAMS numbers, W1 (64 x 8,
 * row j = hidden unit j), b1 (64), W2 (64 x 64), b2 (64), w3 (64), b3 (1).
 * Forward, gradient and Adam run in the library's own kernels; training is
 * deterministic for a given seed.  A model lives on the device that was
 * current when it first ran a kernel.
 */
#define MPM_MODEL_INPUTS 8
#define MPM_MODEL_HIDDEN 64
#define MPM_MODEL_PARAMS 4801

typedef struct mpm_model mpm_model;

typedef struct {
    float lr;            /* Adam step size; 0 = 1e-3                     */
    float beta1, beta2;  /* 0 = 0.9, 0.999                               */
    float eps;           /* 0 = 1e-8                                     */
    int epochs;          /* 0 = 200                                      */
    int batch;           /* samples per step; 0 = 256                    */
    uint64_t seed;       /* the order of each epoch is a function of (seed, epoch) */
} mpm_train_opts;

/* A new model: He-uniform weights from SplitMix64(seed), zero biases, unit
 * normalisation, a fresh Adam state.  NULL on error.  Host only. */
mpm_model *mpm_model_create(uint64_t seed);
void mpm_model_free(mpm_model *model);
/* Input/output normalisation (8 means, 8 deviations > 0, output mean and
 * deviation > 0).  Host only. */
int mpm_model_set_norm(mpm_model *model, const float *in_mean, const float *in_std,
                       float out_mean, float out_std);
int mpm_model_get_norm(const mpm_model *model, float *in_mean, float *in_std, float *out_mean,
                       float *out_std);
/* Copy the MPM_MODEL_PARAMS parameters out of / into the model (host
 * arrays); setting them resets the Adam state. */
int mpm_model_get_params(const mpm_model *model, float *theta);
int mpm_model_set_params(mpm_model *model, const float *theta);
/* y[i] = predicted ln(ms) for the raw features X[i*8 .. i*8+8).  X and y
 * are host or device arrays.  N = 0 is allowed. */
int mpm_model_predict(mpm_model *model, const float *X, size_t N, float *y);
/* Mean squared error of the standardised outputs against the standardised
 * targets y (raw ln(ms)) over all N samples, and its gradient (host array of
 * MPM_MODEL_PARAMS; may be NULL).  No parameter changes. */
int mpm_model_loss_grad(mpm_model *model, const float *X, const float *y, size_t N, float *loss,
                        float *grad);
/* One Adam step with the given gradient (host array). */
int mpm_model_adam_step(mpm_model *model, const float *grad, const mpm_train_opts *opts);
/* Mini-batch Adam on (X, y): opts->epochs passes, each over a permutation of
 * the samples; epoch_loss (may be NULL) receives each epoch's mean loss. */
int mpm_model_train(mpm_model *model, const float *X, const float *y, size_t N,
                    const mpm_train_opts *opts, float *epoch_loss);
/* Checkpoint: parameters, normalisation and Adam state (little-endian
 * binary).  Host only. */
int mpm_model_save(const mpm_model *model, const char *path);
mpm_model *mpm_model_load(const char *path);
/* The feasible points of the model's parameter grid for a pattern set: q in
 * 2..6 with sigma' in {2, 4, 8, 16} (the planner's mapping for that sigma'),
 * q in 2..5 with q-gram hashing into 2^12, 2^14 or 2^16 bins, every feasible
 * k <= 8, tables of at most 16 MiB and at most max_positions filter positions
 * (0 = 64).  *count receives the number of points; up to cap of them are
 * written to out (and info, which may be NULL).  Host only. */
int mpm_model_grid(const uint8_t *P, size_t r, size_t m, int sigma, int max_positions,
                   mpm_params *out, mpm_table_info *info, size_t cap, size_t *count);
/* Raw model inputs for `count` parameter sets of one pattern set (r patterns
 * of length m, declared alphabet sigma) searched in texts of n bytes whose
 * symbol entropy is `entropy` bits: X[i*8 ..] = [sigma, entropy, log2 m,
 * log10 r, log2 n, q, log2 sigma', k].  Host only. */
int mpm_model_features(int sigma, double entropy, size_t m, size_t r, size_t n,
                       const mpm_params *params, size_t count, float *X);
/* The grid point (at most 32 positions: the batched kernel's limit; a mask
 * table of at most max_table_bytes, 0 = no limit beyond the grid's) with the
 * smallest predicted time for a pattern set searched in texts of n bytes
 * whose symbol entropy is `entropy` bits.  *pred receives its ln(ms).
 * MPM_EINVAL when no grid point qualifies. */
int mpm_model_choose(mpm_model *model, const uint8_t *P, size_t r, size_t m, int sigma,
                     double entropy, size_t n, size_t max_table_bytes, mpm_params *best,
                     float *pred);

/* ------------------------------------------------------------ test hook */

/*
 * Failure detection without a GPU fault: fault = 1 arms the next launch of a
 * specialised scan (MPM_KERNEL_SPECIALISED or SPLIT, rows read through TMA)
 * so that one warp's first stage barrier expects 16 bytes more than its copy
 * brings; that warp's bounded wait gives up after about a second, it records
 * MPM_ETIMEOUT, waits (bounded) for its other copies and returns, and the
 * search returns MPM_ETIMEOUT.  The handle stays usable.  One-shot; 0
 * disarms.  MPM_EINVAL for other values.  Host only.
 */
int mpm_test_inject(int fault);

/* ------------------------------------------- search that allocates nothing */

/*
 * The paper has no counterpart to this call; it exists for callers of this
 * library that must not allocate device memory when they search: programs
 * whose GPU memory is all handed out by their own pool or caching allocator
 * (a stray cudaMalloc there can fail or fragment the pool), and
 * latency-sensitive servers, where cudaMalloc and cudaFree can synchronise
 * the device and stall every other stream.  mpm_search grows its scratch
 * buffers with cudaMalloc on first use and when a search needs more; this
 * call instead keeps all of its scratch (counters, candidate records and
 * occurrence keys) in one fixed array of device memory inside the library,
 * MPM_NOALLOC_SCRATCH_BYTES bytes, that every GPU which loads the library
 * holds until the process exits.  It calls no cudaMalloc, cudaFree or other
 * allocating routine.
 *
 * Arguments and results are those of mpm_search, except: T, out_pos and
 * out_pid must be device memory (host memory would need a staging buffer:
 * MPM_EINVAL), the handle must not use SMAG (MPM_ENOTSUP), and a search that
 * produces more than MPM_NOALLOC_MAX_CANDIDATES candidate records or more
 * than MPM_NOALLOC_MAX_OCCURRENCES occurrences is rejected with
 * MPM_ESCRATCH (*z is then the occurrence count when it is known, else 0);
 * mpm_search handles such searches.
 *
 * The first call on a device looks up that device's address of the array
 * (cudaGetSymbolAddress, with the device current); make that first call
 * before any stream capture.  Every call on a device shares the one array
 * and leaves its contents behind; each call clears the counters it needs.
 * Calls whose work overlaps on the GPU (different streams, threads or
 * handles on the same device) race on the array and must be serialised by
 * the caller.
 */
#define MPM_NOALLOC_MAX_CANDIDATES  (1u << 21)
#define MPM_NOALLOC_MAX_OCCURRENCES 8192u
#define MPM_NOALLOC_SCRATCH_BYTES   (256u + 8u * (MPM_NOALLOC_MAX_CANDIDATES + MPM_NOALLOC_MAX_OCCURRENCES))

int mpm_search_noalloc(mpm_handle *h, const uint8_t *T, size_t n, uint32_t *out_pos,
                       uint32_t *out_pid, size_t *z);

#ifdef __cplusplus
}
#endif

#endif /* MPM_H */
