/*
 * cxbwt — multi-string Burrows-Wheeler transform of short DNA reads on one
 * NVIDIA GB300 (sm_103a).
 *
 * The operation (Section 2 of Liu, Luo & Lam, "GPU-Accelerated BWT Construction
 * for Large Collection of Short Reads", arXiv 1401.7457):
 *
 *   R = {S_0 .. S_{n-1}} is a collection of reads over A < C < G < T.  Read i
 *   has L_i bases and is terminated by its own end marker $_i; every $ sorts
 *   below every base and $_i < $_j whenever i < j.  All N = sum_i (L_i + 1)
 *   suffixes (the terminator-only ones included) are sorted; B_R[r] is the
 *   symbol that precedes the r-th smallest suffix in its read, or $ when that
 *   suffix is the whole read.
 *
 * The method on the device is the paper's Section 3.2 (radix sort of suffixes
 * by fixed-width "stringwords", moving indices instead of strings, with the
 * variable-length / distinct-$ problem solved by padding plus a stable sort),
 * with the stringword gathered on the GPU from a resident 2-bit read store
 * instead of being copied from the host every iteration.
 *
 * Conventions used by every call below
 * ------------------------------------
 *  - Packed bases ("2-bit words"): base codes A=0, C=1, G=2, T=3 (the
 *    2-bit-per-base representation of Section 3).  Base j of a packed string
 *    occupies bits [31-2(j%16) .. 30-2(j%16)] of 32-bit word j/16 (most
 *    significant first, so a window of bases read as an integer orders like
 *    the string).  Reads are concatenated without padding: read i starts at
 *    base sum_{r<i} L_r.  The buffer holds ceil(sum L / 16) words; bits past
 *    the last base are ignored.
 *  - Lengths: 1 <= L_i <= 65535 (the paper's reads all have m >= 1 bases).
 *  - Pointers: every array argument may point to device memory (cudaMalloc,
 *    cudaMallocAsync, a torch CUDA tensor) or to host memory (pageable or
 *    pinned).  The library tells them apart with cudaPointerGetAttributes;
 *    device inputs are used in place, never copied.
 *  - Ownership: the caller owns every buffer passed in or out.  The library
 *    never frees, keeps or aliases them after the call has completed.
 *  - Streams: `stream` is a cudaStream_t passed as void* (NULL = the legacy
 *    default stream).  All device work of a call is ordered on it.  Unless the
 *    context option `async` is set, a call returns only after its work is
 *    complete; with it, a call returns after enqueueing when every output
 *    is device memory; errors raised on the device by such a call are
 *    reported by cxbwt_sync.  Calls on one context share its workspace, so
 *    they must be issued on one stream (or synchronised in between).
 *  - Errors: a negative cxbwt_status; cxbwt_last_error(ctx) gives a message.
 *    Nothing throws or aborts across this boundary.  On an error the outputs
 *    are unspecified.
 *  - Threads: a context may be used by one host thread at a time.
 */
#ifndef CXBWT_H
#define CXBWT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define CXBWT_ABI_VERSION 3

typedef enum {
  CXBWT_OK = 0,
  CXBWT_EINVAL = -1,        /* bad argument: NULL pointer, n_reads == 0, a length of 0 or > 65535 */
  CXBWT_ENOMEM = -2,        /* device memory or the context's device budget is exhausted */
  CXBWT_ECUDA = -3,         /* a CUDA runtime call failed */
  CXBWT_ETIMEOUT = -4,      /* a device-side wait gave up after its time limit (no hang, no trap) */
  CXBWT_EUNSUPPORTED = -5,  /* a size the current build does not handle */
  CXBWT_EBUSY = -6,         /* serving: no slot or budget free (only from non-blocking calls) */
  CXBWT_EINTERNAL = -7      /* an internal consistency check failed */
} cxbwt_status;

typedef struct cxbwt_ctx cxbwt_ctx;

/* Options of a context.  Zero in any field selects the default. */
typedef struct {
  uint64_t device_budget_bytes; /* cap on device memory the context may hold; 0 = 90% of free memory */
  int device;                   /* CUDA device ordinal */
  int prefix_len;               /* l of the group plan (Section 3.1: suffixes sharing their first l bases
                                   form one partition): its LSD passes sort the first l bases and each
                                   partition is finished on chip.  0 = automatic (the autotuned value for
                                   the build's size class, else 16), 12 or 16; other values give
                                   CXBWT_EUNSUPPORTED.  Slices and parts are planned from buckets of 4 or
                                   8 bases (16 when refined) whatever l is */
  int digit_bits;               /* radix digit width; 8 is the only width built (0 = 8, others give
                                   CXBWT_EUNSUPPORTED) */
  int tile_items;               /* items per radix tile: 0 = automatic (4096); 4096 or 8192 with 32-bit
                                   suffix ids, 2048, 3072 or 4096 with 64-bit ones */
  int async;                    /* nonzero: calls return after enqueue when outputs are on the device */
  int timing;                   /* nonzero: record CUDA events around every phase (see cxbwt_stats) */
  int algorithm;                /* CXBWT_ALGO_*: how the suffixes are sorted (all give identical output) */
  int plan_flags;               /* CXBWT_PLAN_* bits: force plan choices normally made by size (testing, tuning) */
  int batch_workers;            /* cxbwt_build_batch: concurrent worker contexts (0 = automatic) */
  int batch_small_mrows;        /* cxbwt_build_batch: collections below this many million suffixes are packed
                                   (0 = automatic, -1 = never) */
  int wait_limit_ms;            /* limit of every device-side wait (radix look-back); 0 = 1000 ms */
  int reserved[3];
} cxbwt_options;

/* plan_flags bits.  None changes the result.
 *  ID64        - carry 64-bit suffix ids even when 32 bits would do.
 *  READ_MAJOR  - when the build needs several slices, enumerate suffixes in
 *                read-major order (store read in address order) even when the
 *                store would fit L2. */
#define CXBWT_PLAN_ID64 1
#define CXBWT_PLAN_READ_MAJOR 2
/*  CARRY_BASE  - for reads of one length, carry the base before each suffix
 *                in its id from the first digit pass on, so that writing B_R
 *                gathers nothing from the store; by default only when the
 *                store is larger than 64 MB (out of L2). */
#define CXBWT_PLAN_CARRY_BASE 8
/*  NO_PREFETCH - carried-key digit passes do not ask for their tiles to be
 *                read into L2 ahead of the CTAs that sort them (by default
 *                they do when their arrays are 16-byte aligned). */
#define CXBWT_PLAN_NO_PREFETCH 16
/*  DIGIT_LISTING - list the suffixes of a build in slices with the general
 *                digit pass (digit = slice and suffix length, ranked by warp
 *                ballots) instead of the listing kernel whose threads each
 *                own one suffix length (reads of one length of at most 255
 *                bases). */
#define CXBWT_PLAN_DIGIT_LISTING 32
/* Test hook for failure handling: in the first digit pass of a build, tile 0
 * does not publish its counts, so tile 1's look-back wait runs out (after
 * wait_limit_ms).  The build then returns CXBWT_ETIMEOUT with unspecified
 * outputs; nothing hangs or faults and the context stays usable. */
#define CXBWT_PLAN_TEST_STALL 4

/* Sort plans.  Every plan computes the same B_R; they differ in speed only.
 *  AUTO     - GROUPS when the reads are at most 528 bases, else LSD.
 *  LSD      - stable LSD radix passes over every 4-base digit of the
 *             A-padded suffixes (Section 3.2 as stated: one pass per digit).
 *  GROUPS   - LSD passes over the first l = 16 (or prefix_len = 12)
 *             bases only (the l-prefix partition of Section 3.1), then each
 *             group of suffixes sharing those bases is finished on chip. */
#define CXBWT_ALGO_AUTO 0
#define CXBWT_ALGO_LSD 1
#define CXBWT_ALGO_GROUPS 2

/* Counters accumulated by a context since creation or cxbwt_reset_stats. */
typedef struct {
  uint64_t builds;              /* completed builds */
  uint64_t bases;               /* sum of read lengths over those builds */
  uint64_t suffixes;            /* sum of N over those builds */
  uint64_t kernel_launches;     /* kernels this library launched */
  uint64_t sort_pass_launches;  /* radix digit passes among them */
  uint64_t sort_pass_items;     /* sum over digit passes of the items each one moved */
  double sort_pass_ms;          /* device time of the digit passes (only with `timing`) */
  double build_ms;              /* device time of whole builds (only with `timing`) */
  uint64_t h2d_bytes;           /* bytes this library copied host -> device */
  uint64_t d2h_bytes;           /* bytes this library copied device -> host */
  uint64_t device_bytes_held;   /* device memory the context holds now */
  double group_ms;              /* device time finishing groups (group plan, only with `timing`) */
  double emit_ms;               /* device time of the emission (only with `timing`) */
  uint64_t slices;              /* device-memory-bounded slices sorted (one per build when it fits) */
  uint64_t cta_groups;          /* groups of equal first 16 bases finished by one CTA (33 .. 2048 rows) */
  uint64_t big_groups;          /* larger groups, finished with more digit passes */
  uint64_t carried_pass_launches; /* digit passes (among sort_pass_launches) that load the key window the
                                     previous pass carried, instead of generating ids or gathering it */
  uint64_t carried_pass_items;  /* sum over those passes of the items each one moved */
  double carried_pass_ms;       /* their device time, each pass between its own events (only with `timing`) */
  uint64_t reserved[2];
} cxbwt_stats;

/* ABI version of the loaded library (CXBWT_ABI_VERSION it was built with). */
int cxbwt_abi_version(void);

/* Fills *opt with the defaults. */
void cxbwt_default_options(cxbwt_options* opt);

/* Creates a context on opt->device (NULL opt = defaults).  The context owns
 * the device workspace (grown on demand within the budget and reused across
 * calls) and the per-call bookkeeping.  *out is set to NULL on failure. */
int cxbwt_create(cxbwt_ctx** out, const cxbwt_options* opt);

/* Waits for the context's outstanding work, frees everything it holds. NULL is a no-op. */
void cxbwt_destroy(cxbwt_ctx* ctx);

/* Message of the last error on ctx ("" if none); with ctx == NULL, the last
 * error of a failed cxbwt_create on this thread.  Valid until the next call. */
const char* cxbwt_last_error(const cxbwt_ctx* ctx);

/* Name of a status code. */
const char* cxbwt_status_string(int status);

/* Sizes of the outputs of a build of n_reads reads with host lengths `lens`:
 * *n_symbols = N = n_reads + sum(lens); *bwt_words = ceil(N / 16).
 * Either output pointer may be NULL. */
int cxbwt_output_size(uint64_t n_reads, const uint32_t* lens_host, uint64_t* n_symbols, uint64_t* bwt_words);

/* Builds the BWT of one read collection (Section 2 definition; Section 3.2 method).
 *
 *   reads_2bit      packed bases of all reads (layout above), ceil(sum L / 16) words
 *   n_reads         n >= 1
 *   lens            n read lengths (uint32)
 *   out_bwt         ceil(N / 16) words: B_R packed 2 bits per symbol in the
 *                   same layout; a $ symbol is stored as code 0 (its position
 *                   is given by out_dollar_pos).  Padding bits are 0.
 *   out_dollar_pos  n entries (may be NULL): out_dollar_pos[i] is the row r of
 *                   B_R holding the $ that precedes read i as a whole suffix,
 *                   i.e. the rank of suffix (i, 0).  These n rows are exactly
 *                   the $ symbols of B_R.
 *   out_counts      5 entries (may be NULL): occurrences of $, A, C, G, T in
 *                   B_R.  The FM-index array C[c] is their exclusive prefix sum.
 *
 * Returns CXBWT_OK, or CXBWT_EINVAL / ENOMEM / ECUDA / ETIMEOUT / EUNSUPPORTED. */
int cxbwt_build(cxbwt_ctx* ctx, const uint32_t* reads_2bit, uint64_t n_reads, const uint32_t* lens,
                uint32_t* out_bwt, uint64_t* out_dollar_pos, uint64_t* out_counts, void* stream);

/* cxbwt_build that also returns the sorted suffix list:
 *   out_sa          N entries: out_sa[r] = (i << 16) | k for the suffix
 *                   S_i[k..] $_i of rank r (k = L_i is the terminator-only one).
 * Meant for verification (a sortedness certificate at any size) and for
 * callers that sample the suffix array; it costs 8 extra bytes per suffix. */
int cxbwt_build_sa(cxbwt_ctx* ctx, const uint32_t* reads_2bit, uint64_t n_reads, const uint32_t* lens,
                   uint32_t* out_bwt, uint64_t* out_dollar_pos, uint64_t* out_counts, uint64_t* out_sa,
                   void* stream);

/* ---- bucket-range parts -----------------------------------------------------
 * Section 3.3 splits the suffixes by their l-prefix into ranges of buckets of
 * about equal size and builds each range on its own (one per GPU or node);
 * Section 3.1 builds such ranges one after the other when memory is bounded
 * (rounds).  B_R is the concatenation of the ranges' parts in bucket order,
 * because every suffix of a lower bucket sorts before every suffix of a
 * higher one.  Here a bucket is the first 8 bases of a suffix, A-padded past
 * the read end (CXBWT_BUCKETS of them).  Parts need reads of at most 528
 * bases (of one length or not).  A part holds whole 8-base buckets (inside a
 * part, a bucket larger than a device-memory slice is split by its next 8
 * bases). */
#define CXBWT_BUCKETS 65536u

/* Suffixes per bucket (Figure 2 step 1): out_counts (host, CXBWT_BUCKETS
 * entries) receives the counts; they sum to N.  Synchronous. */
int cxbwt_bucket_counts(cxbwt_ctx* ctx, const uint32_t* reads_2bit, uint64_t n_reads, const uint32_t* lens,
                        uint64_t* out_counts, void* stream);

/* Host only.  Splits buckets [0, n_buckets) into n_parts consecutive ranges
 * of about N / n_parts suffixes each: part j is buckets
 * [bucket_bounds[j], bucket_bounds[j+1]) and rows [row_bounds[j],
 * row_bounds[j+1]) of B_R (both arrays n_parts + 1 entries, non-decreasing,
 * from 0 to n_buckets and N).  A part is empty (equal bounds) when there are
 * more parts than buckets with suffixes.  EINVAL on NULL or n_parts == 0. */
int cxbwt_split_parts(const uint64_t* counts, uint32_t n_buckets, uint32_t n_parts, uint32_t* bucket_bounds,
                      uint64_t* row_bounds);

/* Builds the part of B_R made of the suffixes in buckets [bucket_lo,
 * bucket_hi), 0 <= bucket_lo < bucket_hi <= CXBWT_BUCKETS.  Its rows are
 * [row0, row0 + rows) of B_R, row0 = the suffixes of the buckets below
 * bucket_lo (both written to *out_row0 and *out_rows, host, may be NULL).
 *   bucket_counts   host, CXBWT_BUCKETS entries, or NULL: the collection's
 *                   counts as cxbwt_bucket_counts gives them (a caller that
 *                   builds several parts passes them to spare a count of
 *                   every suffix per part); EINVAL when they do not sum to N
 *   out_words       host or device, (row0 % 16 + rows + 15) / 16 words:
 *                   word j holds global BWT word row0 / 16 + j with only the
 *                   part's symbols set (the rest of the first and last word
 *                   is 0), so parts merge by OR (cxbwt_merge_part)
 *   out_dollar_pos  n_reads entries (may be NULL): as cxbwt_build for reads
 *                   whose $ row falls in the part, ~0 for the others; the
 *                   parts' arrays merge by element-wise minimum
 *   out_counts      5 entries (may be NULL): the part's symbol counts (they
 *                   add up over the parts)
 * The caller owns every buffer.  Returns as cxbwt_build; EINVAL for a bad
 * bucket range. */
int cxbwt_build_part(cxbwt_ctx* ctx, const uint32_t* reads_2bit, uint64_t n_reads, const uint32_t* lens,
                     uint32_t bucket_lo, uint32_t bucket_hi, const uint64_t* bucket_counts, uint32_t* out_words,
                     uint64_t* out_dollar_pos, uint64_t* out_counts, uint64_t* out_row0, uint64_t* out_rows,
                     void* stream);

/* Host only.  ORs a part's words (as cxbwt_build_part writes them, rows
 * [row0, row0 + rows)) into bwt_words, a zero-initialised host buffer of
 * n_words words of the whole B_R.  EINVAL when the part does not fit. */
int cxbwt_merge_part(uint32_t* bwt_words, uint64_t n_words, const uint32_t* part_words, uint64_t row0, uint64_t rows);

/* One collection of a batch. */
typedef struct {
  const uint32_t* reads_2bit;   /* packed bases, host or device (layout above) */
  uint64_t n_reads;
  const uint32_t* lens;         /* n_reads lengths, host or device */
  uint32_t* out_bwt;            /* as cxbwt_build */
  uint64_t* out_dollar_pos;     /* as cxbwt_build, may be NULL */
  uint64_t* out_counts;         /* as cxbwt_build, may be NULL */
} cxbwt_collection;

/* Builds the BWT of each of k independent collections (each result is
 * exactly what cxbwt_build gives for that collection alone).  Collections of
 * one read length are packed, up to a device-memory cap, into one sort: the
 * sorted order of the union restricted to one collection is that
 * collection's own order (the comparator of Section 2 is the same and the
 * union keeps each collection's read order), so one set of launches sorts
 * the pack, one stable pass by collection index separates it, and each
 * collection is emitted from its contiguous rows.  Collections too large for
 * a pack, or with reads of different lengths, are built one by one.
 * Returns after every result is complete; on an error, results of
 * collections not yet built are unspecified. */
int cxbwt_build_batch(cxbwt_ctx* ctx, const cxbwt_collection* colls, uint64_t k, void* stream);

/* ---- serving: continuous batching of build requests --------------------------
 *
 * A server runs `workers` builds at once, each on its own context (its share
 * of the device budget) and CUDA stream.  Requests queue in arrival order; a
 * free worker takes the oldest one.  A small one (under 2M suffixes) is
 * packed with every queued small request of the same read length that fits
 * the worker's pack cap (requests that arrive while others run join the next
 * pack) and built with them (cxbwt_build_batch); a larger one is built alone.
 * Each result is written into the request's host buffers and is exactly what
 * cxbwt_build gives for that request alone. */
typedef struct cxbwt_server cxbwt_server;

typedef struct {
  uint64_t device_budget_bytes; /* device memory all workers may hold together; 0 = min(120 GB, 90% of free) */
  int device;
  int workers;                  /* concurrent builds; 0 = 2 */
  uint64_t max_pack_suffixes;   /* suffixes built together at most; 0 = derived from the budget */
  int reserved[8];
} cxbwt_server_options;

/* A request: every pointer is host memory that must stay valid (and, for the
 * outputs, unread) until the request is done.  Pinned host memory makes the
 * copies faster. */
typedef struct {
  const uint32_t* reads_2bit;   /* packed bases (layout above) */
  uint64_t n_reads;
  const uint32_t* lens;
  uint32_t* out_bwt;            /* ceil(N / 16) words */
  uint64_t* out_dollar_pos;     /* n_reads entries, may be NULL */
  uint64_t* out_counts;         /* 5 entries, may be NULL */
} cxbwt_request;

void cxbwt_default_server_options(cxbwt_server_options* opt);
/* Creates the server and starts its workers (each creates a context). */
int cxbwt_server_create(cxbwt_server** out, const cxbwt_server_options* opt);
/* Finishes every submitted request, stops the workers, frees everything. */
void cxbwt_server_destroy(cxbwt_server* s);
/* Queues a request; *ticket names it.  EINVAL for a bad request, EBUSY while
 * the server is stopping.  Never blocks on the GPU.  Tickets (and their
 * times) are kept until the server is destroyed. */
int cxbwt_submit(cxbwt_server* s, const cxbwt_request* req, uint64_t* ticket);
/* *done = 1 once the request finished (then returns its status), else 0 (returns CXBWT_OK). */
int cxbwt_poll(cxbwt_server* s, uint64_t ticket, int* done);
/* Blocks until the request finished; returns its status. */
int cxbwt_wait(cxbwt_server* s, uint64_t ticket);
/* Of a finished request: time from submission to the start of its build and
 * to its completion (host clock, milliseconds).  EINVAL if not finished. */
int cxbwt_ticket_times(cxbwt_server* s, uint64_t ticket, double* queued_ms, double* latency_ms);
/* Requests completed, packs built, bases built so far (any pointer may be NULL). */
int cxbwt_server_counters(cxbwt_server* s, uint64_t* completed, uint64_t* packs, uint64_t* bases);

/* ---- autotuning -------------------------------------------------------------
 * Times every candidate plan on one collection (device or host buffers) and
 * keeps the fastest in the context for builds of the same maximum read
 * length and size class (N within a factor of two) whose options leave
 * tile_items, algorithm and prefix_len automatic.  Candidates: tiles of
 * 4096 or 8192 items (2048, 3072 or 4096 when the build carries 64-bit
 * suffix ids) x the group plan with l = 16 (reads of at most 528 bases) or
 * l = 12 (at most 524), or the LSD plan.  The radix digit is 8 bits (the
 * only width built).  scratch_bwt (ceil(N / 16) words) and
 * scratch_dollar_pos (n_reads, may be NULL) receive the BWT; every candidate
 * produces the same one. */
typedef struct {
  int tile_items;
  int algorithm;   /* CXBWT_ALGO_GROUPS or CXBWT_ALGO_LSD */
  int digit_bits;
  float best_ms;   /* device time of one build with the chosen plan */
  int prefix_len;  /* l of the chosen group plan (12 or 16); 0 for the LSD plan */
} cxbwt_tuning;
int cxbwt_autotune(cxbwt_ctx* ctx, const uint32_t* reads_2bit, uint64_t n_reads, const uint32_t* lens,
                   uint32_t* scratch_bwt, uint64_t* scratch_dollar_pos, void* stream, cxbwt_tuning* out);

/* Waits for the context's outstanding work and returns the first error a
 * device-side check recorded since the last call (CXBWT_OK if none). */
int cxbwt_sync(cxbwt_ctx* ctx);

/* Statistics (see cxbwt_stats). */
int cxbwt_get_stats(const cxbwt_ctx* ctx, cxbwt_stats* out);
int cxbwt_reset_stats(cxbwt_ctx* ctx);

/* ---- a build that allocates nothing ---------------------------------------
 *
 * The paper has no counterpart to this call; it serves callers that cannot
 * allocate device memory while they run: an application whose own pool
 * allocator owns all device memory and forbids allocations behind its back,
 * or a latency-bound loop where cudaFree's implicit device-wide
 * synchronisation would stall its other streams.
 *
 * It computes exactly what cxbwt_build computes, with every intermediate
 * buffer in one static device array of the library (about 34 MB, held by
 * every GPU that loads the library until the process exits).  No context is
 * needed and no memory is allocated: it calls no cudaMalloc, cudaFree,
 * cudaMallocHost or other allocating routine.
 *
 *   reads_2bit      device pointer, packed bases (layout above)
 *   lens_host       host pointer, n_reads lengths, all equal
 *   out_bwt         device pointer, ceil(N / 16) words (as cxbwt_build)
 *   out_dollar_pos  device pointer, n_reads entries (as cxbwt_build)
 *   out_counts      device or host pointer, 5 entries (as cxbwt_build)
 *   stream          cudaStream_t as void*; the call returns after the build
 *                   has completed on it
 *
 * Limits: N = n_reads * (L + 1) <= CXBWT_NOALLOC_MAX_SUFFIXES and
 * L <= CXBWT_NOALLOC_MAX_READ_LEN, one read length.  Returns CXBWT_OK;
 * CXBWT_EINVAL for a NULL pointer, n_reads == 0 or a length of 0 or above
 * 65535; CXBWT_EUNSUPPORTED for sizes beyond those limits or reads of
 * different lengths (both checked before any device work); CXBWT_ECUDA,
 * CXBWT_ETIMEOUT or CXBWT_EINTERNAL as cxbwt_build.
 *
 * The array is shared by every call on a device and keeps the previous
 * call's contents (each call clears what must start at zero).  Calls whose
 * device work overlaps - from two host threads, or on two streams without
 * synchronisation between them - race on it: callers must serialise them.
 * The first call on a device does that device's set-up (it looks up the
 * array's device address and clears it); make it before any stream capture.
 * Every call waits for its stream: it reads small results (the group-finish
 * counts, the error word) back to the host before it returns. */
#define CXBWT_NOALLOC_MAX_SUFFIXES (1u << 21)
#define CXBWT_NOALLOC_MAX_READ_LEN 272
int cxbwt_build_noalloc(const uint32_t* reads_2bit, uint64_t n_reads, const uint32_t* lens_host, uint32_t* out_bwt,
                        uint64_t* out_dollar_pos, uint64_t* out_counts, void* stream);

/* ---- host helpers (no device work) ---------------------------------------- */

/* Packs n_bases base codes (uint8 0..3) into ceil(n_bases/16) words, layout
 * above.  EINVAL on a code > 3. */
int cxbwt_pack_codes(const uint8_t* codes, uint64_t n_bases, uint32_t* out_words);

/* Same from ASCII "ACGT" (upper case).  EINVAL on any other character
 * (reads must be pre-filtered: the paper's reads contain only A, C, G, T). */
int cxbwt_pack_ascii(const char* acgt, uint64_t n_bases, uint32_t* out_words);

/* Expands a packed BWT of n_symbols symbols to ASCII over "$ACGT": symbol r is
 * '$' if r is one of the n_dollars entries of dollar_pos (any order), else
 * the base its code names.  out holds n_symbols bytes (no terminator).
 * EINVAL on a dollar position >= n_symbols. */
int cxbwt_unpack_ascii(const uint32_t* bwt_words, const uint64_t* dollar_pos, uint64_t n_symbols,
                       uint64_t n_dollars, char* out);

#ifdef __cplusplus
}
#endif

#endif /* CXBWT_H */
