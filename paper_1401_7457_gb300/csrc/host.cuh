// Host-side internals shared by the C ABI translation units: the context,
// device workspace helpers, and the plan / slice / run structures of a build.
#pragma once
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/cxbwt.h"
#include "group.cuh"
#include "kernels.cuh"

namespace cxbwt {
namespace host {


struct DevBuf {
  void* p = nullptr;
  size_t cap = 0;
};

constexpr uint64_t kTimeoutNs = 1000000000ull;  // look-back waits give up after 1 s

// An autotuned plan for builds of one maximum read length and size class
// (key: tune_key): tile items, algorithm, and the group plan's depth l.
struct TunedPlan {
  uint64_t key;
  int tile, algo, depth;
};

}  // namespace host
}  // namespace cxbwt

struct cxbwt_ctx {
  using DevBuf = cxbwt::host::DevBuf;
  cxbwt_options opt{};
  int device = 0;
  int sm_count = 0;
  uint64_t budget = 0;
  uint64_t held = 0;
  std::string err;

  DevBuf vals[2], keys[2], status, P, base, lenhist, desc, misc, store, out_bwt, out_dollar, out_sa, seglist, rhist,
      bhist;
  uint32_t epoch = 0;
  cudaStream_t side = nullptr;            // device -> host streaming of finished slices
  cudaEvent_t slice_done[2] = {nullptr, nullptr};
  std::vector<cudaEvent_t> tev;           // timing events, 4 per slice (timing option)
  std::vector<cudaEvent_t> pev;           // timing events, 2 per digit pass of a build (timing option)
  unsigned long long* h_small = nullptr;  // pinned: device error word, length stats
  cudaStream_t last_stream = nullptr;
  cudaEvent_t ev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
  cxbwt_stats stats{};
  // Autotuner choices (autotune.cu), one per maximum read length and size
  // class.  Used when the options leave tile, algorithm and depth automatic.
  std::vector<cxbwt::host::TunedPlan> tuned;
  void* batch_pool = nullptr;             // worker contexts of cxbwt_build_batch (batch.cu), created on first use
  void (*batch_pool_free)(void*) = nullptr;
};

namespace cxbwt {
namespace host {

inline int fail(cxbwt_ctx* c, int status, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  c->err = buf;
  return status;
}

#define CX_CUDA(ctx, call)                                                                          \
  do {                                                                                              \
    cudaError_t e_ = (call);                                                                        \
    if (e_ != cudaSuccess) {                                                                        \
      return fail((ctx), e_ == cudaErrorMemoryAllocation ? CXBWT_ENOMEM : CXBWT_ECUDA, "%s: %s (%s:%d)", \
                  #call, cudaGetErrorString(e_), __FILE__, __LINE__);                               \
    }                                                                                               \
  } while (0)

#define CX_TRY(expr)          \
  do {                        \
    int s_ = (expr);          \
    if (s_ != CXBWT_OK) return s_; \
  } while (0)

// Grow-only device buffer within the context's budget.
inline int ensure(cxbwt_ctx* c, DevBuf& b, size_t bytes, const char* what) {
  if (b.cap >= bytes) return CXBWT_OK;
  // Large buffers grow in 2 MB steps (fewer regrows), small ones in 64 KB steps.
  const size_t step = bytes >= (size_t(64) << 20) ? (size_t(1) << 21) : (size_t(1) << 16);
  const size_t want = std::max<size_t>((bytes + step - 1) & ~(step - 1), step);
  if (c->held - b.cap + want > c->budget)
    return fail(c, CXBWT_ENOMEM, "device budget of %llu bytes exceeded growing %s to %zu bytes",
                (unsigned long long)c->budget, what, want);
  if (b.p) {
    CX_CUDA(c, cudaFree(b.p));
    c->held -= b.cap;
    b.p = nullptr;
    b.cap = 0;
  }
  void* p = nullptr;
  cudaError_t e = cudaMalloc(&p, want);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(c, CXBWT_ENOMEM, "cudaMalloc(%zu) for %s: %s", want, what, cudaGetErrorString(e));
  }
  b.p = p;
  b.cap = want;
  c->held += want;
  return CXBWT_OK;
}

inline void release(cxbwt_ctx* c, DevBuf& b) {
  if (b.p) cudaFree(b.p);
  c->held -= b.cap;
  b.p = nullptr;
  b.cap = 0;
}

inline bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

inline bool is_pinned_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeHost;
}

// misc buffer layout (bytes)
constexpr size_t kMiscTileCounter = 0;   // uint32
constexpr size_t kMiscErr = 4;           // uint32
constexpr size_t kMiscCounts = 64;       // 5 x uint64
constexpr size_t kMiscLenStats = 128;    // 4 x uint64
constexpr size_t kMiscSeg = 192;         // 8 x uint32: group-finish list lengths and work counters
constexpr size_t kMiscBytes = 256;

inline uint32_t bits_for(uint32_t x) {  // smallest s with 2^s > x
  uint32_t s = 0;
  while (s < 32 && (uint64_t(1) << s) <= x) ++s;
  return s;
}

constexpr uint32_t kBucketBits = 16;  // parts (and slices when 4-base buckets are too coarse): first 8 bases

struct Plan {
  uint64_t n = 0, sum = 0, N = 0;
  uint32_t Lmin = 0, Lmax = 0, shift = 0;
  bool uniform = true;
  uint32_t D = 0;         // char digit positions (4 bases each)
  uint32_t W = 0;         // 16-base windows
  uint32_t len_passes = 0;
  uint64_t n_words = 0;
  int idb = 4;            // suffix id bytes
  uint32_t sym = 0;       // id bits holding the preceding base (0 or 2)
  bool groups = false;
  uint32_t depth = 16;    // group plan: bases sorted by the LSD passes (l of Section 3.1: 12 or 16)
  int seg_words = 0;
  uint32_t w_last = 0;    // windows [0, w_last] are sorted by LSD passes over all rows of a slice
};

// Id layout of a build: (read << shift) | (k << sym) | preceding base.  The
// preceding base rides along (sym = 2) when the emission would otherwise
// gather it from a store in HBM (want_sym: a store larger than L2) and the
// reads have one length (the first digit pass generates their ids), unless
// those two bits would push 32-bit ids to 64 bits; ids are 64-bit only when
// 32 bits cannot hold (read, k).  (With the store in L2 the gather is cheaper
// than carrying the base through the first pass.)
inline void plan_ids(Plan& pl, bool force64, bool want_sym) {
  const uint32_t len_bits = bits_for(pl.Lmax);
  const bool sym_ok = want_sym && pl.uniform;
  auto fits32 = [&](uint32_t sh) { return sh <= 31 && ((pl.n - 1) >> (32 - sh)) == 0; };
  if (!force64 && sym_ok && fits32(len_bits + 2)) {
    pl.idb = 4;
    pl.sym = 2;
  } else if (!force64 && fits32(len_bits)) {
    pl.idb = 4;
    pl.sym = 0;
  } else {
    pl.idb = 8;
    pl.sym = sym_ok ? 2 : 0;
  }
  pl.shift = len_bits + pl.sym;
}

struct Slice {
  bool whole = true;          // every suffix (no bucket filter)
  uint32_t key_lo = 0;        // when not whole: the suffixes whose first window (16 bases, A-padded)
  uint64_t key_hi = 0;        //   lies in [key_lo, key_hi), a range of buckets of 4, 8 or 16 bases
  uint32_t rows = 0;          // suffixes in the slice
  uint64_t row0 = 0;          // global BWT row of its first suffix
  bool pregen = false;        // its ids and first windows are already listed, in (length, read) order, in
                              // r.vals[0] / r.keys[0] (the split pass of a build in several slices)
  uint64_t arr0 = 0;          // split pass: its first row in the listing arrays (a multiple of 4, so
                              //   that its keys and ids start on 16-byte boundaries)
};

// A bucket-range part of a build (Section 3.3): only the suffixes whose first
// 8 bases (A-padded) fall in buckets [lo, hi) are sorted and emitted, into an
// output that starts at the part's first global word.  counts_only: return
// the per-bucket suffix counts (Figure 2 step 1) and build nothing.
struct PartSpec {
  uint32_t lo = 0, hi = 0;
  bool counts_only = false;
  uint64_t* bucket_counts = nullptr;  // host, 2^kBucketBits entries (counts_only)
  const uint64_t* given_counts = nullptr;  // host, 2^kBucketBits entries, or null: counted on the device
  uint64_t* row0 = nullptr;           // host: the part's first global row
  uint64_t* rows = nullptr;           // host: its number of rows
};

// Per-build device state shared by the slices.
struct Run {
  cudaStream_t st = nullptr;
  Plan pl;
  ReadIndex R{};
  TileShape shape{};
  void* vals[2] = {nullptr, nullptr};
  uint32_t* keys[2] = {nullptr, nullptr};
  uint32_t* base = nullptr;
  uint32_t* d_err = nullptr;
  uint32_t* d_counter = nullptr;
  uint32_t* d_seg = nullptr;
  unsigned long long* d_counts = nullptr;
  uint32_t* d_bwt = nullptr;      // global word w at d_bwt[w]
  uint64_t* d_dollar = nullptr;
  uint64_t* d_sa = nullptr;       // global rows
  bool read_major = false;        // multi-slice first pass in read-major order
  uint32_t bucket_bits = kBucketBits;  // slices are ranges of buckets of the first bucket_bits / 2 bases
  uint64_t launches = 0, sort_launches = 0, sort_items = 0, d2h = 0;
  uint64_t carried_launches = 0, carried_items = 0;
  // Per-pass timing (timing option): pass j ran between events pev[2j] and
  // pev[2j+1]; pev_carried[j] says whether it was a carried-key pass.
  uint32_t n_pev = 0;
  std::vector<uint8_t> pev_carried;  // 1: carried-key pass; 2: the split pass (outside every slice); 0: other
};

// Records the start event of one timed digit pass (grows the context's pool).
inline int pass_event_begin(cxbwt_ctx* c, Run& r) {
  while (c->pev.size() < 2 * size_t(r.n_pev + 1)) {
    cudaEvent_t ev;
    CX_CUDA(c, cudaEventCreate(&ev));
    c->pev.push_back(ev);
  }
  CX_CUDA(c, cudaEventRecord(c->pev[2 * size_t(r.n_pev)], r.st));
  return CXBWT_OK;
}

// Records the end event of the pass begun last.
inline int pass_event_end(cxbwt_ctx* c, Run& r, int kind) {
  CX_CUDA(c, cudaEventRecord(c->pev[2 * size_t(r.n_pev) + 1], r.st));
  r.pev_carried.push_back(uint8_t(kind));
  ++r.n_pev;
  return CXBWT_OK;
}

// Reads the device error word (already copied to h_small[4] by a completed
// call), clears it, and turns it into a status.  The word is sticky on the
// device until read here, so an error of an asynchronous build is not lost.
inline int take_device_error(cxbwt_ctx* c) {
  const uint32_t derr = *reinterpret_cast<volatile uint32_t*>(reinterpret_cast<char*>(c->h_small + 4));
  if (!derr) return CXBWT_OK;
  *reinterpret_cast<volatile uint32_t*>(reinterpret_cast<char*>(c->h_small + 4)) = 0;
  CX_CUDA(c, cudaMemset(static_cast<char*>(c->misc.p) + kMiscErr, 0, 4));
  if (derr & kErrTimeout) return fail(c, CXBWT_ETIMEOUT, "a radix look-back wait exceeded its limit");
  if (derr & kErrBounds)
    return fail(c, CXBWT_EINTERNAL, "a sort pass or the emission met an out-of-range row or suffix id");
  return fail(c, CXBWT_EINTERNAL, "device check failed (error word 0x%x)", derr);
}

inline void* vptr(void* base, int idb, uint64_t row) { return static_cast<char*>(base) + row * uint64_t(idb); }

inline uint64_t tune_key(uint32_t max_len, uint64_t n_suffixes) {
  uint32_t cls = 0;
  while (cls < 63 && (uint64_t(1) << (cls + 1)) <= n_suffixes) ++cls;
  return (uint64_t(max_len) << 8) | cls;
}

// The autotuned (tile items, algorithm, depth) of a build, or false.
inline bool tuned_choice(const cxbwt_ctx* c, uint32_t max_len, uint64_t n_suffixes, int* tile, int* algo,
                         int* depth) {
  const uint64_t k = tune_key(max_len, n_suffixes);
  for (const auto& e : c->tuned)
    if (e.key == k) {
      *tile = e.tile;
      *algo = e.algo;
      *depth = e.depth;
      return true;
    }
  return false;
}

// Sort one slice into r.vals[*cur_out] (api.cu).
int sort_slice(cxbwt_ctx* c, Run& r, const Slice& sl, int* cur_out, cudaEvent_t* tev);
// One whole build (api.cu).
int build_impl(cxbwt_ctx* c, const uint32_t* reads, uint64_t n, const uint32_t* lens, uint32_t* out_bwt,
               uint64_t* out_dollar, uint64_t* out_counts, uint64_t* out_sa, void* stream_v,
               const PartSpec* part = nullptr);

}  // namespace host
}  // namespace cxbwt
