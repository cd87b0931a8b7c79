// The C ABI of include/cxbwt.h: validation, device workspace, the pass plan
// of the LSD suffix sort, launches, and the host helpers.
//
// A build runs, on the caller's stream:
//   1. the all-digit histogram (k_poscount + k_digitbase): Figure 2 step 1's
//      scan of all suffixes, turned into the first output row of every digit
//      value of every pass;
//   2. for reads of different lengths, the (suffix length, read) start order
//      (k_identity + one or two length passes); for one common length that
//      order is generated inside the first digit pass;
//   3. the LSD digit passes (Section 3.2), least significant 4-base digit
//      first, each 16-base stringword window gathered once and carried in the
//      key array for its remaining passes;
//   4. emission (Figure 2 step 3(c)(iii)).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/cxbwt.h"
#include "group.cuh"
#include "kernels.cuh"

using namespace cxbwt;

namespace {

thread_local std::string g_create_error;

struct DevBuf {
  void* p = nullptr;
  size_t cap = 0;
};

constexpr uint64_t kTimeoutNs = 1000000000ull;  // look-back waits give up after 1 s

}  // namespace

struct cxbwt_ctx {
  cxbwt_options opt{};
  int device = 0;
  int sm_count = 0;
  uint64_t budget = 0;
  uint64_t held = 0;
  std::string err;

  DevBuf vals[2], keys[2], status, P, base, lenhist, desc, misc, store, out_bwt, out_dollar, out_sa, seglist, rhist;
  uint32_t epoch = 0;
  unsigned long long* h_small = nullptr;  // pinned: device error word, length stats
  cudaStream_t last_stream = nullptr;
  cudaEvent_t ev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
  cxbwt_stats stats{};
};

namespace {

int fail(cxbwt_ctx* c, int status, const char* fmt, ...) {
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
int ensure(cxbwt_ctx* c, DevBuf& b, size_t bytes, const char* what) {
  if (b.cap >= bytes) return CXBWT_OK;
  const size_t want = std::max<size_t>((bytes + (1u << 21) - 1) & ~size_t((1u << 21) - 1), 1u << 21);
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

void release(cxbwt_ctx* c, DevBuf& b) {
  if (b.p) cudaFree(b.p);
  c->held -= b.cap;
  b.p = nullptr;
  b.cap = 0;
}

bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// misc buffer layout (bytes)
constexpr size_t kMiscTileCounter = 0;   // uint32
constexpr size_t kMiscErr = 4;           // uint32
constexpr size_t kMiscCounts = 64;       // 5 x uint64
constexpr size_t kMiscLenStats = 128;    // 4 x uint64
constexpr size_t kMiscSeg = 192;         // 4 x uint32: group-finish list lengths and work counter
constexpr size_t kMiscBytes = 256;

uint32_t bits_for(uint32_t x) {  // smallest s with 2^s > x
  uint32_t s = 0;
  while (s < 32 && (uint64_t(1) << s) <= x) ++s;
  return s;
}

struct Plan {
  uint64_t n = 0, sum = 0, N = 0;
  uint32_t Lmin = 0, Lmax = 0, shift = 0;
  bool uniform = true;
  uint32_t D = 0;         // char digit positions (4 bases each)
  uint32_t W = 0;         // 16-base windows
  uint32_t len_passes = 0;
  uint64_t n_words = 0;
};

// Reads the device error word (already copied to h_small[4] by a completed
// call), clears it, and turns it into a status.  The word is sticky on the
// device until read here, so an error of an asynchronous build is not lost.
int take_device_error(cxbwt_ctx* c) {
  const uint32_t derr = *reinterpret_cast<volatile uint32_t*>(reinterpret_cast<char*>(c->h_small + 4));
  if (!derr) return CXBWT_OK;
  *reinterpret_cast<volatile uint32_t*>(reinterpret_cast<char*>(c->h_small + 4)) = 0;
  CX_CUDA(c, cudaMemset(static_cast<char*>(c->misc.p) + kMiscErr, 0, 4));
  if (derr & kErrTimeout)
    return fail(c, CXBWT_ETIMEOUT, "a radix look-back wait exceeded %.1f s", double(kTimeoutNs) * 1e-9);
  if (derr & kErrBounds)
    return fail(c, CXBWT_EINTERNAL, "a sort pass or the emission met an out-of-range row or suffix id");
  return fail(c, CXBWT_EINTERNAL, "device check failed (error word 0x%x)", derr);
}

int build_impl(cxbwt_ctx* c, const uint32_t* reads, uint64_t n, const uint32_t* lens, uint32_t* out_bwt,
               uint64_t* out_dollar, uint64_t* out_counts, uint64_t* out_sa, void* stream_v) {
  if (!c) return CXBWT_EINVAL;
  c->err.clear();
  if (!reads || !lens || !out_bwt) return fail(c, CXBWT_EINVAL, "reads_2bit, lens and out_bwt must not be NULL");
  if (n == 0) return fail(c, CXBWT_EINVAL, "n_reads must be at least 1");
  if (n >= (uint64_t(1) << 32)) return fail(c, CXBWT_EUNSUPPORTED, "more than 2^32 - 1 reads in one build");
  CX_CUDA(c, cudaSetDevice(c->device));
  cudaStream_t st = static_cast<cudaStream_t>(stream_v);
  c->last_stream = st;

  const bool reads_dev = is_device_ptr(reads), lens_dev = is_device_ptr(lens);
  const bool bwt_dev = is_device_ptr(out_bwt);
  const bool dollar_dev = out_dollar && is_device_ptr(out_dollar);
  const bool counts_dev = out_counts && is_device_ptr(out_counts);
  const bool sa_dev = out_sa && is_device_ptr(out_sa);
  uint64_t launches = 0, h2d = 0, d2h = 0;

  CX_TRY(ensure(c, c->misc, kMiscBytes, "scratch words"));
  char* misc = static_cast<char*>(c->misc.p);
  auto* d_err = reinterpret_cast<uint32_t*>(misc + kMiscErr);
  auto* d_counter = reinterpret_cast<uint32_t*>(misc + kMiscTileCounter);
  auto* d_counts = reinterpret_cast<unsigned long long*>(misc + kMiscCounts);
  auto* d_lstats = reinterpret_cast<unsigned long long*>(misc + kMiscLenStats);

  // ---- read lengths ------------------------------------------------------
  Plan pl;
  pl.n = n;
  std::vector<uint32_t> lens_copy;
  const uint32_t* hlens = nullptr;
  if (!lens_dev) {
    hlens = lens;
  }
  uint64_t mn = ~0ull, mx = 0, sum = 0, bad = 0;
  if (hlens) {
    for (uint64_t i = 0; i < n; ++i) {
      const uint32_t L = hlens[i];
      mn = std::min<uint64_t>(mn, L);
      mx = std::max<uint64_t>(mx, L);
      sum += L;
      bad += (L == 0 || L > 65535) ? 1 : 0;
    }
  } else {
    const unsigned long long init[4] = {~0ull, 0, 0, 0};
    CX_CUDA(c, cudaMemcpyAsync(d_lstats, init, sizeof init, cudaMemcpyHostToDevice, st));
    CX_CUDA(c, launch_lenstats(lens, n, d_lstats, st));
    ++launches;
    CX_CUDA(c, cudaMemcpyAsync(c->h_small, d_lstats, 4 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
    CX_CUDA(c, cudaStreamSynchronize(st));
    d2h += 32;
    mn = c->h_small[0];
    mx = c->h_small[1];
    sum = c->h_small[2];
    bad = c->h_small[3];
  }
  if (bad) return fail(c, CXBWT_EINVAL, "%llu read lengths are 0 or above 65535", (unsigned long long)bad);
  pl.Lmin = uint32_t(mn);
  pl.Lmax = uint32_t(mx);
  pl.sum = sum;
  pl.N = sum + n;
  pl.uniform = (mn == mx);
  pl.shift = bits_for(pl.Lmax);
  pl.D = (pl.Lmax + 3) / 4;
  pl.W = (pl.Lmax + 15) / 16;
  pl.len_passes = pl.uniform ? 0 : (pl.Lmax > 255 ? 2 : 1);
  pl.n_words = (sum + 15) / 16;
  const int seg_words = segsort_words(pl.Lmax);
  bool groups;
  switch (c->opt.algorithm) {
    case CXBWT_ALGO_LSD: groups = false; break;
    case CXBWT_ALGO_GROUPS:
      if (!seg_words) return fail(c, CXBWT_EUNSUPPORTED, "the group plan handles reads of at most 272 bases");
      groups = true;
      break;
    case CXBWT_ALGO_AUTO: groups = seg_words != 0; break;
    default: return fail(c, CXBWT_EINVAL, "unknown algorithm %d", c->opt.algorithm);
  }
  // Windows [0, w_last] are sorted by LSD passes over all rows; with the
  // group plan only window 0 is, and the groups are finished on chip.
  const uint32_t w_last = groups ? 0u : pl.W - 1;
  const uint32_t d_sorted = std::min<uint32_t>(pl.D, 4 * (w_last + 1));
  const uint64_t max_value = ((n - 1) << pl.shift) | pl.Lmax;
  if (pl.shift > 31 || ((n - 1) >> (32 - pl.shift)) != 0 || max_value > 0xFFFFFFFFull)
    return fail(c, CXBWT_EUNSUPPORTED, "n_reads x 2^%u exceeds the 32-bit suffix id space of one sort", pl.shift);
  if (pl.N >= (uint64_t(1) << 32)) return fail(c, CXBWT_EUNSUPPORTED, "more than 2^32 - 1 suffixes in one sort");

  // ---- inputs on the device ----------------------------------------------
  const uint32_t* d_reads = reads;
  if (!reads_dev) {
    CX_TRY(ensure(c, c->store, pl.n_words * 4, "read store"));
    CX_CUDA(c, cudaMemcpyAsync(c->store.p, reads, pl.n_words * 4, cudaMemcpyHostToDevice, st));
    h2d += pl.n_words * 4;
    d_reads = static_cast<const uint32_t*>(c->store.p);
  }
  const uint32_t TILE = uint32_t(onesweep_shape(c->opt.tile_items).tile());
  const uint64_t n_tiles = (pl.N + TILE - 1) / TILE;
  std::vector<uint32_t> len_bases;
  const uint64_t* d_desc = nullptr;
  const uint32_t* d_lenhist = nullptr;
  if (!pl.uniform) {
    if (!hlens) {
      lens_copy.resize(n);
      CX_CUDA(c, cudaMemcpyAsync(lens_copy.data(), lens, n * 4, cudaMemcpyDeviceToHost, st));
      CX_CUDA(c, cudaStreamSynchronize(st));
      d2h += n * 4;
      hlens = lens_copy.data();
    }
    std::vector<uint64_t> desc(n);
    std::vector<uint32_t> lh(pl.Lmax + 1, 0);
    uint64_t off = 0;
    for (uint64_t i = 0; i < n; ++i) {
      desc[i] = (off << 16) | hlens[i];
      off += hlens[i];
      ++lh[hlens[i]];
    }
    // Length passes: digit j of the suffix length t = L_i - k; there are
    // cnt(t) = #{i : L_i >= t} suffixes of length t.
    std::vector<uint64_t> cnt(pl.Lmax + 1, 0);
    uint64_t run = 0;
    for (int64_t t = pl.Lmax; t >= 0; --t) {
      run += lh[t];
      cnt[t] = run;
    }
    len_bases.assign(size_t(pl.len_passes) * kRadix, 0);
    for (uint32_t j = 0; j < pl.len_passes; ++j) {
      std::vector<uint64_t> h(kRadix, 0);
      for (uint32_t t = 0; t <= pl.Lmax; ++t) h[(t >> (8 * j)) & 255] += cnt[t];
      uint64_t acc = 0;
      for (int v = 0; v < kRadix; ++v) {
        len_bases[size_t(j) * kRadix + v] = uint32_t(acc);
        acc += h[v];
      }
    }
    CX_TRY(ensure(c, c->desc, n * 8, "read descriptors"));
    CX_TRY(ensure(c, c->lenhist, (pl.Lmax + 1) * 4, "length histogram"));
    CX_CUDA(c, cudaMemcpyAsync(c->desc.p, desc.data(), n * 8, cudaMemcpyHostToDevice, st));
    CX_CUDA(c, cudaMemcpyAsync(c->lenhist.p, lh.data(), (pl.Lmax + 1) * 4, cudaMemcpyHostToDevice, st));
    h2d += n * 8 + (pl.Lmax + 1) * 4;
    d_desc = static_cast<const uint64_t*>(c->desc.p);
    d_lenhist = static_cast<const uint32_t*>(c->lenhist.p);
  }

  // ---- workspace ---------------------------------------------------------
  CX_TRY(ensure(c, c->vals[0], pl.N * 4, "suffix ids"));
  CX_TRY(ensure(c, c->vals[1], pl.N * 4, "suffix ids"));
  CX_TRY(ensure(c, c->keys[0], pl.N * 4, "keys"));
  CX_TRY(ensure(c, c->keys[1], pl.N * 4, "keys"));
  const void* status_before = c->status.p;
  CX_TRY(ensure(c, c->status, n_tiles * kRadix * 8, "look-back words"));
  if (c->status.p != status_before) {
    // Fresh memory could hold any flag value: clear it so no stale word looks published.
    CX_CUDA(c, cudaMemsetAsync(c->status.p, 0, c->status.cap, st));
  }
  CX_TRY(ensure(c, c->P, uint64_t(pl.Lmax) * kRadix * 4, "position counts"));
  CX_TRY(ensure(c, c->base, uint64_t(pl.D + pl.len_passes) * kRadix * 4, "digit bases"));
  uint32_t* d_base = static_cast<uint32_t*>(c->base.p);
  if (pl.len_passes) {
    CX_CUDA(c, cudaMemcpyAsync(d_base + size_t(pl.D) * kRadix, len_bases.data(), len_bases.size() * 4,
                               cudaMemcpyHostToDevice, st));
    h2d += len_bases.size() * 4;
  }
  const uint32_t passes = pl.D + pl.len_passes;
  if (uint64_t(c->epoch) + passes + 2 >= (uint64_t(1) << 30)) {
    // Look-back flags are 2*epoch and 2*epoch+1 in 32 bits: restart the epochs.
    CX_CUDA(c, cudaMemsetAsync(c->status.p, 0, c->status.cap, st));
    c->epoch = 0;
  }
  CX_CUDA(c, cudaMemsetAsync(c->P.p, 0, uint64_t(pl.Lmax) * kRadix * 4, st));
  CX_CUDA(c, cudaMemsetAsync(d_counts, 0, 5 * 8, st));

  const bool timing = c->opt.timing != 0;
  if (timing) CX_CUDA(c, cudaEventRecord(c->ev[0], st));

  ReadIndex R{d_reads, pl.n_words, d_desc, pl.shift, pl.uniform ? pl.Lmax : 0u, uint32_t(n),
              (reinterpret_cast<uintptr_t>(d_reads) & 15u) == 0 ? 1u : 0u};

  // ---- 1. all-digit histogram -----------------------------------------------
  CX_CUDA(c, launch_poscount(R, uint32_t(n), pl.Lmax, static_cast<uint32_t*>(c->P.p), c->sm_count, st));
  CX_CUDA(c, launch_digitbase(static_cast<const uint32_t*>(c->P.p), pl.Lmax, d_sorted, pl.uniform ? 1 : 0,
                              uint32_t(n), pl.Lmax, d_lenhist, d_base, st));
  launches += 2;

  // ---- 2./3. digit passes ----------------------------------------------------
  uint32_t* vals[2] = {static_cast<uint32_t*>(c->vals[0].p), static_cast<uint32_t*>(c->vals[1].p)};
  uint32_t* keys[2] = {static_cast<uint32_t*>(c->keys[0].p), static_cast<uint32_t*>(c->keys[1].p)};
  int cur = 0, kin = 0;
  const TileShape shape = onesweep_shape(c->opt.tile_items);
  PassArgs a{};
  a.status = static_cast<unsigned long long*>(c->status.p);
  a.tile_counter = d_counter;
  a.err = d_err;
  a.R = R;
  a.n_items = uint32_t(pl.N);
  a.n_tiles = uint32_t(n_tiles);
  a.n_reads = uint32_t(n);
  a.timeout_ns = kTimeoutNs;

  if (!pl.uniform) {
    CX_CUDA(c, launch_identity(R, uint32_t(n), nullptr, vals[0], st));
    ++launches;
  }
  if (timing) CX_CUDA(c, cudaEventRecord(c->ev[1], st));
  uint64_t sort_launches = 0, sort_items = 0;
  for (uint32_t j = 0; j < pl.len_passes; ++j) {
    a.vals_in = vals[cur];
    a.vals_out = vals[cur ^ 1];
    a.keys_in = nullptr;
    a.keys_out = nullptr;
    a.digit_base = d_base + size_t(pl.D + j) * kRadix;
    a.key_shift = 8 * j;
    a.window_c0 = 0;
    a.epoch = ++c->epoch;
    CX_CUDA(c, launch_onesweep(a, kSrcLength, false, shape, st));
    cur ^= 1;
    ++sort_launches;
    sort_items += pl.N;
  }
  bool first = pl.uniform;
  for (int64_t w = int64_t(w_last); w >= 0; --w) {
    const uint32_t d_lo = uint32_t(4 * w);
    const uint32_t d_hi = std::min<uint32_t>(d_lo + 3, pl.D - 1);
    for (int64_t d = d_hi; d >= int64_t(d_lo); --d) {
      const bool first_in_window = (uint32_t(d) == d_hi);
      const bool last_in_window = (uint32_t(d) == d_lo);
      const int mode = first_in_window ? (first ? kSrcInitUniform : kSrcExtract) : kSrcCarried;
      // The group plan keeps the window-0 keys of the final order: groups are runs of equal keys.
      const bool write_key = !last_in_window || groups;
      a.vals_in = vals[cur];
      a.vals_out = vals[cur ^ 1];
      a.keys_in = (mode == kSrcCarried) ? keys[kin] : nullptr;
      const int kout = (mode == kSrcCarried) ? (kin ^ 1) : kin;
      a.keys_out = write_key ? keys[kout] : nullptr;
      a.digit_base = d_base + size_t(d) * kRadix;
      a.key_shift = 24u - 8u * uint32_t(d - d_lo);
      a.window_c0 = uint32_t(16 * w);
      a.epoch = ++c->epoch;
      CX_CUDA(c, launch_onesweep(a, mode, write_key, shape, st));
      cur ^= 1;
      if (write_key) kin = kout;
      first = false;
      ++sort_launches;
      sort_items += pl.N;
    }
  }
  if (timing) CX_CUDA(c, cudaEventRecord(c->ev[2], st));
  launches += sort_launches;

  // ---- 3b. group plan: finish every group of equal first windows on chip ------
  if (groups && pl.Lmax > 16) {
    const uint64_t cta_cap = pl.N / 33 + 1, big_cap = pl.N / kCtaMax + 1;
    CX_TRY(ensure(c, c->seglist, (cta_cap + big_cap) * 8, "group lists"));
    auto* d_seg = reinterpret_cast<uint32_t*>(misc + kMiscSeg);
    CX_CUDA(c, cudaMemsetAsync(d_seg, 0, 16, st));
    SegArgs g{};
    g.keys = keys[kin];
    g.vals = vals[cur];
    g.n_items = uint32_t(pl.N);
    g.R = R;
    g.depth = 16;
    g.cta_list = static_cast<uint2*>(c->seglist.p);
    g.cta_cap = uint32_t(cta_cap);
    g.big_list = g.cta_list + cta_cap;
    g.big_cap = uint32_t(big_cap);
    g.counts = d_seg;
    g.err = d_err;
    CX_CUDA(c, launch_segsort(g, seg_words, c->sm_count, st));
    launches += 2;
    // Remainders too large for one CTA (rare: long runs of equal bases) are
    // finished here with LSD passes over bases 16.. restricted to their rows.
    CX_CUDA(c, cudaMemcpyAsync(c->h_small + 5, d_seg, 8, cudaMemcpyDeviceToHost, st));
    CX_CUDA(c, cudaStreamSynchronize(st));
    const uint32_t n_big = std::min<uint32_t>(reinterpret_cast<const uint32_t*>(c->h_small + 5)[1], g.big_cap);
    if (n_big) {
      std::vector<uint2> big(n_big);
      CX_CUDA(c, cudaMemcpyAsync(big.data(), g.big_list, n_big * 8, cudaMemcpyDeviceToHost, st));
      CX_CUDA(c, cudaStreamSynchronize(st));
      d2h += n_big * 8;
      const uint32_t n_win = pl.W - 1;
      CX_TRY(ensure(c, c->rhist, size_t(n_win) * 4 * kRadix * 4, "group digit counts"));
      auto* rh = static_cast<uint32_t*>(c->rhist.p);
      for (const uint2& bg : big) {
        const uint32_t s0 = bg.x, m = bg.y;
        CX_CUDA(c, cudaMemsetAsync(rh, 0, size_t(n_win) * 4 * kRadix * 4, st));
        CX_CUDA(c, launch_range_hist(vals[cur] + s0, m, R, n_win, rh, c->sm_count, st));
        launches += 2;
        uint32_t* gv[2] = {vals[cur] + s0, vals[cur ^ 1] + s0};
        uint32_t* gk[2] = {keys[0] + s0, keys[1] + s0};
        int gc = 0, gki = 0;
        PassArgs b = a;
        b.n_items = m;
        b.n_tiles = uint32_t((m + TILE - 1) / TILE);
        for (uint32_t w = pl.W - 1; w >= 1; --w) {
          const uint32_t d_lo = 4 * w;
          const uint32_t d_hi = std::min<uint32_t>(d_lo + 3, pl.D - 1);
          for (int64_t d = d_hi; d >= int64_t(d_lo); --d) {
            const bool first_in_window = (uint32_t(d) == d_hi);
            const bool last_in_window = (uint32_t(d) == d_lo);
            const int mode = first_in_window ? kSrcExtract : kSrcCarried;
            const bool write_key = !last_in_window;
            b.vals_in = gv[gc];
            b.vals_out = gv[gc ^ 1];
            b.keys_in = (mode == kSrcCarried) ? gk[gki] : nullptr;
            const int kout = (mode == kSrcCarried) ? (gki ^ 1) : gki;
            b.keys_out = write_key ? gk[kout] : nullptr;
            b.digit_base = rh + size_t((w - 1) * 4 + (uint32_t(d) - d_lo)) * kRadix;
            b.key_shift = 24u - 8u * (uint32_t(d) - d_lo);
            b.window_c0 = 16 * w;
            b.epoch = ++c->epoch;
            CX_CUDA(c, launch_onesweep(b, mode, write_key, shape, st));
            gc ^= 1;
            if (write_key) gki = kout;
            ++launches;
            ++sort_launches;
            sort_items += m;
          }
        }
        if (gc) CX_CUDA(c, cudaMemcpyAsync(gv[0], gv[1], size_t(m) * 4, cudaMemcpyDeviceToDevice, st));
      }
    }
  }

  if (timing) CX_CUDA(c, cudaEventRecord(c->ev[4], st));

  // ---- 4. emission -----------------------------------------------------------
  const uint64_t bwt_words = (pl.N + 15) / 16;
  uint32_t* d_bwt = out_bwt;
  if (!bwt_dev) {
    CX_TRY(ensure(c, c->out_bwt, bwt_words * 4, "BWT output"));
    d_bwt = static_cast<uint32_t*>(c->out_bwt.p);
  }
  uint64_t* d_dollar = out_dollar;
  if (out_dollar && !dollar_dev) {
    CX_TRY(ensure(c, c->out_dollar, n * 8, "dollar positions"));
    d_dollar = static_cast<uint64_t*>(c->out_dollar.p);
  }
  uint64_t* d_sa = out_sa;
  if (out_sa && !sa_dev) {
    CX_TRY(ensure(c, c->out_sa, pl.N * 8, "suffix array output"));
    d_sa = static_cast<uint64_t*>(c->out_sa.p);
  }
  EmitArgs e{vals[cur], uint32_t(pl.N), R, d_bwt, d_dollar, d_counts, d_sa, d_err};
  CX_CUDA(c, launch_emit(e, st));
  ++launches;
  if (out_counts) {
    CX_CUDA(c, cudaMemcpyAsync(out_counts, d_counts, 5 * 8, counts_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                               st));
    if (!counts_dev) d2h += 40;
  }
  if (timing) CX_CUDA(c, cudaEventRecord(c->ev[3], st));
  if (!bwt_dev) {
    CX_CUDA(c, cudaMemcpyAsync(out_bwt, d_bwt, bwt_words * 4, cudaMemcpyDeviceToHost, st));
    d2h += bwt_words * 4;
  }
  if (out_dollar && !dollar_dev) {
    CX_CUDA(c, cudaMemcpyAsync(out_dollar, d_dollar, n * 8, cudaMemcpyDeviceToHost, st));
    d2h += n * 8;
  }
  if (out_sa && !sa_dev) {
    CX_CUDA(c, cudaMemcpyAsync(out_sa, d_sa, pl.N * 8, cudaMemcpyDeviceToHost, st));
    d2h += pl.N * 8;
  }
  CX_CUDA(c, cudaMemcpyAsync(c->h_small + 4, d_err, 4, cudaMemcpyDeviceToHost, st));

  c->stats.kernel_launches += launches;
  c->stats.sort_pass_launches += sort_launches;
  c->stats.sort_pass_items += sort_items;
  c->stats.h2d_bytes += h2d;
  c->stats.d2h_bytes += d2h;
  c->stats.device_bytes_held = c->held;

  const bool host_out = !bwt_dev || (out_dollar && !dollar_dev) || (out_counts && !counts_dev) || (out_sa && !sa_dev);
  if (c->opt.async && !host_out) {
    // Completed (and checked) by the next call on this context or cxbwt_sync.
    c->stats.builds += 1;
    c->stats.bases += pl.sum;
    c->stats.suffixes += pl.N;
    return CXBWT_OK;
  }
  CX_CUDA(c, cudaStreamSynchronize(st));
  CX_TRY(take_device_error(c));
  if (timing) {
    float ms_sort = 0, ms_all = 0, ms_group = 0, ms_emit = 0;
    CX_CUDA(c, cudaEventElapsedTime(&ms_sort, c->ev[1], c->ev[2]));
    CX_CUDA(c, cudaEventElapsedTime(&ms_group, c->ev[2], c->ev[4]));
    CX_CUDA(c, cudaEventElapsedTime(&ms_emit, c->ev[4], c->ev[3]));
    CX_CUDA(c, cudaEventElapsedTime(&ms_all, c->ev[0], c->ev[3]));
    c->stats.sort_pass_ms += ms_sort;
    c->stats.group_ms += ms_group;
    c->stats.emit_ms += ms_emit;
    c->stats.build_ms += ms_all;
  }
  c->stats.builds += 1;
  c->stats.bases += pl.sum;
  c->stats.suffixes += pl.N;
  return CXBWT_OK;
}

}  // namespace

extern "C" {

int cxbwt_abi_version(void) { return CXBWT_ABI_VERSION; }

void cxbwt_default_options(cxbwt_options* opt) {
  if (!opt) return;
  std::memset(opt, 0, sizeof *opt);
  opt->digit_bits = 8;
}

int cxbwt_create(cxbwt_ctx** out, const cxbwt_options* opt) {
  g_create_error.clear();
  if (!out) {
    g_create_error = "out must not be NULL";
    return CXBWT_EINVAL;
  }
  *out = nullptr;
  cxbwt_options o;
  cxbwt_default_options(&o);
  if (opt) o = *opt;
  if (o.digit_bits == 0) o.digit_bits = 8;
  if (o.digit_bits != 8) {
    g_create_error = "digit_bits: only 8-bit digits are built";
    return CXBWT_EUNSUPPORTED;
  }
  int ndev = 0;
  cudaError_t e = cudaGetDeviceCount(&ndev);
  if (e != cudaSuccess || ndev == 0) {
    cudaGetLastError();
    g_create_error = std::string("no CUDA device: ") + cudaGetErrorString(e);
    return CXBWT_ECUDA;
  }
  if (o.device < 0 || o.device >= ndev) {
    g_create_error = "device ordinal out of range";
    return CXBWT_EINVAL;
  }
  e = cudaSetDevice(o.device);
  if (e != cudaSuccess) {
    g_create_error = std::string("cudaSetDevice: ") + cudaGetErrorString(e);
    return CXBWT_ECUDA;
  }
  auto* c = new cxbwt_ctx();
  c->opt = o;
  c->device = o.device;
  cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, o.device);
  size_t free_b = 0, total_b = 0;
  cudaMemGetInfo(&free_b, &total_b);
  c->budget = o.device_budget_bytes ? o.device_budget_bytes : uint64_t(double(free_b) * 0.9);
  bool ok = cudaMallocHost(reinterpret_cast<void**>(&c->h_small), 64) == cudaSuccess;
  for (auto& ev : c->ev) ok = ok && cudaEventCreate(&ev) == cudaSuccess;
  if (ok) ok = ensure(c, c->misc, kMiscBytes, "scratch words") == CXBWT_OK;
  if (ok) ok = cudaMemset(c->misc.p, 0, kMiscBytes) == cudaSuccess;
  if (!ok) {
    g_create_error = c->err.empty() ? std::string("context set-up failed: ") + cudaGetErrorString(cudaGetLastError())
                                    : c->err;
    cxbwt_destroy(c);
    return CXBWT_ECUDA;
  }
  *out = c;
  return CXBWT_OK;
}

void cxbwt_destroy(cxbwt_ctx* c) {
  if (!c) return;
  cudaSetDevice(c->device);
  cudaDeviceSynchronize();
  DevBuf* bufs[] = {&c->vals[0], &c->vals[1], &c->keys[0], &c->keys[1], &c->status, &c->P, &c->base,
                    &c->lenhist, &c->desc, &c->misc, &c->store, &c->out_bwt, &c->out_dollar, &c->out_sa,
                    &c->seglist, &c->rhist};
  for (DevBuf* b : bufs) release(c, *b);
  for (auto& ev : c->ev)
    if (ev) cudaEventDestroy(ev);
  if (c->h_small) cudaFreeHost(c->h_small);
  delete c;
}

const char* cxbwt_last_error(const cxbwt_ctx* c) { return c ? c->err.c_str() : g_create_error.c_str(); }

const char* cxbwt_status_string(int s) {
  switch (s) {
    case CXBWT_OK: return "CXBWT_OK";
    case CXBWT_EINVAL: return "CXBWT_EINVAL";
    case CXBWT_ENOMEM: return "CXBWT_ENOMEM";
    case CXBWT_ECUDA: return "CXBWT_ECUDA";
    case CXBWT_ETIMEOUT: return "CXBWT_ETIMEOUT";
    case CXBWT_EUNSUPPORTED: return "CXBWT_EUNSUPPORTED";
    case CXBWT_EBUSY: return "CXBWT_EBUSY";
    case CXBWT_EINTERNAL: return "CXBWT_EINTERNAL";
    default: return "CXBWT_UNKNOWN";
  }
}

int cxbwt_output_size(uint64_t n_reads, const uint32_t* lens, uint64_t* n_symbols, uint64_t* bwt_words) {
  if (n_reads && !lens) return CXBWT_EINVAL;
  uint64_t N = n_reads;
  for (uint64_t i = 0; i < n_reads; ++i) N += lens[i];
  if (n_symbols) *n_symbols = N;
  if (bwt_words) *bwt_words = (N + 15) / 16;
  return CXBWT_OK;
}

int cxbwt_build(cxbwt_ctx* ctx, const uint32_t* reads_2bit, uint64_t n_reads, const uint32_t* lens,
                uint32_t* out_bwt, uint64_t* out_dollar_pos, uint64_t* out_counts, void* stream) {
  return build_impl(ctx, reads_2bit, n_reads, lens, out_bwt, out_dollar_pos, out_counts, nullptr, stream);
}

int cxbwt_build_sa(cxbwt_ctx* ctx, const uint32_t* reads_2bit, uint64_t n_reads, const uint32_t* lens,
                   uint32_t* out_bwt, uint64_t* out_dollar_pos, uint64_t* out_counts, uint64_t* out_sa,
                   void* stream) {
  if (ctx && !out_sa) return fail(ctx, CXBWT_EINVAL, "out_sa must not be NULL");
  return build_impl(ctx, reads_2bit, n_reads, lens, out_bwt, out_dollar_pos, out_counts, out_sa, stream);
}

int cxbwt_sync(cxbwt_ctx* c) {
  if (!c) return CXBWT_EINVAL;
  c->err.clear();
  CX_CUDA(c, cudaSetDevice(c->device));
  CX_CUDA(c, cudaStreamSynchronize(c->last_stream));
  CX_CUDA(c, cudaMemcpy(c->h_small + 4, static_cast<char*>(c->misc.p) + kMiscErr, 4, cudaMemcpyDeviceToHost));
  return take_device_error(c);
}

int cxbwt_get_stats(const cxbwt_ctx* c, cxbwt_stats* out) {
  if (!c || !out) return CXBWT_EINVAL;
  *out = c->stats;
  out->device_bytes_held = c->held;
  return CXBWT_OK;
}

int cxbwt_reset_stats(cxbwt_ctx* c) {
  if (!c) return CXBWT_EINVAL;
  c->stats = cxbwt_stats{};
  return CXBWT_OK;
}

int cxbwt_pack_codes(const uint8_t* codes, uint64_t n_bases, uint32_t* out) {
  if ((!codes || !out) && n_bases) return CXBWT_EINVAL;
  const uint64_t words = (n_bases + 15) / 16;
  for (uint64_t w = 0; w < words; ++w) {
    uint32_t x = 0;
    const uint64_t b0 = w * 16;
    const uint64_t m = std::min<uint64_t>(16, n_bases - b0);
    for (uint64_t j = 0; j < m; ++j) {
      const uint8_t cd = codes[b0 + j];
      if (cd > 3) return CXBWT_EINVAL;
      x |= uint32_t(cd) << (30 - 2 * j);
    }
    out[w] = x;
  }
  return CXBWT_OK;
}

int cxbwt_pack_ascii(const char* acgt, uint64_t n_bases, uint32_t* out) {
  if ((!acgt || !out) && n_bases) return CXBWT_EINVAL;
  const uint64_t words = (n_bases + 15) / 16;
  for (uint64_t w = 0; w < words; ++w) {
    uint32_t x = 0;
    const uint64_t b0 = w * 16;
    const uint64_t m = std::min<uint64_t>(16, n_bases - b0);
    for (uint64_t j = 0; j < m; ++j) {
      uint32_t cd;
      switch (acgt[b0 + j]) {
        case 'A': cd = 0; break;
        case 'C': cd = 1; break;
        case 'G': cd = 2; break;
        case 'T': cd = 3; break;
        default: return CXBWT_EINVAL;
      }
      x |= cd << (30 - 2 * j);
    }
    out[w] = x;
  }
  return CXBWT_OK;
}

int cxbwt_unpack_ascii(const uint32_t* words, const uint64_t* dollar_pos, uint64_t n_symbols, uint64_t n_dollars,
                       char* out) {
  if ((!words || !out) && n_symbols) return CXBWT_EINVAL;
  if (n_dollars && !dollar_pos) return CXBWT_EINVAL;
  static const char kBase[4] = {'A', 'C', 'G', 'T'};
  for (uint64_t r = 0; r < n_symbols; ++r) out[r] = kBase[(words[r >> 4] >> (30 - 2 * (r & 15))) & 3u];
  for (uint64_t i = 0; i < n_dollars; ++i) {
    if (dollar_pos[i] >= n_symbols) return CXBWT_EINVAL;
    out[dollar_pos[i]] = '$';
  }
  return CXBWT_OK;
}

}  // extern "C"
