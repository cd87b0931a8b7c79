// cxbwt_build_noalloc: a BWT build that allocates no memory.
//
// Some callers cannot allocate device memory while they run: an application
// whose own pool allocator owns all device memory and forbids allocations
// behind its back (a framework's caching allocator, a fixed memory plan on a
// shared GPU), or a latency-bound loop where cudaFree's implicit device-wide
// synchronisation would stall its other streams.  For them this entry point
// does a whole build (same kernels, same result as cxbwt_build) with every
// intermediate buffer carved out of one file-scope static device array.  It
// calls no cudaMalloc, cudaFree, cudaMallocHost or other allocating routine;
// the caller passes device inputs and outputs.
//
// The first call on a device does the set-up for that device (it looks up
// the array's device address and clears it), so that first call should come
// before any stream capture.
//
// The static array is part of the module: every GPU that loads the library
// holds it (kNoallocScratchBytes, about 34 MB) until the process exits.
// Every call on a device shares it, and it keeps the previous call's
// contents, so everything that must start at zero is cleared by each call.
// Calls whose device work overlaps (two host threads, or two streams without
// synchronisation between the calls) race on the array and corrupt each
// other's results: callers must serialise them.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>

#include "../../include/cxbwt.h"
#include "group.cuh"
#include "kernels.cuh"

using namespace cxbwt;

namespace {

constexpr uint64_t kMaxRows = CXBWT_NOALLOC_MAX_SUFFIXES;
constexpr uint32_t kMaxLen = CXBWT_NOALLOC_MAX_READ_LEN;
constexpr uint32_t kTile = 4096;                       // onesweep_shape(0, 4).tile(), checked at each call
constexpr uint64_t kMaxTiles = (kMaxRows + kTile - 1) / kTile;
constexpr uint32_t kMaxD = (kMaxLen + 3) / 4;
constexpr uint32_t kMaxW = (kMaxLen + 15) / 16;

constexpr uint64_t align256(uint64_t x) { return (x + 255) & ~uint64_t(255); }

// Byte offsets of the pieces of the scratch array.
constexpr uint64_t kOffVals0 = 0;
constexpr uint64_t kOffVals1 = align256(kOffVals0 + kMaxRows * 4);
constexpr uint64_t kOffKeys0 = align256(kOffVals1 + kMaxRows * 4);
constexpr uint64_t kOffKeys1 = align256(kOffKeys0 + kMaxRows * 4);
constexpr uint64_t kOffStatus = align256(kOffKeys1 + kMaxRows * 4);
constexpr uint64_t kOffP = align256(kOffStatus + kMaxTiles * kRadix * 8);
constexpr uint64_t kOffBase = align256(kOffP + uint64_t(kMaxLen) * kRadix * 4);
// Reads of at most kMaxLen bases finish their groups with keys of at most
// 16 words (segsort_words), which sets the CTA size of the group finish.
static_assert((kMaxLen - 16 + 15) / 16 <= 16, "the group lists below assume keys of at most 16 words");
constexpr uint64_t kCtaCap = cta_list_cap(kMaxRows), kBigCap = big_list_cap(kMaxRows, 16);
// Look-back epochs one call may use: the four window-0 passes, then at most
// 4 per window for every big group.
constexpr uint32_t kEpochsPerCall = uint32_t(4 + 4 * kMaxW * kBigCap);
constexpr uint64_t kOffSeg = align256(kOffBase + uint64_t(kMaxD + 5) * kRadix * 4);
constexpr uint64_t kOffRhist = align256(kOffSeg + (kCtaCap + kBigCap) * 8);
constexpr uint64_t kOffMisc = align256(kOffRhist + uint64_t(kMaxW) * 4 * kRadix * 4);
// misc: [0] tile counter, [4] error word, [64] 5 x u64 counts, [128] 5 x u32 group-finish counters
constexpr uint64_t kNoallocScratchBytes = align256(kOffMisc + 256);

__device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch[kMaxDevices] = {};     // device address of g_noalloc_scratch, per device
uint32_t g_epoch[kMaxDevices] = {};    // look-back epoch, per device

#define NA_CUDA(call)                   \
  do {                                  \
    if ((call) != cudaSuccess) {        \
      cudaGetLastError();               \
      return CXBWT_ECUDA;               \
    }                                   \
  } while (0)

uint32_t bits_for(uint32_t x) {
  uint32_t s = 0;
  while (s < 32 && (uint64_t(1) << s) <= x) ++s;
  return s;
}

}  // namespace

extern "C" int cxbwt_build_noalloc(const uint32_t* reads_2bit, uint64_t n_reads, const uint32_t* lens_host,
                                   uint32_t* out_bwt, uint64_t* out_dollar_pos, uint64_t* out_counts,
                                   void* stream_v) {
  if (!reads_2bit || !lens_host || !out_bwt || !out_dollar_pos || !out_counts) return CXBWT_EINVAL;
  if (n_reads == 0) return CXBWT_EINVAL;
  uint64_t sum = 0;
  const uint32_t L = lens_host[0];
  for (uint64_t i = 0; i < n_reads; ++i) {
    if (lens_host[i] == 0 || lens_host[i] > 65535) return CXBWT_EINVAL;
    if (lens_host[i] != L) return CXBWT_EUNSUPPORTED;  // reads of one length only
    sum += lens_host[i];
  }
  const uint64_t N = sum + n_reads;
  // Sizes beyond what the static array holds are rejected before any device work.
  if (N > kMaxRows || L > kMaxLen) return CXBWT_EUNSUPPORTED;
  const int seg_words = segsort_words(L, 16);
  if (!seg_words) return CXBWT_EUNSUPPORTED;

  int dev = 0;
  NA_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return CXBWT_EUNSUPPORTED;
  cudaStream_t st = static_cast<cudaStream_t>(stream_v);
  char* base;
  uint32_t epoch;
  {
    // Once per device, with that device current: the device address of the
    // static array (its host-side name is only a stand-in, not an address a
    // kernel may use).
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch[dev]) {
      void* p = nullptr;
      NA_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
      NA_CUDA(cudaMemsetAsync(static_cast<char*>(p) + kOffStatus, 0, kMaxTiles * kRadix * 8, st));
      g_scratch[dev] = p;
    }
    base = static_cast<char*>(g_scratch[dev]);
    // Look-back flags are 2*epoch and 2*epoch+1 in 32 bits.  The call takes
    // its whole range of epochs now, whatever happens later: a call that
    // fails half-way leaves flags of its own epochs in the status words, and
    // no later call uses those epochs again.
    if (g_epoch[dev] >= (1u << 29) - kEpochsPerCall) {
      NA_CUDA(cudaMemsetAsync(base + kOffStatus, 0, kMaxTiles * kRadix * 8, st));
      g_epoch[dev] = 0;
    }
    epoch = g_epoch[dev];
    g_epoch[dev] += kEpochsPerCall;
  }
  char* misc = base + kOffMisc;
  auto* d_counter = reinterpret_cast<uint32_t*>(misc);
  auto* d_err = reinterpret_cast<uint32_t*>(misc + 4);
  auto* d_counts = reinterpret_cast<unsigned long long*>(misc + 64);
  auto* d_seg = reinterpret_cast<uint32_t*>(misc + 128);
  // The previous call's contents stay in the array: clear what must start at zero.
  NA_CUDA(cudaMemsetAsync(misc, 0, 256, st));
  NA_CUDA(cudaMemsetAsync(base + kOffP, 0, uint64_t(L) * kRadix * 4, st));

  const uint32_t shift = bits_for(L);
  const uint64_t n_words = (sum + 15) / 16;
  ReadIndex R{reads_2bit, n_words, nullptr, shift, L, uint32_t(n_reads),
              (reinterpret_cast<uintptr_t>(reads_2bit) & 15u) == 0 ? 1u : 0u};
  const uint32_t D = (L + 3) / 4, W = (L + 15) / 16;
  const uint32_t d_sorted = std::min<uint32_t>(D, 4);
  uint32_t* d_base = reinterpret_cast<uint32_t*>(base + kOffBase);
  int sm_count = 0;
  NA_CUDA(cudaDeviceGetAttribute(&sm_count, cudaDevAttrMultiProcessorCount, dev));
  NA_CUDA(launch_poscount(R, uint32_t(n_reads), L, reinterpret_cast<uint32_t*>(base + kOffP), sm_count, st));
  NA_CUDA(launch_digitbase(reinterpret_cast<const uint32_t*>(base + kOffP), L, d_sorted, 1, uint32_t(n_reads), L,
                           nullptr, d_base, st));

  void* vals[2] = {base + kOffVals0, base + kOffVals1};
  uint32_t* keys[2] = {reinterpret_cast<uint32_t*>(base + kOffKeys0), reinterpret_cast<uint32_t*>(base + kOffKeys1)};
  const TileShape shape = onesweep_shape(0, 4);
  if (uint32_t(shape.tile()) != kTile) return CXBWT_EINTERNAL;  // the array was sized for kTile-item tiles
  PassArgs a{};
  a.status = reinterpret_cast<unsigned long long*>(base + kOffStatus);
  a.tile_counter = d_counter;
  a.err = d_err;
  a.R = R;
  a.n_reads = uint32_t(n_reads);
  a.timeout_ns = 1000000000ull;
  a.n_gen = N;
  a.n_out = uint32_t(N);
  a.n_tiles = uint32_t((N + kTile - 1) / kTile);
  // Window 0 (bases 0..15): digit passes, least significant first; the first
  // generates the (length, read) start order.
  int cur = 0, kin = 0;
  const uint32_t d_hi = std::min<uint32_t>(3, D - 1);
  for (int64_t d = d_hi; d >= 0; --d) {
    const bool first = uint32_t(d) == d_hi;
    const int mode = first ? kSrcInitUniform : kSrcCarried;
    a.vals_in = first ? nullptr : vals[cur];
    a.vals_out = vals[cur ^ 1];
    a.keys_in = first ? nullptr : keys[kin];
    const int kout = first ? kin : (kin ^ 1);
    a.keys_out = keys[kout];
    a.digit_base = d_base + size_t(d) * kRadix;
    a.key_shift = 24u - 8u * uint32_t(d);
    a.window_c0 = 0;
    a.epoch = ++epoch;
    NA_CUDA(launch_onesweep(a, mode, true, false, 4, shape, st));
    cur ^= 1;
    kin = kout;
  }
  if (L > 16) {
    SegArgs g{};
    g.keys = keys[kin];
    g.vals = vals[cur];
    g.n_items = uint32_t(N);
    g.R = R;
    g.depth = 16;
    g.key_mask = depth_mask(16);
    g.cta_list = reinterpret_cast<uint2*>(base + kOffSeg);
    g.cta_cap = uint32_t(kCtaCap);
    g.big_list = g.cta_list + kCtaCap;
    g.big_cap = uint32_t(kBigCap);
    g.counts = d_seg;
    g.err = d_err;
    NA_CUDA(launch_segsort(g, seg_words, 4, sm_count, false, st));
    uint32_t seg_counts[2] = {0, 0};
    NA_CUDA(cudaMemcpyAsync(seg_counts, d_seg, 8, cudaMemcpyDeviceToHost, st));
    NA_CUDA(cudaStreamSynchronize(st));
    const uint32_t n_big = std::min<uint32_t>(seg_counts[1], g.big_cap);
    uint32_t* rh = reinterpret_cast<uint32_t*>(base + kOffRhist);
    for (uint32_t b = 0; b < n_big; ++b) {
      uint2 bg;
      NA_CUDA(cudaMemcpyAsync(&bg, g.big_list + b, 8, cudaMemcpyDeviceToHost, st));
      NA_CUDA(cudaStreamSynchronize(st));
      const uint32_t s0 = bg.x, m = bg.y, n_win = W - 1;
      NA_CUDA(cudaMemsetAsync(rh, 0, size_t(n_win) * 4 * kRadix * 4, st));
      NA_CUDA(launch_range_hist(static_cast<uint32_t*>(vals[cur]) + s0, 4, m, R, 16, n_win, rh, sm_count, st));
      void* gv[2] = {static_cast<uint32_t*>(vals[cur]) + s0, static_cast<uint32_t*>(vals[cur ^ 1]) + s0};
      uint32_t* gk[2] = {keys[0] + s0, keys[1] + s0};
      int gc = 0, gki = 0;
      PassArgs b2 = a;
      b2.n_gen = m;
      b2.n_out = m;
      b2.n_tiles = (m + kTile - 1) / kTile;
      for (uint32_t w = W - 1; w >= 1; --w) {
        const uint32_t lo = 4 * w, hi = std::min<uint32_t>(lo + 3, D - 1);
        for (int64_t d = hi; d >= int64_t(lo); --d) {
          const bool first_in = uint32_t(d) == hi, last_in = uint32_t(d) == lo;
          const int mode = first_in ? kSrcExtract : kSrcCarried;
          b2.vals_in = gv[gc];
          b2.vals_out = gv[gc ^ 1];
          b2.keys_in = mode == kSrcCarried ? gk[gki] : nullptr;
          const int kout = mode == kSrcCarried ? (gki ^ 1) : gki;
          b2.keys_out = last_in ? nullptr : gk[kout];
          b2.digit_base = rh + size_t((w - 1) * 4 + (uint32_t(d) - lo)) * kRadix;
          b2.key_shift = 24u - 8u * (uint32_t(d) - lo);
          b2.window_c0 = 16 * w;
          b2.epoch = ++epoch;
          NA_CUDA(launch_onesweep(b2, mode, !last_in, false, 4, shape, st));
          gc ^= 1;
          if (!last_in) gki = kout;
        }
      }
      if (gc) NA_CUDA(cudaMemcpyAsync(gv[0], gv[1], size_t(m) * 4, cudaMemcpyDeviceToDevice, st));
    }
  }
  EmitArgs e{};
  e.sa = vals[cur];
  e.n = uint32_t(N);
  e.row0 = 0;
  e.n_total = N;
  e.R = R;
  e.bwt = out_bwt;
  e.word_base = 0;
  e.dollar_pos = out_dollar_pos;
  e.counts = d_counts;
  e.sa_out = nullptr;
  e.err = d_err;
  e.id_bytes = 4;
  e.read_base = 0;
  e.n_reads_out = uint32_t(n_reads);
  NA_CUDA(launch_emit(e, st));
  NA_CUDA(cudaMemcpyAsync(out_counts, d_counts, 40, cudaMemcpyDefault, st));
  uint32_t derr = 0;
  NA_CUDA(cudaMemcpyAsync(&derr, d_err, 4, cudaMemcpyDeviceToHost, st));
  NA_CUDA(cudaStreamSynchronize(st));
  if (derr & kErrTimeout) return CXBWT_ETIMEOUT;
  if (derr) return CXBWT_EINTERNAL;
  return CXBWT_OK;
}
