// The listing pass of a build in slices (Figure 2 step 3(a)): every suffix
// of a collection of reads of one length L is enumerated from the read
// store, its first window (bases 0..15, A-padded) gathered, and the suffixes
// whose window falls in one of S key ranges (the slices) are written to that
// slice's arrays, ordered by suffix length and then read - the start order
// of the slice's LSD passes (Section 3.2: suffixes listed in read order and
// sorted stably).
//
// The general digit pass (onesweep.cuh) can do this with digit = (slice,
// suffix length), but it ranks every item with eight warp ballots.  Here a
// tile is a run of whole reads and thread k of the CTA handles offset k of
// the tile's reads (of one half of them, for reads of at most 127 bases: the
// CTA's two halves of 128 threads take the two halves of the reads), so the
// digits (s, L - k) belong to one thread per half: a thread counts its own
// digits in registers, in read order; the tile's count of a digit is the two
// halves' sum, and the second half's rows follow the first half's.  Per tile:
//   0. stage the tile's store words in shared memory (every load in flight
//      at once; the tile one resident grid ahead is asked into L2);
//   1. count: thread k takes the window of suffix (i, k) for each of its
//      reads i and counts it in its slice (none when no slice keeps it);
//   2. publish the counts (decoupled look-back words, one per digit), scan
//      them into tile-local first rows, and walk back over the predecessors'
//      counts (every digit's wait bounded by a wall-clock limit, as in
//      onesweep.cuh);
//   3. take the windows again, and write each kept (window, id) into shared memory at
//      its tile-local row (thread k's items of one digit are consecutive);
//   4. write the staged rows out: consecutive rows of one digit go to
//      consecutive addresses of their slice's arrays.
// The ids are (read << shift) | (k << sym_bits) | preceding base, as the
// digit passes produce them.  Bounds: every output row is checked against
// its slice's size (kErrBounds, nothing written out of range).
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>

#include "kernels.cuh"

namespace cxbwt {
namespace {

constexpr int kSlots = kRadix;  // digit slots of the look-back words: S * (L + 1) <= 256

// First word of the staged ids: after the keys, rounded up to 16 bytes (the
// row count is odd for some read lengths; 8-byte ids need 8-byte alignment).
__host__ __device__ constexpr uint32_t stage_ids_at(uint32_t rows) { return (rows + 3u) & ~3u; }

// Store words a tile stages: its reads' bases plus the word after them.
constexpr uint32_t kListWords = kListMaxStage / 16 + 8;

__device__ __forceinline__ void prefetch_l2(const void* p, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// The first window of suffix (read at store offset off, position k) of a
// read of L bases, A-padded, from the tile's store words sw (store word w_lo
// at sw[0]); *prev = the base before it (0 when k = 0).  The same arithmetic
// as window16_pair_prev, on shared memory.
__device__ __forceinline__ uint32_t window_staged(const uint32_t* sw, uint64_t w_lo, uint64_t off, uint32_t k,
                                                  uint32_t L, uint32_t* prev) {
  const bool inside = k < L;
  const uint32_t rem = inside ? L - k : 0u;
  const uint64_t q = off + (inside ? k : 0u);
  const uint32_t w = uint32_t((q >> 4) - w_lo);
  const uint32_t sh = uint32_t(q & 15u) * 2u;
  const uint32_t w0 = sw[w];
  const uint32_t key = __funnelshift_l(sw[w + 1], w0, sh);
  const uint32_t keep = rem >= 16u ? 0xFFFFFFFFu : ~(0xFFFFFFFFu >> (2u * rem));
  if (prev) {
    uint32_t p = 0;
    if (k != 0) {
      const uint64_t qp = off + k - 1;
      const uint32_t wp = uint32_t((qp >> 4) - w_lo);
      p = ((wp == w ? w0 : sw[wp]) >> (30u - 2u * uint32_t(qp & 15u))) & 3u;
    }
    *prev = p;
  }
  return key & keep;
}

__device__ __forceinline__ uint32_t slice_of(const ListArgs& a, uint32_t key) {
  uint32_t s = kMaxSplit;
#pragma unroll
  for (int j = kMaxSplit - 1; j >= 0; --j)
    if (uint32_t(j) < a.n_slices && key - a.key_lo[j] <= a.key_last[j]) s = uint32_t(j);
  return s;
}

template <class V, int THREADS>
__global__ void __launch_bounds__(THREADS) k_list(const ListArgs a) {
  constexpr int WARPS = THREADS / 32;
  constexpr int PER = kSlots / THREADS;  // slots per thread in the scan and the look-back
  static_assert(kSlots % THREADS == 0, "threads divide the slots");
  extern __shared__ __align__(16) uint32_t s_stage[];  // keys [stage_rows], then ids from a 16-byte boundary
  __shared__ uint32_t s_cnt[kSlots];    // tile count of each digit, then its first tile-local row
  __shared__ uint32_t s_gbase[kSlots];  // output row of tile-local row 0 of each digit
  __shared__ uint32_t s_scan[WARPS];
  __shared__ uint32_t s_tile;
  __shared__ uint32_t s_words[kListWords];  // the tile's store words
  __shared__ uint32_t s_half0[kSlots];      // count of each digit in the first half of the tile's reads

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint32_t L = a.R.uniform_len, L1 = L + 1u, S = a.n_slices;
  for (int x = tid; x < kSlots; x += THREADS) s_cnt[x] = 0u;
  if (tid == 0) {
    const uint32_t t = atomicAdd(a.tile_counter, 1u);
    if (t == a.n_tiles - 1) atomicExch(a.tile_counter, 0u);  // every id handed out: reset for the next pass
    s_tile = t;
  }
  __syncthreads();
  const uint32_t tile = s_tile;
  const uint32_t i0 = tile * a.reads_per_tile;
  const uint32_t i1 = min(i0 + a.reads_per_tile, a.n_reads);
  // Reads of at most 127 bases: threads [128h, 128h + 128) take half h of
  // the tile's reads, so two threads own each suffix length; longer reads:
  // one thread per suffix length, every read of the tile.
  const bool halves = L1 <= 128u;
  const uint32_t half = halves ? uint32_t(tid) >> 7 : 0u;
  const uint32_t k = halves ? uint32_t(tid) & 127u : uint32_t(tid);
  const bool act = k <= L;
  const uint32_t i_mid = halves ? i0 + (i1 - i0 + 1u) / 2u : i1;
  const uint32_t ra = half ? i_mid : i0, rb = half ? i1 : i_mid;  // this thread's reads
  if (tid == 0 && a.prefetch) {
    // The store words of the tile one resident grid ahead, into L2 (whole
    // 16-byte units inside the store).
    const uint64_t ahead = uint64_t(tile) + a.prefetch;
    if (ahead < a.n_tiles) {
      const uint64_t r0 = ahead * a.reads_per_tile;
      const uint64_t r1 = min(r0 + a.reads_per_tile, uint64_t(a.n_reads));
      const uint64_t lo = ((r0 * L) >> 4) & ~uint64_t(3);
      const uint64_t hi = min((((r1 * L) >> 4) + 4) & ~uint64_t(3), a.R.n_words & ~uint64_t(3));
      if (hi > lo) prefetch_l2(a.R.words + lo, uint32_t(hi - lo) * 4u);
    }
  }
  // Stage the tile's store words: bases [i0 * L, i1 * L) and the word after
  // them (a window reads its word and the next), all loads in flight at once.
  const uint64_t w_lo = (uint64_t(i0) * L) >> 4;
  const uint32_t n_w = uint32_t(((uint64_t(i1) * L + 15u) >> 4) + 1u - w_lo);
  for (uint32_t x = uint32_t(tid); x < n_w && x < kListWords; x += THREADS) s_words[x] = load_word(a.R, w_lo + x);
  if (n_w > kListWords && tid == 0) atomicOr(a.err, kErrBounds);  // not reached: the host sizes tiles to fit
  __syncthreads();

  // ---- 1. count ------------------------------------------------------------------
  uint32_t cnt[kMaxSplit];
#pragma unroll
  for (int s = 0; s < kMaxSplit; ++s) cnt[s] = 0u;
  if (act) {
    for (uint32_t i = ra; i < rb; ++i) {
      const uint32_t s = slice_of(a, window_staged(s_words, w_lo, uint64_t(i) * L, k, L, nullptr));
#pragma unroll
      for (int j = 0; j < kMaxSplit; ++j) cnt[j] += (s == uint32_t(j)) ? 1u : 0u;
    }
    // The tile's count of each digit: the two halves' counts added; the
    // first half's alone is where the second half's rows start.
#pragma unroll
    for (int j = 0; j < kMaxSplit; ++j) {
      if (uint32_t(j) < S) {
        const uint32_t d = uint32_t(j) * L1 + (L - k);
        atomicAdd(&s_cnt[d], cnt[j]);
        if (half == 0) s_half0[d] = cnt[j];
      }
    }
  }
  __syncthreads();
  // ---- 2. publish; exclusive scan of the slots (thread t holds slots
  // [t * PER, t * PER + PER)) -----------------------------------------------------
  uint32_t mine[PER], tot = 0;
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    const uint32_t d = uint32_t(tid * PER + q);
    mine[q] = s_cnt[d];
    tot += mine[q];
    if (d < S * L1) {
      const unsigned long long flag = (unsigned long long)(tile == 0 ? 2u * a.epoch + 1u : 2u * a.epoch) << 32;
      store_relaxed_u64(a.status + uint64_t(tile) * kSlots + d, flag | mine[q]);
    }
  }
  uint32_t incl = tot;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) s_scan[warp] = incl;
  __syncthreads();
  uint32_t run = incl - tot;
#pragma unroll
  for (int w = 0; w < WARPS; ++w)
    if (w < warp) run += s_scan[w];
  uint32_t excl[PER];
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    excl[q] = run;
    s_cnt[tid * PER + q] = run;
    run += mine[q];
  }
  // Look-back: thread t walks back for its slots (only the S * (L + 1) in use).
  const uint32_t used = S * L1;
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    const uint32_t d = uint32_t(tid * PER + q);
    if (d >= used) continue;
    uint32_t before = 0;
    if (tile > 0) {
      const uint32_t agg = 2u * a.epoch, pre = 2u * a.epoch + 1u;
      uint32_t p = tile - 1;
      uint64_t t0 = 0;
      uint32_t spins = 0;
      unsigned long long st = load_relaxed_u64(a.status + uint64_t(p) * kSlots + d);
      while (true) {
        const uint32_t flag = uint32_t(st >> 32);
        if (flag != agg && flag != pre) {
          ++spins;
          if (spins > 4) __nanosleep(64);
          if ((spins & 63u) == 0u) {
            const uint64_t now = global_timer_ns();
            if (t0 == 0) {
              t0 = now;
            } else if (now - t0 > a.timeout_ns) {
              atomicOr(a.err, kErrTimeout);
              break;
            }
          }
          st = load_relaxed_u64(a.status + uint64_t(p) * kSlots + d);
          continue;
        }
        before += uint32_t(st);
        if (flag == pre || p == 0) break;
        --p;
        st = load_relaxed_u64(a.status + uint64_t(p) * kSlots + d);
      }
      store_relaxed_u64(a.status + uint64_t(tile) * kSlots + d,
                        ((unsigned long long)(2u * a.epoch + 1u) << 32) | (before + mine[q]));
    }
    s_gbase[d] = __ldg(a.digit_base + d) + before - excl[q];
  }
  __syncthreads();
  uint32_t rows_kept = 0;  // rows of this tile that are written: the scan's total
#pragma unroll
  for (int w = 0; w < WARPS; ++w) rows_kept += s_scan[w];

  // ---- 3. stage -----------------------------------------------------------------
  uint32_t* s_keys = s_stage;
  V* s_vals = reinterpret_cast<V*>(s_stage + stage_ids_at(a.stage_rows));
  if (act) {
    uint32_t next[kMaxSplit];
#pragma unroll
    for (int j = 0; j < kMaxSplit; ++j) {
      const uint32_t d = uint32_t(j) * L1 + (L - k);
      next[j] = uint32_t(j) < S ? s_cnt[d] + (half ? s_half0[d] : 0u) : 0u;
    }
    const V kbits = V(k) << a.R.sym_bits;
    auto place = [&](uint32_t i, uint32_t key, uint32_t prev) {
      const uint32_t s = slice_of(a, key);
      if (s < S) {
        uint32_t r = 0;
#pragma unroll
        for (int j = 0; j < kMaxSplit; ++j)
          if (s == uint32_t(j)) r = next[j]++;
        s_keys[r] = key;
        s_vals[r] = (V(i) << a.R.shift) | kbits | (a.R.sym_bits ? V(prev) : V(0));
      }
    };
    for (uint32_t i = ra; i < rb; ++i) {
      uint32_t prev;
      const uint32_t key = window_staged(s_words, w_lo, uint64_t(i) * L, k, L, &prev);
      place(i, key, prev);
    }
  }
  __syncthreads();

  // ---- 4. write out -------------------------------------------------------------
  bool bad = false;
  const uint32_t kmask = (1u << a.R.shift) - 1u;
  for (uint32_t r = uint32_t(tid); r < rows_kept; r += THREADS) {
    const uint32_t key = s_keys[r];
    const V v = s_vals[r];
    const uint32_t s = slice_of(a, key);
    const uint32_t kk = (uint32_t(v) & kmask) >> a.R.sym_bits;
    const uint32_t d = s * L1 + (L - kk);
    const bool ok = s < S && kk <= L;
    const uint32_t g = ok ? s_gbase[d] + r : 0u;
    const bool in = ok && g < a.rows[s < kMaxSplit ? s : 0];
    if (in) {
      static_cast<V*>(a.vals[s])[g] = v;
      a.keys[s][g] = key;
    }
    bad = bad || !in;
  }
  if (bad) atomicOr(a.err, kErrBounds);
}

template <class V, int THREADS>
cudaError_t launch_t(const ListArgs& a, cudaStream_t st) {
  const size_t smem = size_t(stage_ids_at(a.stage_rows)) * 4 + size_t(a.stage_rows) * sizeof(V);
  auto kern = k_list<V, THREADS>;
  static std::atomic<unsigned long long> configured{0};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const unsigned long long bit = 1ull << (dev & 63);
  if (!(configured.load(std::memory_order_acquire) & bit)) {
    // Attributes sized for the largest staging a launch may ask for.
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(kListMaxStage * (4 + sizeof(V))));
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if (e != cudaSuccess) return e;
    configured.fetch_or(bit, std::memory_order_release);
  }
  // Tiles ahead to prefetch: the CTAs resident on the GPU (once per device).
  static std::atomic<uint32_t> resident[64];
  uint32_t grid_resident = resident[dev & 63].load(std::memory_order_acquire);
  if (grid_resident == 0) {
    int per_sm = 0, sms = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, THREADS, kListMaxStage * (4 + sizeof(V)));
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    grid_resident = uint32_t(std::max(per_sm, 1) * std::max(sms, 1));
    resident[dev & 63].store(grid_resident, std::memory_order_release);
  }
  ListArgs b = a;
  b.prefetch = (a.prefetch && a.R.words_aligned) ? grid_resident : 0u;
  kern<<<a.n_tiles, THREADS, smem, st>>>(b);
  return cudaGetLastError();
}

}  // namespace

uint32_t list_reads_per_tile(uint32_t read_len) { return std::max<uint32_t>(1u, kListMaxStage / (read_len + 1)); }

cudaError_t launch_list(const ListArgs& a, int id_bytes, cudaStream_t st) {
  if (a.n_tiles == 0) return cudaSuccess;
  const uint32_t L1 = a.R.uniform_len + 1;
  if (a.n_slices == 0 || a.n_slices > kMaxSplit || a.n_slices * L1 > uint32_t(kSlots) ||
      a.stage_rows > kListMaxStage || a.stage_rows < a.reads_per_tile * L1 ||
      (uint64_t(a.reads_per_tile) * a.R.uniform_len + 15) / 16 + 2 > kListWords)
    return cudaErrorInvalidValue;
  return id_bytes == 8 ? launch_t<uint64_t, 256>(a, st) : launch_t<uint32_t, 256>(a, st);
}

}  // namespace cxbwt
