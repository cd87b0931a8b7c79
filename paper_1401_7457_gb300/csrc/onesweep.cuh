// One stable LSD digit pass over (key, value) items: the "onesweep" scheme
// (Adinets & Merrill 2022) written for sm_103a.
//
// This is the radix sort at the core of Section 3.2 of the paper ("sort by
// index": the values are 32-bit suffix ids; the keys are 16-base stringwords,
// 8 bits = 4 bases per pass, least significant first).  The paper called a
// library sort and permuted each new stringword by index on the host side of
// PCIe; here the stringword is gathered from the device-resident read store
// inside the first pass of each 16-base window (kSrcExtract), and carried in
// the key array for the other passes of that window.
//
// One CTA sorts one tile of threads*IPT items:
//   1. take a tile id from an atomic counter (so every lower tile is already
//      running: the look-back below always makes progress),
//   2. load the tile (warp-striped, coalesced) and compute each item's digit,
//   3. count the tile's digits (shared-memory atomics) and publish the
//      counts at once, so that successors rarely wait for them; then rank
//      items inside the tile: warp-level ballots (one per digit bit) group
//      equal digits; a per-warp shared-memory histogram accumulates counts in
//      item order, so the ranking is stable,
//   4. stage the tile in shared memory in sorted order, and walk back over
//      the predecessors' published counts
//      (decoupled look-back) to find, for each digit, how many items of
//      earlier tiles precede this tile (the first look-back load is issued
//      before the staging, so the two overlap); the first row of each digit
//      comes from the all-tile histogram computed before the pass
//      (digit_base),
//   5. write the staged tile out, so that runs of equal digits go to
//      consecutive addresses.
// The only wait is in step 4.  It is bounded by a wall-clock limit; when the
// limit passes the kernel records kErrTimeout and finishes (it never traps).
#pragma once
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <type_traits>

#include "kernels.cuh"

namespace cxbwt {
namespace onesweep {

template <int THREADS>
__device__ __forceinline__ uint32_t block_exclusive_scan_256(uint32_t x, uint32_t* scratch /*[8]*/) {
  // Threads 0..255 hold one value each; returns their exclusive prefix sum.
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  uint32_t incl = x;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
    if (lane >= o) incl += y;
  }
  if (tid < 256 && lane == 31) scratch[warp] = incl;
  __syncthreads();
  uint32_t warp_prefix = 0;
  if (tid < 256) {
#pragma unroll
    for (int w = 0; w < 8; ++w)
      if (w < warp) warp_prefix += scratch[w];
  }
  return warp_prefix + incl - x;
}

// Asks the bulk-copy engine to bring `bytes` (a multiple of 16, 16-byte
// aligned) of this GPU's memory into L2; nothing waits for it.
__device__ __forceinline__ void prefetch_l2(const void* p, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

template <class V, int THREADS, int IPT, int MIN_BLOCKS, int MODE, bool WRITE_KEY, bool FILTER>
__global__ void __launch_bounds__(THREADS, MIN_BLOCKS) k_onesweep(const PassArgs a) {
  constexpr int TILE = THREADS * IPT;
  constexpr int WARPS = THREADS / 32;
  constexpr bool SPLIT = (MODE == kSrcInitSplit);  // digit = (slice, suffix length), per-slice outputs
  constexpr bool MIXED = (MODE == kSrcInitMixed);  // read-major over reads of any lengths
  constexpr bool GEN = (MODE == kSrcInitUniform || MODE == kSrcInitReadMajor || SPLIT || MIXED);
  constexpr bool CARRY_KEY = (MODE == kSrcCarried || MODE == kSrcCarriedLength);
  constexpr bool LEN_DIGIT = (MODE == kSrcInitReadMajor);  // digit = suffix length, key = window 0
  constexpr bool READ_MAJOR = (MODE == kSrcInitReadMajor || SPLIT);
  using I = typename std::conditional<GEN, uint64_t, uint32_t>::type;  // generated inputs may exceed 2^32 rows
  static_assert(THREADS >= 256 && THREADS % 32 == 0, "one thread per digit value is needed");
  static_assert(!FILTER || GEN, "the bucket filter applies to generated inputs");

  extern __shared__ __align__(16) uint32_t s_stage[];  // keys [TILE], then ids [TILE]
  uint32_t* s_keys = s_stage;
  V* s_vals = reinterpret_cast<V*>(s_stage + TILE);
  // Per-warp digit counts; after the look-back, the tile-local row of the
  // warp's first item of each digit.
  __shared__ uint32_t s_whist[WARPS][kRadix];
  __shared__ uint32_t s_thist[kRadix];
  __shared__ uint32_t s_gbase[kRadix];  // global row of tile-local row 0 of each digit
  __shared__ uint32_t s_scan[8];
  __shared__ uint32_t s_tile, s_kept;
  __shared__ uint32_t s_coll[MODE == kSrcCollection ? kMaxPackCollections + 1 : 1];
  __shared__ uint8_t s_split[SPLIT ? kRadix : 1];  // slice of each 4-base bucket

  const V* vals_in = static_cast<const V*>(a.vals_in);
  V* vals_out = static_cast<V*>(a.vals_out);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int i = tid; i < WARPS * kRadix; i += THREADS) (&s_whist[0][0])[i] = 0u;
  for (int i = tid; i < kRadix; i += THREADS) s_thist[i] = 0u;
  if (MODE == kSrcCollection)
    for (uint32_t i = tid; i <= a.n_coll; i += THREADS) s_coll[i] = a.coll_start[i];
  if (SPLIT)
    for (int i = tid; i < kRadix; i += THREADS) s_split[i] = a.split_of[i];
  if (tid == 0) {
    const uint32_t t = atomicAdd(a.tile_counter, 1u);
    // Every id has been handed out once the last one is: reset for the next pass.
    if (t == a.n_tiles - 1) atomicExch(a.tile_counter, 0u);
    s_tile = t;
  }
  __syncthreads();
  const uint32_t tile = s_tile;
  if (CARRY_KEY && a.prefetch && tid == 0) {
    // Tiles are taken in order, about one resident grid at a time: the tile
    // that the CTA starting one grid later takes is read from HBM into L2
    // now, so that its loads wait on L2 instead of HBM (whole tiles only).
    const uint64_t ahead = uint64_t(tile) + a.prefetch;
    if (ahead + 1 < a.n_tiles) {
      prefetch_l2(a.keys_in + ahead * TILE, uint32_t(TILE) * 4u);
      prefetch_l2(vals_in + ahead * TILE, uint32_t(TILE) * uint32_t(sizeof(V)));
    }
  }
  const I tile_base = I(tile) * I(TILE);
  const I warp_base = tile_base + I(warp) * 32u * IPT + lane;
  const I n_in = I(a.n_gen);

  // A tile with a dropped row (the last one, or any when filtering) ranks a
  // 9th digit bit and checks rows against the input's end; every other tile
  // skips both.
  auto tile_body = [&](auto ninth_c) {
    constexpr bool NINTH = decltype(ninth_c)::value;
    uint32_t key[IPT], digit[IPT];
    V val[IPT];

    // ---- 2. load ------------------------------------------------------------
    if (MODE == kSrcInitUniform) {
      // Row idx of the (suffix length, read) order: length idx / n, read
      // idx % n.  One division per thread; its next rows (idx + 32, ...) step
      // the remainder and carry into the quotient.
      const uint32_t L = a.R.uniform_len, n = a.n_reads;
      const I slen0 = warp_base / n;
      uint32_t slen = uint32_t(min(slen0, I(L + 1)));
      uint32_t i = uint32_t(warp_base - slen0 * n);
  #pragma unroll
      for (int j = 0; j < IPT; ++j) {
        val[j] = (V(i) << a.R.shift) | (V(L - min(slen, L)) << a.R.sym_bits);
        i += 32;
        while (i >= n) {  // once per step when n >= 32
          i -= n;
          slen = min(slen + 1, L + 1);
        }
      }
    } else if (MIXED) {
      // Row idx of the read-major order over reads of any lengths: lane 0
      // finds the read holding the warp's first row (a binary search over
      // the read starts off_i + i), every lane steps to its own rows.
      uint32_t i = 0;
      if (lane == 0) {
        uint32_t lo = 0, hi = a.n_reads;
        while (hi - lo > 1) {
          const uint32_t mid = (lo + hi) >> 1;
          if ((__ldg(a.R.desc + mid) >> 16) + mid <= warp_base - lane) lo = mid; else hi = mid;
        }
        i = lo;
      }
      i = __shfl_sync(0xFFFFFFFFu, i, 0);
      uint64_t d = __ldg(a.R.desc + i);
      uint32_t len = uint32_t(d & 0xFFFFu);
      uint64_t k64 = uint64_t(warp_base) - ((d >> 16) + i);
      while (k64 > len && i + 1 < a.n_reads) {
        k64 -= len + 1;
        d = __ldg(a.R.desc + ++i);
        len = uint32_t(d & 0xFFFFu);
      }
      uint32_t k = uint32_t(k64);
  #pragma unroll
      for (int j = 0; j < IPT; ++j) {
        val[j] = (V(i) << a.R.shift) | (V(k) << a.R.sym_bits);
        k += 32;
        while (k > len && i + 1 < a.n_reads) {  // rows past the last read are dropped below
          k -= len + 1;
          d = __ldg(a.R.desc + ++i);
          len = uint32_t(d & 0xFFFFu);
        }
      }
    } else if (READ_MAJOR) {
      // Row idx of the read-major order: read idx / (L+1), offset idx % (L+1),
      // stepped the same way.
      const uint32_t L1 = a.R.uniform_len + 1;
      const I i0 = warp_base / L1;
      uint32_t k = uint32_t(warp_base - i0 * L1);
      V i = V(i0);
  #pragma unroll
      for (int j = 0; j < IPT; ++j) {
        val[j] = (i << a.R.shift) | (V(k) << a.R.sym_bits);
        k += 32;
        while (k >= L1) {
          k -= L1;
          ++i;
        }
      }
    } else {
  #pragma unroll
      for (int j = 0; j < IPT; ++j) {
        const I idx = warp_base + j * 32;
        val[j] = (!NINTH || idx < n_in) ? __ldg(vals_in + idx) : V(0);
      }
    }
    if (CARRY_KEY) {
  #pragma unroll
      for (int j = 0; j < IPT; ++j) {
        const I idx = warp_base + j * 32;
        key[j] = (!NINTH || idx < n_in) ? __ldg(a.keys_in + idx) : 0u;
      }
    } else if (MODE == kSrcLength) {
  #pragma unroll
      for (int j = 0; j < IPT; ++j) {
        const Suffix s = decode(a.R, val[j]);
        key[j] = s.len - s.k;
      }
    } else if (MODE == kSrcCollection) {
  #pragma unroll
      for (int j = 0; j < IPT; ++j) {
        // Collection of the id's read: the last c with s_coll[c] <= read.
        const uint32_t read = uint32_t(val[j] >> a.R.shift);
        uint32_t lo = 0, hi = a.n_coll;
        while (hi - lo > 1) {
          const uint32_t mid = (lo + hi) >> 1;
          if (s_coll[mid] <= read) lo = mid; else hi = mid;
        }
        key[j] = lo;
      }
    } else if (GEN && a.R.sym_bits) {
      // Generated ids take the base before the suffix into their low bits
      // (one branch per tile: the plain gather below keeps its own loop).
  #pragma unroll
      for (int j = 0; j < IPT; ++j) {
        const I idx = warp_base + j * 32;
        key[j] = 0u;
        if (!NINTH || idx < n_in) {
          const Suffix sfx = decode(a.R, val[j]);
          uint32_t prev;
          if (a.window_c0 == 0) {
            key[j] = window16_pair_prev(a.R, sfx, &prev);
          } else {
            key[j] = window16_pair(a.R, sfx, a.window_c0);
            prev = sfx.k ? base_at(a.R, sfx.off + sfx.k - 1) : 0u;
          }
          val[j] |= V(prev);
        }
      }
    } else {
  #pragma unroll
      for (int j = 0; j < IPT; ++j) {
        const I idx = warp_base + j * 32;
        key[j] = (!NINTH || idx < n_in) ? window16_pair(a.R, decode(a.R, val[j]), a.window_c0) : 0u;
      }
    }
  #pragma unroll
    for (int j = 0; j < IPT; ++j) {
      const I idx = warp_base + j * 32;
      bool keep = !NINTH || idx < n_in;
      if (FILTER) keep = keep && (key[j] - a.key_lo) <= a.key_last;
      uint32_t d;
      if (LEN_DIGIT) d = a.R.uniform_len - ((uint32_t(val[j]) & ((1u << a.R.shift) - 1u)) >> a.R.sym_bits);
      else if (MIXED || MODE == kSrcCarriedLength) {
        const Suffix sx = decode(a.R, val[j]);
        d = ((sx.len - sx.k) >> (MIXED ? 0u : a.key_shift)) & (kRadix - 1);
      } else if (SPLIT)
        d = uint32_t(s_split[key[j] >> 24]) * (a.R.uniform_len + 1u) + a.R.uniform_len -
            ((uint32_t(val[j]) & ((1u << a.R.shift) - 1u)) >> a.R.sym_bits);
      else d = (key[j] >> a.key_shift) & (kRadix - 1);
      // Rows past the end (or filtered out) get a value no digit has, so they
      // match only each other and are neither counted nor written.
      digit[j] = keep ? d : uint32_t(kRadix);
    }
    // Tile counts first, published before the ranking: a successor's
    // look-back then finds them already written.
  #pragma unroll
    for (int j = 0; j < IPT; ++j)
      if (!NINTH || digit[j] < kRadix) atomicAdd(&s_thist[digit[j]], 1u);
    __syncthreads();
    uint32_t tile_cnt = 0;
    if (tid < kRadix) {
      tile_cnt = s_thist[tid];
      const unsigned long long agg_flag = (unsigned long long)(2u * a.epoch) << 32;
      const unsigned long long pre_flag = (unsigned long long)(2u * a.epoch + 1u) << 32;
      if (!(tile == 0 && a.stall_tile0))
        store_relaxed_u64(a.status + uint64_t(tile) * kRadix + tid, (tile == 0 ? pre_flag : agg_flag) | tile_cnt);
    }

    // ---- 3. stable rank inside the warp, in item order ------------------------
    // Lanes holding the same digit are found with one ballot per digit bit (a
    // 9th bit separates dropped rows: only in the last tile unless filtering):
    // cheaper on sm_103a than __match_any_sync.  Every lane reads its digit's
    // running count; the lowest lane of each digit adds the group's size.
    // digit[j] becomes (rank of the item among the warp's items of its digit)
    // << 9 | digit.
    const uint32_t lt = lanemask_lt();
  #pragma unroll
    for (int j = 0; j < IPT; ++j) {
      const uint32_t d = digit[j];
      uint32_t peers = 0xFFFFFFFFu;
  #pragma unroll
      for (int b = 0; b < kRadixBits; ++b) {
        const uint32_t bit = (d >> b) & 1u;
        const uint32_t m = __ballot_sync(0xFFFFFFFFu, bit);
        peers &= bit ? m : ~m;
      }
      if (NINTH) {
        const uint32_t bit = d >> kRadixBits;
        const uint32_t m = __ballot_sync(0xFFFFFFFFu, bit);
        peers &= bit ? m : ~m;
      }
      const uint32_t prior = s_whist[warp][d & (kRadix - 1)];  // dropped rows read a count they never use
      if ((peers & lt) == 0 && (!NINTH || d < kRadix)) s_whist[warp][d] = prior + __popc(peers);
      digit[j] = ((prior + __popc(peers & lt)) << 9) | d;
      __syncwarp();
    }
    __syncthreads();

    // ---- 4. stage sorted while the first look-back load is out ---------------
    unsigned long long prev = 0;  // predecessor's status word, fetched before the staging
    if (tid < kRadix) {
      uint32_t sum = 0;
  #pragma unroll
      for (int w = 0; w < WARPS; ++w) {
        const uint32_t c = s_whist[w][tid];
        s_whist[w][tid] = sum;
        sum += c;
      }
    }
    const uint32_t local_excl = block_exclusive_scan_256<THREADS>(tile_cnt, s_scan);
    if (tid == kRadix - 1) s_kept = local_excl + tile_cnt;  // rows of this tile that are written
    if (tid < kRadix) {
  #pragma unroll
      for (int w = 0; w < WARPS; ++w) s_whist[w][tid] += local_excl;
      if (tile > 0) prev = load_relaxed_u64(a.status + uint64_t(tile - 1) * kRadix + tid);
    }
    __syncthreads();
    // The tile-local sorted order needs only the tile's own counts: write it to
    // shared memory now, so the staging overlaps the look-back's first load.
  #pragma unroll
    for (int j = 0; j < IPT; ++j) {
      const uint32_t d = digit[j] & 0x1FFu;
      if (!NINTH || d < kRadix) {
        const uint32_t r = s_whist[warp][d] + (digit[j] >> 9);
        s_keys[r] = key[j];
        s_vals[r] = val[j];
      }
    }
    if (tid < kRadix) {
      uint32_t before = 0;  // items with this digit in tiles 0 .. tile-1
      if (tile > 0) {
        const uint32_t agg = 2u * a.epoch, pre = 2u * a.epoch + 1u;
        uint32_t p = tile - 1;
        uint64_t t0 = 0;
        uint32_t spins = 0;
        unsigned long long st = prev;
        while (true) {
          const uint32_t flag = uint32_t(st >> 32);
          if (flag != agg && flag != pre) {  // not yet published in this pass
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
            st = load_relaxed_u64(a.status + uint64_t(p) * kRadix + tid);
            continue;
          }
          before += uint32_t(st);
          if (flag == pre || p == 0) break;
          --p;
          st = load_relaxed_u64(a.status + uint64_t(p) * kRadix + tid);
        }
        store_relaxed_u64(a.status + uint64_t(tile) * kRadix + tid,
                          ((unsigned long long)(2u * a.epoch + 1u) << 32) | (before + tile_cnt));
        // (after a wait that ran out, `before` is short: the outputs are then
        // unspecified but every write stays in bounds, and the error word says so)
      }
      s_gbase[tid] = __ldg(a.digit_base + tid) + before - local_excl;
    }

    // ---- 5. write out the staged tile ----------------------------------------
    __syncthreads();
    const uint32_t n_valid = NINTH ? s_kept : uint32_t(TILE);  // a full tile keeps every row
    bool bad = false;
  #pragma unroll
    for (int j = 0; j < IPT; ++j) {
      const uint32_t r = j * THREADS + tid;
      if (!NINTH || r < n_valid) {
        const uint32_t k = s_keys[r];
        const V v = s_vals[r];
        const uint32_t kpos = (uint32_t(v) & ((1u << a.R.shift) - 1u)) >> a.R.sym_bits;
        uint32_t d;
        if (LEN_DIGIT) d = a.R.uniform_len - kpos;
        else if (MIXED || MODE == kSrcCarriedLength) {
          const Suffix sx = decode(a.R, v);
          d = ((sx.len - sx.k) >> (MIXED ? 0u : a.key_shift)) & (kRadix - 1);
        }
        else if (SPLIT) d = uint32_t(s_split[k >> 24]) * (a.R.uniform_len + 1u) + a.R.uniform_len - kpos;
        else d = (k >> a.key_shift) & (kRadix - 1);
        const uint32_t g = s_gbase[d] + r;
        if (SPLIT) {
          // Rows of slice sl go to its own arrays, counted from 0 there.
          const uint32_t sl = s_split[k >> 24];
          const bool ok = sl < kMaxSplit && g < a.split_rows[sl < kMaxSplit ? sl : 0];
          if (ok) {
            static_cast<V*>(a.split_vals[sl])[g] = v;
            a.split_keys[sl][g] = k;
          }
          bad = bad || !ok;
        } else {
          const bool ok = g < a.n_out;
          if (ok) vals_out[g] = v;
          if (WRITE_KEY && ok) a.keys_out[g] = k;
          bad = bad || !ok;
        }
      }
    }
    // Digit bases that disagree with the items: nothing was written out of bounds.
    if (bad) atomicOr(a.err, kErrBounds);
  };
  if (FILTER || tile == a.n_tiles - 1) tile_body(std::true_type{});
  else tile_body(std::false_type{});
}

// Tile shapes compiled in (threads, items per thread, CTAs per SM the register
// budget is sized for).
template <int T, int I, int B>
struct Shape {
  static constexpr int threads = T, ipt = I, min_blocks = B;
};
using ShapeMid = Shape<256, 16, 4>;    // 4096 items
using ShapeLarge = Shape<512, 16, 2>;  // 8192 items (32-bit ids)
using Shape64x16 = Shape<256, 16, 3>;  // 4096 items, 64-bit ids: 48 KB staged holds an SM to three CTAs,
                                       // so the registers are sized for three (no spills)
using Shape64x12 = Shape<256, 12, 4>;  // 3072 items (64-bit ids: 36 KB staged, four CTAs per SM)
using Shape64x8 = Shape<256, 8, 5>;    // 2048 items (64-bit ids: 24 KB staged, five CTAs per SM)

template <class V, class S, int MODE, bool WK, bool F>
cudaError_t launch_mode(const PassArgs& a, cudaStream_t st) {
  const size_t smem = size_t(S::threads) * S::ipt * (sizeof(uint32_t) + sizeof(V));
  auto kern = k_onesweep<V, S::threads, S::ipt, S::min_blocks, MODE, WK, F>;
  // Attributes are set once per instantiation and device (a bit per device;
  // threads that race here both set the same values).
  // CTAs resident on the whole GPU, per device (set with the attributes, once;
  // threads that race here store the same values).
  static std::atomic<uint32_t> resident[64];
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  uint32_t grid_resident = resident[dev & 63].load(std::memory_order_acquire);
  if (grid_resident == 0) {
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if (e != cudaSuccess) return e;
    int per_sm = 0, sms = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, S::threads, smem);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    grid_resident = uint32_t(std::max(per_sm, 1) * std::max(sms, 1));
    resident[dev & 63].store(grid_resident, std::memory_order_release);
  }
  PassArgs b = a;
  b.prefetch = 0;
  if (MODE == kSrcCarried && a.prefetch && (reinterpret_cast<uintptr_t>(a.keys_in) & 15u) == 0 &&
      (reinterpret_cast<uintptr_t>(a.vals_in) & 15u) == 0)
    b.prefetch = grid_resident;
  kern<<<a.n_tiles, S::threads, smem, st>>>(b);
  return cudaGetLastError();
}

template <class V, class S>
cudaError_t launch_shape(const PassArgs& a, int mode, bool wk, bool filter, cudaStream_t st) {
  switch (mode) {
    case kSrcInitUniform:
      if (filter) return wk ? launch_mode<V, S, kSrcInitUniform, true, true>(a, st)
                            : launch_mode<V, S, kSrcInitUniform, false, true>(a, st);
      return wk ? launch_mode<V, S, kSrcInitUniform, true, false>(a, st)
                : launch_mode<V, S, kSrcInitUniform, false, false>(a, st);
    case kSrcInitReadMajor:
      if (!wk) return cudaErrorInvalidValue;  // it exists to carry window 0
      return filter ? launch_mode<V, S, kSrcInitReadMajor, true, true>(a, st)
                    : launch_mode<V, S, kSrcInitReadMajor, true, false>(a, st);
    case kSrcExtract:
      if (filter) return cudaErrorInvalidValue;
      return wk ? launch_mode<V, S, kSrcExtract, true, false>(a, st) : launch_mode<V, S, kSrcExtract, false, false>(a, st);
    case kSrcCarried:
      if (filter) return cudaErrorInvalidValue;
      return wk ? launch_mode<V, S, kSrcCarried, true, false>(a, st) : launch_mode<V, S, kSrcCarried, false, false>(a, st);
    case kSrcLength:
      if (filter || wk) return cudaErrorInvalidValue;
      return launch_mode<V, S, kSrcLength, false, false>(a, st);
    case kSrcCollection:
      if (filter || wk) return cudaErrorInvalidValue;
      return launch_mode<V, S, kSrcCollection, false, false>(a, st);
    case kSrcInitSplit:
      if (filter || !wk) return cudaErrorInvalidValue;  // it writes every slice's ids and keys
      return launch_mode<V, S, kSrcInitSplit, true, false>(a, st);
    case kSrcInitMixed:
      if (!wk) return cudaErrorInvalidValue;  // it exists to list window 0
      return filter ? launch_mode<V, S, kSrcInitMixed, true, true>(a, st)
                    : launch_mode<V, S, kSrcInitMixed, true, false>(a, st);
    case kSrcCarriedLength:
      if (filter || !wk) return cudaErrorInvalidValue;
      return launch_mode<V, S, kSrcCarriedLength, true, false>(a, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace onesweep
}  // namespace cxbwt
