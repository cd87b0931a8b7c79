// Finishing the sort inside groups of suffixes that share their first 16 bases.
//
// After the stable LSD passes over the first 16-base window, the suffix ids
// are ordered by those 16 bases (A-padded) and, among equal windows, by
// (suffix length, read): a "group" is a maximal run of equal windows.  This
// is the partition step of Section 3.1 (suffixes with the same l-prefix form
// one partition, l = 16 here) followed by sorting each partition; groups are
// small for reads (about the coverage), so each one is finished on chip
// instead of with more passes over HBM:
//
//   * the members of a group whose suffix has at most 16 bases are final:
//     their whole A-padded key is the window, they tie with each other and
//     with every longer member's padded key only when that member continues
//     with A's, and then the shorter one is smaller - the group is already in
//     (length, read) order, so they form its prefix and stay where they are;
//   * the rest of the group (the "remainder") is sorted by bases 16.. of the
//     suffix, A-padded, ties kept in the current order (stable): one warp
//     with a register bitonic network when it has at most 32 members, one CTA
//     with a shared-memory bitonic network up to kCtaMax members, and larger
//     ones are listed for the host, which finishes them with more LSD passes
//     restricted to their rows (k_range_hist gives those passes' digit bases).
//
// Each warp scans a chunk of rows for group heads, so no group list is
// materialised for the common case.
#include <cuda_runtime.h>

#include "group.cuh"

namespace cxbwt {
namespace {

constexpr int kChunk = 256;  // rows scanned per warp task

// Bases [c0, c0 + 16*NW) of suffix s (A-padded past the read end) as NW words.
template <int NW>
__device__ __forceinline__ void gather_words(const ReadIndex& R, const Suffix& s, uint32_t c0, uint32_t (&w)[NW]) {
  const uint32_t rel = s.k + c0;
  const uint32_t rem = rel < s.len ? s.len - rel : 0u;  // real bases from c0 on
  const uint64_t q = s.off + rel;
  const uint64_t w0 = q >> 4;
  const uint32_t sh = uint32_t(q & 15u) * 2u;
  uint32_t prev = rem ? load_word(R, w0) : 0u;
#pragma unroll
  for (int i = 0; i < NW; ++i) {
    const uint32_t need = 16u * i;  // bases of the read before word i
    uint32_t x = 0;
    if (need < rem) {
      const uint32_t next = load_word(R, w0 + i + 1);
      x = __funnelshift_l(next, prev, sh);
      prev = next;
      const uint32_t left = rem - need;
      if (left < 16u) x &= ~(0xFFFFFFFFu >> (2u * left));
    }
    w[i] = x;
  }
}

// (a < b) on (words, position): lexicographic words, then position.
template <int NW>
__device__ __forceinline__ bool key_less(const uint32_t (&a)[NW], uint32_t pa, const uint32_t (&b)[NW], uint32_t pb) {
#pragma unroll
  for (int i = 0; i < NW; ++i)
    if (a[i] != b[i]) return a[i] < b[i];
  return pa < pb;
}

__device__ __forceinline__ uint32_t suffix_len(const ReadIndex& R, uint32_t v) {
  const Suffix s = decode(R, v);
  return s.len - s.k;
}

// Sort rows [s, s + m) (m <= 32) of vals by bases 16.. with one warp.
template <int NW>
__device__ void warp_sort_rows(const SegArgs& a, uint32_t s, uint32_t m, int lane) {
  uint32_t w[NW];
  uint32_t v = 0, p = uint32_t(lane);
  if (uint32_t(lane) < m) {
    v = a.vals[s + lane];
    gather_words<NW>(a.R, decode(a.R, v), a.depth, w);
  } else {
#pragma unroll
    for (int i = 0; i < NW; ++i) w[i] = 0xFFFFFFFFu;  // past the group: sorts last (its position is larger)
  }
#pragma unroll
  for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
    for (int j = k >> 1; j > 0; j >>= 1) {
      uint32_t ow[NW];
#pragma unroll
      for (int i = 0; i < NW; ++i) ow[i] = __shfl_xor_sync(0xFFFFFFFFu, w[i], j);
      const uint32_t ov = __shfl_xor_sync(0xFFFFFFFFu, v, j);
      const uint32_t op = __shfl_xor_sync(0xFFFFFFFFu, p, j);
      const bool ascending = (lane & k) == 0;
      const bool lower = (lane & j) == 0;
      const bool other_less = key_less<NW>(ow, op, w, p);
      // The lower lane of an ascending pair keeps the smaller item.
      const bool take = (lower == ascending) ? other_less : !other_less;
      if (take) {
#pragma unroll
        for (int i = 0; i < NW; ++i) w[i] = ow[i];
        v = ov;
        p = op;
      }
    }
  }
  if (uint32_t(lane) < m) a.vals[s + lane] = v;
}

template <int NW>
__global__ void __launch_bounds__(256) k_segsort_warp(const SegArgs a) {
  const int lane = threadIdx.x & 31;
  const uint32_t warps = (gridDim.x * blockDim.x) >> 5;
  const uint32_t n_chunks = (a.n_items + kChunk - 1) / kChunk;
  for (uint32_t c = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; c < n_chunks; c += warps) {
    const uint32_t base = c * kChunk;
    for (uint32_t t = 0; t < kChunk; t += 32) {
      const uint32_t r = base + t + lane;
      bool head = false;
      uint32_t key = 0;
      if (r < a.n_items) {
        key = a.keys[r];
        head = (r == 0) || (a.keys[r - 1] != key);
      }
      uint32_t heads = __ballot_sync(0xFFFFFFFFu, head);
      while (heads) {
        const int hl = __ffs(heads) - 1;
        heads &= heads - 1;
        const uint32_t gs = base + t + hl;
        const uint32_t gk = __shfl_sync(0xFFFFFFFFu, key, hl);
        // End of the group: first row after gs whose window differs.
        uint32_t ge = a.n_items;
        for (uint32_t x = gs + 1;; x += 32) {
          const uint32_t y = x + lane;
          const bool differs = (y >= a.n_items) || (a.keys[y] != gk);
          const uint32_t m = __ballot_sync(0xFFFFFFFFu, differs);
          if (m) {
            ge = x + __ffs(m) - 1;
            break;
          }
          if (x - gs > 64) {  // long group: binary search over the sorted windows
            uint32_t lo = x + 32, hi = a.n_items;
            if (lane == 0) {
              while (lo < hi) {
                const uint32_t mid = lo + (hi - lo) / 2;
                if (a.keys[mid] == gk) lo = mid + 1; else hi = mid;
              }
            }
            ge = __shfl_sync(0xFFFFFFFFu, lo, 0);
            break;
          }
        }
        if (ge - gs < 2) continue;
        // Skip the finished prefix: members with at most `depth` bases.
        uint32_t gsr;
        if (ge - gs <= 32) {
          const uint32_t y = gs + lane;
          const bool longer = (y < ge) && suffix_len(a.R, a.vals[y]) > a.depth;
          const uint32_t m = __ballot_sync(0xFFFFFFFFu, longer);
          gsr = m ? gs + __ffs(m) - 1 : ge;
        } else {
          uint32_t lo = gs, hi = ge;
          if (lane == 0) {
            while (lo < hi) {
              const uint32_t mid = lo + (hi - lo) / 2;
              if (suffix_len(a.R, a.vals[mid]) > a.depth) hi = mid; else lo = mid + 1;
            }
          }
          gsr = __shfl_sync(0xFFFFFFFFu, lo, 0);
        }
        const uint32_t m = ge - gsr;
        if (m < 2) continue;
        if (m <= 32) {
          warp_sort_rows<NW>(a, gsr, m, lane);
        } else if (lane == 0) {
          const bool cta = m <= kCtaMax;
          const uint32_t slot = atomicAdd(a.counts + (cta ? 0 : 1), 1u);
          if (slot < (cta ? a.cta_cap : a.big_cap)) (cta ? a.cta_list : a.big_list)[slot] = make_uint2(gsr, m);
          else atomicOr(a.err, kErrBounds);
        }
      }
    }
  }
}

// Shared-memory bitonic sort of one listed group per CTA (33 .. kCtaMax members).
template <int NW>
__global__ void __launch_bounds__(512) k_segsort_cta(const SegArgs a) {
  extern __shared__ __align__(16) uint32_t sm[];
  uint32_t* s_w = sm;                       // [NW][kCtaMax]
  uint32_t* s_v = sm + NW * kCtaMax;        // [kCtaMax]
  uint16_t* s_perm = reinterpret_cast<uint16_t*>(s_v + kCtaMax);  // [kCtaMax]
  __shared__ uint32_t s_item;
  const uint32_t n_list = min(*(volatile uint32_t*)(a.counts + 0), a.cta_cap);
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) s_item = atomicAdd(a.counts + 2, 1u);
    __syncthreads();
    const uint32_t it = s_item;
    if (it >= n_list) break;
    const uint2 g = a.cta_list[it];
    const uint32_t s = g.x, m = g.y;
    uint32_t P = 64;
    while (P < m) P <<= 1;
    for (uint32_t x = threadIdx.x; x < P; x += blockDim.x) {
      s_perm[x] = uint16_t(x);
      if (x < m) {
        const uint32_t v = a.vals[s + x];
        uint32_t w[NW];
        gather_words<NW>(a.R, decode(a.R, v), a.depth, w);
#pragma unroll
        for (int i = 0; i < NW; ++i) s_w[i * kCtaMax + x] = w[i];
        s_v[x] = v;
      }
    }
    __syncthreads();
    for (uint32_t k = 2; k <= P; k <<= 1) {
      for (uint32_t j = k >> 1; j > 0; j >>= 1) {
        for (uint32_t x = threadIdx.x; x < P; x += blockDim.x) {
          const uint32_t y = x ^ j;
          if (y > x) {
            const uint32_t px = s_perm[x], py = s_perm[y];
            // y_less: item at y orders before item at x (rows >= m sort last, by row).
            bool y_less;
            if (px >= m || py >= m) {
              y_less = (py >= m) ? (px >= m && py < px) : true;
            } else {
              y_less = py < px;
#pragma unroll
              for (int i = 0; i < NW; ++i) {
                const uint32_t a0 = s_w[i * kCtaMax + px], b0 = s_w[i * kCtaMax + py];
                if (a0 != b0) {
                  y_less = b0 < a0;
                  break;
                }
              }
            }
            const bool ascending = (x & k) == 0;
            if (y_less == ascending) {
              s_perm[x] = uint16_t(py);
              s_perm[y] = uint16_t(px);
            }
          }
        }
        __syncthreads();
      }
    }
    for (uint32_t x = threadIdx.x; x < m; x += blockDim.x) a.vals[s + x] = s_v[s_perm[x]];
  }
}

// Digit counts of bases [16, 16 * (1 + NWIN)) over rows [0, n) of vals: the
// per-pass histograms of the LSD passes that finish one big group.
// hist[(w * 4 + j) * 256 + digit] for window w (bases 16(w+1) ..) and digit j.
__global__ void k_range_hist(const uint32_t* vals, uint32_t n, ReadIndex R, uint32_t n_win, uint32_t* hist) {
  extern __shared__ uint32_t sh[];
  const uint32_t bins = n_win * 4 * kRadix;
  for (uint32_t x = threadIdx.x; x < bins; x += blockDim.x) sh[x] = 0;
  __syncthreads();
  for (uint32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
    const Suffix s = decode(R, vals[r]);
    for (uint32_t w = 0; w < n_win; ++w) {
      const uint32_t key = window16(R, s, 16u * (w + 1));
#pragma unroll
      for (int j = 0; j < 4; ++j) atomicAdd(&sh[(w * 4 + j) * kRadix + ((key >> (24 - 8 * j)) & 255u)], 1u);
    }
  }
  __syncthreads();
  for (uint32_t x = threadIdx.x; x < bins; x += blockDim.x)
    if (sh[x]) atomicAdd(&hist[x], sh[x]);
}

// In-place exclusive scan of `rows` histograms of 256 bins (one CTA each).
__global__ void __launch_bounds__(kRadix) k_scan256(uint32_t* hist) {
  __shared__ uint32_t s[kRadix];
  const uint32_t row = blockIdx.x, v = threadIdx.x;
  s[v] = hist[row * kRadix + v];
  __syncthreads();
  if (v == 0) {
    uint32_t acc = 0;
    for (int i = 0; i < kRadix; ++i) {
      const uint32_t c = s[i];
      s[i] = acc;
      acc += c;
    }
  }
  __syncthreads();
  hist[row * kRadix + v] = s[v];
}

template <int NW>
cudaError_t launch_nw(const SegArgs& a, int sm_count, cudaStream_t st) {
  const uint32_t n_chunks = (a.n_items + kChunk - 1) / kChunk;
  uint32_t blocks = (n_chunks + 7) / 8;
  const uint32_t cap = uint32_t(sm_count) * 16;
  if (blocks > cap) blocks = cap;
  if (blocks == 0) blocks = 1;
  k_segsort_warp<NW><<<blocks, 256, 0, st>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const size_t smem = size_t(NW + 1) * kCtaMax * 4 + kCtaMax * 2;
  static bool configured = false;
  if (!configured) {
    e = cudaFuncSetAttribute(k_segsort_cta<NW>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess) return e;
    configured = true;
  }
  k_segsort_cta<NW><<<sm_count * 2, 512, smem, st>>>(a);
  return cudaGetLastError();
}

}  // namespace

int segsort_words(uint32_t max_len) {
  const uint32_t rest = max_len > 16 ? max_len - 16 : 0;  // bases after the first window
  const uint32_t nw = (rest + 15) / 16;
  if (nw <= 2) return 2;
  if (nw <= 4) return 4;
  if (nw <= 6) return 6;
  if (nw <= 8) return 8;
  if (nw <= 12) return 12;
  if (nw <= 16) return 16;
  return 0;  // reads too long for the on-chip finish
}

cudaError_t launch_segsort(const SegArgs& a, int nw, int sm_count, cudaStream_t st) {
  switch (nw) {
    case 2: return launch_nw<2>(a, sm_count, st);
    case 4: return launch_nw<4>(a, sm_count, st);
    case 6: return launch_nw<6>(a, sm_count, st);
    case 8: return launch_nw<8>(a, sm_count, st);
    case 12: return launch_nw<12>(a, sm_count, st);
    case 16: return launch_nw<16>(a, sm_count, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_range_hist(const uint32_t* vals, uint32_t n, const ReadIndex& R, uint32_t n_win, uint32_t* hist,
                              int sm_count, cudaStream_t st) {
  if (n == 0 || n_win == 0) return cudaSuccess;
  const size_t smem = size_t(n_win) * 4 * kRadix * 4;
  cudaError_t e = cudaFuncSetAttribute(k_range_hist, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  if (e != cudaSuccess) return e;
  uint32_t blocks = (n + 255) / 256;
  if (blocks > uint32_t(sm_count) * 2) blocks = sm_count * 2;
  k_range_hist<<<blocks, 256, smem, st>>>(vals, n, R, n_win, hist);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_scan256<<<n_win * 4, kRadix, 0, st>>>(hist);
  return cudaGetLastError();
}

}  // namespace cxbwt
