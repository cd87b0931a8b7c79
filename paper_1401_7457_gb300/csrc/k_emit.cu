// BWT emission: Figure 2 step 3(c)(iii) of the paper, where the suffixes are
// walked in sorted order and each one contributes the base just before it to
// the BWT, with the Section 2 rule that a suffix starting at position 0 is
// preceded by $.
//
// Each thread owns one packed output word (16 consecutive global rows), so it
// assembles the word by itself: up to 16 sorted ids, the preceding base of
// each (carried in the id when the ids were generated with it, else gathered
// from the read store), one 4-byte store.  A
// slice of the BWT (one HBM-bounded pass) may start or end inside a word:
// those two words are merged with atomicOr into a word the host zeroed.
// Alongside it records where each read's $ landed and counts the symbols.
#include <cuda_runtime.h>

#include "kernels.cuh"

namespace cxbwt {
namespace {

constexpr int kEmitThreads = 256;

template <class V>
__global__ void __launch_bounds__(kEmitThreads) k_emit(const EmitArgs a) {
  __shared__ unsigned long long s_cnt[5];
  if (threadIdx.x < 5) s_cnt[threadIdx.x] = 0;
  __syncthreads();
  const V* sa = static_cast<const V*>(a.sa);
  const uint64_t w = (a.row0 >> 4) + uint64_t(blockIdx.x) * blockDim.x + threadIdx.x;  // global word
  const uint64_t end = a.row0 + a.n;
  // Symbol counts of this thread's (at most 16) rows, 8 bits per symbol:
  // byte 0 = $, bytes 1..4 = A, C, G, T.
  unsigned long long cpack = 0;
  if (16 * w < end) {
    const uint64_t g0 = 16 * w;
    // The slice owns the word when every row of it that exists is in the slice.
    const bool whole = g0 >= a.row0 && min(g0 + 16, a.n_total) <= end;
    V v[16];
    // 16-byte loads only when all 16 rows are in the slice and the address is
    // 16-byte aligned (a collection inside a pack, or a slice's part of the
    // listed rows, may start at any row).
    const bool full16 = g0 >= a.row0 && g0 + 16 <= end;
    const bool aligned16 = (reinterpret_cast<uintptr_t>(sa + (g0 - a.row0)) & 15u) == 0;
    if (full16 && aligned16 && sizeof(V) == 4) {
      const uint4* p = reinterpret_cast<const uint4*>(sa + (g0 - a.row0));
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const uint4 x = __ldg(p + q);
        v[4 * q] = V(x.x); v[4 * q + 1] = V(x.y); v[4 * q + 2] = V(x.z); v[4 * q + 3] = V(x.w);
      }
    } else if (full16 && aligned16 && sizeof(V) == 8) {
      // Two 64-bit ids per 16-byte load (little-endian halves).
      const uint4* p = reinterpret_cast<const uint4*>(sa + (g0 - a.row0));
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const uint4 x = __ldg(p + q);
        v[2 * q] = V((uint64_t(x.y) << 32) | x.x);
        v[2 * q + 1] = V((uint64_t(x.w) << 32) | x.z);
      }
    } else {
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const uint64_t g = g0 + j;
        v[j] = (g >= a.row0 && g < end) ? sa[g - a.row0] : V(0);
      }
    }
    uint32_t word = 0;
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      const uint64_t g = g0 + j;
      if (g >= a.row0 && g < end) {
        const Suffix s = decode(a.R, v[j]);
        uint32_t sym;
        if (s.read - a.read_base >= a.n_reads_out || s.k > s.len) {
          atomicOr(a.err, kErrBounds);  // not a suffix id: record, write nothing through it
          sym = 0;
        } else if (s.k == 0) {
          sym = 0;  // $ is stored as code 0; its row is reported separately
          cpack += 1ull;
          if (a.dollar_pos) a.dollar_pos[s.read - a.read_base] = g;
        } else {
          // The id carries the preceding base when the ids were generated with it.
          sym = a.R.sym_bits ? uint32_t(v[j]) & 3u : base_at(a.R, s.off + s.k - 1);
          cpack += 1ull << (8 * (sym + 1));
        }
        word |= sym << (30 - 2 * j);
        if (a.sa_out) a.sa_out[g - a.row0] = (uint64_t(s.read - a.read_base) << 16) | s.k;
      }
    }
    if (whole) a.bwt[w - a.word_base] = word;
    else atomicOr(a.bwt + (w - a.word_base), word);
  }
#pragma unroll
  for (int q = 0; q < 5; ++q) {
    const uint32_t x = __reduce_add_sync(0xFFFFFFFFu, uint32_t(cpack >> (8 * q)) & 0xFFu);
    if ((threadIdx.x & 31) == 0 && x) atomicAdd(&s_cnt[q], (unsigned long long)x);
  }
  __syncthreads();
  if (threadIdx.x < 5 && s_cnt[threadIdx.x]) atomicAdd(a.counts + threadIdx.x, s_cnt[threadIdx.x]);
}

}  // namespace

cudaError_t launch_emit(const EmitArgs& a, cudaStream_t st) {
  if (a.n == 0) return cudaSuccess;
  const uint64_t words = ((a.row0 + a.n + 15) >> 4) - (a.row0 >> 4);
  const uint64_t blocks = (words + kEmitThreads - 1) / kEmitThreads;
  if (a.id_bytes == 8) k_emit<uint64_t><<<uint32_t(blocks), kEmitThreads, 0, st>>>(a);
  else k_emit<uint32_t><<<uint32_t(blocks), kEmitThreads, 0, st>>>(a);
  return cudaGetLastError();
}

}  // namespace cxbwt
