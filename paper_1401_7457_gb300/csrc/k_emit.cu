// BWT emission: Figure 2 step 3(c)(iii) of the paper ("for each suffix in the
// sorted order, output its preceding character"), with the Section 2 rule
// that a suffix starting at position 0 is preceded by $.
//
// Each thread owns 16 consecutive rows, so it assembles one packed output word
// by itself: one 64-byte read of sorted values, 16 gathers of the preceding
// base from the (L2-resident) read store, one 4-byte store.  Alongside it
// records where each read's $ landed and counts the five symbols.
#include <cuda_runtime.h>

#include "kernels.cuh"

namespace cxbwt {
namespace {

constexpr int kEmitThreads = 256;

__global__ void __launch_bounds__(kEmitThreads) k_emit(const EmitArgs a) {
  __shared__ unsigned long long s_cnt[5];
  if (threadIdx.x < 5) s_cnt[threadIdx.x] = 0;
  __syncthreads();
  const uint64_t t = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  const uint64_t r0 = t * 16;
  uint32_t c[5] = {0, 0, 0, 0, 0};
  if (r0 < a.n) {
    uint32_t v[16];
    if (r0 + 16 <= a.n) {
      const uint4* p = reinterpret_cast<const uint4*>(a.sa + r0);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const uint4 x = __ldg(p + q);
        v[4 * q] = x.x; v[4 * q + 1] = x.y; v[4 * q + 2] = x.z; v[4 * q + 3] = x.w;
      }
    } else {
#pragma unroll
      for (int j = 0; j < 16; ++j) v[j] = (r0 + j < a.n) ? __ldg(a.sa + r0 + j) : 0u;
    }
    uint32_t word = 0;
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      if (r0 + j < a.n) {
        const Suffix s = decode(a.R, v[j]);
        uint32_t sym;
        if (s.read >= a.R.n_reads || s.k > s.len) {
          atomicOr(a.err, kErrBounds);  // not a suffix id: record, write nothing through it
          sym = 0;
        } else if (s.k == 0) {
          sym = 0;  // $ is stored as code 0; its row is reported separately
          ++c[0];
          if (a.dollar_pos) a.dollar_pos[s.read] = r0 + j;
        } else {
          sym = base_at(a.R, s.off + s.k - 1);
          ++c[sym + 1];
        }
        word |= sym << (30 - 2 * j);
        if (a.sa_out) a.sa_out[r0 + j] = (uint64_t(s.read) << 16) | s.k;
      }
    }
    a.bwt[t] = word;
  }
#pragma unroll
  for (int q = 0; q < 5; ++q) {
    const uint32_t w = __reduce_add_sync(0xFFFFFFFFu, c[q]);
    if ((threadIdx.x & 31) == 0 && w) atomicAdd(&s_cnt[q], (unsigned long long)w);
  }
  __syncthreads();
  if (threadIdx.x < 5 && s_cnt[threadIdx.x]) atomicAdd(a.counts + threadIdx.x, s_cnt[threadIdx.x]);
}

}  // namespace

cudaError_t launch_emit(const EmitArgs& a, cudaStream_t st) {
  if (a.n == 0) return cudaSuccess;
  const uint64_t words = (uint64_t(a.n) + 15) / 16;
  const uint64_t blocks = (words + kEmitThreads - 1) / kEmitThreads;
  k_emit<<<uint32_t(blocks), kEmitThreads, 0, st>>>(a);
  return cudaGetLastError();
}

}  // namespace cxbwt
