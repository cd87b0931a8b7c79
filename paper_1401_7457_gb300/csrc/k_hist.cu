// Whole-collection counts computed before the digit passes.
//
// Step 1 of the paper's Figure 2 scans every suffix once to size its
// partitions; here one scan of the read store yields, for every digit
// position d of the LSD sort, how many suffixes carry each digit value.  That
// is the all-digit histogram of onesweep: each pass then knows the first
// output row of every digit value before it starts.
//
// Counting suffixes directly would cost N * D digit extractions.  Instead:
// the digit d of suffix (i, k) is the 4-mer of read i at position q = k + 4d
// (A-padded), so with P[q][v] = #{reads i : q < L_i, 4-mer_i(q) = v},
//   hist_d[v] = sum_{q >= 4d} P[q][v] + [v = 0] * Z_d,
//   Z_d       = sum_i (L_i + 1 - max(0, L_i - 4d))   (suffixes whose digit d
//               lies wholly past the end of the read),
// which needs one pass over the bases (sum L_i counter increments).
#include <cuda_runtime.h>

#include "kernels.cuh"

namespace cxbwt {
namespace {

constexpr int kSlab = 64;            // read positions per CTA slab: 64 x 256 counters = 64 KB
constexpr int kCountThreads = 512;

__device__ uint32_t block_exclusive_scan(uint32_t x, uint32_t* scratch /*[blockDim/32]*/) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  uint32_t incl = x;
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) scratch[warp] = incl;
  __syncthreads();
  uint32_t pre = 0;
  for (int w = 0; w < nw; ++w)
    if (w < warp) pre += scratch[w];
  return pre + incl - x;
}

__global__ void __launch_bounds__(kCountThreads) k_poscount(const ReadIndex R, uint32_t n_reads, uint32_t q_max,
                                                            uint32_t* __restrict__ P) {
  extern __shared__ uint32_t sP[];
  const uint32_t q0 = blockIdx.y * kSlab;
  const uint32_t qn = min(uint32_t(kSlab), q_max - q0);
  for (uint32_t x = threadIdx.x; x < qn * kRadix; x += blockDim.x) sP[x] = 0u;
  __syncthreads();
  for (uint32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < n_reads; r += gridDim.x * blockDim.x) {
    Suffix s = decode(R, uint64_t(r) << R.shift);  // whole read (k = 0)
    const uint32_t qe = min(q0 + qn, s.len);
    for (uint32_t q = q0; q < qe; q += 16) {
      // Bases q .. q+31 (A-padded): every 4-mer starting in q .. q+15.
      const uint64_t win = (uint64_t(window16(R, s, q)) << 32) | window16(R, s, q + 16);
      const uint32_t tn = min(16u, qe - q);
      for (uint32_t t = 0; t < tn; ++t) {
        const uint32_t mer = uint32_t(win >> (56 - 2 * t)) & (kRadix - 1);
        atomicAdd(&sP[(q + t - q0) * kRadix + mer], 1u);
      }
    }
  }
  __syncthreads();
  for (uint32_t x = threadIdx.x; x < qn * kRadix; x += blockDim.x) {
    const uint32_t v = sP[x];
    if (v) atomicAdd(&P[uint64_t(q0) * kRadix + x], v);
  }
}

__global__ void __launch_bounds__(kRadix) k_digitbase(const uint32_t* __restrict__ P, uint32_t q_max, int uniform,
                                                      uint32_t n_reads, uint32_t uniform_len,
                                                      const uint32_t* __restrict__ lenhist, uint32_t* __restrict__ base) {
  __shared__ unsigned long long s_z[kRadix / 32];
  __shared__ uint32_t s_scan[kRadix / 32];
  const uint32_t d = blockIdx.x, v = threadIdx.x;
  const uint32_t lo = 4u * d;
  uint32_t h = 0;
  for (uint32_t q = lo; q < q_max; ++q) h += P[uint64_t(q) * kRadix + v];
  // Z_d: suffixes whose digit d is entirely padding.
  unsigned long long z = 0;
  if (uniform) {
    z = (unsigned long long)n_reads * (uniform_len + 1u - (uniform_len > lo ? uniform_len - lo : 0u));
  } else {
    for (uint32_t l = v; l <= q_max; l += blockDim.x)
      z += (unsigned long long)lenhist[l] * (l + 1u - (l > lo ? l - lo : 0u));
    for (int o = 16; o > 0; o >>= 1) z += __shfl_down_sync(0xFFFFFFFFu, z, o);
    if ((v & 31) == 0) s_z[v >> 5] = z;
    __syncthreads();
    z = 0;
    for (int w = 0; w < kRadix / 32; ++w) z += s_z[w];
  }
  if (v == 0) h += uint32_t(z);
  base[uint64_t(d) * kRadix + v] = block_exclusive_scan(h, s_scan);
}

template <class V>
__global__ void k_identity(const ReadIndex R, uint32_t n_reads, V* __restrict__ vals) {
  // One warp per read: vals[off_i + i + k] = (i << shift) | k, k = 0 .. L_i.
  const uint32_t warps = (gridDim.x * blockDim.x) >> 5;
  const uint32_t lane = threadIdx.x & 31;
  for (uint32_t i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < n_reads; i += warps) {
    const Suffix s = decode(R, V(i) << R.shift);
    const uint64_t row0 = s.off + i;
    for (uint32_t k = lane; k <= s.len; k += 32) vals[row0 + k] = (V(i) << R.shift) | V(k);
  }
}

// Suffixes per bucket (first `bucket_bits` bits of the A-padded first window,
// i.e. the first bucket_bits/2 bases) over every suffix of every read: the
// "size" array of Figure 2 step 1.  One thread per read walks its suffixes
// in address order; CTAs own 16384-bucket slabs (grid.y) in shared memory.
constexpr uint32_t kBucketSlab = 16384;

__global__ void __launch_bounds__(512) k_bucket_hist(const ReadIndex R, uint32_t n_reads, uint32_t bucket_bits,
                                                     unsigned long long* __restrict__ hist) {
  extern __shared__ uint32_t sh[];  // kBucketSlab counters
  const uint32_t slab0 = blockIdx.y * kBucketSlab;
  for (uint32_t x = threadIdx.x; x < kBucketSlab; x += blockDim.x) sh[x] = 0;
  __syncthreads();
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n_reads; i += gridDim.x * blockDim.x) {
    Suffix s = decode(R, uint64_t(i) << R.shift);
    const uint32_t L = s.len;
    for (uint32_t k = 0; k <= L; ++k) {
      s.k = k;
      const uint32_t b = window16(R, s, 0) >> (32 - bucket_bits);
      if (b - slab0 < kBucketSlab) atomicAdd(&sh[b - slab0], 1u);
    }
  }
  __syncthreads();
  const uint32_t n_buckets = 1u << bucket_bits;
  for (uint32_t x = threadIdx.x; x < kBucketSlab && slab0 + x < n_buckets; x += blockDim.x)
    if (sh[x]) atomicAdd(&hist[slab0 + x], (unsigned long long)sh[x]);
}

// Suffixes of one 8-base bucket (first window >> 16 == prefix) per value of
// their next 8 bases: when one 8-base bucket holds more suffixes than a
// slice, Section 3.1 refines it by the characters that follow.  Same walk as
// k_bucket_hist; CTAs own 16384-counter slabs of the 65536 sub-buckets.
__global__ void __launch_bounds__(512) k_sub_bucket_hist(const ReadIndex R, uint32_t n_reads, uint32_t prefix,
                                                         unsigned long long* __restrict__ hist) {
  extern __shared__ uint32_t sh[];  // kBucketSlab counters
  const uint32_t slab0 = blockIdx.y * kBucketSlab;
  for (uint32_t x = threadIdx.x; x < kBucketSlab; x += blockDim.x) sh[x] = 0;
  __syncthreads();
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n_reads; i += gridDim.x * blockDim.x) {
    Suffix s = decode(R, uint64_t(i) << R.shift);
    const uint32_t L = s.len;
    for (uint32_t k = 0; k <= L; ++k) {
      s.k = k;
      const uint32_t w = window16(R, s, 0);
      if ((w >> 16) == prefix && (w & 0xFFFFu) - slab0 < kBucketSlab) atomicAdd(&sh[(w & 0xFFFFu) - slab0], 1u);
    }
  }
  __syncthreads();
  for (uint32_t x = threadIdx.x; x < kBucketSlab; x += blockDim.x)
    if (sh[x]) atomicAdd(&hist[slab0 + x], (unsigned long long)sh[x]);
}

// Digit counts of the suffixes of one HBM-bounded pass (first window w with
// w - key_lo <= key_last): row 0 = low byte of the suffix length (the
// read-major start order's length digit), rows 1..4 = the four 8-bit digits
// of the first window (most significant first), row 5 = high byte of the
// suffix length.  Figure 2 step 3(a)'s rescan of all suffixes for the
// selected partitions.
__global__ void __launch_bounds__(512) k_pass_hist(const ReadIndex R, uint32_t n_reads, uint32_t key_lo,
                                                   uint32_t key_last, uint32_t* __restrict__ hist) {
  __shared__ uint32_t sh[6 * kRadix];
  for (uint32_t x = threadIdx.x; x < 6 * kRadix; x += blockDim.x) sh[x] = 0;
  __syncthreads();
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n_reads; i += gridDim.x * blockDim.x) {
    Suffix s = decode(R, uint64_t(i) << R.shift);
    const uint32_t L = s.len;
    for (uint32_t k = 0; k <= L; ++k) {
      s.k = k;
      const uint32_t key = window16(R, s, 0);
      if (key - key_lo <= key_last) {
        atomicAdd(&sh[(L - k) & 255u], 1u);
        atomicAdd(&sh[5 * kRadix + ((L - k) >> 8)], 1u);
#pragma unroll
        for (int j = 0; j < 4; ++j) atomicAdd(&sh[(1 + j) * kRadix + ((key >> (24 - 8 * j)) & 255u)], 1u);
      }
    }
  }
  __syncthreads();
  for (uint32_t x = threadIdx.x; x < 6 * kRadix; x += blockDim.x)
    if (sh[x]) atomicAdd(&hist[x], sh[x]);
}

// Counts of the four 8-bit digits of n keys already in HBM (a slice's first
// windows, written by the pass that listed it): 4 bytes read per key, where
// a rescan of the store would decode and gather every suffix of the
// collection again.  Each warp counts into its own shared copy.
constexpr int kKeyHistThreads = 512;

__global__ void __launch_bounds__(kKeyHistThreads) k_key_hist(const uint32_t* __restrict__ keys, uint64_t n,
                                                              uint32_t* __restrict__ hist) {
  extern __shared__ uint32_t sk[];  // [warps][4 * 256]
  constexpr int kWarps = kKeyHistThreads / 32;
  for (uint32_t x = threadIdx.x; x < kWarps * 4 * kRadix; x += blockDim.x) sk[x] = 0;
  __syncthreads();
  uint32_t* mine = sk + (threadIdx.x >> 5) * 4 * kRadix;
  const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
  // Eight independent loads in flight per thread (coalesced across the
  // warp for each of them), then their 32 counter increments.
  constexpr int kUnroll = 8;
  for (uint64_t r0 = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; r0 < n; r0 += stride * kUnroll) {
    uint32_t k[kUnroll];
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      const uint64_t r = r0 + uint64_t(u) * stride;
      k[u] = r < n ? __ldg(keys + r) : 0u;
    }
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      if (r0 + uint64_t(u) * stride >= n) break;
#pragma unroll
      for (int j = 0; j < 4; ++j) atomicAdd(&mine[j * kRadix + ((k[u] >> (24 - 8 * j)) & 255u)], 1u);
    }
  }
  __syncthreads();
  for (uint32_t x = threadIdx.x; x < 4 * kRadix; x += blockDim.x) {
    uint32_t sum = 0;
    for (int w = 0; w < kWarps; ++w) sum += sk[w * 4 * kRadix + x];
    if (sum) atomicAdd(&hist[x], sum);
  }
}

__global__ void __launch_bounds__(kRadix) k_scan_rows(uint32_t* hist) {
  __shared__ uint32_t s_scan[kRadix / 32];
  const uint32_t row = blockIdx.x, v = threadIdx.x;
  const uint32_t x = hist[row * kRadix + v];
  hist[row * kRadix + v] = block_exclusive_scan(x, s_scan);
}

__global__ void k_lenstats(const uint32_t* __restrict__ lens, uint64_t n, unsigned long long* out) {
  unsigned long long mn = ~0ull, mx = 0, sum = 0, bad = 0;
  for (uint64_t i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += uint64_t(gridDim.x) * blockDim.x) {
    const uint32_t L = lens[i];
    mn = min(mn, (unsigned long long)L);
    mx = max(mx, (unsigned long long)L);
    sum += L;
    bad += (L == 0u || L > 65535u) ? 1u : 0u;
  }
  for (int o = 16; o > 0; o >>= 1) {
    mn = min(mn, __shfl_down_sync(0xFFFFFFFFu, mn, o));
    mx = max(mx, __shfl_down_sync(0xFFFFFFFFu, mx, o));
    sum += __shfl_down_sync(0xFFFFFFFFu, sum, o);
    bad += __shfl_down_sync(0xFFFFFFFFu, bad, o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMin(out + 0, mn);
    atomicMax(out + 1, mx);
    atomicAdd(out + 2, sum);
    atomicAdd(out + 3, bad);
  }
}

}  // namespace

cudaError_t launch_poscount(const ReadIndex& R, uint32_t n_reads, uint32_t q_max, uint32_t* P, int sm_count,
                            cudaStream_t st) {
  if (q_max == 0 || n_reads == 0) return cudaSuccess;
  const size_t smem = size_t(kSlab) * kRadix * sizeof(uint32_t);
  cudaError_t e = cudaFuncSetAttribute(k_poscount, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  if (e != cudaSuccess) return e;
  const uint32_t slabs = (q_max + kSlab - 1) / kSlab;
  uint32_t gx = (n_reads + kCountThreads - 1) / kCountThreads;
  const uint32_t cap = max(1u, uint32_t(2 * sm_count) / slabs);
  if (gx > cap) gx = cap;
  k_poscount<<<dim3(gx, slabs), kCountThreads, smem, st>>>(R, n_reads, q_max, P);
  return cudaGetLastError();
}

cudaError_t launch_digitbase(const uint32_t* P, uint32_t q_max, uint32_t D, int uniform, uint32_t n_reads,
                             uint32_t uniform_len, const uint32_t* lenhist, uint32_t* base, cudaStream_t st) {
  if (D == 0) return cudaSuccess;
  k_digitbase<<<D, kRadix, 0, st>>>(P, q_max, uniform, n_reads, uniform_len, lenhist, base);
  return cudaGetLastError();
}

cudaError_t launch_identity(const ReadIndex& R, uint32_t n_reads, void* vals, int id_bytes, cudaStream_t st) {
  if (n_reads == 0) return cudaSuccess;
  const uint32_t threads = 256;
  uint64_t blocks = (uint64_t(n_reads) * 32 + threads - 1) / threads;
  if (blocks > 65535u * 4u) blocks = 65535u * 4u;
  if (id_bytes == 8) k_identity<uint64_t><<<uint32_t(blocks), threads, 0, st>>>(R, n_reads, static_cast<uint64_t*>(vals));
  else k_identity<uint32_t><<<uint32_t(blocks), threads, 0, st>>>(R, n_reads, static_cast<uint32_t*>(vals));
  return cudaGetLastError();
}

cudaError_t launch_bucket_hist(const ReadIndex& R, uint32_t n_reads, uint32_t bucket_bits, unsigned long long* hist,
                               int sm_count, cudaStream_t st) {
  const uint32_t slabs = ((1u << bucket_bits) + kBucketSlab - 1) / kBucketSlab;
  uint32_t gx = (n_reads + 511) / 512;
  const uint32_t cap = max(1u, uint32_t(2 * sm_count) / slabs);
  if (gx > cap) gx = cap;
  if (gx == 0) gx = 1;
  const int smem = int(kBucketSlab * sizeof(uint32_t));
  cudaError_t e = cudaFuncSetAttribute(k_bucket_hist, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  k_bucket_hist<<<dim3(gx, slabs), 512, smem, st>>>(R, n_reads, bucket_bits, hist);
  return cudaGetLastError();
}

cudaError_t launch_sub_bucket_hist(const ReadIndex& R, uint32_t n_reads, uint32_t prefix, unsigned long long* hist,
                                   int sm_count, cudaStream_t st) {
  const uint32_t slabs = 65536u / kBucketSlab;
  uint32_t gx = (n_reads + 511) / 512;
  const uint32_t cap = max(1u, uint32_t(2 * sm_count) / slabs);
  if (gx > cap) gx = cap;
  if (gx == 0) gx = 1;
  const int smem = int(kBucketSlab * sizeof(uint32_t));
  cudaError_t e = cudaFuncSetAttribute(k_sub_bucket_hist, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  k_sub_bucket_hist<<<dim3(gx, slabs), 512, smem, st>>>(R, n_reads, prefix, hist);
  return cudaGetLastError();
}

cudaError_t launch_pass_hist(const ReadIndex& R, uint32_t n_reads, uint32_t key_lo, uint32_t key_last,
                             uint32_t* hist, int sm_count, cudaStream_t st) {
  uint32_t gx = (n_reads + 511) / 512;
  if (gx > uint32_t(2 * sm_count)) gx = 2 * sm_count;
  if (gx == 0) gx = 1;
  k_pass_hist<<<gx, 512, 0, st>>>(R, n_reads, key_lo, key_last, hist);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_scan_rows<<<6, kRadix, 0, st>>>(hist);
  return cudaGetLastError();
}

cudaError_t launch_key_hist(const uint32_t* keys, uint64_t n, uint32_t* hist, int sm_count, cudaStream_t st) {
  if (n > 0) {
    const int smem = int(kKeyHistThreads / 32 * 4 * kRadix * sizeof(uint32_t));
    cudaError_t e = cudaFuncSetAttribute(k_key_hist, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    uint64_t gx = (n + kKeyHistThreads - 1) / kKeyHistThreads;
    if (gx > uint64_t(3 * sm_count)) gx = 3 * sm_count;  // three 64 KB CTAs per SM
    k_key_hist<<<uint32_t(gx), kKeyHistThreads, smem, st>>>(keys, n, hist);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  k_scan_rows<<<4, kRadix, 0, st>>>(hist);
  return cudaGetLastError();
}

cudaError_t launch_lenstats(const uint32_t* lens, uint64_t n, unsigned long long* out, cudaStream_t st) {
  const uint32_t threads = 256;
  uint64_t blocks = (n + threads - 1) / threads;
  if (blocks > 1024) blocks = 1024;
  if (blocks == 0) blocks = 1;
  k_lenstats<<<uint32_t(blocks), threads, 0, st>>>(lens, n, out);
  return cudaGetLastError();
}

}  // namespace cxbwt
