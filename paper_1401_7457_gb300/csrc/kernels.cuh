// Host-side launchers of the cxbwt kernels (one translation unit per group).
#pragma once
#include <cuda_runtime.h>

#include "device.cuh"

namespace cxbwt {

// Where a digit pass takes its items from.
enum SrcMode : int {
  // Position j of the initial order is generated, not loaded: suffix length
  // j / n, read j % n (every read of one length).  The key window is gathered.
  kSrcInitUniform = 0,
  // Values are loaded; the key window is gathered from the store by value.
  kSrcExtract = 1,
  // Values and the key window carried from the previous pass are loaded.
  kSrcCarried = 2,
  // Values are loaded; the key is the suffix length (the (length, read) start
  // order of reads of different lengths).
  kSrcLength = 3,
};

struct PassArgs {
  const uint32_t* vals_in;
  const uint32_t* keys_in;
  uint32_t* vals_out;
  uint32_t* keys_out;                // nullptr when the next pass gathers a new window
  const uint32_t* digit_base;        // [256] first output row of each digit value
  unsigned long long* status;        // [n_tiles * 256] look-back words of this pass
  uint32_t* tile_counter;            // zero on entry; the kernel leaves it zero
  uint32_t* err;                     // device error word
  ReadIndex R;
  uint32_t n_items;
  uint32_t n_tiles;
  uint32_t epoch;                    // look-back flags of this pass: 2*epoch, 2*epoch+1
  uint32_t key_shift;                // digit = (key >> key_shift) & 255
  uint32_t window_c0;                // gathered window: suffix bases [c0, c0 + 16)
  uint32_t n_reads;                  // kSrcInitUniform
  uint64_t timeout_ns;               // look-back wait limit
};

// Tile geometry of the digit pass (threads x items per thread).
struct TileShape {
  int threads;
  int items_per_thread;
  int tile() const { return threads * items_per_thread; }
};
TileShape onesweep_shape(int tile_items_hint);
size_t onesweep_smem_bytes(const TileShape& s);
cudaError_t launch_onesweep(const PassArgs& a, int mode, bool write_key, const TileShape& shape, cudaStream_t st);

// Per-position 4-mer counts P[q][v] (q < q_max) over all reads.
cudaError_t launch_poscount(const ReadIndex& R, uint32_t n_reads, uint32_t q_max, uint32_t* P, int sm_count,
                            cudaStream_t st);
// First output row of every digit value for char digit positions 0..D-1:
// base[d][v].  lenhist (q_max+1 entries) is used when not uniform.
cudaError_t launch_digitbase(const uint32_t* P, uint32_t q_max, uint32_t D, int uniform, uint32_t n_reads,
                             uint32_t uniform_len, const uint32_t* lenhist, uint32_t* base, cudaStream_t st);
// vals[soff_i + k] = (i << shift) | k for every read i and k in [0, L_i].
cudaError_t launch_identity(const ReadIndex& R, uint32_t n_reads, const uint64_t* soff, uint32_t* vals,
                            cudaStream_t st);
// min / max / sum of n lengths and the number of invalid ones (0 or > 65535):
// out[0] = min, out[1] = max, out[2] = sum, out[3] = invalid (out zeroed by caller
// except out[0] = UINT64_MAX).
cudaError_t launch_lenstats(const uint32_t* lens, uint64_t n, unsigned long long* out, cudaStream_t st);

struct EmitArgs {
  const uint32_t* sa;        // sorted values
  uint32_t n;                // N
  ReadIndex R;
  uint32_t* bwt;             // ceil(N/16) words
  uint64_t* dollar_pos;      // per read, may be null
  unsigned long long* counts;// [5], zeroed by the caller
  uint64_t* sa_out;          // (i << 16) | k per rank, may be null
  uint32_t* err;             // device error word
};
cudaError_t launch_emit(const EmitArgs& a, cudaStream_t st);

}  // namespace cxbwt
