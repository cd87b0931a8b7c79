// Host-side launchers of the cxbwt kernels (one translation unit per group).
#pragma once
#include <cuda_runtime.h>

#include "device.cuh"

namespace cxbwt {

// Where a digit pass takes its items from.
enum SrcMode : int {
  // Item j of the (suffix length, read) start order is generated, not loaded:
  // suffix length j / n, read j % n (every read of one length).  The key
  // window is gathered.
  kSrcInitUniform = 0,
  // Ids are loaded; the key window is gathered from the store by id.
  kSrcExtract = 1,
  // Ids and the key window carried from the previous pass are loaded.
  kSrcCarried = 2,
  // Ids are loaded; the digit is a byte of the suffix length (the (length,
  // read) start order for reads of different lengths).
  kSrcLength = 3,
  // Item j of the read-major order (read j / (L+1), offset j % (L+1)) is
  // generated; the first window is gathered and carried; the digit is the
  // suffix length (at most 255).  Gathers walk the store in address order.
  kSrcInitReadMajor = 4,
  // Ids are loaded; the digit is the index of the id's collection in a batch
  // pack (coll_start: first read of each collection, ascending).
  kSrcCollection = 5,
  // Item j of the read-major order is generated as in kSrcInitReadMajor and
  // its first window gathered; the digit is (slice of the window's first 4
  // bases, suffix length), slice * (L+1) + L - k, and each slice's rows go
  // to that slice's own output arrays (split_vals / split_keys, rows counted
  // from 0 there).  One pass lists every slice of a build that runs in
  // several bucket slices.
  kSrcInitSplit = 6,
  // Item j of the read-major order over reads of any lengths (read i holds
  // rows [off_i + i, off_i + i + L_i]) is generated and its first window
  // gathered; the digit is the low byte of the suffix length.  Lists one
  // slice (bucket filter) of a collection of mixed read lengths.
  kSrcInitMixed = 7,
  // Ids and the key window carried from the previous pass are loaded; the
  // digit is byte key_shift / 8 of the suffix length (the high byte, after a
  // kSrcInitMixed pass over reads longer than 255 bases).
  kSrcCarriedLength = 8,
};
constexpr uint32_t kMaxPackCollections = 256;
constexpr uint32_t kMaxSplit = 4;  // slices one kSrcInitSplit pass writes

struct PassArgs {
  const void* vals_in;               // suffix ids (uint32 or uint64)
  const uint32_t* keys_in;
  void* vals_out;
  uint32_t* keys_out;                // nullptr when the next pass gathers a new window
  const uint32_t* digit_base;        // [256] first output row of each digit value
  unsigned long long* status;        // [n_tiles * 256] look-back words of this pass
  uint32_t* tile_counter;            // zero on entry; the kernel leaves it zero
  uint32_t* err;                     // device error word
  ReadIndex R;
  uint64_t n_gen;                    // input rows (loaded or generated)
  uint32_t n_out;                    // output rows (n_gen unless a bucket filter drops some)
  uint32_t n_tiles;
  uint32_t epoch;                    // look-back flags of this pass: 2*epoch, 2*epoch+1
  uint32_t key_shift;                // digit = (key >> key_shift) & 255
  uint32_t window_c0;                // gathered window: suffix bases [c0, c0 + 16)
  uint32_t n_reads;                  // generated modes
  uint32_t key_lo, key_last;         // filter: keep rows whose first window w has w - key_lo <= key_last
  const uint32_t* coll_start;        // kSrcCollection: n_coll + 1 read starts
  uint32_t n_coll;
  uint32_t stall_tile0;              // test hook: tile 0 publishes nothing (its successor's wait runs out)
  uint64_t timeout_ns;               // look-back wait limit
  uint32_t prefetch;                 // host: carried passes may prefetch into L2; kernel: tiles ahead (0 = none)
  // kSrcInitSplit: slice of every 4-base bucket (first window >> 24), and
  // each slice's outputs and rows.
  const uint8_t* split_of;
  void* split_vals[kMaxSplit];
  uint32_t* split_keys[kMaxSplit];
  uint32_t split_rows[kMaxSplit];
};

// The listing pass of a build in slices (k_list.cu): suffixes of reads of
// one length L, enumerated read by read, kept when their first window lies
// in one of n_slices key ranges, written to their slice's arrays in
// (suffix length, read) order.  Digit d = s * (L + 1) + suffix length.
constexpr uint32_t kListMaxStage = 4096;  // rows one tile stages in shared memory
struct ListArgs {
  ReadIndex R;                  // reads of one length (R.uniform_len = L, at most 255)
  uint32_t n_reads;
  uint32_t reads_per_tile;      // list_reads_per_tile(L)
  uint32_t n_tiles;             // ceil(n_reads / reads_per_tile)
  uint32_t stage_rows;          // reads_per_tile * (L + 1), at most kListMaxStage
  uint32_t n_slices;            // S in 1 .. kMaxSplit, with S * (L + 1) <= 256
  uint32_t key_lo[kMaxSplit];   // slice s keeps the suffixes whose first window w has
  uint32_t key_last[kMaxSplit]; //   w - key_lo[s] <= key_last[s] (ranges do not overlap)
  void* vals[kMaxSplit];        // slice s's ids (uint32 or uint64) and first windows, rows from 0
  uint32_t* keys[kMaxSplit];
  uint32_t rows[kMaxSplit];     // rows of slice s (writes beyond are refused: kErrBounds)
  const uint32_t* digit_base;   // [S * (L + 1)]: row, in its slice, of the first suffix of digit d
  unsigned long long* status;   // look-back words, [n_tiles * 256]
  uint32_t* tile_counter;       // zero on entry; the kernel leaves it zero
  uint32_t* err;                // device error word
  uint32_t epoch;               // look-back flags of this pass: 2*epoch, 2*epoch+1
  uint64_t timeout_ns;          // look-back wait limit
  uint32_t prefetch;            // host: nonzero asks for the store words of later tiles to be read into L2
};
uint32_t list_reads_per_tile(uint32_t read_len);
cudaError_t launch_list(const ListArgs& a, int id_bytes, cudaStream_t st);

// Tile geometry of the digit pass (threads x items per thread).
struct TileShape {
  int threads;
  int items_per_thread;
  int tile() const { return threads * items_per_thread; }
};
TileShape onesweep_shape(int tile_items_hint, int id_bytes);
// id_bytes: 4 or 8.  filter: drop rows outside the bucket range (generated modes only).
cudaError_t launch_onesweep(const PassArgs& a, int mode, bool write_key, bool filter, int id_bytes,
                            const TileShape& shape, cudaStream_t st);
template <class V>
cudaError_t launch_onesweep_t(const PassArgs& a, int mode, bool write_key, bool filter, const TileShape& shape,
                              cudaStream_t st);

// Per-position 4-mer counts P[q][v] (q < q_max) over all reads.
cudaError_t launch_poscount(const ReadIndex& R, uint32_t n_reads, uint32_t q_max, uint32_t* P, int sm_count,
                            cudaStream_t st);
// First output row of every digit value for char digit positions 0..D-1:
// base[d][v].  lenhist (q_max+1 entries) is used when not uniform.
cudaError_t launch_digitbase(const uint32_t* P, uint32_t q_max, uint32_t D, int uniform, uint32_t n_reads,
                             uint32_t uniform_len, const uint32_t* lenhist, uint32_t* base, cudaStream_t st);
// vals[off_i + i + k] = (i << shift) | k for every read i and k in [0, L_i].
cudaError_t launch_identity(const ReadIndex& R, uint32_t n_reads, void* vals, int id_bytes, cudaStream_t st);
// Suffixes per bucket of the first bucket_bits / 2 bases (hist: 2^bucket_bits
// zeroed uint64 counters).
cudaError_t launch_bucket_hist(const ReadIndex& R, uint32_t n_reads, uint32_t bucket_bits, unsigned long long* hist,
                               int sm_count, cudaStream_t st);
// First output row of each digit value, for the suffixes whose first
// window w has w - key_lo <= key_last: row 0 = low byte of the suffix
// length, rows 1..4 = first-window digits, row 5 = high byte of the suffix
// length (hist: 6 x 256 zeroed counters, replaced by exclusive sums).
cudaError_t launch_pass_hist(const ReadIndex& R, uint32_t n_reads, uint32_t key_lo, uint32_t key_last,
                             uint32_t* hist, int sm_count, cudaStream_t st);
// Suffixes whose first 8 bases (A-padded) are `prefix` (16 bits), counted by
// their next 8 bases (hist: 65536 zeroed counters): the refinement of one
// 8-base bucket by the characters that follow (Section 3.1).
cudaError_t launch_sub_bucket_hist(const ReadIndex& R, uint32_t n_reads, uint32_t prefix, unsigned long long* hist,
                                   int sm_count, cudaStream_t st);
// First output row of each value of the four 8-bit digits of n keys (most
// significant digit first): hist (4 x 256 zeroed counters) is replaced by
// exclusive sums.
cudaError_t launch_key_hist(const uint32_t* keys, uint64_t n, uint32_t* hist, int sm_count, cudaStream_t st);
// min / max / sum of n lengths and the number of invalid ones (0 or > 65535):
// out[0] = min, out[1] = max, out[2] = sum, out[3] = invalid (out zeroed by caller
// except out[0] = UINT64_MAX).
cudaError_t launch_lenstats(const uint32_t* lens, uint64_t n, unsigned long long* out, cudaStream_t st);

struct EmitArgs {
  const void* sa;            // sorted ids of this slice's rows (uint32 or uint64)
  uint32_t n;                // rows in the slice
  uint64_t row0;             // global BWT row of the slice's row 0
  uint64_t n_total;          // rows of the whole BWT
  ReadIndex R;
  uint32_t* bwt;             // global word w is bwt[w - word_base]
  uint64_t word_base;
  uint64_t* dollar_pos;      // per read (global rows), may be null
  unsigned long long* counts;// [5], accumulated
  uint64_t* sa_out;          // (i << 16) | k per slice row (sa_out[r]), may be null
  uint32_t read_base;        // dollar_pos and sa_out use read index - read_base (a collection inside a pack)
  uint32_t n_reads_out;      // reads of the slice's collection: read - read_base must be below it
  uint32_t* err;             // device error word
  int id_bytes;              // 4 or 8
};
cudaError_t launch_emit(const EmitArgs& a, cudaStream_t st);

}  // namespace cxbwt
