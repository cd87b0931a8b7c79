// Launchers of the group-finishing kernels (k_group.cu).
#pragma once
#include <cuda_runtime.h>

#include "device.cuh"

namespace cxbwt {

constexpr uint32_t kCtaMax = 2048;  // largest group remainder finished by one CTA (keys of at most 16 words)
constexpr uint32_t kSmallCta = 256; // remainders up to this size go to small CTAs (128 threads, many per SM)
// The CTA finish holds (id, key words, index) per row in shared memory: wide
// keys (long reads) get fewer rows.
constexpr uint32_t cta_rows_for(int nw) { return nw <= 16 ? kCtaMax : kCtaMax / 2; }
template <int NW>
struct CtaRows {
  static constexpr uint32_t value = cta_rows_for(NW);
};
// Entries the two group lists need for `rows` rows finished with key width
// nw: every listed CTA remainder holds more than 32 rows, every big one more
// than cta_rows_for(nw).
constexpr uint64_t cta_list_cap(uint64_t rows) { return rows / 33 + 1; }
constexpr uint64_t big_list_cap(uint64_t rows, int nw) { return rows / (uint64_t(cta_rows_for(nw)) + 1) + 1; }

struct SegArgs {
  const uint32_t* keys;   // first 16-base window of each row; ascending under key_mask
  void* vals;             // suffix ids (uint32 or uint64), sorted by that window; finished in place
  uint32_t n_items;
  ReadIndex R;
  uint32_t depth;         // bases already sorted: l of the group plan (12 or 16)
  uint32_t key_mask;      // the window bits of those bases: rows are in one group when their masked keys are equal
  uint2* cta_list;        // (first row, rows) of remainders of 33 .. kCtaMax rows
  uint32_t cta_cap;
  uint2* big_list;        // remainders of more rows, finished by the host
  uint32_t big_cap;
  uint32_t* counts;       // zero on entry: [0] small remainders (cta_list front), [1] big_list length,
                          // [2] small work counter, [3] larger CTA remainders (cta_list back), [4] their work counter
  uint32_t* err;
};

// Key words a group remainder is sorted by for reads of at most max_len bases
// when the first `depth` bases are sorted already (a compiled width >=
// ceil((max_len - depth) / 16)), or 0 if too long.
int segsort_words(uint32_t max_len, uint32_t depth);
// The bits of a 16-base window that hold its first `depth` bases.
constexpr uint32_t depth_mask(uint32_t depth) { return depth >= 16 ? 0xFFFFFFFFu : ~(0xFFFFFFFFu >> (2u * depth)); }
// wide: warp windows of 64 rows (two per lane) instead of 32, for read
// stores out of L2.
cudaError_t launch_segsort(const SegArgs& a, int nw, int id_bytes, int sm_count, bool wide, cudaStream_t st);
// Digit bases (exclusive, per digit position) of the n_win windows of bases
// [c0, c0 + 16), [c0 + 16, c0 + 32), ... over n rows of vals.
cudaError_t launch_range_hist(const void* vals, int id_bytes, uint32_t n, const ReadIndex& R, uint32_t c0,
                              uint32_t n_win, uint32_t* hist, int sm_count, cudaStream_t st);

}  // namespace cxbwt
