// Finishing the sort inside groups of suffixes that share their first l
// bases (l = 16, or 12: the depth of the group plan).
//
// After the stable LSD passes over the first l bases of the 16-base window,
// the suffix ids are ordered by those bases (A-padded) and, among equal
// ones, by (suffix length, read): a "group" is a maximal run of rows whose
// windows agree on their first l bases (keys equal under key_mask).  This is
// the partition step of Section 3.1 (suffixes with the same l-prefix form
// one partition) followed by sorting each partition; groups are small for
// reads (about the coverage), so each one is finished on chip instead of
// with more passes over HBM:
//
//   * the members of a group whose suffix has at most l bases are final:
//     their whole A-padded key is the prefix, they tie with each other and
//     with every longer member's padded key only when that member continues
//     with A's, and then the shorter one is smaller - the group is already in
//     (length, read) order, so they form its prefix and stay where they are;
//   * the rest of the group (the "remainder") is sorted by bases l.. of the
//     suffix, A-padded, ties kept in the current order (stable): by one warp
//     when it has at most 64 members (32 for the widest keys) - each member
//     counts the members that order before it -, by one CTA with a
//     shared-memory bitonic network up to kCtaMax members, and larger ones
//     are listed for the host, which finishes them with more LSD passes
//     restricted to their rows (k_range_hist gives those passes' digit bases).
//
// Each warp walks the groups that start in its chunk of rows in windows of
// at most 64 rows made of whole groups (two rows per lane), and ranks a
// window's rows against their groups in per-warp shared memory, so no group
// list is materialised for the common case.
#include <cuda_runtime.h>

#include <atomic>

#include "group.cuh"

namespace cxbwt {
namespace {

constexpr int kChunk = 256;  // rows scanned per warp task

// Bases [c0, c0 + 16*NW) of suffix s (A-padded past the read end) as NW words,
// from the NW + 1 store words they span (4-byte loads: fewer registers held
// per load in flight than 16-byte chunks, and no realignment of the chunks).
// Only the store words that hold some of the suffix's bases are loaded (the
// loads are predicated, not branched around, so the lanes of a warp stay
// together): a suffix near its read's end, or one that ends inside the
// first window (no load at all), moves fewer DRAM sectors when the store is
// out of L2.  The words past the read's end are masked to zero.
template <int NW>
__device__ __forceinline__ void gather_words(const ReadIndex& R, const Suffix& s, uint32_t c0, uint32_t (&w)[NW]) {
  const uint32_t rel = s.k + c0;
  const bool inside = rel < s.len;
  const uint32_t rem = inside ? s.len - rel : 0u;  // real bases from c0 on
  const uint64_t q = s.off + (inside ? rel : 0u);
  const uint64_t w0 = q >> 4;
  const uint32_t sh = uint32_t(q & 15u) * 2u;
  // Store words holding bases q .. q + rem - 1 (none when rem == 0).
  const uint32_t n_load = rem ? uint32_t(((q + rem - 1) >> 4) - w0) + 1u : 0u;
  uint32_t b[NW + 1];
#pragma unroll
  for (int i = 0; i <= NW; ++i) b[i] = uint32_t(i) < n_load ? load_word(R, w0 + i) : 0u;
#pragma unroll
  for (int i = 0; i < NW; ++i) {
    const uint32_t need = 16u * i;
    const uint32_t left = rem > need ? rem - need : 0u;
    const uint32_t keep = left >= 16u ? 0xFFFFFFFFu : ~(0xFFFFFFFFu >> (2u * left));
    w[i] = __funnelshift_l(b[i + 1], b[i], sh) & keep;
  }
}

// Lexicographic comparison as a multiword subtraction: x < y (word 0 most
// significant) exactly when x - y borrows out of its most significant word.
// The borrow ripples through the words least significant first, one
// subtract-with-borrow per word, with no compare-and-select per word.
// sub_borrow<P> continues a chain over P word pairs given in ascending
// significance, from a borrow-in b (0 or ~0u), and returns the borrow-out in
// the same form.  Pairs of equal words (zero padding) pass the borrow on.
template <int P>
__device__ __forceinline__ uint32_t sub_borrow(uint32_t b, const uint32_t* x, const uint32_t* y);

template <>
__device__ __forceinline__ uint32_t sub_borrow<4>(uint32_t b, const uint32_t* x, const uint32_t* y) {
  uint32_t r;
  asm("{\n\t.reg .u32 t;\n\t"
      "sub.cc.u32 t, 0, %1;\n\t"
      "subc.cc.u32 t, %2, %3;\n\t"
      "subc.cc.u32 t, %4, %5;\n\t"
      "subc.cc.u32 t, %6, %7;\n\t"
      "subc.cc.u32 t, %8, %9;\n\t"
      "subc.u32 %0, 0, 0;\n\t}"
      : "=r"(r)
      : "r"(b), "r"(x[0]), "r"(y[0]), "r"(x[1]), "r"(y[1]), "r"(x[2]), "r"(y[2]), "r"(x[3]), "r"(y[3]));
  return r;
}

template <>
__device__ __forceinline__ uint32_t sub_borrow<8>(uint32_t b, const uint32_t* x, const uint32_t* y) {
  uint32_t r;
  asm("{\n\t.reg .u32 t;\n\t"
      "sub.cc.u32 t, 0, %1;\n\t"
      "subc.cc.u32 t, %2, %3;\n\t"
      "subc.cc.u32 t, %4, %5;\n\t"
      "subc.cc.u32 t, %6, %7;\n\t"
      "subc.cc.u32 t, %8, %9;\n\t"
      "subc.cc.u32 t, %10, %11;\n\t"
      "subc.cc.u32 t, %12, %13;\n\t"
      "subc.cc.u32 t, %14, %15;\n\t"
      "subc.cc.u32 t, %16, %17;\n\t"
      "subc.u32 %0, 0, 0;\n\t}"
      : "=r"(r)
      : "r"(b), "r"(x[0]), "r"(y[0]), "r"(x[1]), "r"(y[1]), "r"(x[2]), "r"(y[2]), "r"(x[3]), "r"(y[3]),
        "r"(x[4]), "r"(y[4]), "r"(x[5]), "r"(y[5]), "r"(x[6]), "r"(y[6]), "r"(x[7]), "r"(y[7]));
  return r;
}

// ~0u if (x words, xi) < (y words, yi): words lexicographic (word 0 first),
// then the row index.  Chains of 8 pairs, the last one of 4 or 8.
template <int NW>
__device__ __forceinline__ uint32_t lex_less_mask(const uint32_t (&x)[NW], uint32_t xi, const uint32_t (&y)[NW],
                                                  uint32_t yi) {
  constexpr int P = NW + 1;                        // pairs: the index, then words NW-1 .. 0
  constexpr int PP = (P % 8 == 0 || P % 8 > 4) ? (P + 7) / 8 * 8 : P / 8 * 8 + 4;
  uint32_t a[PP], c[PP];
  a[0] = xi;
  c[0] = yi;
#pragma unroll
  for (int i = 0; i < NW; ++i) {
    a[1 + i] = x[NW - 1 - i];
    c[1 + i] = y[NW - 1 - i];
  }
#pragma unroll
  for (int i = P; i < PP; ++i) a[i] = c[i] = 0u;
  uint32_t b = 0u;
#pragma unroll
  for (int k = 0; k + 8 <= PP; k += 8) b = sub_borrow<8>(b, a + k, c + k);
  if (PP % 8) b = sub_borrow<4>(b, a + PP / 8 * 8, c + PP / 8 * 8);
  return b;
}

template <class V>
__device__ __forceinline__ uint32_t suffix_len(const ReadIndex& R, V v) {
  const Suffix s = decode(R, v);
  return s.len - s.k;
}

// Finish the groups of a window of up to SPAN rows (SPAN = 32 or 64) made
// of whole groups: lane l holds rows l, l + 32, ... (ROUNDS = SPAN / 32 of
// them).  Each row counts the members of its group that order before it -
// smaller bases 16.. (A-padded), or equal bases and an earlier row (stable) -
// and moves to its group's first row + that count.  Rows of at most 16 bases
// gather all-zero words, so they keep their place at the front of their
// group; a row alone in its group neither gathers nor moves.  heads bit r
// says that row r of the window starts a group (bit 0 is always set).
//
// The ranking runs in ROUNDS rounds of 32 rows, each as long as the largest
// group among its rows: a window of several groups of 20 or so rows (reads
// at tens-fold coverage) keeps most lanes busy, where windows of 32 rows
// would hold one such group each.
template <int NW, int SPAN>
struct RowWords {
  static constexpr int kStride = (NW + 3) / 4 * 4;  // words per row, a whole number of uint4
  uint4 r[SPAN][kStride / 4];
};

template <int SPAN>
struct Heads;
template <>
struct Heads<32> {
  using T = uint32_t;
};
template <>
struct Heads<64> {
  using T = unsigned long long;
};

template <int NW, int SPAN, class V>
__device__ void warp_rank_window(const SegArgs& a, uint32_t cur, uint32_t n_rows, typename Heads<SPAN>::T heads,
                                 int lane, RowWords<NW, SPAN>& sw) {
  using H = typename Heads<SPAN>::T;
  constexpr int ROUNDS = SPAN / 32;
  constexpr int Q = RowWords<NW, SPAN>::kStride / 4;
  V* vals = static_cast<V*>(a.vals);
  V v[ROUNDS];
  uint32_t gid[ROUNDS], gsize[ROUNDS];
#pragma unroll
  for (int h = 0; h < ROUNDS; ++h) {
    const uint32_t row = uint32_t(lane) + 32u * h;
    const bool live = row < n_rows;
    // The row's group: from the last head at or before it to the next head after it.
    const H upto = heads & (row + 1 >= uint32_t(SPAN) ? ~H(0) : ((H(2) << row) - 1));
    const uint32_t g0 = uint32_t(8 * sizeof(H) - 1) - (sizeof(H) == 8 ? __clzll((long long)upto) : __clz(uint32_t(upto)));
    const H after = heads & ~upto;
    const uint32_t ge = after ? min(uint32_t(sizeof(H) == 8 ? __ffsll((long long)after) : __ffs(uint32_t(after))) - 1,
                                    n_rows)
                              : n_rows;
    gid[h] = g0;
    gsize[h] = live ? ge - g0 : 0u;
    uint32_t w[Q * 4];
#pragma unroll
    for (int i = 0; i < Q * 4; ++i) w[i] = 0u;
    v[h] = 0;
    if (live) {
      v[h] = vals[cur + row];
      if (gsize[h] > 1) {
        uint32_t g[NW];
        gather_words<NW>(a.R, decode(a.R, v[h]), a.depth, g);
#pragma unroll
        for (int i = 0; i < NW; ++i) w[i] = g[i];
      }
    }
    // Publish this row's words for the other members of its group.
#pragma unroll
    for (int q = 0; q < Q; ++q) sw.r[row][q] = make_uint4(w[4 * q], w[4 * q + 1], w[4 * q + 2], w[4 * q + 3]);
  }
  __syncwarp();
  uint32_t rank[ROUNDS];
#pragma unroll
  for (int h = 0; h < ROUNDS; ++h) {
    const uint32_t row = uint32_t(lane) + 32u * h;
    uint32_t mine[NW];
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      const uint4 o = sw.r[row][q];
      if (4 * q < NW) mine[4 * q] = o.x;
      if (4 * q + 1 < NW) mine[4 * q + 1] = o.y;
      if (4 * q + 2 < NW) mine[4 * q + 2] = o.z;
      if (4 * q + 3 < NW) mine[4 * q + 3] = o.w;
    }
    uint32_t rk = 0;
    const uint32_t n_cmp = gsize[h] > 1 ? gsize[h] : 0u;
    for (uint32_t t = 0; t < n_cmp; ++t) {
      const uint32_t src = gid[h] + t;
      // Row src orders before this row: smaller words, or equal words and an
      // earlier row.  Lanes of one group read one row: a broadcast.
      uint32_t ov[NW];
#pragma unroll
      for (int q = 0; q < Q; ++q) {
        const uint4 o = sw.r[src][q];
        if (4 * q < NW) ov[4 * q] = o.x;
        if (4 * q + 1 < NW) ov[4 * q + 1] = o.y;
        if (4 * q + 2 < NW) ov[4 * q + 2] = o.z;
        if (4 * q + 3 < NW) ov[4 * q + 3] = o.w;
      }
      rk -= lex_less_mask<NW>(ov, src, mine, row);  // ~0u is -1
    }
    rank[h] = rk;
  }
  __syncwarp();  // every lane has read its rows and the shared words before any write
#pragma unroll
  for (int h = 0; h < ROUNDS; ++h) {
    const uint32_t row = uint32_t(lane) + 32u * h;
    if (gsize[h] > 1 && gid[h] + rank[h] != row) vals[cur + gid[h] + rank[h]] = v[h];
  }
  __syncwarp();  // the next window reuses the shared rows
}

// First row r >= from (r < n) whose window differs from row r-1, or n.
__device__ uint32_t next_head(const SegArgs& a, uint32_t from, int lane) {
  if (from >= a.n_items) return a.n_items;
  for (uint32_t x = from;; x += 32) {
    const uint32_t y = x + lane;
    const bool head = (y < a.n_items) && (y == 0 || ((a.keys[y] ^ a.keys[y - 1]) & a.key_mask) != 0u);
    const bool stop = head || y >= a.n_items;
    const uint32_t m = __ballot_sync(0xFFFFFFFFu, stop);
    if (m) return min(x + __ffs(m) - 1, a.n_items);
    if (x - from >= 64) {  // a long run of equal windows: binary search for its end
      const uint32_t key = a.keys[x + 31] & a.key_mask;
      uint32_t lo = x + 32, hi = a.n_items;
      while (lo < hi) {
        const uint32_t mid = lo + (hi - lo) / 2;
        if ((a.keys[mid] & a.key_mask) == key) lo = mid + 1; else hi = mid;
      }
      return lo;
    }
  }
}

// Finish one group of more than SPAN rows [gs, ge): skip its finished
// prefix, sort a remainder of at most SPAN rows here, list a larger one.
template <int NW, int SPAN, class V>
__device__ void finish_long_group(const SegArgs& a, uint32_t gs, uint32_t ge, int lane, RowWords<NW, SPAN>& sw) {
  const V* vals = static_cast<const V*>(a.vals);
  uint32_t lo = gs, hi = ge;
  while (lo < hi) {
    const uint32_t mid = lo + (hi - lo) / 2;
    if (suffix_len(a.R, vals[mid]) > a.depth) hi = mid; else lo = mid + 1;
  }
  const uint32_t m = ge - lo;
  if (m < 2) return;
  if (m <= uint32_t(SPAN)) {
    warp_rank_window<NW, SPAN, V>(a, lo, m, typename Heads<SPAN>::T(1), lane, sw);
  } else if (lane == 0) {
    // Up to kSmallCta rows: cta_list from the front (counts[0]); up to
    // CtaRows: cta_list from the back (counts[3]; the two never meet, as each
    // listed group holds more than 32 of the n_items rows); larger: big_list.
    if (m <= CtaRows<NW>::value) {
      const bool small = m <= kSmallCta;
      const uint32_t slot = atomicAdd(a.counts + (small ? 0 : 3), 1u);
      if (slot < a.cta_cap) a.cta_list[small ? slot : a.cta_cap - 1 - slot] = make_uint2(lo, m);
      else atomicOr(a.err, kErrBounds);
    } else {
      const uint32_t slot = atomicAdd(a.counts + 1, 1u);
      if (slot < a.big_cap) a.big_list[slot] = make_uint2(lo, m);
      else atomicOr(a.err, kErrBounds);
    }
  }
}

// Each warp owns the groups whose first row lies in its chunk of kChunk rows
// and walks them in windows of up to SPAN rows made of whole groups.  SPAN is
// 64 (two rows per lane) when the read store is out of L2: the gathers of a
// window then wait on DRAM, and a window of two rows per lane puts twice as
// many in flight and spends fewer rounds on groups of 20 to 30 rows (reads at
// tens-fold coverage); with the store in L2 the ranking's instructions
// dominate and 32-row windows, with fewer of them, are faster (measured).
template <int NW, class V, int SPAN>
__device__ __forceinline__ void segsort_warp_body(const SegArgs& a) {
  using H = typename Heads<SPAN>::T;
  const int lane = threadIdx.x & 31;
  __shared__ RowWords<NW, SPAN> s_rows[8];
  RowWords<NW, SPAN>& sw = s_rows[threadIdx.x >> 5];
  const uint32_t warps = (gridDim.x * blockDim.x) >> 5;
  const uint32_t n_chunks = (a.n_items + kChunk - 1) / kChunk;
  for (uint32_t c = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; c < n_chunks; c += warps) {
    const uint32_t limit = min((c + 1) * kChunk, a.n_items);
    uint32_t cur = next_head(a, c * kChunk, lane);
    while (cur < limit) {
      // Heads among rows cur+1 .. cur+SPAN (bit r-1 for row cur+r); row
      // limit and beyond belong to the next chunk's groups, so the first
      // head at or after limit ends this chunk's last group.
      H hm = 0, past = 0;
#pragma unroll
      for (int h = 0; h < SPAN / 32; ++h) {
        const uint32_t y = cur + 1 + lane + 32u * h;
        const bool head = (y >= a.n_items) || (((a.keys[y] ^ a.keys[y - 1]) & a.key_mask) != 0u);
        hm |= H(__ballot_sync(0xFFFFFFFFu, head)) << (32 * h);
        past |= H(__ballot_sync(0xFFFFFFFFu, head && y >= limit)) << (32 * h);
      }
      if (past) hm &= (past & (~past + 1)) * 2u - 1u;  // keep bits up to the lowest one in past
      if (hm == 0) {  // the group at cur has more than SPAN rows
        const uint32_t ge = next_head(a, cur + SPAN + 1, lane);
        finish_long_group<NW, SPAN, V>(a, cur, ge, lane, sw);
        cur = ge;
        continue;
      }
      // Rows up to the last usable head; heads bit r: row cur+r starts a group.
      const uint32_t n_rows =
          uint32_t(SPAN) - (sizeof(H) == 8 ? __clzll((long long)hm) : __clz(uint32_t(hm)));
      const H heads = (hm << 1) | H(1);
      // A window of only one-row groups is already sorted.
      const H full = n_rows == uint32_t(SPAN) ? ~H(0) : ((H(1) << n_rows) - 1);
      if ((heads & full) != full) warp_rank_window<NW, SPAN, V>(a, cur, n_rows, heads, lane, sw);
      cur += n_rows;
    }
  }
}

template <int NW, class V>
__global__ void __launch_bounds__(256) k_segsort_warp(const SegArgs a) {
  segsort_warp_body<NW, V, 32>(a);
}

// The 64-row windows wait on DRAM gathers: resident warps hide that wait, so
// the registers are capped for kWideBlocks CTAs of 256 threads per SM (40
// registers; the 16 KB of shared rows per CTA allow more CTAs).  Measured on
// 5.05G repeat-rich suffixes: 145.4 ms per build uncapped (45 registers, 5
// CTAs), 137.1 ms for 6 CTAs, 141.4 ms for 8 (32 registers, more spilled).
constexpr int kWideBlocks = 6;
template <int NW, class V>
__global__ void __launch_bounds__(256, kWideBlocks) k_segsort_warp_wide(const SegArgs a) {
  segsort_warp_body<NW, V, 64>(a);
}

// Shared-memory bitonic sort of one listed group per CTA, for groups of up to
// ROWS members.  The groups come from a list of n_ptr[0] entries, read from
// the front (dir > 0) or from the back of a list of cap entries (dir < 0);
// *work hands them out.  Groups of up to kSmallCta rows run in small CTAs,
// many per SM, so that the latency of their loads and barriers overlaps.
template <int NW, class V, uint32_t ROWS, int THREADS>
__global__ void __launch_bounds__(THREADS) k_segsort_cta(const SegArgs a, const uint2* list, const uint32_t* n_ptr,
                                                         uint32_t cap, int dir, uint32_t* work) {
  constexpr uint32_t kRows = ROWS;
  extern __shared__ __align__(16) uint32_t sm[];
  V* vals = static_cast<V*>(a.vals);
  V* s_v = reinterpret_cast<V*>(sm);                                // [kRows]
  uint32_t* s_w = reinterpret_cast<uint32_t*>(s_v + kRows);         // [NW][kRows]
  uint16_t* s_perm = reinterpret_cast<uint16_t*>(s_w + NW * kRows);  // [kRows]
  __shared__ uint32_t s_item;
  const uint32_t n_list = min(*(volatile const uint32_t*)n_ptr, cap);
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) s_item = atomicAdd(work, 1u);
    __syncthreads();
    const uint32_t it = s_item;
    if (it >= n_list) break;
    const uint2 g = dir > 0 ? list[it] : list[cap - 1 - it];
    const uint32_t s = g.x, m = g.y;
    uint32_t P = 64;
    while (P < m) P <<= 1;
    for (uint32_t x = threadIdx.x; x < P; x += blockDim.x) {
      s_perm[x] = uint16_t(x);
      if (x < m) {
        const V v = vals[s + x];
        uint32_t w[NW];
        gather_words<NW>(a.R, decode(a.R, v), a.depth, w);
#pragma unroll
        for (int i = 0; i < NW; ++i) s_w[i * kRows + x] = w[i];
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
                const uint32_t a0 = s_w[i * kRows + px], b0 = s_w[i * kRows + py];
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
    for (uint32_t x = threadIdx.x; x < m; x += blockDim.x) vals[s + x] = s_v[s_perm[x]];
  }
}

// Digit counts of bases [c0, c0 + 16 * n_win) over rows [0, n) of vals: the
// per-pass histograms of the LSD passes that finish one big group.
// hist[(w * 4 + j) * 256 + digit] for window w (bases c0 + 16w ..) and digit j.
template <class V>
__global__ void k_range_hist(const V* vals, uint32_t n, ReadIndex R, uint32_t c0, uint32_t n_win, uint32_t* hist) {
  extern __shared__ uint32_t sh[];
  const uint32_t bins = n_win * 4 * kRadix;
  for (uint32_t x = threadIdx.x; x < bins; x += blockDim.x) sh[x] = 0;
  __syncthreads();
  for (uint32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
    const Suffix s = decode(R, vals[r]);
    for (uint32_t w = 0; w < n_win; ++w) {
      const uint32_t key = window16(R, s, c0 + 16u * w);
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

template <int NW, class V, uint32_t ROWS, int THREADS>
cudaError_t launch_cta_nw(const SegArgs& a, uint32_t grid, const uint2* list, const uint32_t* n_ptr, uint32_t cap,
                          int dir, uint32_t* work, cudaStream_t st) {
  const size_t smem = size_t(ROWS) * (sizeof(V) + NW * 4 + 2);
  auto kern = k_segsort_cta<NW, V, ROWS, THREADS>;
  // Set once per instantiation and device (a bit per device; racing threads
  // set the same value).
  static std::atomic<unsigned long long> configured{0};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const unsigned long long bit = 1ull << (dev & 63);
  if (!(configured.load(std::memory_order_acquire) & bit)) {
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess) return e;
    configured.fetch_or(bit, std::memory_order_release);
  }
  kern<<<grid, THREADS, smem, st>>>(a, list, n_ptr, cap, dir, work);
  return cudaGetLastError();
}

// The warp kernel, then the small-group and the large-group CTA kernels over
// the two ends of the list it fills.
template <int NW, class V>
cudaError_t launch_nw(const SegArgs& a, int sm_count, bool wide, cudaStream_t st) {
  const uint32_t n_chunks = (a.n_items + kChunk - 1) / kChunk;
  uint32_t blocks = (n_chunks + 7) / 8;
  const uint32_t cap = uint32_t(sm_count) * 16;
  if (blocks > cap) blocks = cap;
  if (blocks == 0) blocks = 1;
  // Rows of the widest keys (long reads) would not fit twice in shared memory.
  if (wide && NW <= 16) k_segsort_warp_wide<NW, V><<<blocks, 256, 0, st>>>(a);
  else k_segsort_warp<NW, V><<<blocks, 256, 0, st>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  e = launch_cta_nw<NW, V, kSmallCta, 128>(a, uint32_t(sm_count) * 16, a.cta_list, a.counts + 0, a.cta_cap, 1,
                                           a.counts + 2, st);
  if (e != cudaSuccess) return e;
  return launch_cta_nw<NW, V, CtaRows<NW>::value, 512>(a, uint32_t(sm_count) * 2, a.cta_list, a.counts + 3,
                                                        a.cta_cap, -1, a.counts + 4, st);
}

template <class V>
cudaError_t launch_v(const SegArgs& a, int nw, int sm_count, bool wide, cudaStream_t st) {
  switch (nw) {
    case 2: return launch_nw<2, V>(a, sm_count, wide, st);
    case 4: return launch_nw<4, V>(a, sm_count, wide, st);
    case 6: return launch_nw<6, V>(a, sm_count, wide, st);
    case 8: return launch_nw<8, V>(a, sm_count, wide, st);
    case 10: return launch_nw<10, V>(a, sm_count, wide, st);
    case 12: return launch_nw<12, V>(a, sm_count, wide, st);
    case 16: return launch_nw<16, V>(a, sm_count, wide, st);
    case 24: return launch_nw<24, V>(a, sm_count, wide, st);
    case 32: return launch_nw<32, V>(a, sm_count, wide, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

int segsort_words(uint32_t max_len, uint32_t depth) {
  const uint32_t rest = max_len > depth ? max_len - depth : 0;  // bases after the sorted ones
  const uint32_t nw = (rest + 15) / 16;
  if (nw <= 2) return 2;
  if (nw <= 4) return 4;
  if (nw <= 6) return 6;
  if (nw <= 8) return 8;
  if (nw <= 10) return 10;
  if (nw <= 12) return 12;
  if (nw <= 16) return 16;
  if (nw <= 24) return 24;
  if (nw <= 32) return 32;
  return 0;  // reads too long for the on-chip finish
}

cudaError_t launch_segsort(const SegArgs& a, int nw, int id_bytes, int sm_count, bool wide, cudaStream_t st) {
  return id_bytes == 8 ? launch_v<uint64_t>(a, nw, sm_count, wide, st) : launch_v<uint32_t>(a, nw, sm_count, wide, st);
}

cudaError_t launch_range_hist(const void* vals, int id_bytes, uint32_t n, const ReadIndex& R, uint32_t c0,
                              uint32_t n_win, uint32_t* hist, int sm_count, cudaStream_t st) {
  if (n == 0 || n_win == 0) return cudaSuccess;
  const size_t smem = size_t(n_win) * 4 * kRadix * 4;
  uint32_t blocks = (n + 255) / 256;
  if (blocks > uint32_t(sm_count) * 2) blocks = sm_count * 2;
  cudaError_t e;
  if (id_bytes == 8) {
    e = cudaFuncSetAttribute(k_range_hist<uint64_t>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess) return e;
    k_range_hist<uint64_t><<<blocks, 256, smem, st>>>(static_cast<const uint64_t*>(vals), n, R, c0, n_win, hist);
  } else {
    e = cudaFuncSetAttribute(k_range_hist<uint32_t>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess) return e;
    k_range_hist<uint32_t><<<blocks, 256, smem, st>>>(static_cast<const uint32_t*>(vals), n, R, c0, n_win, hist);
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_scan256<<<n_win * 4, kRadix, 0, st>>>(hist);
  return cudaGetLastError();
}

}  // namespace cxbwt
