// CPU oracle for the multi-string Burrows-Wheeler transform.
//
// TEST INFRASTRUCTURE ONLY.  Nothing in the product path links, loads or calls
// this file; it is used by tests/, by the smoke check and by the CPU-baseline
// leg of the benchmark.  It shares no code with the CUDA library.
//
// What it computes is the definition of Section 2 ("Preliminaries") of
// Liu, Luo & Lam, "GPU-Accelerated BWT Construction for Large Collection of
// Short Reads" (arXiv 1401.7457), written out directly:
//
//   * R = {S_0 .. S_{n-1}}; read S_i has L_i bases over A<C<G<T and is
//     terminated by its own end marker $_i.  Every $ is smaller than every
//     base, and $_i < $_j whenever i < j (Section 2).
//   * All sum_i (L_i + 1) suffixes are listed, the terminator-only suffix of
//     each read included (Section 2; Figure 1 shows three such rows), and
//     sorted lexicographically.
//   * B_R[r] is the symbol preceding the r-th smallest suffix in its own
//     read, and $ when that suffix starts at position 0 (Section 2).
//
// The paper fixes one read length m; the same comparator is used unchanged for
// reads of different lengths.  Reads are given as ASCII over {A,C,G,T}
// (concatenated, read i at offset read_off[i]); 'A'<'C'<'G'<'T' in ASCII, so
// memcmp orders bases exactly as the alphabet does.
//
// The sort itself is a library primitive (std::sort, or the libstdc++
// parallel-mode sort when more than one thread is asked for); both produce the
// same result because the comparator is a strict total order: no two distinct
// suffixes compare equal.
//
// Entry points (extern "C", plain pointers):
//   cxo_sort      - the sorted suffix list, the BWT and nothing else.
//   cxo_rank      - how many suffixes are smaller than one given suffix.
//   cxo_check_sa  - certifies that a given suffix list is every suffix once,
//                   in strictly increasing order (a proof of sortedness that
//                   holds at any size).
//   cxo_prefix_counts, cxo_sort_range
//                 - the same sort one range of prefix buckets at a time, for
//                   collections whose whole suffix list does not fit in host
//                   memory.  Section 3.1 partitions the suffixes by their
//                   first l symbols: two suffixes whose first l symbols differ
//                   are ordered by those symbols alone, so sorting every
//                   bucket on its own and concatenating the buckets in bucket
//                   order gives the whole order.  Here a bucket is the first p
//                   symbols over $ < A < C < G < T (every position from the $
//                   on reads as $), and within a bucket the comparator below
//                   decides, unchanged.
#include <algorithm>
#include <cstdint>
#include <cstring>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#include <parallel/algorithm>
#endif

namespace {

struct Reads {
  const char* seq;        // concatenated ASCII bases
  const uint64_t* off;    // off[i] = start of read i in seq
  const uint32_t* len;    // len[i] = L_i (number of bases, no terminator)
};

struct Suffix {
  uint64_t read;  // i
  uint32_t pos;   // k in [0, L_i]; k == L_i is the terminator-only suffix
};

// Strict "less than" between suffix S_i[k..] $_i and S_j[l..] $_j (Section 2).
inline bool suffix_less(const Reads& R, const Suffix& a, const Suffix& b) {
  const uint32_t la = R.len[a.read] - a.pos;  // bases before $_i
  const uint32_t lb = R.len[b.read] - b.pos;
  const uint32_t m = la < lb ? la : lb;
  const int c = std::memcmp(R.seq + R.off[a.read] + a.pos, R.seq + R.off[b.read] + b.pos, m);
  if (c != 0) return c < 0;
  // The first m symbols agree.  The shorter suffix now shows its $, which is
  // smaller than any base.
  if (la != lb) return la < lb;
  // Both show their $ at the same place: $_i < $_j iff i < j.
  return a.read < b.read;
}

// Writes the sorted list: the suffix of each rank and its BWT symbol, the
// symbol preceding the suffix in its own read, or $ at position 0 (Section 2).
inline void write_sorted(const Reads& R, const std::vector<Suffix>& list, uint64_t* out_read, uint32_t* out_pos,
                         char* out_bwt) {
  const uint64_t total = list.size();
  for (uint64_t r = 0; r < total; ++r) {
    const Suffix& s = list[r];
    if (out_read) out_read[r] = s.read;
    if (out_pos) out_pos[r] = s.pos;
    if (out_bwt) out_bwt[r] = s.pos == 0 ? '$' : R.seq[R.off[s.read] + s.pos - 1];
  }
}

}  // namespace

extern "C" {

// Sorts every suffix of the collection and writes, for rank r = 0 .. N-1:
//   out_read[r], out_pos[r]  the suffix (i, k) of rank r   (either may be NULL)
//   out_bwt[r]               the BWT symbol, one of '$','A','C','G','T' (may be NULL)
// N = n + sum(len).  Returns N, or -1 on a bad argument.
int64_t cxo_sort(const char* seq, const uint64_t* off, const uint32_t* len, uint64_t n,
                 uint64_t* out_read, uint32_t* out_pos, char* out_bwt, int threads) {
  if (!seq || !off || !len) return -1;
  const Reads R{seq, off, len};
  std::vector<Suffix> list;
  uint64_t total = 0;
  for (uint64_t i = 0; i < n; ++i) total += uint64_t(len[i]) + 1;
  list.reserve(total);
  for (uint64_t i = 0; i < n; ++i)
    for (uint32_t k = 0; k <= len[i]; ++k) list.push_back(Suffix{i, k});
  auto cmp = [&R](const Suffix& a, const Suffix& b) { return suffix_less(R, a, b); };
#ifdef _OPENMP
  if (threads > 1) {
    omp_set_num_threads(threads);
    __gnu_parallel::sort(list.begin(), list.end(), cmp);
  } else {
    std::sort(list.begin(), list.end(), cmp);
  }
#else
  (void)threads;
  std::sort(list.begin(), list.end(), cmp);
#endif
  write_sorted(R, list, out_read, out_pos, out_bwt);
  return int64_t(total);
}

// Number of suffixes of the collection strictly smaller than suffix (read, pos),
// i.e. its rank in the sorted list.  Returns -1 on a bad argument.
int64_t cxo_rank(const char* seq, const uint64_t* off, const uint32_t* len, uint64_t n,
                 uint64_t read, uint32_t pos, int threads) {
  if (!seq || !off || !len || read >= n || pos > len[read]) return -1;
  const Reads R{seq, off, len};
  const Suffix q{read, pos};
  int64_t count = 0;
#ifdef _OPENMP
  if (threads > 0) omp_set_num_threads(threads);
#pragma omp parallel for reduction(+ : count) schedule(dynamic, 4096)
#endif
  for (int64_t i = 0; i < int64_t(n); ++i)
    for (uint32_t k = 0; k <= len[i]; ++k)
      if (suffix_less(R, Suffix{uint64_t(i), k}, q)) ++count;
  (void)threads;
  return count;
}

// Certificate of a claimed suffix order (sa_read[r], sa_pos[r]), r < N:
//   every entry names a suffix of the collection, every suffix appears exactly
//   once (N = n + sum(len) entries, none repeated), and each entry is strictly
//   smaller than the next under the definition's order.
// Returns -1 when all holds; otherwise the first rank r at which it fails
// (for the order check, r is the index of the left element of the bad pair),
// or -2 for a bad argument or a wrong N.
int64_t cxo_check_sa(const char* seq, const uint64_t* off, const uint32_t* len, uint64_t n,
                     const uint64_t* sa_read, const uint32_t* sa_pos, uint64_t N, int threads) {
  if (!seq || !off || !len || !sa_read || !sa_pos) return -2;
  uint64_t total = 0;
  for (uint64_t i = 0; i < n; ++i) total += uint64_t(len[i]) + 1;
  if (N != total) return -2;
  const Reads R{seq, off, len};
  // Suffix (i, k) owns slot off[i] + i + k of a bitmap over all N suffixes.
  std::vector<uint8_t> seen(N, 0);
  for (uint64_t r = 0; r < N; ++r) {
    const uint64_t i = sa_read[r];
    if (i >= n || sa_pos[r] > len[i]) return int64_t(r);
    uint8_t& s = seen[off[i] + i + sa_pos[r]];
    if (s) return int64_t(r);
    s = 1;
  }
  int64_t first_bad = -1;
  const int64_t last = int64_t(N) - 1;  // pairs (r, r + 1) for r < last
#ifdef _OPENMP
  if (threads > 0) omp_set_num_threads(threads);
#pragma omp parallel for schedule(static, 65536)
#endif
  for (int64_t r = 0; r < last; ++r) {
    if (!suffix_less(R, Suffix{sa_read[r], sa_pos[r]}, Suffix{sa_read[r + 1], sa_pos[r + 1]})) {
#ifdef _OPENMP
#pragma omp critical
#endif
      {
        if (first_bad < 0 || r < first_bad) first_bad = r;
      }
    }
  }
  (void)threads;
  return first_bad;
}

// Bucket of suffix (i, k): its first p symbols, each $ = 0, A = 1, C = 2,
// G = 3, T = 4, as a base-5 number with the first symbol most significant;
// every position from the $ on is 0 (the suffix has ended there).
static inline uint64_t prefix_bucket(const char* seq, const uint64_t* off, const uint32_t* len, uint64_t i,
                                     uint32_t k, int p) {
  uint64_t code = 0;
  for (int t = 0; t < p; ++t) {
    uint64_t s = 0;
    if (k + uint32_t(t) < len[i]) {
      switch (seq[off[i] + k + t]) {
        case 'A': s = 1; break;
        case 'C': s = 2; break;
        case 'G': s = 3; break;
        default: s = 4; break;  // 'T'
      }
    }
    code = code * 5 + s;
  }
  return code;
}

// counts[b] = number of suffixes in bucket b, for b < 5^p (1 <= p <= 12).
// Returns N, or -1 on a bad argument.
int64_t cxo_prefix_counts(const char* seq, const uint64_t* off, const uint32_t* len, uint64_t n, int p,
                          uint64_t* counts, int threads) {
  if (!seq || !off || !len || !counts || p < 1 || p > 12) return -1;
  uint64_t buckets = 1;
  for (int t = 0; t < p; ++t) buckets *= 5;
  std::memset(counts, 0, buckets * sizeof(uint64_t));
  uint64_t total = 0;
#ifdef _OPENMP
  if (threads > 0) omp_set_num_threads(threads);
#pragma omp parallel
#endif
  {
    std::vector<uint64_t> mine(buckets, 0);
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 4096) nowait
#endif
    for (int64_t i = 0; i < int64_t(n); ++i)
      for (uint32_t k = 0; k <= len[i]; ++k) ++mine[prefix_bucket(seq, off, len, uint64_t(i), k, p)];
#ifdef _OPENMP
#pragma omp critical
#endif
    for (uint64_t b = 0; b < buckets; ++b) counts[b] += mine[b];
  }
  (void)threads;
  for (uint64_t b = 0; b < buckets; ++b) total += counts[b];
  return int64_t(total);
}

// Sorts the suffixes whose bucket (first p symbols, as above) lies in
// [bucket_lo, bucket_hi) and writes them, smallest first, as cxo_sort does
// (out_read, out_pos, out_bwt: `capacity` entries each, any may be NULL).
// Their ranks in the whole order are those of cxo_sort offset by the number
// of suffixes in the buckets below bucket_lo.  Returns the number written,
// -1 on a bad argument, or -2 when they are more than `capacity`.
int64_t cxo_sort_range(const char* seq, const uint64_t* off, const uint32_t* len, uint64_t n, int p,
                       uint64_t bucket_lo, uint64_t bucket_hi, uint64_t capacity, uint64_t* out_read,
                       uint32_t* out_pos, char* out_bwt, int threads) {
  if (!seq || !off || !len || p < 1 || p > 12 || bucket_lo > bucket_hi) return -1;
  const Reads R{seq, off, len};
  std::vector<Suffix> list;
  // List the range's suffixes (in read order; the sort decides the rest).
  {
    int nt = 1;
#ifdef _OPENMP
    if (threads > 0) omp_set_num_threads(threads);
    nt = threads > 0 ? threads : omp_get_max_threads();
#endif
    std::vector<std::vector<Suffix>> parts(static_cast<size_t>(nt));
#ifdef _OPENMP
#pragma omp parallel num_threads(nt)
#endif
    {
      int me = 0;
#ifdef _OPENMP
      me = omp_get_thread_num();
#endif
      std::vector<Suffix>& mine = parts[size_t(me)];
      const uint64_t lo = n * uint64_t(me) / uint64_t(nt), hi = n * uint64_t(me + 1) / uint64_t(nt);
      for (uint64_t i = lo; i < hi; ++i)
        for (uint32_t k = 0; k <= len[i]; ++k) {
          const uint64_t b = prefix_bucket(seq, off, len, i, k, p);
          if (b >= bucket_lo && b < bucket_hi) mine.push_back(Suffix{i, k});
        }
    }
    uint64_t total = 0;
    for (const auto& v : parts) total += v.size();
    if (total > capacity) return -2;
    list.reserve(total);
    for (auto& v : parts) {
      list.insert(list.end(), v.begin(), v.end());
      std::vector<Suffix>().swap(v);
    }
  }
  auto cmp = [&R](const Suffix& a, const Suffix& b) { return suffix_less(R, a, b); };
#ifdef _OPENMP
  if (threads > 1) {
    omp_set_num_threads(threads);
    __gnu_parallel::sort(list.begin(), list.end(), cmp);
  } else {
    std::sort(list.begin(), list.end(), cmp);
  }
#else
  std::sort(list.begin(), list.end(), cmp);
#endif
  write_sorted(R, list, out_read, out_pos, out_bwt);
  return int64_t(list.size());
}

}  // extern "C"
