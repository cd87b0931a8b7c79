// Device-side building blocks shared by the cxbwt kernels.
//
// Suffix encoding.  A suffix S_i[k..] $_i is carried through the sort as one
// id v = (i << shift) | (k << sym_bits) | sym, with 2^(shift - sym_bits) >
// max L_i so that k in [0, L_i] fits; the id is 32 bits while n * 2^shift <
// 2^32, else 64 bits.  Moving these values instead of the suffixes is the
// paper's "sort by index" (Section 3.2).  When sym_bits is 2 (reads of one
// length: the first digit pass generates the ids), sym is the code of the
// base before the suffix, S_i[k-1] (0 when k = 0), gathered while the ids are
// made, so that writing the BWT needs no second gather.
//
// Read store.  Bases are 2-bit codes, most significant first, reads
// concatenated (the ABI layout).  The offset and length of read i are either
// i * L and L (every read of one length L) or come from a per-read descriptor
// (offset << 16 | length).
//
// Padding.  Positions past the end of a read read as A (code 0).  An A-padded
// suffix is the smallest string that extends it, and suffixes whose padded
// keys tie are put in (length, read) order before the first pass; a stable
// LSD sort keeps that order, which realises "$ below every base" and
// "$_i < $_j for i < j" of Section 2 (the paper pads with $ and lists suffixes
// in read order, Section 3.2; with 2-bit keys there is no code left for $).
#pragma once
#include <cstdint>

namespace cxbwt {

constexpr int kRadixBits = 8;
constexpr int kRadix = 1 << kRadixBits;

// Device error word bits.
constexpr uint32_t kErrTimeout = 1u;
constexpr uint32_t kErrBounds = 2u;

struct ReadIndex {
  const uint32_t* words;  // packed store
  uint64_t n_words;
  const uint64_t* desc;   // per read: (base offset << 16) | length; nullptr when uniform
  uint32_t shift;         // v = (read << shift) | offset
  uint32_t uniform_len;   // L when desc == nullptr
  uint32_t n_reads;
  uint32_t words_aligned; // nonzero when `words` is 16-byte aligned (vector loads allowed)
  uint32_t sym_bits;      // 2 when ids carry the preceding base in their low bits, else 0
};

struct Suffix {
  uint64_t off;  // base offset of the read in the store
  uint32_t len;  // L_i
  uint32_t k;    // start position in the read
  uint32_t read; // i
};

template <class V>
__device__ __forceinline__ Suffix decode(const ReadIndex& R, V v) {
  Suffix s;
  s.read = uint32_t(v >> R.shift);
  s.k = (uint32_t(v) & ((1u << R.shift) - 1u)) >> R.sym_bits;
  if (R.desc) {
    // The clamp only matters for a corrupted value; it keeps the load in bounds.
    const uint64_t d = __ldg(R.desc + min(s.read, R.n_reads - 1u));
    s.off = d >> 16;
    s.len = uint32_t(d & 0xFFFFu);
  } else {
    s.off = uint64_t(s.read) * R.uniform_len;
    s.len = R.uniform_len;
  }
  return s;
}

__device__ __forceinline__ uint32_t load_word(const ReadIndex& R, uint64_t w) {
  return w < R.n_words ? __ldg(R.words + w) : 0u;
}

// 16 bases of suffix s starting at suffix position c0 (bases c0 .. c0+15),
// A-padded past the end of the read, as a 32-bit integer (first base in the
// top two bits).  This is the paper's "stringword" (Section 3.2), gathered by
// index from the resident store with one funnel shift.
__device__ __forceinline__ uint32_t window16(const ReadIndex& R, const Suffix& s, uint32_t c0) {
  const uint32_t rel = s.k + c0;
  if (rel >= s.len) return 0u;
  const uint32_t rem = s.len - rel;
  const uint64_t q = s.off + rel;
  const uint64_t w = q >> 4;
  const uint32_t sh = uint32_t(q & 15u) * 2u;
  uint32_t first, next;
  const uint32_t o = uint32_t(w & 3u);
  if (R.words_aligned && o < 3 && (w | 3u) < R.n_words) {
    // Both words sit in one aligned 16-byte chunk that lies wholly inside the
    // store: one load.
    const uint4 c = __ldg(reinterpret_cast<const uint4*>(R.words) + (w >> 2));
    first = o == 0 ? c.x : o == 1 ? c.y : c.z;
    next = o == 0 ? c.y : o == 1 ? c.z : c.w;
  } else {
    first = load_word(R, w);
    next = sh ? load_word(R, w + 1) : 0u;
  }
  // top 32 bits of (first:next) << sh
  uint32_t key = __funnelshift_l(next, first, sh);
  if (rem < 16u) key &= ~(0xFFFFFFFFu >> (2u * rem));
  return key;
}

// window16 for kernels that issue many gathers at once (a digit pass gathers
// one window per item, 16 per thread): two 4-byte loads, no 16-byte chunk
// (fewer registers held per load in flight) and no branch on the suffix (a
// window past the read's end reads the read's first word and is masked to
// zero), so the lanes of a warp stay together.
__device__ __forceinline__ uint32_t window16_pair(const ReadIndex& R, const Suffix& s, uint32_t c0) {
  const uint32_t rel = s.k + c0;
  const bool inside = rel < s.len;
  const uint32_t rem = inside ? s.len - rel : 0u;
  const uint64_t q = s.off + (inside ? rel : 0u);
  const uint64_t w = q >> 4;
  const uint32_t sh = uint32_t(q & 15u) * 2u;
  const uint32_t key = __funnelshift_l(load_word(R, w + 1), load_word(R, w), sh);
  // Keep the first rem bases (none when rem == 0: the shift by 0 keeps all ones).
  const uint32_t keep = rem >= 16u ? 0xFFFFFFFFu : ~(0xFFFFFFFFu >> (2u * rem));
  return key & keep;
}

// window16_pair of the suffix's first window (c0 = 0) that also returns the
// base before the suffix (S_i[k-1], 0 when k = 0).  It lies in the first word
// the window already loaded unless the suffix starts a store word (or is the
// terminator-only one): only then is one more word loaded.
__device__ __forceinline__ uint32_t window16_pair_prev(const ReadIndex& R, const Suffix& s, uint32_t* prev) {
  const bool inside = s.k < s.len;
  const uint32_t rem = inside ? s.len - s.k : 0u;
  const uint64_t q = s.off + (inside ? s.k : 0u);
  const uint64_t w = q >> 4;
  const uint32_t sh = uint32_t(q & 15u) * 2u;
  const uint32_t w0 = load_word(R, w);
  const uint32_t key = __funnelshift_l(load_word(R, w + 1), w0, sh);
  const uint32_t keep = rem >= 16u ? 0xFFFFFFFFu : ~(0xFFFFFFFFu >> (2u * rem));
  const uint64_t qp = s.off + s.k - 1;  // meaningful for k > 0
  const uint64_t wp = qp >> 4;
  const uint32_t wordp = (s.k == 0u || wp == w) ? w0 : load_word(R, wp);
  *prev = s.k ? (wordp >> (30u - 2u * uint32_t(qp & 15u))) & 3u : 0u;
  return key & keep;
}

// Code (0..3) of the base at store position q.
__device__ __forceinline__ uint32_t base_at(const ReadIndex& R, uint64_t q) {
  return (load_word(R, q >> 4) >> (30u - 2u * uint32_t(q & 15u))) & 3u;
}

__device__ __forceinline__ uint32_t lanemask_lt() {
  uint32_t m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

__device__ __forceinline__ uint64_t global_timer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void store_relaxed_u64(unsigned long long* p, unsigned long long v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ unsigned long long load_relaxed_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

}  // namespace cxbwt
