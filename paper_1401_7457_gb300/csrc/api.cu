// The C ABI of include/cxbwt.h: validation, device workspace, the plan of a
// build, launches, and the host helpers.
//
// A build sorts one or more "slices" of the suffixes and emits each slice's
// part of the BWT at its global row offset.  A slice is the whole collection
// when its workspace fits the device budget; otherwise the planner of Figure
// 2 steps 1-3 applies: the suffixes of every bucket are counted (first 4
// bases, summed from the per-position 4-mer counts; first 8 bases, one count
// per suffix, when a 4-base bucket is larger than a slice, and always for a
// bucket-range part), consecutive buckets are packed into slices of at most
// m1 suffixes (m1 from the budget), and each slice rescans all suffixes
// keeping those of its buckets (the listing of step 3(a)).  Per slice, on the
// caller's stream:
//   1. digit histograms: k_poscount + k_digitbase (whole collection) or
//      k_pass_hist (the slice's buckets) - the first output row of every digit
//      value of every pass;
//   2. the (suffix length, read) start order: generated inside the first
//      digit pass for reads of one length (in read-major order plus a
//      suffix-length digit when the store is too big for L2), or k_identity
//      plus length passes for mixed lengths;
//   3. the LSD digit passes (Section 3.2), least significant 4-base digit
//      first, each 16-base stringword window gathered once and carried in the
//      key array for its remaining passes - every window (LSD plan) or only
//      the first (group plan, followed by the on-chip group finish);
//   4. emission (Figure 2 step 3(c)(iii)), with the preceding base carried
//      in the ids when the store is out of L2; with host outputs, the
//      finished words of each slice stream to the host on a side stream while
//      the next slice sorts.
#include "host.cuh"

using namespace cxbwt;
using namespace cxbwt::host;

namespace {
thread_local std::string g_create_error;
}  // namespace


namespace cxbwt {
namespace host {

// The listing kernel (k_list.cu) lists a build's slices: reads of one length
// of at most 255 bases, unless the plan flags ask for the digit pass.
static bool list_kernel(const cxbwt_ctx* c, const Plan& pl) {
  return pl.uniform && pl.Lmax <= 255 && !(c->opt.plan_flags & CXBWT_PLAN_DIGIT_LISTING);
}

// Tiles of the pass with the most of them: the generating digit passes
// (every suffix, TILE per tile) or the listing kernel (whole reads per tile).
static uint64_t status_tiles(const cxbwt_ctx* c, const Plan& pl, uint32_t TILE) {
  uint64_t t = (pl.N + TILE - 1) / TILE;
  if (list_kernel(c, pl)) {
    const uint64_t rpt = list_reads_per_tile(pl.Lmax);
    t = std::max<uint64_t>(t, (pl.n + rpt - 1) / rpt);
  }
  return t;
}

// Sort the slice's suffixes into r.vals[cur]; returns cur (0 or 1) through
// *cur_out.  tev (or nullptr): events recorded before the digit passes and
// after them.
int sort_slice(cxbwt_ctx* c, Run& r, const Slice& sl, int* cur_out, cudaEvent_t* tev) {
  const Plan& pl = r.pl;
  cudaStream_t st = r.st;
  const uint32_t TILE = uint32_t(r.shape.tile());
  PassArgs a{};
  a.status = static_cast<unsigned long long*>(c->status.p);
  a.tile_counter = r.d_counter;
  a.err = r.d_err;
  a.R = r.R;
  a.n_reads = uint32_t(pl.n);
  a.timeout_ns = c->opt.wait_limit_ms > 0 ? uint64_t(c->opt.wait_limit_ms) * 1000000ull : kTimeoutNs;
  a.key_lo = sl.key_lo;
  a.key_last = uint32_t(sl.key_hi - 1 - sl.key_lo);  // the offset of its last key (a part may span every key)
  a.prefetch = (c->opt.plan_flags & CXBWT_PLAN_NO_PREFETCH) ? 0u : 1u;
  const uint32_t d_sorted = std::min<uint32_t>(pl.D, 4 * (pl.w_last + 1));

  // ---- digit bases -----------------------------------------------------------
  // whole: rows 0..d_sorted-1 = char digits d, rows D.. = length digits.
  // slice: row 0 = suffix length (its low byte), rows 1..4 = window-0 digits
  // (most significant first), row 5 = the high byte of the suffix length.
  if (sl.pregen) {
    // The slice's first windows are listed already: count their digits (rows 1..4).
    CX_CUDA(c, cudaMemsetAsync(r.base + kRadix, 0, 4 * kRadix * 4, st));
    CX_CUDA(c, launch_key_hist(r.keys[0], sl.rows, r.base + kRadix, c->sm_count, st));
    r.launches += 2;
  } else if (sl.whole) {
    CX_CUDA(c, cudaMemsetAsync(c->P.p, 0, uint64_t(pl.Lmax) * kRadix * 4, st));
    CX_CUDA(c, launch_poscount(r.R, uint32_t(pl.n), pl.Lmax, static_cast<uint32_t*>(c->P.p), c->sm_count, st));
    CX_CUDA(c, launch_digitbase(static_cast<const uint32_t*>(c->P.p), pl.Lmax, d_sorted, pl.uniform ? 1 : 0,
                                uint32_t(pl.n), pl.Lmax, static_cast<const uint32_t*>(c->lenhist.p), r.base, st));
    r.launches += 2;
  } else {
    CX_CUDA(c, cudaMemsetAsync(r.base, 0, 6 * kRadix * 4, st));
    CX_CUDA(c, launch_pass_hist(r.R, uint32_t(pl.n), sl.key_lo, uint32_t(sl.key_hi - 1 - sl.key_lo), r.base,
                                c->sm_count, st));
    r.launches += 2;
  }
  auto digit_base = [&](uint32_t d) -> const uint32_t* {  // char digit d of window 0 (or any window when whole)
    if (sl.whole) return r.base + size_t(d) * kRadix;
    return r.base + size_t(1 + d) * kRadix;  // d in 0..3
  };

  if (tev) CX_CUDA(c, cudaEventRecord(tev[0], st));
  int cur = 0, kin = 0;
  const int idb = pl.idb;
  bool first = pl.uniform;  // the first digit pass generates the start order
  bool listed = sl.pregen;  // window 0 is already in the key array, in (length, read) order
  a.n_gen = pl.N;  // generated passes enumerate every suffix (a slice's pass filters them)
  a.n_out = sl.rows;
  a.n_tiles = uint32_t((pl.N + TILE - 1) / TILE);
  if (!pl.uniform && !sl.whole) {
    // A slice of a collection of mixed read lengths: every suffix listed in
    // read-major order, the slice's kept with window 0, stably ordered by the
    // low byte of the suffix length, then by its high byte.
    a.vals_in = nullptr;
    a.vals_out = r.vals[cur ^ 1];
    a.keys_in = nullptr;
    a.keys_out = r.keys[kin];
    a.digit_base = r.base;  // row 0: low byte of the suffix length
    a.key_shift = 0;
    a.window_c0 = 0;
    a.epoch = ++c->epoch;
    if (tev) CX_TRY(pass_event_begin(c, r));
    CX_CUDA(c, launch_onesweep(a, kSrcInitMixed, true, true, idb, r.shape, st));
    if (tev) CX_TRY(pass_event_end(c, r, 0));
    cur ^= 1;
    ++r.sort_launches;
    r.sort_items += sl.rows;
    if (pl.Lmax > 255) {
      a.n_gen = sl.rows;
      a.n_tiles = uint32_t((uint64_t(sl.rows) + TILE - 1) / TILE);
      a.vals_in = r.vals[cur];
      a.vals_out = r.vals[cur ^ 1];
      a.keys_in = r.keys[kin];
      a.keys_out = r.keys[kin ^ 1];
      a.digit_base = r.base + 5 * size_t(kRadix);  // row 5: high byte of the suffix length
      a.key_shift = 8;
      a.epoch = ++c->epoch;
      CX_CUDA(c, launch_onesweep(a, kSrcCarriedLength, true, false, idb, r.shape, st));
      cur ^= 1;
      kin ^= 1;
      ++r.sort_launches;
      r.sort_items += sl.rows;
    }
    listed = true;
    first = false;
  } else if (!pl.uniform) {
    // Mixed lengths (whole collection only): id list in read order, then
    // stable passes over the suffix length.
    CX_CUDA(c, launch_identity(r.R, uint32_t(pl.n), r.vals[0], idb, st));
    ++r.launches;
    a.n_gen = sl.rows;
    a.n_tiles = uint32_t((uint64_t(sl.rows) + TILE - 1) / TILE);
    for (uint32_t j = 0; j < pl.len_passes; ++j) {
      a.vals_in = r.vals[cur];
      a.vals_out = r.vals[cur ^ 1];
      a.keys_in = nullptr;
      a.keys_out = nullptr;
      a.digit_base = r.base + size_t(pl.D + j) * kRadix;
      a.key_shift = 8 * j;
      a.window_c0 = 0;
      a.epoch = ++c->epoch;
      CX_CUDA(c, launch_onesweep(a, kSrcLength, false, false, idb, r.shape, st));
      cur ^= 1;
      ++r.sort_launches;
      r.sort_items += sl.rows;
    }
  } else if (r.read_major && !sl.pregen && list_kernel(c, pl)) {
    // Read-major listing of the slice's suffixes (the store read in address
    // order), ordered by suffix length, window 0 carried: the listing kernel
    // with one key range.
    ListArgs la{};
    la.R = r.R;
    la.n_reads = uint32_t(pl.n);
    la.reads_per_tile = list_reads_per_tile(pl.Lmax);
    la.n_tiles = uint32_t((pl.n + la.reads_per_tile - 1) / la.reads_per_tile);
    la.stage_rows = la.reads_per_tile * (pl.Lmax + 1);
    la.n_slices = 1;
    la.key_lo[0] = sl.key_lo;
    la.key_last[0] = a.key_last;
    la.vals[0] = r.vals[cur ^ 1];
    la.keys[0] = r.keys[kin];
    la.rows[0] = sl.rows;
    la.digit_base = r.base;  // row 0: suffix length
    la.status = a.status;
    la.tile_counter = a.tile_counter;
    la.err = a.err;
    la.epoch = ++c->epoch;
    la.timeout_ns = a.timeout_ns;
    la.prefetch = a.prefetch;
    if (tev) CX_TRY(pass_event_begin(c, r));
    CX_CUDA(c, launch_list(la, idb, st));
    if (tev) CX_TRY(pass_event_end(c, r, 0));
    cur ^= 1;
    ++r.sort_launches;
    r.sort_items += sl.rows;
    first = false;
  } else if (r.read_major && !sl.pregen) {
    // Read-major generated order (the store is read in address order),
    // filtered to the slice, stably sorted by suffix length, window 0 carried.
    a.vals_in = nullptr;
    a.vals_out = r.vals[cur ^ 1];
    a.keys_in = nullptr;
    a.keys_out = r.keys[kin];
    a.digit_base = r.base;  // row 0: suffix length
    a.key_shift = 0;
    a.window_c0 = 0;
    a.epoch = ++c->epoch;
    if (tev) CX_TRY(pass_event_begin(c, r));
    CX_CUDA(c, launch_onesweep(a, kSrcInitReadMajor, true, !sl.whole, idb, r.shape, st));
    if (tev) CX_TRY(pass_event_end(c, r, 0));
    cur ^= 1;
    ++r.sort_launches;
    r.sort_items += sl.rows;
    first = false;
  }
  for (int64_t w = int64_t(pl.w_last); w >= 0; --w) {
    // The group plan sorts the first l = depth bases of window 0 (4 bases per
    // digit): 4 passes for l = 16, 3 for l = 12.
    const uint32_t w_digits = (pl.groups && w == 0) ? pl.depth / 4 : 4u;
    const uint32_t d_lo = uint32_t(4 * w);
    const uint32_t d_hi = std::min<uint32_t>(d_lo + w_digits - 1, pl.D - 1);
    for (int64_t d = d_hi; d >= int64_t(d_lo); --d) {
      const bool first_in_window = (uint32_t(d) == d_hi);
      const bool last_in_window = (uint32_t(d) == d_lo);
      const bool carried = !first_in_window || (w == 0 && (listed || (r.read_major && pl.uniform)));
      const int mode = carried ? kSrcCarried : (first ? kSrcInitUniform : kSrcExtract);
      // The group plan keeps the window-0 keys of the final order: groups are runs of equal keys.
      const bool write_key = !last_in_window || pl.groups;
      const bool generated = (mode == kSrcInitUniform);
      a.n_gen = generated ? pl.N : sl.rows;
      a.n_tiles = uint32_t((a.n_gen + TILE - 1) / TILE);
      a.vals_in = generated ? nullptr : r.vals[cur];
      a.vals_out = r.vals[cur ^ 1];
      a.keys_in = (mode == kSrcCarried) ? r.keys[kin] : nullptr;
      const int kout = (mode == kSrcCarried) ? (kin ^ 1) : kin;
      a.keys_out = write_key ? r.keys[kout] : nullptr;
      a.digit_base = digit_base(uint32_t(d));
      a.key_shift = 24u - 8u * uint32_t(d - d_lo);
      a.window_c0 = uint32_t(16 * w);
      a.epoch = ++c->epoch;
      a.stall_tile0 = (c->opt.plan_flags & CXBWT_PLAN_TEST_STALL) && r.sort_launches == 0 ? 1u : 0u;
      if (tev) CX_TRY(pass_event_begin(c, r));
      CX_CUDA(c, launch_onesweep(a, mode, write_key, generated && !sl.whole, idb, r.shape, st));
      if (tev) CX_TRY(pass_event_end(c, r, mode == kSrcCarried ? 1 : 0));
      a.stall_tile0 = 0;
      if (mode == kSrcCarried) {
        ++r.carried_launches;
        r.carried_items += sl.rows;
      }
      cur ^= 1;
      if (write_key) kin = kout;
      first = false;
      ++r.sort_launches;
      r.sort_items += sl.rows;
    }
  }
  if (tev) CX_CUDA(c, cudaEventRecord(tev[1], st));

  // ---- group plan: finish every group of equal first l bases on chip --------
  if (pl.groups && pl.Lmax > pl.depth) {
    const uint64_t cta_cap = cta_list_cap(sl.rows), big_cap = big_list_cap(sl.rows, pl.seg_words);
    CX_CUDA(c, cudaMemsetAsync(r.d_seg, 0, 32, st));
    SegArgs g{};
    g.keys = r.keys[kin];
    g.vals = r.vals[cur];
    g.n_items = sl.rows;
    g.R = r.R;
    g.depth = pl.depth;
    g.key_mask = depth_mask(pl.depth);
    g.cta_list = static_cast<uint2*>(c->seglist.p);
    g.cta_cap = uint32_t(cta_cap);
    g.big_list = g.cta_list + cta_cap;
    g.big_cap = uint32_t(big_cap);
    g.counts = r.d_seg;
    g.err = r.d_err;
    CX_CUDA(c, launch_segsort(g, pl.seg_words, idb, c->sm_count, pl.n_words * 4 > (64u << 20), st));
    r.launches += 2;
    // Remainders too large for one CTA (rare: long runs of equal bases) are
    // finished here with LSD passes over bases l.. restricted to their rows.
    CX_CUDA(c, cudaMemcpyAsync(c->h_small + 5, r.d_seg, 16, cudaMemcpyDeviceToHost, st));
    CX_CUDA(c, cudaStreamSynchronize(st));
    const uint32_t n_big = std::min<uint32_t>(reinterpret_cast<const uint32_t*>(c->h_small + 5)[1], g.big_cap);
    c->stats.cta_groups += uint64_t(reinterpret_cast<const uint32_t*>(c->h_small + 5)[0]) +
                           reinterpret_cast<const uint32_t*>(c->h_small + 5)[3];
    c->stats.big_groups += n_big;
    if (n_big) {
      std::vector<uint2> big(n_big);
      CX_CUDA(c, cudaMemcpyAsync(big.data(), g.big_list, n_big * 8, cudaMemcpyDeviceToHost, st));
      CX_CUDA(c, cudaStreamSynchronize(st));
      r.d2h += n_big * 8;
      // Windows of bases [l + 16u, l + 16u + 16), u < n_win, cover bases l .. Lmax-1.
      const uint32_t n_win = (pl.Lmax - pl.depth + 15) / 16;
      auto* rh = static_cast<uint32_t*>(c->rhist.p);
      for (const uint2& bg : big) {
        const uint32_t s0 = bg.x, m = bg.y;
        CX_CUDA(c, cudaMemsetAsync(rh, 0, size_t(n_win) * 4 * kRadix * 4, st));
        CX_CUDA(c, launch_range_hist(vptr(r.vals[cur], idb, s0), idb, m, r.R, pl.depth, n_win, rh, c->sm_count, st));
        r.launches += 2;
        void* gv[2] = {vptr(r.vals[cur], idb, s0), vptr(r.vals[cur ^ 1], idb, s0)};
        uint32_t* gk[2] = {r.keys[0] + s0, r.keys[1] + s0};
        int gc = 0, gki = 0;
        PassArgs b = a;
        b.n_gen = m;
        b.n_out = m;
        b.n_tiles = uint32_t((m + TILE - 1) / TILE);
        for (uint32_t u = n_win; u-- > 0;) {
          const uint32_t c0 = pl.depth + 16 * u;
          const uint32_t n_dig = std::min<uint32_t>(4, (pl.Lmax - c0 + 3) / 4);  // digits holding bases < Lmax
          for (int64_t j = int64_t(n_dig) - 1; j >= 0; --j) {
            const bool first_in_window = (uint32_t(j) == n_dig - 1);
            const bool last_in_window = (j == 0);
            const int mode = first_in_window ? kSrcExtract : kSrcCarried;
            const bool write_key = !last_in_window;
            b.vals_in = gv[gc];
            b.vals_out = gv[gc ^ 1];
            b.keys_in = (mode == kSrcCarried) ? gk[gki] : nullptr;
            const int kout = (mode == kSrcCarried) ? (gki ^ 1) : gki;
            b.keys_out = write_key ? gk[kout] : nullptr;
            b.digit_base = rh + size_t(u * 4 + uint32_t(j)) * kRadix;
            b.key_shift = 24u - 8u * uint32_t(j);
            b.window_c0 = c0;
            b.epoch = ++c->epoch;
            CX_CUDA(c, launch_onesweep(b, mode, write_key, false, idb, r.shape, st));
            gc ^= 1;
            if (write_key) gki = kout;
            ++r.sort_launches;
            r.sort_items += m;
          }
        }
        if (gc) CX_CUDA(c, cudaMemcpyAsync(gv[0], gv[1], size_t(m) * idb, cudaMemcpyDeviceToDevice, st));
      }
    }
  }
  *cur_out = cur;
  return CXBWT_OK;
}

// The one generating pass of a build in several slices of 4-base buckets:
// every suffix is listed, in read-major order with its first window, into
// its slice's part of r.vals[0] / r.keys[0] (slice s at rows [row0_s,
// row0_s + rows_s)), stably ordered by suffix length inside the slice, which
// with the read-major order gives the (suffix length, read) start order the
// slice's window passes need.  The digit is (slice, suffix length); its
// first output rows follow from the per-position 4-mer counts P that planned
// the slices: suffix (i, k) has length L - k and first 4 bases = the 4-mer of
// read i at position k, and the n terminator-only suffixes fall in bucket 0.
int split_pass(cxbwt_ctx* c, Run& r, const std::vector<Slice>& slices, const std::vector<uint32_t>& P, bool timing) {
  const Plan& pl = r.pl;
  const uint32_t L = pl.Lmax, L1 = L + 1, S = uint32_t(slices.size());
  std::vector<uint8_t> split_of(kRadix, 0);
  for (uint32_t si = 0; si < S; ++si)
    for (uint64_t b = slices[si].key_lo >> 24; b < (slices[si].key_hi >> 24); ++b) split_of[b] = uint8_t(si);
  std::vector<uint64_t> cnt(size_t(S) * L1, 0);
  cnt[size_t(split_of[0]) * L1] += pl.n;
  for (uint32_t t = 1; t <= L; ++t)
    for (int v = 0; v < kRadix; ++v) cnt[size_t(split_of[v]) * L1 + t] += P[size_t(L - t) * kRadix + v];
  std::vector<uint32_t> sbase(kRadix, 0);
  for (uint32_t si = 0; si < S; ++si) {
    uint64_t acc = 0;
    for (uint32_t t = 0; t < L1; ++t) {
      sbase[si * L1 + t] = uint32_t(acc);
      acc += cnt[size_t(si) * L1 + t];
    }
    if (acc != slices[si].rows)
      return fail(c, CXBWT_EINTERNAL, "slice %u: %llu listed suffixes, %u planned", si, (unsigned long long)acc,
                  slices[si].rows);
  }
  uint32_t* d_sbase = r.base + size_t(std::max<uint32_t>(pl.D + pl.len_passes, 5)) * kRadix;
  uint8_t* d_split = reinterpret_cast<uint8_t*>(d_sbase + kRadix);
  CX_CUDA(c, cudaMemcpyAsync(d_sbase, sbase.data(), kRadix * 4, cudaMemcpyHostToDevice, r.st));
  if (list_kernel(c, pl)) {
    ListArgs la{};
    la.R = r.R;
    la.n_reads = uint32_t(pl.n);
    la.reads_per_tile = list_reads_per_tile(L);
    la.n_tiles = uint32_t((pl.n + la.reads_per_tile - 1) / la.reads_per_tile);
    la.stage_rows = la.reads_per_tile * L1;
    la.n_slices = S;
    for (uint32_t si = 0; si < S; ++si) {
      la.key_lo[si] = slices[si].key_lo;
      la.key_last[si] = uint32_t(slices[si].key_hi - 1 - slices[si].key_lo);
      la.vals[si] = vptr(c->vals[0].p, pl.idb, slices[si].arr0);
      la.keys[si] = static_cast<uint32_t*>(c->keys[0].p) + slices[si].arr0;
      la.rows[si] = slices[si].rows;
    }
    la.digit_base = d_sbase;
    la.status = static_cast<unsigned long long*>(c->status.p);
    la.tile_counter = r.d_counter;
    la.err = r.d_err;
    la.epoch = ++c->epoch;
    la.timeout_ns = c->opt.wait_limit_ms > 0 ? uint64_t(c->opt.wait_limit_ms) * 1000000ull : kTimeoutNs;
    la.prefetch = (c->opt.plan_flags & CXBWT_PLAN_NO_PREFETCH) ? 0u : 1u;
    if (timing) CX_TRY(pass_event_begin(c, r));
    CX_CUDA(c, launch_list(la, pl.idb, r.st));
    if (timing) CX_TRY(pass_event_end(c, r, 2));
    ++r.sort_launches;
    r.sort_items += pl.N;
    r.read_major = true;
    return CXBWT_OK;
  }
  CX_CUDA(c, cudaMemcpyAsync(d_split, split_of.data(), kRadix, cudaMemcpyHostToDevice, r.st));
  const uint32_t TILE = uint32_t(r.shape.tile());
  PassArgs a{};
  a.status = static_cast<unsigned long long*>(c->status.p);
  a.tile_counter = r.d_counter;
  a.err = r.d_err;
  a.R = r.R;
  a.n_reads = uint32_t(pl.n);
  a.timeout_ns = c->opt.wait_limit_ms > 0 ? uint64_t(c->opt.wait_limit_ms) * 1000000ull : kTimeoutNs;
  a.n_gen = pl.N;
  a.n_out = 0;  // every row goes to a slice's own arrays
  a.n_tiles = uint32_t((pl.N + TILE - 1) / TILE);
  a.digit_base = d_sbase;
  a.split_of = d_split;
  for (uint32_t si = 0; si < S; ++si) {
    a.split_vals[si] = vptr(c->vals[0].p, pl.idb, slices[si].arr0);
    a.split_keys[si] = static_cast<uint32_t*>(c->keys[0].p) + slices[si].arr0;
    a.split_rows[si] = slices[si].rows;
  }
  a.epoch = ++c->epoch;
  if (timing) CX_TRY(pass_event_begin(c, r));
  CX_CUDA(c, launch_onesweep(a, kSrcInitSplit, true, false, pl.idb, r.shape, r.st));
  if (timing) CX_TRY(pass_event_end(c, r, 2));
  ++r.sort_launches;
  r.sort_items += pl.N;
  r.read_major = true;
  return CXBWT_OK;
}

int build_impl(cxbwt_ctx* c, const uint32_t* reads, uint64_t n, const uint32_t* lens, uint32_t* out_bwt,
               uint64_t* out_dollar, uint64_t* out_counts, uint64_t* out_sa, void* stream_v, const PartSpec* part) {
  if (!c) return CXBWT_EINVAL;
  c->err.clear();
  const bool counts_only = part && part->counts_only;
  if (!reads || !lens || (!out_bwt && !counts_only))
    return fail(c, CXBWT_EINVAL, "reads_2bit, lens and out_bwt must not be NULL");
  if (part && !counts_only && (part->lo >= part->hi || part->hi > (1u << kBucketBits) || out_sa))
    return fail(c, CXBWT_EINVAL, "a part needs buckets lo < hi <= %u and no suffix array output", 1u << kBucketBits);
  if (n == 0) return fail(c, CXBWT_EINVAL, "n_reads must be at least 1");
  // (the generated start order steps read indices by 32 in 32 bits)
  if (n > (uint64_t(1) << 32) - 64) return fail(c, CXBWT_EUNSUPPORTED, "more than 2^32 - 64 reads in one build");
  CX_CUDA(c, cudaSetDevice(c->device));
  cudaStream_t st = static_cast<cudaStream_t>(stream_v);
  c->last_stream = st;

  const bool reads_dev = is_device_ptr(reads), lens_dev = is_device_ptr(lens);
  const bool bwt_dev = out_bwt && is_device_ptr(out_bwt);
  const bool dollar_dev = out_dollar && is_device_ptr(out_dollar);
  const bool counts_dev = out_counts && is_device_ptr(out_counts);
  const bool sa_dev = out_sa && is_device_ptr(out_sa);
  Run r;
  r.st = st;
  uint64_t h2d = 0;

  CX_TRY(ensure(c, c->misc, kMiscBytes, "scratch words"));
  char* misc = static_cast<char*>(c->misc.p);
  r.d_err = reinterpret_cast<uint32_t*>(misc + kMiscErr);
  r.d_counter = reinterpret_cast<uint32_t*>(misc + kMiscTileCounter);
  r.d_counts = reinterpret_cast<unsigned long long*>(misc + kMiscCounts);
  r.d_seg = reinterpret_cast<uint32_t*>(misc + kMiscSeg);
  auto* d_lstats = reinterpret_cast<unsigned long long*>(misc + kMiscLenStats);

  // ---- read lengths ------------------------------------------------------
  Plan& pl = r.pl;
  pl.n = n;
  std::vector<uint32_t> lens_copy;
  const uint32_t* hlens = lens_dev ? nullptr : lens;
  // Lengths in pinned host memory are scanned on the device (one fast copy
  // and a reduction instead of a serial host loop); pageable ones on the host.
  const uint32_t* dlens = lens_dev ? lens : nullptr;
  if (hlens && is_pinned_ptr(hlens)) {
    CX_TRY(ensure(c, c->desc, n * 4, "read lengths"));
    CX_CUDA(c, cudaMemcpyAsync(c->desc.p, hlens, n * 4, cudaMemcpyHostToDevice, st));
    h2d += n * 4;
    dlens = static_cast<const uint32_t*>(c->desc.p);
  }
  uint64_t mn = ~0ull, mx = 0, sum = 0, bad = 0;
  if (!dlens) {
    for (uint64_t i = 0; i < n; ++i) {
      const uint32_t L = hlens[i];
      mn = std::min<uint64_t>(mn, L);
      mx = std::max<uint64_t>(mx, L);
      sum += L;
      bad += (L == 0 || L > 65535) ? 1 : 0;
    }
  } else {
    const unsigned long long init[4] = {~0ull, 0, 0, 0};
    CX_CUDA(c, cudaMemcpyAsync(d_lstats, init, sizeof init, cudaMemcpyHostToDevice, st));
    CX_CUDA(c, launch_lenstats(dlens, n, d_lstats, st));
    ++r.launches;
    CX_CUDA(c, cudaMemcpyAsync(c->h_small, d_lstats, 4 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
    CX_CUDA(c, cudaStreamSynchronize(st));
    r.d2h += 32;
    mn = c->h_small[0];
    mx = c->h_small[1];
    sum = c->h_small[2];
    bad = c->h_small[3];
  }
  if (bad) return fail(c, CXBWT_EINVAL, "%llu read lengths are 0 or above 65535", (unsigned long long)bad);
  pl.Lmin = uint32_t(mn);
  pl.Lmax = uint32_t(mx);
  pl.sum = sum;
  pl.N = sum + n;
  pl.uniform = (mn == mx);
  pl.shift = bits_for(pl.Lmax);
  pl.D = (pl.Lmax + 3) / 4;
  pl.W = (pl.Lmax + 15) / 16;
  pl.len_passes = pl.uniform ? 0 : (pl.Lmax > 255 ? 2 : 1);
  pl.n_words = (sum + 15) / 16;
  int algorithm = c->opt.algorithm, tile_items = c->opt.tile_items, depth = c->opt.prefix_len;
  {
    int t_tile = 0, t_algo = 0, t_depth = 0;
    if (tuned_choice(c, pl.Lmax, pl.N, &t_tile, &t_algo, &t_depth)) {
      if (algorithm == CXBWT_ALGO_AUTO) algorithm = t_algo;
      if (tile_items == 0) tile_items = t_tile;
      if (depth == 0) depth = t_depth;
    }
  }
  pl.depth = depth ? uint32_t(depth) : 16u;
  pl.seg_words = segsort_words(pl.Lmax, pl.depth);
  switch (algorithm) {
    case CXBWT_ALGO_LSD: pl.groups = false; break;
    case CXBWT_ALGO_GROUPS:
      if (!pl.seg_words)
        return fail(c, CXBWT_EUNSUPPORTED, "the group plan handles reads of at most %u bases with l = %u",
                    pl.depth + 512, pl.depth);
      pl.groups = true;
      break;
    case CXBWT_ALGO_AUTO: pl.groups = pl.seg_words != 0; break;
    default: return fail(c, CXBWT_EINVAL, "unknown algorithm %d", algorithm);
  }
  // Windows [0, w_last] are sorted by LSD passes over all rows; with the
  // group plan only window 0 is, and the groups are finished on chip.
  pl.w_last = pl.groups ? 0u : pl.W - 1;
  plan_ids(pl, (c->opt.plan_flags & CXBWT_PLAN_ID64) != 0,
           pl.n_words * 4 > (64u << 20) || (c->opt.plan_flags & CXBWT_PLAN_CARRY_BASE));
  r.shape = onesweep_shape(tile_items, pl.idb);
  const uint32_t TILE = uint32_t(r.shape.tile());

  // ---- inputs on the device ----------------------------------------------
  const uint32_t* d_reads = reads;
  if (!reads_dev) {
    CX_TRY(ensure(c, c->store, pl.n_words * 4, "read store"));
    CX_CUDA(c, cudaMemcpyAsync(c->store.p, reads, pl.n_words * 4, cudaMemcpyHostToDevice, st));
    h2d += pl.n_words * 4;
    d_reads = static_cast<const uint32_t*>(c->store.p);
  }
  std::vector<uint32_t> len_bases;
  const uint64_t* d_desc = nullptr;
  if (!pl.uniform) {
    if (!hlens) {
      lens_copy.resize(n);
      CX_CUDA(c, cudaMemcpyAsync(lens_copy.data(), lens, n * 4, cudaMemcpyDeviceToHost, st));
      CX_CUDA(c, cudaStreamSynchronize(st));
      r.d2h += n * 4;
      hlens = lens_copy.data();
    }
    std::vector<uint64_t> desc(n);
    std::vector<uint32_t> lh(pl.Lmax + 1, 0);
    uint64_t off = 0;
    for (uint64_t i = 0; i < n; ++i) {
      desc[i] = (off << 16) | hlens[i];
      off += hlens[i];
      ++lh[hlens[i]];
    }
    // Length passes: digit j of the suffix length t = L_i - k; there are
    // cnt(t) = #{i : L_i >= t} suffixes of length t.
    std::vector<uint64_t> cnt(pl.Lmax + 1, 0);
    uint64_t run = 0;
    for (int64_t t = pl.Lmax; t >= 0; --t) {
      run += lh[t];
      cnt[t] = run;
    }
    len_bases.assign(size_t(pl.len_passes) * kRadix, 0);
    for (uint32_t j = 0; j < pl.len_passes; ++j) {
      std::vector<uint64_t> h(kRadix, 0);
      for (uint32_t t = 0; t <= pl.Lmax; ++t) h[(t >> (8 * j)) & 255] += cnt[t];
      uint64_t acc = 0;
      for (int v = 0; v < kRadix; ++v) {
        len_bases[size_t(j) * kRadix + v] = uint32_t(acc);
        acc += h[v];
      }
    }
    CX_TRY(ensure(c, c->desc, n * 8, "read descriptors"));
    CX_TRY(ensure(c, c->lenhist, (pl.Lmax + 1) * 4, "length histogram"));
    CX_CUDA(c, cudaMemcpyAsync(c->desc.p, desc.data(), n * 8, cudaMemcpyHostToDevice, st));
    CX_CUDA(c, cudaMemcpyAsync(c->lenhist.p, lh.data(), (pl.Lmax + 1) * 4, cudaMemcpyHostToDevice, st));
    h2d += n * 8 + (pl.Lmax + 1) * 4;
    d_desc = static_cast<const uint64_t*>(c->desc.p);
  }
  r.R = ReadIndex{d_reads, pl.n_words, d_desc, pl.shift, pl.uniform ? pl.Lmax : 0u, uint32_t(n),
                  (reinterpret_cast<uintptr_t>(d_reads) & 15u) == 0 ? 1u : 0u, pl.sym};

  // ---- slices --------------------------------------------------------------
  // Device bytes per suffix of a slice: ids and keys (double-buffered),
  // look-back words, group lists; plus the SA staging when it goes to the host.
  // The look-back words cover every tile of a generated enumeration of all N
  // suffixes, so they are a fixed cost, not a per-row one.
  const double per_row = 2.0 * pl.idb + 8.0 + 8.0 / 33 + (out_sa && !sa_dev ? 8.0 : 0.0);
  const uint64_t status_bytes = status_tiles(c, pl, TILE) * kRadix * 8;
  const uint64_t fixed = uint64_t(pl.Lmax) * kRadix * 4 + uint64_t(pl.D + pl.len_passes + 5) * kRadix * 4 +
                         uint64_t(pl.W) * 4 * kRadix * 4 + (uint64_t(1) << kBucketBits) * 8 + status_bytes + (1u << 20);
  // Buffers sized per slice are reused (or regrown) by this build: they do
  // not count against what it may take.
  const uint64_t reusable = c->vals[0].cap + c->vals[1].cap + c->keys[0].cap + c->keys[1].cap + c->status.cap +
                            c->seglist.cap + c->out_sa.cap;
  const uint64_t held_fixed = c->held - reusable;
  // Output staging for host buffers is granted below, after the slices are
  // planned: count what it will add to what is held now (a whole build's size
  // bounds a part's).
  uint64_t out_more = 0;
  if (!bwt_dev && !counts_only) {
    const uint64_t need = ((pl.N + 15) / 16 + 1) * 4;
    out_more += need > c->out_bwt.cap ? need - c->out_bwt.cap + (2u << 20) : 0;
  }
  if (out_dollar && !dollar_dev) out_more += n * 8 > c->out_dollar.cap ? n * 8 - c->out_dollar.cap + (2u << 20) : 0;
  const uint64_t avail =
      c->budget > held_fixed + fixed + out_more ? c->budget - held_fixed - fixed - out_more : 0;
  uint64_t m1 = uint64_t(double(avail) / per_row);
  // A slice must fit 32-bit row counts; every workspace buffer below is
  // granted in 2 MB steps, so leave room for that rounding.
  m1 = std::min<uint64_t>(m1 > (64u << 20) ? m1 - (1u << 20) : (m1 > 32768 ? m1 - 16384 : m1), 0xFFFFFFF0ull);
  std::vector<Slice> slices;
  uint64_t part_row0 = 0, part_rows = pl.N;  // global rows this call emits
  std::vector<uint32_t> P_host;  // per-position 4-mer counts, when the slices were planned from them
  bool refined = false;          // an 8-base bucket was split into 16-base ones
  if (pl.N <= m1 && !part) {
    Slice sl;
    sl.rows = uint32_t(pl.N);
    slices.push_back(sl);
  } else {
    if (!pl.groups)
      return fail(c, CXBWT_EUNSUPPORTED, "device-memory-bounded slices and parts use the group plan (reads of at most 528 bases)");
    // Figure 2 step 1: suffixes per bucket; then consecutive buckets packed
    // into slices of at most m1 suffixes.  A build first tries buckets of the
    // first 4 bases: their counts are sums of the per-position 4-mer counts
    // (one pass over the bases instead of one per suffix), plus the n
    // terminator-only suffixes in bucket 0.  When one of them holds more than
    // a slice, and for parts (whose buckets are 8 bases by definition), the
    // suffixes are counted per 8-base bucket.
    std::vector<uint64_t> bh;
    if (!part) {
      CX_TRY(ensure(c, c->P, uint64_t(pl.Lmax) * kRadix * 4, "position counts"));
      CX_CUDA(c, cudaMemsetAsync(c->P.p, 0, uint64_t(pl.Lmax) * kRadix * 4, st));
      CX_CUDA(c, launch_poscount(r.R, uint32_t(n), pl.Lmax, static_cast<uint32_t*>(c->P.p), c->sm_count, st));
      ++r.launches;
      std::vector<uint32_t>& P = P_host;
      P.resize(size_t(pl.Lmax) * kRadix);
      CX_CUDA(c, cudaMemcpyAsync(P.data(), c->P.p, P.size() * 4, cudaMemcpyDeviceToHost, st));
      CX_CUDA(c, cudaStreamSynchronize(st));
      r.d2h += P.size() * 4;
      std::vector<uint64_t> b4(kRadix, 0);
      for (uint32_t q = 0; q < pl.Lmax; ++q)
        for (int v = 0; v < kRadix; ++v) b4[v] += P[size_t(q) * kRadix + v];
      b4[0] += n;
      if (*std::max_element(b4.begin(), b4.end()) <= m1) {
        bh.swap(b4);
        r.bucket_bits = 8;
      }
    }
    if (bh.empty() && part && part->given_counts) {
      r.bucket_bits = kBucketBits;
      bh.assign(part->given_counts, part->given_counts + (size_t(1) << kBucketBits));
      uint64_t total = 0;
      for (uint64_t x : bh) total += x;
      if (total != pl.N)
        return fail(c, CXBWT_EINVAL, "bucket counts sum to %llu, not the collection's %llu suffixes",
                    (unsigned long long)total, (unsigned long long)pl.N);
    }
    if (bh.empty()) {
      r.bucket_bits = kBucketBits;
      CX_TRY(ensure(c, c->bhist, (uint64_t(1) << kBucketBits) * 8, "bucket counts"));
      CX_CUDA(c, cudaMemsetAsync(c->bhist.p, 0, (uint64_t(1) << kBucketBits) * 8, st));
      CX_CUDA(c, launch_bucket_hist(r.R, uint32_t(n), kBucketBits, static_cast<unsigned long long*>(c->bhist.p),
                                    c->sm_count, st));
      ++r.launches;
      bh.resize(size_t(1) << kBucketBits);
      CX_CUDA(c, cudaMemcpyAsync(bh.data(), c->bhist.p, bh.size() * 8, cudaMemcpyDeviceToHost, st));
      CX_CUDA(c, cudaStreamSynchronize(st));
      r.d2h += bh.size() * 8;
    }
    if (counts_only) {
      std::memcpy(part->bucket_counts, bh.data(), bh.size() * 8);
      return CXBWT_OK;
    }
    const uint32_t b_lo = part ? part->lo : 0u, b_hi = part ? part->hi : uint32_t(bh.size());
    uint64_t row = 0, acc = 0;
    for (uint32_t b = 0; b < b_lo; ++b) row += bh[b];
    part_row0 = row;
    // Units of consecutive first windows, in key order: the buckets, except
    // that an 8-base bucket holding more suffixes than a slice is refined by
    // its next 8 bases (Section 3.1: a partition larger than the GPU takes is
    // split by the characters that follow its prefix) into 16-base units.
    struct Unit {
      uint64_t key_lo, key_hi, cnt;
    };
    std::vector<Unit> units;
    const uint32_t ush = 32 - r.bucket_bits;
    for (uint32_t b = b_lo; b < b_hi; ++b) {
      if (bh[b] <= m1) {
        units.push_back(Unit{uint64_t(b) << ush, uint64_t(b + 1) << ush, bh[b]});
        continue;
      }
      if (r.bucket_bits != kBucketBits)
        return fail(c, CXBWT_EINTERNAL, "a %u-base bucket exceeds a slice", r.bucket_bits / 2);
      refined = true;
      CX_TRY(ensure(c, c->bhist, (uint64_t(1) << kBucketBits) * 8, "bucket counts"));
      CX_CUDA(c, cudaMemsetAsync(c->bhist.p, 0, (uint64_t(1) << kBucketBits) * 8, st));
      CX_CUDA(c, launch_sub_bucket_hist(r.R, uint32_t(n), b, static_cast<unsigned long long*>(c->bhist.p), c->sm_count,
                                        st));
      ++r.launches;
      std::vector<uint64_t> sub(size_t(1) << 16);
      CX_CUDA(c, cudaMemcpyAsync(sub.data(), c->bhist.p, sub.size() * 8, cudaMemcpyDeviceToHost, st));
      CX_CUDA(c, cudaStreamSynchronize(st));
      r.d2h += sub.size() * 8;
      uint64_t total = 0;
      for (uint32_t x = 0; x < sub.size(); ++x) {
        total += sub[x];
        if (sub[x] > m1)
          return fail(c, CXBWT_ENOMEM,
                      "one 16-base prefix holds %llu suffixes, more than the %llu a slice can hold (refining by the "
                      "bases after the first 16 is not built)",
                      (unsigned long long)sub[x], (unsigned long long)m1);
        units.push_back(Unit{(uint64_t(b) << 16) | x, ((uint64_t(b) << 16) | x) + 1, sub[x]});
      }
      if (total != bh[b])
        return fail(c, CXBWT_EINTERNAL, "8-base bucket %u: %llu suffixes refined, %llu counted", b,
                    (unsigned long long)total, (unsigned long long)bh[b]);
    }
    // Slices of about equal size: as few as m1 allows, each closed once it
    // reaches the average (smaller slices need less workspace).
    uint64_t range_rows = 0;
    for (const Unit& u : units) range_rows += u.cnt;
    const uint64_t n_min = std::max<uint64_t>(1, (range_rows + m1 - 1) / std::max<uint64_t>(m1, 1));
    const uint64_t target = (range_rows + n_min - 1) / n_min;
    size_t lo = 0;
    for (size_t u = 0; u <= units.size(); ++u) {
      const bool end = (u == units.size());
      const uint64_t cnt = end ? 0 : units[u].cnt;
      if (end || acc + cnt > m1 || acc >= target) {
        if (acc) {
          Slice sl;
          sl.whole = false;
          sl.key_lo = uint32_t(units[lo].key_lo);
          sl.key_hi = units[u - 1].key_hi;
          sl.rows = uint32_t(acc);
          sl.row0 = row;
          slices.push_back(sl);
          row += acc;
        }
        lo = u;
        acc = 0;
      }
      acc += cnt;
    }
    part_rows = row - part_row0;
    if (!part) {
      if (row != pl.N) return fail(c, CXBWT_EINTERNAL, "bucket counts sum to %llu, not N", (unsigned long long)row);
    } else {
      uint64_t total = row;
      for (uint32_t b = b_hi; b < bh.size(); ++b) total += bh[b];
      if (total != pl.N) return fail(c, CXBWT_EINTERNAL, "bucket counts sum to %llu, not N", (unsigned long long)total);
    }
    // Gathers walk the store in address order when it is too big for L2.
    r.read_major = pl.Lmax <= 255 && (pl.n_words * 4 > (64u << 20) || (c->opt.plan_flags & CXBWT_PLAN_READ_MAJOR));
  }
  if (part) {
    if (part->row0) *part->row0 = part_row0;
    if (part->rows) *part->rows = part_rows;
  }

  // ---- outputs on the device ---------------------------------------------
  // The output holds global words [word0, word0 + bwt_words): all of them for
  // a whole build, those the part's rows touch for a part.
  const uint64_t word0 = part_row0 / 16;
  const uint64_t bwt_words = (part_row0 + part_rows + 15) / 16 - word0;
  r.d_bwt = out_bwt;
  if (!bwt_dev) {
    CX_TRY(ensure(c, c->out_bwt, bwt_words * 4, "BWT output"));
    r.d_bwt = static_cast<uint32_t*>(c->out_bwt.p);
  }
  r.d_dollar = out_dollar;
  if (out_dollar && !dollar_dev) {
    CX_TRY(ensure(c, c->out_dollar, n * 8, "dollar positions"));
    r.d_dollar = static_cast<uint64_t*>(c->out_dollar.p);
  }

  if (slices.size() > 1 || part) {
    CX_CUDA(c, cudaMemsetAsync(r.d_bwt, 0, bwt_words * 4, st));  // slice edges are merged with atomicOr
  }
  if (part && r.d_dollar) {
    CX_CUDA(c, cudaMemsetAsync(r.d_dollar, 0xFF, n * 8, st));  // reads whose $ row is in another part
  }

  uint32_t max_rows = 0;
  for (const Slice& sl : slices) max_rows = std::max(max_rows, sl.rows);
  const uint64_t gen_tiles = status_tiles(c, pl, TILE);  // look-back words: the most tiles any pass has

  // A build in a few slices of 4-base buckets lists every slice in one
  // generating pass (kSrcInitSplit: digit = (slice, suffix length)) into its
  // own part of one array of N rows, instead of one pass over all N suffixes
  // per slice; each slice then sorts between its part and one spare array.
  // That needs (N + largest slice) rows of ids and keys instead of twice the
  // largest slice, so it is taken only when the budget holds them.
  bool split = false;
  if (!part && slices.size() > 1 && slices.size() <= kMaxSplit && pl.uniform && r.bucket_bits == 8 && !refined &&
      !P_host.empty() && slices.size() * (pl.Lmax + 1) <= uint64_t(kRadix)) {
    const uint64_t need = (pl.N + 4 * slices.size() + max_rows) * uint64_t(pl.idb + 4) +
                          uint64_t(double(max_rows) * (8.0 / 33 + 8.0 / 1025)) +
                          (out_sa && !sa_dev ? uint64_t(max_rows) * 8 : 0);
    split = need <= avail;
  }

  // ---- workspace ---------------------------------------------------------
  uint64_t rows0 = uint64_t(max_rows);
  if (split) {
    uint64_t at = 0;
    for (Slice& sl : slices) {
      sl.arr0 = at;
      at = (at + sl.rows + 3) & ~uint64_t(3);
    }
    rows0 = at;
  }
  CX_TRY(ensure(c, c->vals[0], rows0 * pl.idb, "suffix ids"));
  CX_TRY(ensure(c, c->vals[1], uint64_t(max_rows) * pl.idb, "suffix ids"));
  CX_TRY(ensure(c, c->keys[0], rows0 * 4, "keys"));
  CX_TRY(ensure(c, c->keys[1], uint64_t(max_rows) * 4, "keys"));
  const void* status_before = c->status.p;
  CX_TRY(ensure(c, c->status, gen_tiles * kRadix * 8, "look-back words"));
  if (c->status.p != status_before) {
    // Fresh memory could hold any flag value: clear it so no stale word looks published.
    CX_CUDA(c, cudaMemsetAsync(c->status.p, 0, c->status.cap, st));
  }
  CX_TRY(ensure(c, c->P, uint64_t(pl.Lmax) * kRadix * 4, "position counts"));
  // digit bases; then the split pass's digit bases and slice of every bucket (two more rows)
  const uint32_t split_row = std::max<uint32_t>(pl.D + pl.len_passes, 5);
  CX_TRY(ensure(c, c->base, uint64_t(split_row + 2) * kRadix * 4, "digit bases"));
  if (pl.uniform && !c->lenhist.p) CX_TRY(ensure(c, c->lenhist, 4, "length histogram"));
  if (pl.groups && pl.Lmax > pl.depth) {
    CX_TRY(ensure(c, c->seglist, (cta_list_cap(max_rows) + big_list_cap(max_rows, pl.seg_words)) * 8, "group lists"));
    CX_TRY(ensure(c, c->rhist, size_t(pl.W) * 4 * kRadix * 4, "group digit counts"));
  }
  r.d_sa = out_sa;
  if (out_sa && !sa_dev) {
    CX_TRY(ensure(c, c->out_sa, uint64_t(max_rows) * 8, "suffix array slice"));
    r.d_sa = static_cast<uint64_t*>(c->out_sa.p);
  }
  r.vals[0] = c->vals[0].p;
  r.vals[1] = c->vals[1].p;
  r.keys[0] = static_cast<uint32_t*>(c->keys[0].p);
  r.keys[1] = static_cast<uint32_t*>(c->keys[1].p);
  r.base = static_cast<uint32_t*>(c->base.p);
  if (pl.len_passes) {
    CX_CUDA(c, cudaMemcpyAsync(r.base + size_t(pl.D) * kRadix, len_bases.data(), len_bases.size() * 4,
                               cudaMemcpyHostToDevice, st));
    h2d += len_bases.size() * 4;
  }
  const uint64_t passes_max = uint64_t(slices.size()) * (pl.D + pl.len_passes + 1) + 4 * pl.W * 64 + 1;
  if (uint64_t(c->epoch) + passes_max + 2 >= (uint64_t(1) << 30)) {
    // Look-back flags are 2*epoch and 2*epoch+1 in 32 bits: restart the epochs.
    CX_CUDA(c, cudaMemsetAsync(c->status.p, 0, c->status.cap, st));
    c->epoch = 0;
  }
  CX_CUDA(c, cudaMemsetAsync(r.d_counts, 0, 5 * 8, st));

  const bool timing = c->opt.timing != 0;
  if (timing) {
    while (c->tev.size() < 4 * slices.size()) {
      cudaEvent_t ev;
      CX_CUDA(c, cudaEventCreate(&ev));
      c->tev.push_back(ev);
    }
    CX_CUDA(c, cudaEventRecord(c->ev[0], st));
  }

  if (split) CX_TRY(split_pass(c, r, slices, P_host, timing));

  uint64_t words_sent = 0;  // BWT words already streamed to the host
  for (size_t si = 0; si < slices.size(); ++si) {
    Slice& sl = slices[si];
    int cur = 0;
    cudaEvent_t* tev = timing ? &c->tev[4 * si] : nullptr;
    if (split) {
      // The slice's part of the listed rows, and the spare array to sort into.
      sl.pregen = true;
      r.vals[0] = vptr(c->vals[0].p, pl.idb, sl.arr0);
      r.keys[0] = static_cast<uint32_t*>(c->keys[0].p) + sl.arr0;
    }
    CX_TRY(sort_slice(c, r, sl, &cur, tev));
    if (tev) CX_CUDA(c, cudaEventRecord(tev[2], st));
    // ---- emission of the slice -------------------------------------------
    EmitArgs e{};
    e.sa = r.vals[cur];
    e.n = sl.rows;
    e.row0 = sl.row0;
    e.n_total = pl.N;
    e.R = r.R;
    e.bwt = r.d_bwt;
    e.word_base = word0;
    e.dollar_pos = r.d_dollar;
    e.counts = r.d_counts;
    e.sa_out = r.d_sa ? (sa_dev ? r.d_sa + sl.row0 : r.d_sa) : nullptr;
    e.err = r.d_err;
    e.id_bytes = pl.idb;
    e.read_base = 0;
    e.n_reads_out = uint32_t(n);
    CX_CUDA(c, launch_emit(e, st));
    ++r.launches;
    if (tev) CX_CUDA(c, cudaEventRecord(tev[3], st));
    if (out_sa && !sa_dev) {
      CX_CUDA(c, cudaMemcpyAsync(out_sa + sl.row0, r.d_sa, uint64_t(sl.rows) * 8, cudaMemcpyDeviceToHost, st));
      r.d2h += uint64_t(sl.rows) * 8;
    }
    if (!bwt_dev) {
      // Words whose 16 rows are all emitted stream to the host while the next slice sorts.
      const bool last = si + 1 == slices.size();
      const uint64_t done = last ? bwt_words : (sl.row0 + sl.rows) / 16 - word0;
      if (done > words_sent) {
        cudaEvent_t ev = c->slice_done[si & 1];
        CX_CUDA(c, cudaEventRecord(ev, st));
        CX_CUDA(c, cudaStreamWaitEvent(c->side, ev, 0));
        CX_CUDA(c, cudaMemcpyAsync(out_bwt + words_sent, r.d_bwt + words_sent, (done - words_sent) * 4,
                                   cudaMemcpyDeviceToHost, c->side));
        r.d2h += (done - words_sent) * 4;
        words_sent = done;
      }
    }
  }
  if (timing) CX_CUDA(c, cudaEventRecord(c->ev[3], st));
  if (!bwt_dev) {
    CX_CUDA(c, cudaEventRecord(c->slice_done[0], c->side));
    CX_CUDA(c, cudaStreamWaitEvent(st, c->slice_done[0], 0));
  }
  if (out_counts) {
    CX_CUDA(c, cudaMemcpyAsync(out_counts, r.d_counts, 5 * 8, counts_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                               st));
    if (!counts_dev) r.d2h += 40;
  }
  if (out_dollar && !dollar_dev) {
    CX_CUDA(c, cudaMemcpyAsync(out_dollar, r.d_dollar, n * 8, cudaMemcpyDeviceToHost, st));
    r.d2h += n * 8;
  }
  CX_CUDA(c, cudaMemcpyAsync(c->h_small + 4, r.d_err, 4, cudaMemcpyDeviceToHost, st));

  c->stats.kernel_launches += r.launches + r.sort_launches;
  c->stats.sort_pass_launches += r.sort_launches;
  c->stats.sort_pass_items += r.sort_items;
  c->stats.h2d_bytes += h2d;
  c->stats.d2h_bytes += r.d2h;
  c->stats.device_bytes_held = c->held;
  c->stats.slices += slices.size();
  c->stats.carried_pass_launches += r.carried_launches;
  c->stats.carried_pass_items += r.carried_items;

  const bool host_out = !bwt_dev || (out_dollar && !dollar_dev) || (out_counts && !counts_dev) || (out_sa && !sa_dev);
  if (c->opt.async && !host_out) {
    // Completed (and checked) by cxbwt_sync.
    c->stats.builds += 1;
    c->stats.bases += pl.sum;
    c->stats.suffixes += pl.N;
    return CXBWT_OK;
  }
  CX_CUDA(c, cudaStreamSynchronize(st));
  CX_TRY(take_device_error(c));
  if (timing) {
    float ms_all = 0;
    CX_CUDA(c, cudaEventElapsedTime(&ms_all, c->ev[0], c->ev[3]));
    for (size_t si = 0; si < slices.size(); ++si) {
      cudaEvent_t* tev = &c->tev[4 * si];
      float ms_sort = 0, ms_group = 0, ms_emit = 0;
      CX_CUDA(c, cudaEventElapsedTime(&ms_sort, tev[0], tev[1]));
      CX_CUDA(c, cudaEventElapsedTime(&ms_group, tev[1], tev[2]));
      CX_CUDA(c, cudaEventElapsedTime(&ms_emit, tev[2], tev[3]));
      c->stats.sort_pass_ms += ms_sort;
      c->stats.group_ms += ms_group;
      c->stats.emit_ms += ms_emit;
    }
    for (uint32_t j = 0; j < r.n_pev; ++j) {
      if (!r.pev_carried[j]) continue;
      float ms = 0;
      CX_CUDA(c, cudaEventElapsedTime(&ms, c->pev[2 * size_t(j)], c->pev[2 * size_t(j) + 1]));
      if (r.pev_carried[j] == 1) c->stats.carried_pass_ms += ms;
      else c->stats.sort_pass_ms += ms;  // the split pass runs before every slice
    }
    c->stats.build_ms += ms_all;
  }
  c->stats.builds += 1;
  c->stats.bases += pl.sum;
  c->stats.suffixes += pl.N;
  return CXBWT_OK;
}

}  // namespace host
}  // namespace cxbwt


extern "C" {

int cxbwt_abi_version(void) { return CXBWT_ABI_VERSION; }

int cxbwt_bucket_counts(cxbwt_ctx* ctx, const uint32_t* reads_2bit, uint64_t n_reads, const uint32_t* lens,
                        uint64_t* out_counts, void* stream) {
  if (!ctx) return CXBWT_EINVAL;
  if (!out_counts) return fail(ctx, CXBWT_EINVAL, "out_counts must not be NULL");
  PartSpec p;
  p.counts_only = true;
  p.bucket_counts = out_counts;
  return build_impl(ctx, reads_2bit, n_reads, lens, nullptr, nullptr, nullptr, nullptr, stream, &p);
}

int cxbwt_split_parts(const uint64_t* counts, uint32_t n_buckets, uint32_t n_parts, uint32_t* bucket_bounds,
                      uint64_t* row_bounds) {
  if (!counts || !bucket_bounds || !row_bounds || n_parts == 0) return CXBWT_EINVAL;
  uint64_t total = 0;
  for (uint32_t b = 0; b < n_buckets; ++b) total += counts[b];
  // Boundary j goes where the running count comes closest to j * N / n_parts.
  uint32_t b = 0;
  uint64_t below = 0;  // suffixes in buckets [0, b)
  bucket_bounds[0] = 0;
  row_bounds[0] = 0;
  for (uint32_t j = 1; j < n_parts; ++j) {
    const uint64_t target = uint64_t((unsigned __int128)total * j / n_parts);
    while (b < n_buckets && below + counts[b] <= target) below += counts[b++];
    // Take bucket b too when that lands closer to the target.
    if (b < n_buckets && below < target && below + counts[b] - target < target - below) below += counts[b++];
    bucket_bounds[j] = b;
    row_bounds[j] = below;
  }
  bucket_bounds[n_parts] = n_buckets;
  row_bounds[n_parts] = total;
  return CXBWT_OK;
}

int cxbwt_build_part(cxbwt_ctx* ctx, const uint32_t* reads_2bit, uint64_t n_reads, const uint32_t* lens,
                     uint32_t bucket_lo, uint32_t bucket_hi, const uint64_t* bucket_counts, uint32_t* out_words,
                     uint64_t* out_dollar_pos, uint64_t* out_counts, uint64_t* out_row0, uint64_t* out_rows,
                     void* stream) {
  PartSpec p;
  p.lo = bucket_lo;
  p.hi = bucket_hi;
  p.given_counts = bucket_counts;
  p.row0 = out_row0;
  p.rows = out_rows;
  return build_impl(ctx, reads_2bit, n_reads, lens, out_words, out_dollar_pos, out_counts, nullptr, stream, &p);
}

int cxbwt_merge_part(uint32_t* bwt_words, uint64_t n_words, const uint32_t* part_words, uint64_t row0, uint64_t rows) {
  if (!bwt_words || (!part_words && rows)) return CXBWT_EINVAL;
  if (rows == 0) return CXBWT_OK;
  const uint64_t w0 = row0 / 16, w1 = (row0 + rows + 15) / 16;
  if (row0 + rows < row0 || w1 > n_words) return CXBWT_EINVAL;
  for (uint64_t w = w0; w < w1; ++w) bwt_words[w] |= part_words[w - w0];
  return CXBWT_OK;
}

void cxbwt_default_options(cxbwt_options* opt) {
  if (!opt) return;
  std::memset(opt, 0, sizeof *opt);
  opt->digit_bits = 8;
}

int cxbwt_create(cxbwt_ctx** out, const cxbwt_options* opt) {
  g_create_error.clear();
  if (!out) {
    g_create_error = "out must not be NULL";
    return CXBWT_EINVAL;
  }
  *out = nullptr;
  cxbwt_options o;
  cxbwt_default_options(&o);
  if (opt) o = *opt;
  if (o.digit_bits == 0) o.digit_bits = 8;
  if (o.digit_bits != 8) {
    g_create_error = "digit_bits: only 8-bit digits are built";
    return CXBWT_EUNSUPPORTED;
  }
  if (o.prefix_len != 0 && o.prefix_len != 12 && o.prefix_len != 16) {
    g_create_error = "prefix_len: the group plan sorts the first 12 or 16 bases (0 = automatic)";
    return CXBWT_EUNSUPPORTED;
  }
  int ndev = 0;
  cudaError_t e = cudaGetDeviceCount(&ndev);
  if (e != cudaSuccess || ndev == 0) {
    cudaGetLastError();
    g_create_error = std::string("no CUDA device: ") + cudaGetErrorString(e);
    return CXBWT_ECUDA;
  }
  if (o.device < 0 || o.device >= ndev) {
    g_create_error = "device ordinal out of range";
    return CXBWT_EINVAL;
  }
  e = cudaSetDevice(o.device);
  if (e != cudaSuccess) {
    g_create_error = std::string("cudaSetDevice: ") + cudaGetErrorString(e);
    return CXBWT_ECUDA;
  }
  auto* c = new cxbwt_ctx();
  c->opt = o;
  c->device = o.device;
  cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, o.device);
  size_t free_b = 0, total_b = 0;
  cudaMemGetInfo(&free_b, &total_b);
  c->budget = o.device_budget_bytes ? o.device_budget_bytes : uint64_t(double(free_b) * 0.9);
  bool ok = cudaMallocHost(reinterpret_cast<void**>(&c->h_small), 64) == cudaSuccess;
  for (auto& ev : c->ev) ok = ok && cudaEventCreate(&ev) == cudaSuccess;
  for (auto& ev : c->slice_done) ok = ok && cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) == cudaSuccess;
  ok = ok && cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking) == cudaSuccess;
  if (ok) ok = ensure(c, c->misc, kMiscBytes, "scratch words") == CXBWT_OK;
  if (ok) ok = cudaMemset(c->misc.p, 0, kMiscBytes) == cudaSuccess;
  if (!ok) {
    g_create_error = c->err.empty() ? std::string("context set-up failed: ") + cudaGetErrorString(cudaGetLastError())
                                    : c->err;
    cxbwt_destroy(c);
    return CXBWT_ECUDA;
  }
  *out = c;
  return CXBWT_OK;
}

void cxbwt_destroy(cxbwt_ctx* c) {
  if (!c) return;
  if (c->batch_pool && c->batch_pool_free) c->batch_pool_free(c->batch_pool);
  cudaSetDevice(c->device);
  cudaDeviceSynchronize();
  DevBuf* bufs[] = {&c->vals[0], &c->vals[1], &c->keys[0], &c->keys[1], &c->status, &c->P, &c->base,
                    &c->lenhist, &c->desc, &c->misc, &c->store, &c->out_bwt, &c->out_dollar, &c->out_sa,
                    &c->seglist, &c->rhist, &c->bhist};
  for (DevBuf* b : bufs) release(c, *b);
  for (auto& ev : c->ev)
    if (ev) cudaEventDestroy(ev);
  for (auto& ev : c->slice_done)
    if (ev) cudaEventDestroy(ev);
  for (auto& ev : c->tev) cudaEventDestroy(ev);
  for (auto& ev : c->pev) cudaEventDestroy(ev);
  if (c->side) cudaStreamDestroy(c->side);
  if (c->h_small) cudaFreeHost(c->h_small);
  delete c;
}

const char* cxbwt_last_error(const cxbwt_ctx* c) { return c ? c->err.c_str() : g_create_error.c_str(); }

const char* cxbwt_status_string(int s) {
  switch (s) {
    case CXBWT_OK: return "CXBWT_OK";
    case CXBWT_EINVAL: return "CXBWT_EINVAL";
    case CXBWT_ENOMEM: return "CXBWT_ENOMEM";
    case CXBWT_ECUDA: return "CXBWT_ECUDA";
    case CXBWT_ETIMEOUT: return "CXBWT_ETIMEOUT";
    case CXBWT_EUNSUPPORTED: return "CXBWT_EUNSUPPORTED";
    case CXBWT_EBUSY: return "CXBWT_EBUSY";
    case CXBWT_EINTERNAL: return "CXBWT_EINTERNAL";
    default: return "CXBWT_UNKNOWN";
  }
}

int cxbwt_output_size(uint64_t n_reads, const uint32_t* lens, uint64_t* n_symbols, uint64_t* bwt_words) {
  if (n_reads && !lens) return CXBWT_EINVAL;
  uint64_t N = n_reads;
  for (uint64_t i = 0; i < n_reads; ++i) N += lens[i];
  if (n_symbols) *n_symbols = N;
  if (bwt_words) *bwt_words = (N + 15) / 16;
  return CXBWT_OK;
}

int cxbwt_build(cxbwt_ctx* ctx, const uint32_t* reads_2bit, uint64_t n_reads, const uint32_t* lens,
                uint32_t* out_bwt, uint64_t* out_dollar_pos, uint64_t* out_counts, void* stream) {
  return build_impl(ctx, reads_2bit, n_reads, lens, out_bwt, out_dollar_pos, out_counts, nullptr, stream);
}

int cxbwt_build_sa(cxbwt_ctx* ctx, const uint32_t* reads_2bit, uint64_t n_reads, const uint32_t* lens,
                   uint32_t* out_bwt, uint64_t* out_dollar_pos, uint64_t* out_counts, uint64_t* out_sa,
                   void* stream) {
  if (ctx && !out_sa) return fail(ctx, CXBWT_EINVAL, "out_sa must not be NULL");
  return build_impl(ctx, reads_2bit, n_reads, lens, out_bwt, out_dollar_pos, out_counts, out_sa, stream);
}

int cxbwt_sync(cxbwt_ctx* c) {
  if (!c) return CXBWT_EINVAL;
  c->err.clear();
  CX_CUDA(c, cudaSetDevice(c->device));
  CX_CUDA(c, cudaStreamSynchronize(c->last_stream));
  CX_CUDA(c, cudaMemcpy(c->h_small + 4, static_cast<char*>(c->misc.p) + kMiscErr, 4, cudaMemcpyDeviceToHost));
  return take_device_error(c);
}

int cxbwt_get_stats(const cxbwt_ctx* c, cxbwt_stats* out) {
  if (!c || !out) return CXBWT_EINVAL;
  *out = c->stats;
  out->device_bytes_held = c->held;
  return CXBWT_OK;
}

int cxbwt_reset_stats(cxbwt_ctx* c) {
  if (!c) return CXBWT_EINVAL;
  c->stats = cxbwt_stats{};
  return CXBWT_OK;
}

int cxbwt_pack_codes(const uint8_t* codes, uint64_t n_bases, uint32_t* out) {
  if ((!codes || !out) && n_bases) return CXBWT_EINVAL;
  const uint64_t words = (n_bases + 15) / 16;
  for (uint64_t w = 0; w < words; ++w) {
    uint32_t x = 0;
    const uint64_t b0 = w * 16;
    const uint64_t m = std::min<uint64_t>(16, n_bases - b0);
    for (uint64_t j = 0; j < m; ++j) {
      const uint8_t cd = codes[b0 + j];
      if (cd > 3) return CXBWT_EINVAL;
      x |= uint32_t(cd) << (30 - 2 * j);
    }
    out[w] = x;
  }
  return CXBWT_OK;
}

int cxbwt_pack_ascii(const char* acgt, uint64_t n_bases, uint32_t* out) {
  if ((!acgt || !out) && n_bases) return CXBWT_EINVAL;
  const uint64_t words = (n_bases + 15) / 16;
  for (uint64_t w = 0; w < words; ++w) {
    uint32_t x = 0;
    const uint64_t b0 = w * 16;
    const uint64_t m = std::min<uint64_t>(16, n_bases - b0);
    for (uint64_t j = 0; j < m; ++j) {
      uint32_t cd;
      switch (acgt[b0 + j]) {
        case 'A': cd = 0; break;
        case 'C': cd = 1; break;
        case 'G': cd = 2; break;
        case 'T': cd = 3; break;
        default: return CXBWT_EINVAL;
      }
      x |= cd << (30 - 2 * j);
    }
    out[w] = x;
  }
  return CXBWT_OK;
}

int cxbwt_unpack_ascii(const uint32_t* words, const uint64_t* dollar_pos, uint64_t n_symbols, uint64_t n_dollars,
                       char* out) {
  if ((!words || !out) && n_symbols) return CXBWT_EINVAL;
  if (n_dollars && !dollar_pos) return CXBWT_EINVAL;
  static const char kBase[4] = {'A', 'C', 'G', 'T'};
  for (uint64_t r = 0; r < n_symbols; ++r) out[r] = kBase[(words[r >> 4] >> (30 - 2 * (r & 15))) & 3u];
  for (uint64_t i = 0; i < n_dollars; ++i) {
    if (dollar_pos[i] >= n_symbols) return CXBWT_EINVAL;
    out[dollar_pos[i]] = '$';
  }
  return CXBWT_OK;
}

}  // extern "C"
