// cxbwt_autotune: choose the tile shape, the sort plan and the group plan's
// depth by timing them.
//
// For one collection (device memory), every candidate (tile of 4096 or 8192
// items with 32-bit suffix ids, of 2048, 3072 or 4096 with 64-bit ones;
// the group plan with its first l = 16 or l = 12 bases sorted by LSD passes
// (four or three passes, then groups sharing those bases finished on chip),
// or the LSD plan, where they apply) is built three times and the last two
// are timed with CUDA events on the caller's stream; the fastest choice is
// kept in the context for builds of the same maximum read length and size
// class (N within a factor of two).  Builds whose options leave the tile,
// the plan and prefix_len automatic then use it.  Every candidate gives the
// same BWT; only speed differs: a smaller l saves a pass over every suffix
// and leaves larger groups to finish, which pays when the collection's
// l-prefixes are still rare (reads of a small genome).  The radix digit
// width is fixed at 8 bits (the only width built).
#include <cuda_runtime.h>

#include "host.cuh"

using namespace cxbwt;
using namespace cxbwt::host;

extern "C" int cxbwt_autotune(cxbwt_ctx* c, const uint32_t* reads_2bit, uint64_t n_reads, const uint32_t* lens,
                              uint32_t* scratch_bwt, uint64_t* scratch_dollar_pos, void* stream, cxbwt_tuning* out) {
  if (!c) return CXBWT_EINVAL;
  if (!reads_2bit || !lens || !scratch_bwt || n_reads == 0) return fail(c, CXBWT_EINVAL, "bad autotune arguments");
  CX_CUDA(c, cudaSetDevice(c->device));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // Sizes (host copy of the lengths when they are on the device).
  std::vector<uint32_t> hl;
  const uint32_t* h = lens;
  if (is_device_ptr(lens)) {
    hl.resize(n_reads);
    CX_CUDA(c, cudaMemcpy(hl.data(), lens, n_reads * 4, cudaMemcpyDeviceToHost));
    h = hl.data();
  }
  uint64_t N = n_reads;
  uint32_t Lmax = 0, Lmin = ~0u;
  for (uint64_t i = 0; i < n_reads; ++i) {
    N += h[i];
    Lmax = std::max(Lmax, h[i]);
    Lmin = std::min(Lmin, h[i]);
  }
  // The id width the build will use decides which tiles exist.
  Plan probe;
  probe.n = n_reads;
  probe.Lmax = Lmax;
  probe.uniform = Lmin == Lmax;
  plan_ids(probe, (c->opt.plan_flags & CXBWT_PLAN_ID64) != 0, false);
  const cxbwt_options saved = c->opt;
  const auto saved_tuned = c->tuned;
  c->tuned.clear();
  struct Cand { int tile, algo, depth; };
  std::vector<Cand> cands;
  const std::vector<int> tiles = probe.idb == 8 ? std::vector<int>{2048, 3072, 4096} : std::vector<int>{4096, 8192};
  for (int t : tiles) {
    if (segsort_words(Lmax, 16)) cands.push_back(Cand{t, CXBWT_ALGO_GROUPS, 16});
    if (segsort_words(Lmax, 12) && Lmax > 12) cands.push_back(Cand{t, CXBWT_ALGO_GROUPS, 12});
    cands.push_back(Cand{t, CXBWT_ALGO_LSD, 0});
  }
  cudaEvent_t e0, e1;
  CX_CUDA(c, cudaEventCreate(&e0));
  CX_CUDA(c, cudaEventCreate(&e1));
  float best = -1.f;
  Cand pick{0, 0, 0};
  int status = CXBWT_OK;
  for (const Cand& cd : cands) {
    c->opt.tile_items = cd.tile;
    c->opt.algorithm = cd.algo;
    c->opt.prefix_len = cd.depth;
    c->opt.async = 0;
    float ms_best = 1e30f;
    int st_c = CXBWT_OK;
    for (int rep = 0; rep < 3 && st_c == CXBWT_OK; ++rep) {
      cudaEventRecord(e0, st);
      st_c = build_impl(c, reads_2bit, n_reads, lens, scratch_bwt, scratch_dollar_pos, nullptr, nullptr, stream);
      cudaEventRecord(e1, st);
      cudaEventSynchronize(e1);
      float ms = 0;
      cudaEventElapsedTime(&ms, e0, e1);
      if (rep > 0) ms_best = std::min(ms_best, ms);  // the first run warms up and sizes the workspace
    }
    if (st_c != CXBWT_OK) {
      status = st_c;
      break;
    }
    if (best < 0 || ms_best < best) {
      best = ms_best;
      pick = cd;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  const std::string err = c->err;
  c->opt = saved;
  c->tuned = saved_tuned;
  if (status != CXBWT_OK) return fail(c, status, "autotune: %s", err.c_str());
  const uint64_t key = tune_key(Lmax, N);
  bool found = false;
  for (auto& e : c->tuned)
    if (e.key == key) {
      e = TunedPlan{key, pick.tile, pick.algo, pick.depth};
      found = true;
    }
  if (!found) c->tuned.push_back(TunedPlan{key, pick.tile, pick.algo, pick.depth});
  if (out) {
    out->tile_items = pick.tile;
    out->algorithm = pick.algo;
    out->digit_bits = 8;
    out->best_ms = best;
    out->prefix_len = pick.depth;
  }
  return CXBWT_OK;
}
