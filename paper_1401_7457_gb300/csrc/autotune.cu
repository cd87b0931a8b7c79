// cxbwt_autotune: choose the tile shape and sort plan by timing them.
//
// For one collection (device memory), every candidate (tile of 4096 or 8192
// items with 32-bit suffix ids, of 2048, 3072 or 4096 with 64-bit ones;
// group plan or LSD plan where both apply) is built twice and timed
// with CUDA events on the caller's stream; the fastest choice is kept in the
// context for builds of the same maximum read length and size class (N
// within a factor of two).  Builds whose options leave the tile and the plan
// automatic then use it.  Every candidate gives the same BWT; only speed
// differs.  The radix digit width is fixed at 8 bits (the only width built),
// and the first-window depth of the group plan at 16 bases.
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
  struct Cand { int tile, algo; };
  std::vector<Cand> cands;
  const std::vector<int> tiles = probe.idb == 8 ? std::vector<int>{2048, 3072, 4096} : std::vector<int>{4096, 8192};
  for (int algo : {CXBWT_ALGO_GROUPS, CXBWT_ALGO_LSD})
    for (int t : tiles) cands.push_back(Cand{t, algo});
  cudaEvent_t e0, e1;
  CX_CUDA(c, cudaEventCreate(&e0));
  CX_CUDA(c, cudaEventCreate(&e1));
  float best = -1.f;
  Cand pick{0, 0};
  int status = CXBWT_OK;
  for (const Cand& cd : cands) {
    if (cd.algo == CXBWT_ALGO_GROUPS && !segsort_words(Lmax)) continue;
    c->opt.tile_items = cd.tile;
    c->opt.algorithm = cd.algo;
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
    if (e.first == key) {
      e.second = {pick.tile, pick.algo};
      found = true;
    }
  if (!found) c->tuned.push_back({key, {pick.tile, pick.algo}});
  if (out) {
    out->tile_items = pick.tile;
    out->algorithm = pick.algo;
    out->digit_bits = 8;
    out->best_ms = best;
  }
  return CXBWT_OK;
}
