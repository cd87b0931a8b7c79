// cxbwt_build_batch: many independent collections, few launches, full GPU.
//
// Small collections (whose own builds would be bound by launch latency)
// whose reads all have one length L (at most 528 bases) are packed, in
// order, into "packs" of that length: up to 255 collections and a cap of
// suffixes per pack.  A pack is built as one collection
// whose reads are the packs' reads in order (read r of collection c is read
// coll_start[c] + r of the pack): the comparator of Section 2 depends only
// on the bases, the suffix length and the read order, so the pack's sorted
// order restricted to collection c is exactly collection c's sorted order.
// One stable digit pass by collection index then makes each collection's
// rows contiguous, and each collection is emitted from its rows (this is the
// paper's merging of small partitions up to the GPU capacity, Section 3.1,
// applied to whole collections).  Every other collection is built alone.
// Packs and lone collections are then run, largest first, by a pool of
// worker contexts (each with its own stream and a share of the budget), so
// independent builds overlap on the GPU.
#include <cuda_runtime.h>

#include <condition_variable>
#include <mutex>
#include <thread>

#include "host.cuh"

using namespace cxbwt;
using namespace cxbwt::host;

namespace {

// desc[r] = (base offset << 16) | L for every read of a pack; collection c's
// packed words start at word cw[c] of the pack store.
__global__ void k_pack_desc(uint64_t* desc, uint32_t n_reads, const uint32_t* cs, const uint64_t* cw, uint32_t n_coll,
                            uint32_t L) {
  __shared__ uint32_t s_cs[kMaxPackCollections + 1];
  __shared__ uint64_t s_cw[kMaxPackCollections];
  for (uint32_t i = threadIdx.x; i <= n_coll; i += blockDim.x) s_cs[i] = cs[i];
  for (uint32_t i = threadIdx.x; i < n_coll; i += blockDim.x) s_cw[i] = cw[i];
  __syncthreads();
  for (uint32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < n_reads; r += gridDim.x * blockDim.x) {
    uint32_t lo = 0, hi = n_coll;
    while (hi - lo > 1) {
      const uint32_t mid = (lo + hi) >> 1;
      if (s_cs[mid] <= r) lo = mid; else hi = mid;
    }
    const uint64_t off = 16 * s_cw[lo] + uint64_t(r - s_cs[lo]) * L;
    desc[r] = (off << 16) | L;
  }
}

struct Coll {
  uint64_t n = 0, sum = 0, N = 0;
  uint32_t L = 0;
  bool uniform = false;
};

int build_pack(cxbwt_ctx* c, const cxbwt_collection* colls, const std::vector<uint32_t>& idx,
               const std::vector<Coll>& info, uint32_t L, cudaStream_t st) {
  const uint32_t k = uint32_t(idx.size());
  Run r;
  r.st = st;
  Plan& pl = r.pl;
  std::vector<uint32_t> cs(k + 1, 0);  // first read of each collection
  std::vector<uint64_t> cw(k, 0);      // first store word of each collection
  std::vector<uint64_t> rows(k + 1, 0);
  uint64_t words = 0;
  for (uint32_t j = 0; j < k; ++j) {
    const Coll& ci = info[idx[j]];
    cs[j + 1] = cs[j] + uint32_t(ci.n);
    cw[j] = words;
    words += (ci.sum + 15) / 16;
    rows[j + 1] = rows[j] + ci.N;
  }
  pl.n = cs[k];
  pl.sum = pl.n * L;
  pl.N = rows[k];
  pl.Lmin = pl.Lmax = L;
  pl.uniform = true;
  pl.shift = bits_for(L);
  pl.D = (L + 3) / 4;
  pl.W = (L + 15) / 16;
  pl.len_passes = 0;
  pl.n_words = words;
  // The group plan's depth l: the option, else the autotuned one for the
  // pack's size class, else 16 (16 also when l = 12 leaves too many bases).
  int depth = c->opt.prefix_len;
  {
    int t_tile = 0, t_algo = 0, t_depth = 0;
    if (!depth && tuned_choice(c, L, pl.N, &t_tile, &t_algo, &t_depth) && t_algo == CXBWT_ALGO_GROUPS)
      depth = t_depth;
  }
  pl.depth = depth ? uint32_t(depth) : 16u;
  pl.seg_words = segsort_words(L, pl.depth);
  if (!pl.seg_words) {
    pl.depth = 16;
    pl.seg_words = segsort_words(L, 16);
  }
  pl.groups = true;
  pl.w_last = 0;
  plan_ids(pl, (c->opt.plan_flags & CXBWT_PLAN_ID64) != 0, (c->opt.plan_flags & CXBWT_PLAN_CARRY_BASE) != 0);
  r.shape = onesweep_shape(c->opt.tile_items, pl.idb);
  const uint32_t TILE = uint32_t(r.shape.tile());

  // ---- pack store, descriptors ---------------------------------------------
  CX_TRY(ensure(c, c->store, words * 4, "pack store"));
  auto* store = static_cast<uint32_t*>(c->store.p);
  uint64_t h2d = 0;
  for (uint32_t j = 0; j < k; ++j) {
    const cxbwt_collection& col = colls[idx[j]];
    const uint64_t w = (info[idx[j]].sum + 15) / 16;
    const bool dev = is_device_ptr(col.reads_2bit);
    CX_CUDA(c, cudaMemcpyAsync(store + cw[j], col.reads_2bit, w * 4, dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                               st));
    if (!dev) h2d += w * 4;
  }
  CX_TRY(ensure(c, c->desc, pl.n * 8, "read descriptors"));
  // Per-pack tables: collection read starts (for the collection pass) and word starts.
  CX_TRY(ensure(c, c->bhist, (k + 1) * 4 + k * 8 + 64, "pack tables"));
  auto* d_cs = static_cast<uint32_t*>(c->bhist.p);
  auto* d_cw = reinterpret_cast<uint64_t*>(static_cast<char*>(c->bhist.p) + ((k + 1) * 4 + 15) / 16 * 16);
  CX_CUDA(c, cudaMemcpyAsync(d_cs, cs.data(), (k + 1) * 4, cudaMemcpyHostToDevice, st));
  CX_CUDA(c, cudaMemcpyAsync(d_cw, cw.data(), k * 8, cudaMemcpyHostToDevice, st));
  const uint32_t desc_blocks = uint32_t(std::min<uint64_t>((pl.n + 255) / 256, uint64_t(c->sm_count) * 8));
  k_pack_desc<<<desc_blocks, 256, 0, st>>>(static_cast<uint64_t*>(c->desc.p), uint32_t(pl.n), d_cs, d_cw, k, L);
  CX_CUDA(c, cudaGetLastError());
  r.R = ReadIndex{store, words, static_cast<const uint64_t*>(c->desc.p), pl.shift, L, uint32_t(pl.n), 1u, pl.sym};

  // ---- workspace ---------------------------------------------------------
  char* misc = static_cast<char*>(c->misc.p);
  r.d_err = reinterpret_cast<uint32_t*>(misc + kMiscErr);
  r.d_counter = reinterpret_cast<uint32_t*>(misc + kMiscTileCounter);
  r.d_seg = reinterpret_cast<uint32_t*>(misc + kMiscSeg);
  CX_TRY(ensure(c, c->vals[0], pl.N * pl.idb, "suffix ids"));
  CX_TRY(ensure(c, c->vals[1], pl.N * pl.idb, "suffix ids"));
  CX_TRY(ensure(c, c->keys[0], pl.N * 4, "keys"));
  CX_TRY(ensure(c, c->keys[1], pl.N * 4, "keys"));
  const void* status_before = c->status.p;
  CX_TRY(ensure(c, c->status, (pl.N + TILE - 1) / TILE * kRadix * 8, "look-back words"));
  if (c->status.p != status_before) CX_CUDA(c, cudaMemsetAsync(c->status.p, 0, c->status.cap, st));
  CX_TRY(ensure(c, c->P, uint64_t(L) * kRadix * 4, "position counts"));
  CX_TRY(ensure(c, c->base, uint64_t(pl.D + 6) * kRadix * 4, "digit bases"));
  CX_TRY(ensure(c, c->lenhist, 4, "length histogram"));
  CX_TRY(ensure(c, c->seglist, (cta_list_cap(pl.N) + big_list_cap(pl.N, pl.seg_words)) * 8, "group lists"));
  CX_TRY(ensure(c, c->rhist, size_t(pl.W) * 4 * kRadix * 4, "group digit counts"));
  // Per-collection counts (5 each) after the pack's own counters.
  CX_TRY(ensure(c, c->out_dollar, uint64_t(k) * 5 * 8, "pack counts"));
  auto* d_counts = static_cast<unsigned long long*>(c->out_dollar.p);
  CX_CUDA(c, cudaMemsetAsync(d_counts, 0, uint64_t(k) * 5 * 8, st));
  r.vals[0] = c->vals[0].p;
  r.vals[1] = c->vals[1].p;
  r.keys[0] = static_cast<uint32_t*>(c->keys[0].p);
  r.keys[1] = static_cast<uint32_t*>(c->keys[1].p);
  r.base = static_cast<uint32_t*>(c->base.p);
  if (uint64_t(c->epoch) + pl.D + 64 * pl.W + 8 >= (uint64_t(1) << 30)) {
    CX_CUDA(c, cudaMemsetAsync(c->status.p, 0, c->status.cap, st));
    c->epoch = 0;
  }

  // ---- sort the pack as one collection -----------------------------------
  Slice sl;
  sl.rows = uint32_t(pl.N);
  int cur = 0;
  CX_TRY(sort_slice(c, r, sl, &cur, nullptr));

  // ---- stable pass by collection index -------------------------------------
  if (k > 1) {
    std::vector<uint32_t> cbase(kRadix, uint32_t(pl.N));
    for (uint32_t j = 0; j < k; ++j) cbase[j] = uint32_t(rows[j]);
    uint32_t* d_cbase = r.base + size_t(pl.D + 5) * kRadix;
    CX_CUDA(c, cudaMemcpyAsync(d_cbase, cbase.data(), kRadix * 4, cudaMemcpyHostToDevice, st));
    PassArgs a{};
    a.vals_in = r.vals[cur];
    a.vals_out = r.vals[cur ^ 1];
    a.digit_base = d_cbase;
    a.status = static_cast<unsigned long long*>(c->status.p);
    a.tile_counter = r.d_counter;
    a.err = r.d_err;
    a.R = r.R;
    a.n_gen = pl.N;
    a.n_out = uint32_t(pl.N);
    a.n_tiles = uint32_t((pl.N + TILE - 1) / TILE);
    a.epoch = ++c->epoch;
    a.key_shift = 0;
    a.n_reads = uint32_t(pl.n);
    a.coll_start = d_cs;
    a.n_coll = k;
    a.timeout_ns = kTimeoutNs;
    CX_CUDA(c, launch_onesweep(a, kSrcCollection, false, false, pl.idb, r.shape, st));
    cur ^= 1;
    ++r.sort_launches;
    r.sort_items += pl.N;
  }

  // ---- emit each collection from its rows ----------------------------------
  std::vector<uint32_t*> host_bwt(k, nullptr);
  for (uint32_t j = 0; j < k; ++j) {
    const cxbwt_collection& col = colls[idx[j]];
    const Coll& ci = info[idx[j]];
    const uint64_t bw = (ci.N + 15) / 16;
    EmitArgs e{};
    e.sa = vptr(r.vals[cur], pl.idb, rows[j]);
    e.n = uint32_t(ci.N);
    e.row0 = 0;
    e.n_total = ci.N;
    e.R = r.R;
    const bool bdev = is_device_ptr(col.out_bwt);
    e.bwt = col.out_bwt;
    if (!bdev) {
      // Host output: emit into the spare key buffer (free after the group finish), then copy.
      e.bwt = r.keys[0];
    }
    e.word_base = 0;
    uint64_t* dpos = col.out_dollar_pos;
    const bool ddev = dpos && is_device_ptr(dpos);
    e.dollar_pos = ddev ? dpos : nullptr;
    e.counts = d_counts + 5 * j;
    e.sa_out = nullptr;
    e.err = r.d_err;
    e.id_bytes = pl.idb;
    e.read_base = cs[j];
    e.n_reads_out = uint32_t(ci.n);
    if (dpos && !ddev) {
      // Host $ rows: emit them into the spare buffer after the BWT words.
      e.dollar_pos = reinterpret_cast<uint64_t*>(static_cast<char*>(c->vals[cur ^ 1].p));
    }
    CX_CUDA(c, launch_emit(e, st));
    ++r.launches;
    if (!bdev) {
      CX_CUDA(c, cudaMemcpyAsync(col.out_bwt, e.bwt, bw * 4, cudaMemcpyDeviceToHost, st));
      r.d2h += bw * 4;
    }
    if (dpos && !ddev) {
      CX_CUDA(c, cudaMemcpyAsync(dpos, e.dollar_pos, ci.n * 8, cudaMemcpyDeviceToHost, st));
      r.d2h += ci.n * 8;
    }
    if (col.out_counts) {
      const bool cdev = is_device_ptr(col.out_counts);
      CX_CUDA(c, cudaMemcpyAsync(col.out_counts, d_counts + 5 * j, 40,
                                 cdev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
    }
    if (!bdev || (dpos && !ddev)) CX_CUDA(c, cudaStreamSynchronize(st));  // spare buffers are reused by the next one
  }
  CX_CUDA(c, cudaMemcpyAsync(c->h_small + 4, r.d_err, 4, cudaMemcpyDeviceToHost, st));
  CX_CUDA(c, cudaStreamSynchronize(st));
  CX_TRY(take_device_error(c));
  c->stats.kernel_launches += r.launches + r.sort_launches + 1;
  c->stats.sort_pass_launches += r.sort_launches;
  c->stats.sort_pass_items += r.sort_items;
  c->stats.h2d_bytes += h2d;
  c->stats.d2h_bytes += r.d2h;
  c->stats.slices += 1;
  c->stats.builds += k;
  c->stats.bases += pl.sum;
  c->stats.suffixes += pl.N;
  return CXBWT_OK;
}

struct Item {
  std::vector<uint32_t> colls;  // a pack (several) or one collection built alone
  bool pack = false;
  uint32_t L = 0;
  uint64_t rows = 0;
};

// Worker contexts and threads of cxbwt_build_batch, kept by the context.
struct Pool {
  std::vector<cxbwt_ctx*> ctxs;
  std::vector<cudaStream_t> streams;
  std::vector<std::thread> threads;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  // the current batch
  const cxbwt_collection* colls = nullptr;
  const std::vector<Coll>* info = nullptr;
  const std::vector<Item>* items = nullptr;
  size_t next = 0, finished = 0;
  int status = CXBWT_OK;
  std::string err;
  bool stop = false;
  uint64_t generation = 0;
};

int run_item(cxbwt_ctx* c, const cxbwt_collection* colls, const std::vector<Coll>& info, const Item& it,
             cudaStream_t st) {
  if (it.pack) return build_pack(c, colls, it.colls, info, it.L, st);
  const cxbwt_collection& col = colls[it.colls[0]];
  return build_impl(c, col.reads_2bit, col.n_reads, col.lens, col.out_bwt, col.out_dollar_pos, col.out_counts,
                    nullptr, st);
}

void pool_worker(Pool* p, int w) {
  cxbwt_ctx* c = p->ctxs[w];
  cudaSetDevice(c->device);
  for (;;) {
    const Item* it = nullptr;
    {
      std::unique_lock<std::mutex> lock(p->mu);
      p->cv_work.wait(lock, [&] { return p->stop || (p->items && p->next < p->items->size()); });
      if (p->stop) return;
      it = &(*p->items)[p->next++];
    }
    int st = p->status == CXBWT_OK ? run_item(c, p->colls, *p->info, *it, p->streams[w]) : CXBWT_OK;
    if (st == CXBWT_OK && cudaStreamSynchronize(p->streams[w]) != cudaSuccess) st = CXBWT_ECUDA;
    {
      std::lock_guard<std::mutex> lock(p->mu);
      if (st != CXBWT_OK && p->status == CXBWT_OK) {
        p->status = st;
        p->err = c->err;
      }
      ++p->finished;
    }
    p->cv_done.notify_all();
  }
}

void pool_free(void* v) {
  auto* p = static_cast<Pool*>(v);
  {
    std::lock_guard<std::mutex> lock(p->mu);
    p->stop = true;
  }
  p->cv_work.notify_all();
  for (auto& t : p->threads) t.join();
  for (auto* c : p->ctxs) cxbwt_destroy(c);
  for (auto s : p->streams) cudaStreamDestroy(s);
  delete p;
}

constexpr int kMaxBatchWorkers = 8;

int get_pool(cxbwt_ctx* c, Pool** out) {
  if (c->batch_pool) {
    *out = static_cast<Pool*>(c->batch_pool);
    return CXBWT_OK;
  }
  auto* p = new Pool();
  const int workers = std::min(std::max(c->opt.batch_workers ? c->opt.batch_workers : 3, 1), kMaxBatchWorkers);
  for (int w = 0; w < workers; ++w) {
    cxbwt_options o = c->opt;
    o.device_budget_bytes = c->budget / workers;
    o.async = 0;
    o.timing = 0;
    cxbwt_ctx* wc = nullptr;
    int st = cxbwt_create(&wc, &o);
    cudaStream_t s = nullptr;
    if (st == CXBWT_OK && cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) st = CXBWT_ECUDA;
    if (st != CXBWT_OK) {
      if (wc) cxbwt_destroy(wc);
      p->stop = true;
      for (auto* x : p->ctxs) cxbwt_destroy(x);
      for (auto x : p->streams) cudaStreamDestroy(x);
      delete p;
      return fail(c, st, "could not create the batch worker contexts: %s", cxbwt_last_error(nullptr));
    }
    p->ctxs.push_back(wc);
    p->streams.push_back(s);
  }
  for (int w = 0; w < workers; ++w) p->threads.emplace_back(pool_worker, p, w);
  c->batch_pool = p;
  c->batch_pool_free = pool_free;
  *out = p;
  return CXBWT_OK;
}

}  // namespace

extern "C" int cxbwt_build_batch(cxbwt_ctx* c, const cxbwt_collection* colls, uint64_t k, void* stream_v) {
  if (!c) return CXBWT_EINVAL;
  c->err.clear();
  if (k == 0) return CXBWT_OK;
  if (!colls) return fail(c, CXBWT_EINVAL, "colls must not be NULL");
  CX_CUDA(c, cudaSetDevice(c->device));
  cudaStream_t st = static_cast<cudaStream_t>(stream_v);
  c->last_stream = st;
  // Length statistics of every collection: host lengths are scanned here,
  // device lengths by k_lenstats (one launch each, one copy back for all).
  std::vector<Coll> info(k);
  std::vector<uint64_t> dev_idx;
  for (uint64_t i = 0; i < k; ++i) {
    const cxbwt_collection& col = colls[i];
    if (!col.reads_2bit || !col.lens || !col.out_bwt || col.n_reads == 0)
      return fail(c, CXBWT_EINVAL, "collection %llu: NULL pointer or no reads", (unsigned long long)i);
    Coll& ci = info[i];
    ci.n = col.n_reads;
    if (is_device_ptr(col.lens)) {
      dev_idx.push_back(i);
      continue;
    }
    const uint32_t* h = col.lens;
    ci.L = h[0];
    ci.uniform = true;
    for (uint64_t r = 0; r < col.n_reads; ++r) {
      if (h[r] == 0 || h[r] > 65535)
        return fail(c, CXBWT_EINVAL, "collection %llu: a read length is 0 or above 65535", (unsigned long long)i);
      ci.uniform = ci.uniform && h[r] == ci.L;
      ci.sum += h[r];
    }
    ci.N = ci.sum + ci.n;
  }
  if (!dev_idx.empty()) {
    const uint64_t m = dev_idx.size();
    CX_TRY(ensure(c, c->rhist, m * 32, "length statistics"));
    auto* d_ls = static_cast<unsigned long long*>(c->rhist.p);
    std::vector<unsigned long long> ls(m * 4);
    for (uint64_t j = 0; j < m; ++j) {
      ls[4 * j] = ~0ull;
      ls[4 * j + 1] = ls[4 * j + 2] = ls[4 * j + 3] = 0;
    }
    CX_CUDA(c, cudaMemcpyAsync(d_ls, ls.data(), m * 32, cudaMemcpyHostToDevice, st));
    for (uint64_t j = 0; j < m; ++j)
      CX_CUDA(c, launch_lenstats(colls[dev_idx[j]].lens, colls[dev_idx[j]].n_reads, d_ls + 4 * j, st));
    CX_CUDA(c, cudaMemcpyAsync(ls.data(), d_ls, m * 32, cudaMemcpyDeviceToHost, st));
    CX_CUDA(c, cudaStreamSynchronize(st));
    for (uint64_t j = 0; j < m; ++j) {
      Coll& ci = info[dev_idx[j]];
      if (ls[4 * j + 3])
        return fail(c, CXBWT_EINVAL, "collection %llu: a read length is 0 or above 65535",
                    (unsigned long long)dev_idx[j]);
      ci.L = uint32_t(ls[4 * j + 1]);
      ci.uniform = ls[4 * j] == ls[4 * j + 1];
      ci.sum = ls[4 * j + 2];
      ci.N = ci.sum + ci.n;
    }
  }
  // Small collections (launch-bound alone) of one read length share packs;
  // the rest are built alone.
  const int sm = c->opt.batch_small_mrows;
  const uint64_t small = sm < 0 ? 0 : uint64_t(sm ? sm : 2) << 20, pack_cap = std::max<uint64_t>(8 * small, 1);
  std::vector<Item> items;
  std::vector<int64_t> open(65536, -1);
  for (uint32_t i = 0; i < k; ++i) {
    const Coll& ci = info[i];
    if (!ci.uniform || !segsort_words(ci.L, 16) || ci.N > small) {
      Item it;
      it.colls.push_back(i);
      it.rows = ci.N;
      items.push_back(it);
      continue;
    }
    int64_t& o = open[ci.L];
    if (o >= 0 && (items[o].rows + ci.N > pack_cap || items[o].colls.size() == kMaxPackCollections - 1)) o = -1;
    if (o < 0) {
      Item it;
      it.pack = true;
      it.L = ci.L;
      items.push_back(it);
      o = int64_t(items.size()) - 1;
    }
    items[o].colls.push_back(i);
    items[o].rows += ci.N;
  }
  // Largest first: the pool then finishes with the small ones.
  std::stable_sort(items.begin(), items.end(), [](const Item& a, const Item& b) { return a.rows > b.rows; });
  // Inputs may come from work queued on the caller's stream.
  CX_CUDA(c, cudaStreamSynchronize(st));
  Pool* p = nullptr;
  CX_TRY(get_pool(c, &p));
  for (auto* wc : p->ctxs) wc->tuned = c->tuned;  // the workers build with the context's autotuned plans
  {
    std::lock_guard<std::mutex> lock(p->mu);
    p->colls = colls;
    p->info = &info;
    p->items = &items;
    p->next = 0;
    p->finished = 0;
    p->status = CXBWT_OK;
    p->err.clear();
  }
  p->cv_work.notify_all();
  int status;
  {
    std::unique_lock<std::mutex> lock(p->mu);
    p->cv_done.wait(lock, [&] { return p->finished == items.size(); });
    status = p->status;
    if (status != CXBWT_OK) c->err = p->err;
    p->items = nullptr;
  }
  for (auto* wc : p->ctxs) {
    c->stats.builds += wc->stats.builds;
    c->stats.bases += wc->stats.bases;
    c->stats.suffixes += wc->stats.suffixes;
    c->stats.kernel_launches += wc->stats.kernel_launches;
    c->stats.sort_pass_launches += wc->stats.sort_pass_launches;
    c->stats.sort_pass_items += wc->stats.sort_pass_items;
    c->stats.h2d_bytes += wc->stats.h2d_bytes;
    c->stats.d2h_bytes += wc->stats.d2h_bytes;
    c->stats.slices += wc->stats.slices;
    wc->stats = cxbwt_stats{};
  }
  return status;
}
