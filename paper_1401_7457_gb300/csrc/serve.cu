// Serving: continuous batching of BWT-build requests.
//
// A server owns W workers; each worker is a host thread with its own context
// (device workspace, within budget / W) and its own CUDA stream, so up to W
// builds are on the GPU at once and overlap there.  Requests queue in arrival
// order.  A free worker takes the oldest request.  When that one is small
// (under kPackRows suffixes, where a lone build is bound by launches and
// histograms rather than by the sort), the worker also takes every other
// queued small request of the same read length that fits its pack cap
// (requests that arrived while others were running join the next pack) and
// builds them as one batch (cxbwt_build_batch: one sort for the pack, split
// by collection); a larger request is built alone (cxbwt_build), so it never
// waits behind another one in the same worker while a second worker is free.
// Each BWT streams back to the caller's host buffers, and each request's
// result is exactly what cxbwt_build gives for it alone.  Admission is by
// device memory: a worker's context never holds more than its share of the
// budget (larger requests are built in slices).
#include <cuda_runtime.h>

#include <chrono>
#include <condition_variable>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>

#include "host.cuh"

using namespace cxbwt;
using namespace cxbwt::host;

namespace {

using Clock = std::chrono::steady_clock;

// Requests below this many suffixes are packed with others of their read
// length (the batch path packs collections below the same size).
constexpr uint64_t kPackRows = uint64_t(2) << 20;

struct Req {
  cxbwt_request r{};
  uint64_t ticket = 0;
  uint64_t N = 0;
  uint32_t L = 0;
  bool uniform = true;
  int status = CXBWT_OK;
  bool done = false;
  Clock::time_point t_submit, t_start, t_done;
};

}  // namespace

struct cxbwt_server {
  cxbwt_server_options opt{};
  std::vector<cxbwt_ctx*> ctxs;
  std::vector<cudaStream_t> streams;
  std::vector<std::thread> threads;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Req*> queue;
  std::unordered_map<uint64_t, std::unique_ptr<Req>> reqs;
  uint64_t next_ticket = 1;
  uint64_t pack_cap = 0;
  bool stop = false;
  uint64_t completed = 0, packs = 0, bases = 0;
};

namespace {

void worker_loop(cxbwt_server* s, int w) {
  cxbwt_ctx* ctx = s->ctxs[w];
  cudaStream_t st = s->streams[w];
  cudaSetDevice(s->opt.device);
  std::vector<Req*> take;
  std::vector<cxbwt_collection> colls;
  for (;;) {
    take.clear();
    {
      std::unique_lock<std::mutex> lock(s->mu);
      s->cv_work.wait(lock, [&] { return s->stop || !s->queue.empty(); });
      if (s->queue.empty()) return;  // stop requested and nothing left
      // The oldest request, then every queued request of its read length while the pack fits.
      Req* first = s->queue.front();
      s->queue.pop_front();
      take.push_back(first);
      uint64_t rows = first->N;
      if (first->uniform && first->N < kPackRows) {
        for (auto it = s->queue.begin(); it != s->queue.end() && take.size() < kMaxPackCollections - 1;) {
          Req* q = *it;
          if (q->uniform && q->L == first->L && q->N < kPackRows && rows + q->N <= s->pack_cap) {
            rows += q->N;
            take.push_back(q);
            it = s->queue.erase(it);
          } else {
            ++it;
          }
        }
      }
      const auto now = Clock::now();
      for (Req* q : take) q->t_start = now;
    }
    colls.clear();
    for (Req* q : take) {
      cxbwt_collection c{};
      c.reads_2bit = q->r.reads_2bit;
      c.n_reads = q->r.n_reads;
      c.lens = q->r.lens;
      c.out_bwt = q->r.out_bwt;
      c.out_dollar_pos = q->r.out_dollar_pos;
      c.out_counts = q->r.out_counts;
      colls.push_back(c);
    }
    int status = take.size() == 1 ? cxbwt_build(ctx, colls[0].reads_2bit, colls[0].n_reads, colls[0].lens,
                                                colls[0].out_bwt, colls[0].out_dollar_pos, colls[0].out_counts, st)
                                  : cxbwt_build_batch(ctx, colls.data(), colls.size(), st);
    if (status == CXBWT_OK) {
      const cudaError_t e = cudaStreamSynchronize(st);
      if (e != cudaSuccess) status = CXBWT_ECUDA;
    }
    {
      std::lock_guard<std::mutex> lock(s->mu);
      const auto now = Clock::now();
      for (Req* q : take) {
        q->status = status;
        q->done = true;
        q->t_done = now;
        s->bases += q->N - q->r.n_reads;
      }
      s->completed += take.size();
      s->packs += 1;
    }
    s->cv_done.notify_all();
  }
}

}  // namespace

extern "C" {

void cxbwt_default_server_options(cxbwt_server_options* o) {
  if (!o) return;
  std::memset(o, 0, sizeof *o);
  // Two concurrent builds: on the served workload (requests of 5M to 750M
  // suffixes) a third one raised p99 latency at every load (measured).
  o->workers = 2;
}

int cxbwt_server_create(cxbwt_server** out, const cxbwt_server_options* opt) {
  if (!out) return CXBWT_EINVAL;
  *out = nullptr;
  cxbwt_server_options o;
  cxbwt_default_server_options(&o);
  if (opt) o = *opt;
  if (o.workers <= 0) o.workers = 2;
  if (o.workers > 16) return CXBWT_EINVAL;
  if (cudaSetDevice(o.device) != cudaSuccess) {
    cudaGetLastError();
    return CXBWT_ECUDA;
  }
  if (!o.device_budget_bytes) {
    size_t free_b = 0, total_b = 0;
    cudaMemGetInfo(&free_b, &total_b);
    o.device_budget_bytes = std::min<uint64_t>(uint64_t(120) << 30, uint64_t(double(free_b) * 0.9));
  }
  auto* s = new cxbwt_server();
  s->opt = o;
  const uint64_t share = o.device_budget_bytes / uint64_t(o.workers);
  // Pack cap: about a third of what one worker's share holds at ~25 bytes per suffix.
  s->pack_cap = o.max_pack_suffixes ? o.max_pack_suffixes : std::max<uint64_t>(share / 25 / 3, 1u << 20);
  for (int w = 0; w < o.workers; ++w) {
    cxbwt_options co;
    cxbwt_default_options(&co);
    co.device = o.device;
    co.device_budget_bytes = share;
    co.batch_workers = 1;  // the server's workers are the concurrency; a pack is built by its own worker
    cxbwt_ctx* c = nullptr;
    int st = cxbwt_create(&c, &co);
    cudaStream_t stream = nullptr;
    if (st == CXBWT_OK && cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking) != cudaSuccess) st = CXBWT_ECUDA;
    if (st != CXBWT_OK) {
      if (c) cxbwt_destroy(c);
      s->stop = true;
      for (auto* x : s->ctxs) cxbwt_destroy(x);
      for (auto x : s->streams) cudaStreamDestroy(x);
      delete s;
      return st;
    }
    s->ctxs.push_back(c);
    s->streams.push_back(stream);
  }
  for (int w = 0; w < o.workers; ++w) s->threads.emplace_back(worker_loop, s, w);
  *out = s;
  return CXBWT_OK;
}

void cxbwt_server_destroy(cxbwt_server* s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lock(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  for (auto& t : s->threads) t.join();
  for (auto* c : s->ctxs) cxbwt_destroy(c);
  for (auto x : s->streams) cudaStreamDestroy(x);
  delete s;
}

int cxbwt_submit(cxbwt_server* s, const cxbwt_request* req, uint64_t* ticket) {
  if (!s || !req || !ticket || !req->reads_2bit || !req->lens || !req->out_bwt || req->n_reads == 0)
    return CXBWT_EINVAL;
  auto q = std::make_unique<Req>();
  q->r = *req;
  q->L = req->lens[0];
  uint64_t sum = 0;
  for (uint64_t i = 0; i < req->n_reads; ++i) {
    const uint32_t L = req->lens[i];
    if (L == 0 || L > 65535) return CXBWT_EINVAL;
    q->uniform = q->uniform && L == q->L;
    sum += L;
  }
  q->N = sum + req->n_reads;
  q->t_submit = Clock::now();
  {
    std::lock_guard<std::mutex> lock(s->mu);
    if (s->stop) return CXBWT_EBUSY;
    q->ticket = s->next_ticket++;
    *ticket = q->ticket;
    s->queue.push_back(q.get());
    s->reqs.emplace(q->ticket, std::move(q));
  }
  s->cv_work.notify_one();
  return CXBWT_OK;
}

int cxbwt_poll(cxbwt_server* s, uint64_t ticket, int* done) {
  if (!s || !done) return CXBWT_EINVAL;
  std::lock_guard<std::mutex> lock(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return CXBWT_EINVAL;
  *done = it->second->done ? 1 : 0;
  return it->second->done ? it->second->status : CXBWT_OK;
}

int cxbwt_wait(cxbwt_server* s, uint64_t ticket) {
  if (!s) return CXBWT_EINVAL;
  std::unique_lock<std::mutex> lock(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return CXBWT_EINVAL;
  Req* q = it->second.get();
  s->cv_done.wait(lock, [&] { return q->done; });
  return q->status;
}

int cxbwt_ticket_times(cxbwt_server* s, uint64_t ticket, double* queued_ms, double* latency_ms) {
  if (!s) return CXBWT_EINVAL;
  std::lock_guard<std::mutex> lock(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end() || !it->second->done) return CXBWT_EINVAL;
  const Req* q = it->second.get();
  using ms = std::chrono::duration<double, std::milli>;
  if (queued_ms) *queued_ms = ms(q->t_start - q->t_submit).count();
  if (latency_ms) *latency_ms = ms(q->t_done - q->t_submit).count();
  return CXBWT_OK;
}

int cxbwt_server_counters(cxbwt_server* s, uint64_t* completed, uint64_t* packs, uint64_t* bases) {
  if (!s) return CXBWT_EINVAL;
  std::lock_guard<std::mutex> lock(s->mu);
  if (completed) *completed = s->completed;
  if (packs) *packs = s->packs;
  if (bases) *bases = s->bases;
  return CXBWT_OK;
}

}  // extern "C"
