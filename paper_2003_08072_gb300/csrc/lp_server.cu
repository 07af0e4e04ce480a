// Serving loop: a stream of LP instances of different sizes solved with continuous batching.
//
// A request is copied at submission and queued.  max_live worker threads each own a
// non-blocking CUDA stream; a free worker admits the request at the head of the queue as soon
// as its device footprint (lp_footprint_bytes) fits into what the admission budget has left,
// creates its context on the worker stream, runs Algorithm 2 and releases the memory.  Work of
// all live instances is in flight on the GPU at the same time (one stream each), so requests
// that arrive while others are being solved start as soon as a slot and memory free up rather
// than after the queue drains.  Contexts draw device memory from the stream-ordered pool, so
// admission and release cost no device-wide synchronisation.  Admission is first come, first
// served: a head request that does not fit waits for memory and holds the later ones back.
#include <chrono>
#include <condition_variable>
#include <deque>
#include <memory>
#include <mutex>
#include <new>
#include <string>
#include <system_error>
#include <thread>
#include <unordered_map>
#include <vector>

#include "lp_batch.cuh"
#include "lp_internal.cuh"

namespace {

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

size_t dtype_bytes(lp_dtype t) { return t == LP_F64 ? 8 : (t == LP_F32 ? 4 : 2); }

struct Request {
  int64_t ticket = 0;
  int32_t m = 0;
  int64_t n = 0;
  lp_layout layout = LP_DENSE_COLMAJOR;
  lp_dtype a_dtype = LP_F32;
  int64_t nnz = 0;
  std::vector<unsigned char> A;
  std::vector<int64_t> indptr;
  std::vector<int32_t> indices;
  std::vector<double> b, c;
  uint64_t footprint = 0;
  std::vector<double> x, y, s;
  lp_info info{};
  lp_status status = LP_OK;
  std::string error;
  double t_submit = 0, t_start = 0, t_done = 0;
  bool done = false;
};

}  // namespace

struct lp_server {
  int dev = 0;
  int num_sms = 0;
  lp_params prm{};
  uint64_t budget = 0;
  int max_live = 1;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Request*> queue;
  std::unordered_map<int64_t, std::unique_ptr<Request>> all;
  std::deque<int64_t> finished;   // completed tickets not yet handed out by lp_server_wait_any
  uint64_t in_use = 0, peak = 0;
  int live = 0, peak_live = 0;
  int64_t next_ticket = 1, submitted = 0, completed = 0, failed = 0;
  bool stop = false;
  std::vector<std::thread> workers;
  CgBatcher* batcher = nullptr;   // shared launches of the live instances' CG iterations
};

namespace {

void solve_one(lp_server* sv, Request* r, cudaStream_t st) {
  lp_ctx* ctx = nullptr;
  // no exception may end a worker thread: a failed host allocation fails the request
  try {
    r->x.assign(r->n, 0.0);
    r->y.assign(r->m, 0.0);
    r->s.assign(r->n, 0.0);
  } catch (const std::bad_alloc&) {
    r->status = LP_ERR_OOM;
    r->info.status = LP_ERR_OOM;
    r->error = "lp_server: host allocation for the result failed";
    return;
  }
  lp_status status = lp_create(&ctx, r->m, r->n, r->layout, r->a_dtype, r->A.data(),
                               r->layout == LP_CSR ? r->indptr.data() : nullptr,
                               r->layout == LP_CSR ? r->indices.data() : nullptr, r->nnz,
                               r->b.data(), r->c.data(), &sv->prm, st);
  if (status == LP_OK) {
    ctx->batcher = sv->batcher;
    status = lp_ipm_solve(ctx, r->x.data(), r->y.data(), r->s.data(), 0, &r->info);
    if (status != LP_OK) r->error = lp_last_error();
  } else {
    r->error = lp_last_error();
  }
  lp_destroy(ctx);
  r->status = status;
  r->info.status = status;
  // the instance's data is no longer needed once solved
  std::vector<unsigned char>().swap(r->A);
  std::vector<int64_t>().swap(r->indptr);
  std::vector<int32_t>().swap(r->indices);
}

void worker_main(lp_server* sv) {
  cudaSetDevice(sv->dev);
  cudaStream_t st = nullptr;
  if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    st = nullptr;
  }
  for (;;) {
    Request* r = nullptr;
    {
      std::unique_lock<std::mutex> lk(sv->mu);
      sv->cv_work.wait(lk, [&] {
        return sv->stop ||
               (!sv->queue.empty() && sv->in_use + sv->queue.front()->footprint <= sv->budget);
      });
      if (sv->stop) break;
      r = sv->queue.front();
      sv->queue.pop_front();
      sv->in_use += r->footprint;
      sv->peak = std::max(sv->peak, sv->in_use);
      ++sv->live;
      sv->peak_live = std::max(sv->peak_live, sv->live);
      r->t_start = now_s();
    }
    solve_one(sv, r, st);
    {
      std::lock_guard<std::mutex> lk(sv->mu);
      sv->in_use -= r->footprint;
      --sv->live;
      r->t_done = now_s();
      r->done = true;
      ++sv->completed;
      if (r->status != LP_OK) ++sv->failed;
      sv->finished.push_back(r->ticket);
    }
    sv->cv_done.notify_all();
    sv->cv_work.notify_all();
  }
  if (st) cudaStreamDestroy(st);
}

}  // namespace

extern "C" {

lp_status lp_server_create(lp_server** out, uint64_t mem_budget_bytes, int32_t max_live,
                           const lp_params* prm) {
  if (!out) return LP_ERR_ARG;
  *out = nullptr;
  if (max_live < 1 || max_live > 256 || mem_budget_bytes == 0) {
    lp_set_error("lp_server_create: need 1 <= max_live <= 256 and a nonzero budget");
    return LP_ERR_ARG;
  }
  std::unique_ptr<lp_server> sv(new (std::nothrow) lp_server());
  if (!sv) {
    lp_set_error("lp_server_create: host allocation failed");
    return LP_ERR_OOM;
  }
  if (prm) sv->prm = *prm; else lp_params_default(&sv->prm);
  // a persistent CG loop holds every SM for its solve, which would serialise the live
  // instances: with several of them each runs its CG solves as CUDA graph launches instead.
  // Likewise the one-launch Cholesky sweep, whose CTAs wait on one another's tiles: next to
  // other instances' kernels those waiting CTAs hold SMs the others could use (measured: 38.4
  // against 43.7 LPs/s for the block-step launches with 16 live instances)
  if (max_live > 1) {
    sv->prm.persistent_cg = 0;
    sv->prm.factor_dag = 0;
  }
  if (cudaGetDevice(&sv->dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sv->num_sms, cudaDevAttrMultiProcessorCount, sv->dev) !=
          cudaSuccess) {
    cudaGetLastError();
    lp_set_error("lp_server_create: no CUDA device");
    return LP_ERR_CUDA;
  }
  sv->budget = mem_budget_bytes;
  sv->max_live = max_live;
  // shared CG launches on request (without the engine, e.g. if its pinned tables cannot be
  // allocated, every instance runs its own CG loop)
  if (sv->prm.shared_cg && max_live > 1) sv->batcher = lpk::cg_batcher_create(sv->dev, sv->num_sms);
  try {
    sv->workers.reserve(max_live);
    for (int i = 0; i < max_live; ++i) sv->workers.emplace_back(worker_main, sv.get());
  } catch (const std::exception&) {
    // could not start every worker (std::system_error or std::bad_alloc): stop the ones running
    lp_server_destroy(sv.release());
    lp_set_error("lp_server_create: could not start the worker threads");
    return LP_ERR_OOM;
  }
  *out = sv.release();
  return LP_OK;
}

lp_status lp_server_submit(lp_server* sv, int32_t m, int64_t n, lp_layout layout,
                           lp_dtype a_dtype, const void* A_vals, const int64_t* indptr,
                           const int32_t* indices, int64_t nnz, const double* b, const double* c,
                           int64_t* ticket) {
  if (!sv || !ticket || !A_vals || !b || !c) {
    lp_set_error("lp_server_submit: NULL argument");
    return LP_ERR_ARG;
  }
  *ticket = 0;
  if (m < 1 || n < m || m > 8192 || (a_dtype != LP_F32 && a_dtype != LP_F64) ||
      (layout == LP_CSR && (!indptr || !indices || nnz < 0))) {
    lp_set_error("lp_server_submit: bad sizes, dtype or CSR arrays");
    return LP_ERR_ARG;
  }
  std::unique_ptr<Request> r(new (std::nothrow) Request());
  if (!r) {
    lp_set_error("lp_server_submit: host allocation failed");
    return LP_ERR_OOM;
  }
  r->m = m;
  r->n = n;
  r->layout = layout;
  r->a_dtype = a_dtype;
  r->nnz = layout == LP_CSR ? nnz : 0;
  const size_t es = dtype_bytes(a_dtype);
  const size_t count = layout == LP_CSR ? (size_t)nnz : (size_t)m * (size_t)n;
  const auto* src = reinterpret_cast<const unsigned char*>(A_vals);
  try {
    r->A.assign(src, src + count * es);
    if (layout == LP_CSR) {
      r->indptr.assign(indptr, indptr + m + 1);
      r->indices.assign(indices, indices + nnz);
    }
    r->b.assign(b, b + m);
    r->c.assign(c, c + n);
  } catch (const std::bad_alloc&) {
    lp_set_error("lp_server_submit: host allocation for the request copy failed");
    return LP_ERR_OOM;
  }
  r->footprint = lp_footprint_bytes(m, n, layout, a_dtype, r->nnz, &sv->prm, sv->num_sms);
  if (r->footprint > sv->budget) {
    lp_set_error("lp_server_submit: the instance alone exceeds the admission budget");
    return LP_ERR_OOM;
  }
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    r->ticket = sv->next_ticket++;
    r->t_submit = now_s();
    Request* raw = r.get();
    try {
      sv->all.emplace(raw->ticket, std::move(r));
      sv->queue.push_back(raw);
    } catch (const std::bad_alloc&) {
      sv->all.erase(raw->ticket);
      lp_set_error("lp_server_submit: host allocation failed");
      return LP_ERR_OOM;
    }
    *ticket = raw->ticket;
    ++sv->submitted;
  }
  sv->cv_work.notify_one();
  return LP_OK;
}

lp_status lp_server_wait_any(lp_server* sv, int32_t timeout_ms, int64_t* ticket) {
  if (!sv || !ticket) return LP_ERR_ARG;
  *ticket = 0;
  std::unique_lock<std::mutex> lk(sv->mu);
  const bool got = sv->cv_done.wait_for(lk, std::chrono::milliseconds(std::max(timeout_ms, 0)),
                                        [&] { return !sv->finished.empty(); });
  if (!got) {
    lp_set_error("lp_server_wait_any: no request finished within the timeout");
    return LP_ERR_TIMEOUT;
  }
  *ticket = sv->finished.front();
  sv->finished.pop_front();
  return LP_OK;
}

lp_status lp_server_result(lp_server* sv, int64_t ticket, double* x, double* y, double* s,
                           lp_info* info, double* times) {
  if (!sv) return LP_ERR_ARG;
  std::unique_ptr<Request> r;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    auto it = sv->all.find(ticket);
    if (it == sv->all.end() || !it->second->done) {
      lp_set_error("lp_server_result: unknown or unfinished ticket");
      return LP_ERR_ARG;
    }
    r = std::move(it->second);
    sv->all.erase(it);
    // a ticket read here is no longer handed out by lp_server_wait_any
    for (auto f = sv->finished.begin(); f != sv->finished.end(); ++f)
      if (*f == ticket) {
        sv->finished.erase(f);
        break;
      }
  }
  if (x) std::copy(r->x.begin(), r->x.end(), x);
  if (y) std::copy(r->y.begin(), r->y.end(), y);
  if (s) std::copy(r->s.begin(), r->s.end(), s);
  if (info) *info = r->info;
  if (times) {
    times[0] = r->t_start - r->t_submit;   // queued
    times[1] = r->t_done - r->t_start;     // on the GPU
    times[2] = r->t_done - r->t_submit;    // latency
  }
  if (r->status != LP_OK) lp_set_error(r->error);
  return r->status;
}

lp_status lp_server_stats(lp_server* sv, lp_server_stats_t* out) {
  if (!sv || !out) return LP_ERR_ARG;
  std::lock_guard<std::mutex> lk(sv->mu);
  out->submitted = sv->submitted;
  out->completed = sv->completed;
  out->failed = sv->failed;
  out->queued = (int64_t)sv->queue.size();
  out->live = sv->live;
  out->peak_live = sv->peak_live;
  out->mem_in_use = sv->in_use;
  out->mem_peak = sv->peak;
  out->mem_budget = sv->budget;
  long long rounds = 0, jobs = 0;
  if (sv->batcher) lpk::cg_batcher_stats(sv->batcher, &rounds, &jobs);
  out->batched_rounds = rounds;
  out->batched_cg_solves = jobs;
  return LP_OK;
}

void lp_server_destroy(lp_server* sv) {
  if (!sv) return;
  {
    // queued requests are dropped; live ones finish first
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->queue.clear();
    sv->stop = true;
  }
  sv->cv_work.notify_all();
  for (auto& t : sv->workers) t.join();
  lpk::cg_batcher_destroy(sv->batcher);
  delete sv;
}

}  // extern "C"
