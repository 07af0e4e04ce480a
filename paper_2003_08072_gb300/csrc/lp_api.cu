// C ABI of the sketch-preconditioned infeasible IPM (include/lp.h): context management and
// the host-side sequencing of the kernels for Algorithms 1 and 2.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <memory>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "lp_batch.cuh"
#include "lp_internal.cuh"

using namespace lpk;

std::atomic<long long> lpk::g_launches{0};

static thread_local std::string g_err;

void lp_set_error(const std::string& msg) { g_err = msg; }

lp_status lp_cuda_fail(cudaError_t e, const char* what) {
  g_err = std::string(what) + ": " + cudaGetErrorString(e);
  cudaGetLastError();
  return LP_ERR_CUDA;
}

static lp_status fail(lp_status st, const std::string& msg) {
  g_err = msg;
  return st;
}

#define LP_TRY(expr)                    \
  do {                                  \
    lp_status s__ = (expr);             \
    if (s__ != LP_OK) return s__;       \
  } while (0)

static size_t dtype_size(lp_dtype t) {
  switch (t) {
    case LP_F64: return 8;
    case LP_F32: return 4;
    case LP_BF16: return 2;
    case LP_F16: return 2;
  }
  return 0;
}

static int round_up(int v, int q) { return (v + q - 1) / q * q; }

extern "C" {

const char* lp_last_error(void) { return g_err.c_str(); }

const char* lp_status_str(lp_status st) {
  switch (st) {
    case LP_OK: return "LP_OK";
    case LP_ERR_ARG: return "LP_ERR_ARG";
    case LP_ERR_OOM: return "LP_ERR_OOM";
    case LP_ERR_CUDA: return "LP_ERR_CUDA";
    case LP_ERR_BREAKDOWN: return "LP_ERR_BREAKDOWN";
    case LP_ERR_NOT_CONVERGED: return "LP_ERR_NOT_CONVERGED";
    case LP_ERR_TIMEOUT: return "LP_ERR_TIMEOUT";
    case LP_ERR_NUMERIC: return "LP_ERR_NUMERIC";
  }
  return "LP_ERR_UNKNOWN";
}

lp_status lp_params_default(lp_params* p) {
  if (!p) return fail(LP_ERR_ARG, "lp_params_default: NULL");
  p->tol = 1e-8;
  p->cg_rel_tol = 1e-6;
  p->sigma = 0.5;
  p->gamma = 0.99;
  p->cg_max_iter = 500;
  p->ipm_max_iter = 200;
  p->refine_max = 6;
  p->sketch_s = 4;
  p->sketch_w = 0;
  p->cg_theory_rule = 1;
  p->seed = 0;
  p->stream_dtype = LP_F64;
  p->cg_batch = 4;
  p->inner_solver = LP_INNER_CG;
  p->sketch_kind = LP_SKETCH_SPARSE;
  p->use_graphs = 1;
  p->gram_tensor_cores = 1;
  p->autotune = 1;
  p->shared_cg = 0;
  p->persistent_cg = 0;
  p->factor_dag = 1;
  return LP_OK;
}

}  // extern "C"

static lp_status check_params(const lp_params& p, int m) {
  if (!(p.tol > 0) || !(p.cg_rel_tol >= 0) || !(p.sigma > 0 && p.sigma < 0.8) ||
      !(p.gamma > 0 && p.gamma < 1))
    return fail(LP_ERR_ARG, "invalid tolerance, sigma (0, 4/5) or gamma (0, 1)");
  if (p.cg_max_iter < 1 || p.ipm_max_iter < 0 || p.refine_max < 0 || p.cg_batch < 1)
    return fail(LP_ERR_ARG, "invalid iteration caps");
  if (p.sketch_s < 1 || p.sketch_w < 0) return fail(LP_ERR_ARG, "invalid sketch size");
  if (p.inner_solver != LP_INNER_CG && p.inner_solver != LP_INNER_RICHARDSON)
    return fail(LP_ERR_ARG, "inner_solver must be LP_INNER_CG or LP_INNER_RICHARDSON");
  if (p.sketch_kind != LP_SKETCH_SPARSE && p.sketch_kind != LP_SKETCH_GAUSSIAN)
    return fail(LP_ERR_ARG, "sketch_kind must be LP_SKETCH_SPARSE or LP_SKETCH_GAUSSIAN");
  const int w = p.sketch_w ? p.sketch_w : 4 * m;
  if (w % p.sketch_s != 0) return fail(LP_ERR_ARG, "sketch_w must be a multiple of sketch_s");
  if (w < m) return fail(LP_ERR_ARG, "sketch_w must be >= m");
  if (w > (1 << 20)) return fail(LP_ERR_ARG, "sketch_w too large");
  return LP_OK;
}

// Device memory of a context comes from the device's stream-ordered pool, allocated and freed
// in order on the context stream (set for the calling thread by AllocStream while lp_create or
// lp_destroy runs).  Creating and destroying contexts, which the serving loop does for every
// request, then neither synchronises the device nor hands memory back to the driver.
static thread_local cudaStream_t t_alloc_stream = nullptr;

struct AllocStream {
  cudaStream_t prev;
  explicit AllocStream(cudaStream_t s) : prev(t_alloc_stream) { t_alloc_stream = s; }
  ~AllocStream() { t_alloc_stream = prev; }
};

// Keep freed pool memory for reuse (once per device).
static void keep_pool_memory(int dev) {
  static std::mutex mu;
  static std::vector<int> done;
  std::lock_guard<std::mutex> lk(mu);
  if (std::find(done.begin(), done.end(), dev) != done.end()) return;
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
    uint64_t thr = UINT64_MAX;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
  }
  cudaGetLastError();
  done.push_back(dev);
}

template <typename T>
static lp_status dalloc(T** p, size_t count) {
  *p = nullptr;
  if (count == 0) count = 1;
  cudaError_t e = cudaMallocAsync((void**)p, count * sizeof(T), t_alloc_stream);
  if (e != cudaSuccess) {
    *p = nullptr;
    cudaGetLastError();
    return fail(LP_ERR_OOM, std::string("cudaMallocAsync: ") + cudaGetErrorString(e));
  }
  return LP_OK;
}

// Small pinned host blocks (the context's scalar mirrors) from a process-wide free list.
static std::mutex g_pin_mu;
static std::vector<void*> g_pin_free;
constexpr size_t kPinBlock = 512;

static void* pinned_block() {
  {
    std::lock_guard<std::mutex> lk(g_pin_mu);
    if (!g_pin_free.empty()) {
      void* p = g_pin_free.back();
      g_pin_free.pop_back();
      return p;
    }
  }
  void* p = nullptr;
  if (cudaMallocHost(&p, kPinBlock) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return p;
}

static void pinned_release(void* p) {
  if (!p) return;
  std::lock_guard<std::mutex> lk(g_pin_mu);
  g_pin_free.push_back(p);
}

static void dfree(void* p) {
  if (p) cudaFreeAsync(p, t_alloc_stream);
}

static void cg_graph_free(lp_ctx::CgGraph& g);

extern "C" void lp_destroy(lp_ctx* c) {
  if (!c) return;
  cudaStreamSynchronize(c->st);
  AllocStream as(c->st);
  if (c->own_As) dfree(c->As_req);
  dfree(c->A);
  dfree(c->cs2);
  if (c->own_svals) dfree(c->svals_req);
  dfree(c->colptr);
  dfree(c->rowidx);
  dfree(c->vals);
  void* bufs[] = {c->gq, c->gtc, c->chtasks, c->chsync, c->pbar, c->Mf64, c->dfc, c->d2f, c->b, c->c, c->x, c->y, c->s, c->d2, c->d, c->rd, c->t, c->wu, c->dx, c->ds,
                  c->rp, c->p, c->dy, c->r, c->z, c->dd, c->q, c->rtil, c->qhat, c->res, c->tm,
                  c->dyacc, c->rhs, c->r_alt, c->d_alt, c->part, c->hb, c->cnt, c->start, c->cursor, c->list, c->coef, c->qf, c->G, c->Gdf,
                  c->u, c->Q, c->M, c->X, c->Qsplit, c->sc, c->fl, c->bpart,
                  c->bcnt, c->X1, c->XF, c->XFT, c->G1df, c->ptmp, c->gdig, c->gex,
                  c->gpart};
  for (void* p : bufs) dfree(p);
  pinned_release(c->pin_blk);
  for (auto& pr : c->ev_pending) {
    if (pr.a) cudaEventDestroy(pr.a);
    if (pr.b) cudaEventDestroy(pr.b);
  }
  for (auto& pr : c->mv_pending) {
    if (pr.a) cudaEventDestroy(pr.a);
    if (pr.b) cudaEventDestroy(pr.b);
  }
  for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
  for (auto& g : c->cg_graphs) cg_graph_free(g);
  if (c->cap_st) cudaStreamDestroy(c->cap_st);
  if (c->batch_ready) cudaEventDestroy(c->batch_ready);
  delete c;
}

static lp_status alloc_workspace(lp_ctx* c) {
  const int m = c->m;
  const int64_t n = c->n;
  double** nvec[] = {&c->x, &c->s, &c->d2, &c->d, &c->rd, &c->t, &c->wu, &c->dx, &c->ds};
  for (double** p : nvec) LP_TRY(dalloc(p, (size_t)n));
  LP_TRY(dalloc(&c->d2f, (size_t)n));
  if (!c->sparse && c->a_dtype == LP_F32) LP_TRY(dalloc(&c->dfc, (size_t)4 * n));
  double** mvec[] = {&c->y, &c->rp, &c->p, &c->dy, &c->r, &c->z, &c->dd, &c->q, &c->rtil,
                     &c->qhat, &c->res, &c->tm, &c->dyacc, &c->rhs, &c->r_alt, &c->d_alt,
                     &c->ptmp};
  for (double** p : mvec) LP_TRY(dalloc(p, (size_t)m));
  const int maxgrid = std::max(coltile_max_grid(c->num_sms), csc_max_grid(c->num_sms));
  c->part_bytes = (size_t)maxgrid * 2 * m * sizeof(double);
  LP_TRY(dalloc((unsigned char**)&c->part, c->part_bytes));
  // sketch
  c->ss = c->prm.sketch_s;
  c->w = c->prm.sketch_w ? c->prm.sketch_w : 4 * m;
  LP_TRY(dalloc(&c->hb, (size_t)n * c->ss));
  LP_TRY(dalloc(&c->list, (size_t)n * c->ss));
  LP_TRY(dalloc(&c->coef, (size_t)n * c->ss));
  LP_TRY(dalloc(&c->qf, (size_t)2 * kQCopies * m));
  LP_TRY(dalloc(&c->cnt, (size_t)c->w + 1));
  LP_TRY(dalloc(&c->start, (size_t)c->w + 1));
  LP_TRY(dalloc(&c->cursor, (size_t)c->w + 1));
  c->ldg = round_up(m, 2);
  LP_TRY(dalloc(&c->G, (size_t)c->ldg * c->w));
  LP_CU(cudaMemsetAsync(c->G, 0, (size_t)c->ldg * c->w * sizeof(double), c->st));
  LP_TRY(dalloc(&c->u, (size_t)c->w));
  LP_TRY(dalloc(&c->Gdf, (size_t)2 * c->ldg * c->w));
  // factor
  c->mp = round_up(m, 64);
  LP_TRY(dalloc(&c->Q, (size_t)c->mp * c->mp));
  LP_TRY(dalloc(&c->M, (size_t)c->mp * c->mp));
  LP_TRY(dalloc(&c->X, (size_t)c->mp * c->mp));
  c->qsplit = gram_split(m, c->w, c->num_sms);
  const int nt = c->mp / 64;
  LP_TRY(dalloc(&c->Qsplit, (size_t)c->qsplit * (nt * (nt + 1) / 2) * 64 * 64));
  // tensor-core Gram product (digits are rewritten completely by every product)
  LP_TRY(dalloc((unsigned char**)&c->gdig, gram_tc_digit_bytes(m, c->w)));
  LP_TRY(dalloc(&c->gex, (size_t)gram_tc_rows(m)));
  LP_TRY(dalloc((unsigned char**)&c->gpart, gram_tc_part_bytes(m, c->mp, c->w, c->num_sms)));
  // quantile table of the Gaussian W (the sketch needs a dense A)
  if (!c->sparse) {
    static std::once_flag once;
    static int16_t table[1 << kGaussBits];
    std::call_once(once, [] { gauss_grid(table); });
    LP_TRY(dalloc(&c->gq, (size_t)1 << kGaussBits));
    LP_CU(cudaMemcpyAsync(c->gq, table, sizeof(table), cudaMemcpyHostToDevice, c->st));
  }
  // scalars
  LP_TRY(dalloc(&c->pbar, 32));
  LP_TRY(dalloc(&c->sc, SC_COUNT));
  LP_TRY(dalloc(&c->fl, FL_COUNT));
  LP_TRY(dalloc(&c->bpart, (size_t)kMaxRedBlocks * 8));
  LP_TRY(dalloc(&c->bcnt, 16));
  LP_CU(cudaMemsetAsync(c->sc, 0, SC_COUNT * sizeof(double), c->st));
  LP_CU(cudaMemsetAsync(c->fl, 0, FL_COUNT * sizeof(int), c->st));
  LP_CU(cudaMemsetAsync(c->bcnt, 0, 16 * sizeof(unsigned), c->st));
  static_assert(SC_COUNT * sizeof(double) + FL_COUNT * sizeof(int) <= kPinBlock, "pinned block");
  c->pin_blk = pinned_block();
  if (!c->pin_blk) return fail(LP_ERR_OOM, "cudaMallocHost of the scalar mirrors failed");
  c->sc_h = reinterpret_cast<double*>(c->pin_blk);
  c->fl_h = reinterpret_cast<int*>(reinterpret_cast<char*>(c->pin_blk) + SC_COUNT * sizeof(double));
  LP_CU(symv_set_smem(m));
  return LP_OK;
}

// ---- profiling: event pairs recorded on the context stream, harvested after a sync --------
static cudaEvent_t ev_get(lp_ctx* c) {
  if (!c->ev_pool.empty()) {
    cudaEvent_t e = c->ev_pool.back();
    c->ev_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return e;
}

static void ev_put(lp_ctx* c, cudaEvent_t e) {
  if (e) c->ev_pool.push_back(e);
}

// Harvests finished phase events (the stream has been synchronized).
static void prof_harvest(lp_ctx* c) {
  for (auto& pr : c->ev_pending) {
    float ms = 0.f;
    if (pr.a && pr.b && cudaEventElapsedTime(&ms, pr.a, pr.b) == cudaSuccess &&
        pr.phase >= 0 && pr.phase < LP_PH_COUNT) {
      c->prof.phase_ms[pr.phase] += ms;
      c->prof.phase_calls[pr.phase] += 1;
    }
    cudaGetLastError();
    ev_put(c, pr.a);
    ev_put(c, pr.b);
  }
  c->ev_pending.clear();
}

// Harvests the CG product events of one batch: the first `real` launches did work, the rest
// found the CG finished and returned at once.
// Algorithmic bytes of one CG product on the copy streamed now: A once, D^2 (FP32 weight or
// FP64), the direction in and the product out (CSC: values, row ids and column pointers).
static double matvec_bytes(const lp_ctx* c) {
  const double wb = c->s_dtype == LP_F64 ? 8.0 : 4.0;
  if (!c->sparse)
    return (double)c->m * (double)c->n * (double)dtype_size(c->s_dtype) + wb * (double)c->n +
           16.0 * c->m;
  return (double)c->nnz * (dtype_size(c->s_dtype) + 4.0) + 8.0 * (c->n + 1) + 8.0 * (double)c->n +
         16.0 * c->m;
}

static void prof_harvest_mv(lp_ctx* c, int real) {
  for (size_t i = 0; i < c->mv_pending.size(); ++i) {
    auto& pr = c->mv_pending[i];
    float ms = 0.f;
    if ((int)i < real && pr.a && pr.b && cudaEventElapsedTime(&ms, pr.a, pr.b) == cudaSuccess) {
      c->prof.matvec_ms += ms;
      c->prof.matvec_count += 1;
      c->mv_bytes_sum += matvec_bytes(c);
    }
    cudaGetLastError();
    ev_put(c, pr.a);
    ev_put(c, pr.b);
  }
  c->mv_pending.clear();
}

struct PhaseScope {
  lp_ctx* c;
  int phase;
  cudaEvent_t a = nullptr;
  PhaseScope(lp_ctx* cc, int ph) : c(cc), phase(ph) {
    if (c->prof_on && (a = ev_get(c))) cudaEventRecord(a, c->st);
  }
  ~PhaseScope() {
    if (!a) return;
    cudaEvent_t b = ev_get(c);
    if (b) cudaEventRecord(b, c->st);
    c->ev_pending.push_back({phase, a, b});
  }
};

static lp_status sync_scalars(lp_ctx* c) {
  LP_CU(cudaMemcpyAsync(c->sc_h, c->sc, SC_COUNT * sizeof(double), cudaMemcpyDeviceToHost, c->st));
  LP_CU(cudaMemcpyAsync(c->fl_h, c->fl, FL_COUNT * sizeof(int), cudaMemcpyDeviceToHost, c->st));
  LP_CU(cudaStreamSynchronize(c->st));
  if (!c->ev_pending.empty()) prof_harvest(c);
  if (c->fl_h[FL_TIMEOUT])
    return fail(LP_ERR_TIMEOUT, "a bounded wait in a kernel gave up (a bulk copy or a task it depends on)");
  return LP_OK;
}

static lp_status check_finite_dev(lp_ctx* c, const void* p, lp_dtype dt, int64_t count,
                                  const char* what) {
  LP_CU(launch_set(nullptr, 0, 0.0, c->fl, FL_NUMERIC, 0, c->st));
  LP_CU(launch_check_finite(p, dt, count, c->fl + FL_NUMERIC, c->st));
  LP_TRY(sync_scalars(c));
  if (c->fl_h[FL_NUMERIC]) return fail(LP_ERR_ARG, std::string(what) + " has NaN or Inf entries");
  return LP_OK;
}

// Autotunes the staged CG product's launch shape for the copy of A of dtype ta (the streamed
// copy, or the master copy a solve may switch to).  Matrices below 64 MB keep the fixed rule
// (the candidates would cost more than they save); results are kept per shape for the process.
static void autotune_cgprod(lp_ctx* c, lp_dtype ta, const void* A, int lda) {
  if (!c->prm.autotune || c->sparse || (ta != LP_F32 && ta != LP_BF16 && ta != LP_F16)) return;
  if ((double)c->m * (double)c->n * (double)dtype_size(ta) < 64e6) return;
  static std::mutex mu;
  static std::vector<std::pair<std::vector<int64_t>, CgTune>> cache;
  const std::vector<int64_t> key{(int64_t)ta, c->m, lda, c->n, c->num_sms, c->dev};
  {
    std::lock_guard<std::mutex> lk(mu);
    for (auto& kv : cache)
      if (kv.first == key) {
        c->tune[(int)ta & 3] = kv.second;
        return;
      }
  }
  if (cudaMemsetAsync(c->d2f, 0, (size_t)c->n * sizeof(float), c->st) != cudaSuccess ||
      cudaMemsetAsync(c->z, 0, (size_t)c->m * sizeof(double), c->st) != cudaSuccess) {
    cudaGetLastError();
    return;
  }
  ColArgs a{};
  a.A = A;
  a.lda = lda;
  a.m = c->m;
  a.n = c->n;
  a.v = c->z;
  a.d2f = c->d2f;
  a.part = c->part;
  a.fl = c->fl;
  a.flw = c->fl;
  CgTune t{};
  if (tune_cgprod(ta, a, c->num_sms, coltile_max_grid(c->num_sms), c->st, &t) == 0) {
    c->tune[(int)ta & 3] = t;
    std::lock_guard<std::mutex> lk(mu);
    cache.push_back({key, t});
  }
  cudaGetLastError();
}

extern "C" lp_status lp_create(lp_ctx** out, int32_t m, int64_t n, lp_layout layout,
                               lp_dtype a_dtype, const void* A_vals, const int64_t* indptr,
                               const int32_t* indices, int64_t nnz, const double* b,
                               const double* cvec, const lp_params* prm, void* stream) {
  if (!out) return fail(LP_ERR_ARG, "lp_create: out is NULL");
  *out = nullptr;
  if (m < 1 || n < m || m > 8192) return fail(LP_ERR_ARG, "lp_create: need 1 <= m <= n, m <= 8192");
  if (n > ((int64_t)1 << 31) - 2) return fail(LP_ERR_ARG, "lp_create: n too large");
  if (!A_vals || !b || !cvec) return fail(LP_ERR_ARG, "lp_create: NULL A, b or c");
  if (a_dtype != LP_F64 && a_dtype != LP_F32)
    return fail(LP_ERR_ARG, "lp_create: A must be LP_F64 or LP_F32");
  if (layout == LP_CSR && prm && prm->sketch_kind == LP_SKETCH_GAUSSIAN)
    return fail(LP_ERR_ARG, "lp_create: the Gaussian sketch needs a dense A");
  if (layout == LP_CSR && (!indptr || !indices || nnz < 0))
    return fail(LP_ERR_ARG, "lp_create: CSR needs indptr, indices and nnz");
  if (layout != LP_CSR && layout != LP_DENSE_COLMAJOR && layout != LP_DENSE_ROWMAJOR)
    return fail(LP_ERR_ARG, "lp_create: unknown layout");
  lp_params p;
  if (prm) p = *prm; else lp_params_default(&p);
  LP_TRY(check_params(p, m));

  // no C++ exception may leave an extern "C" entry point: host allocations are nothrow
  lp_ctx* c = new (std::nothrow) lp_ctx();
  if (!c) return fail(LP_ERR_OOM, "lp_create: host allocation failed");
  c->m = m;
  c->n = n;
  c->prm = p;
  c->st = (cudaStream_t)stream;
  c->sparse = (layout == LP_CSR);
  c->a_dtype = a_dtype;
  lp_status st = LP_OK;
  auto bail = [&](lp_status s) {
    lp_destroy(c);
    return s;
  };
  AllocStream as(c->st);
  cudaError_t e = cudaGetDevice(&c->dev);
  if (e != cudaSuccess) return bail(lp_cuda_fail(e, "cudaGetDevice"));
  keep_pool_memory(c->dev);
  e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->dev);
  if (e != cudaSuccess) return bail(lp_cuda_fail(e, "cudaDeviceGetAttribute"));

  if ((st = alloc_workspace(c)) != LP_OK) return bail(st);
  if ((st = dalloc(&c->b, m)) != LP_OK || (st = dalloc(&c->c, n)) != LP_OK) return bail(st);
  e = cudaMemcpyAsync(c->b, b, m * sizeof(double), cudaMemcpyDefault, c->st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(c->c, cvec, n * sizeof(double), cudaMemcpyDefault, c->st);
  if (e != cudaSuccess) return bail(lp_cuda_fail(e, "copy b, c"));
  if ((st = check_finite_dev(c, c->b, LP_F64, m, "b")) != LP_OK) return bail(st);
  if ((st = check_finite_dev(c, c->c, LP_F64, n, "c")) != LP_OK) return bail(st);

  const size_t es = dtype_size(a_dtype);
  if (!c->sparse) {
    // master copy: column-major, columns 16-byte aligned
    c->lda = round_up(m, (int)(16 / es));
    if ((st = dalloc((unsigned char**)&c->A, (size_t)c->lda * n * es)) != LP_OK) return bail(st);
    if (layout == LP_DENSE_COLMAJOR) {
      if (c->lda != m) {
        e = cudaMemsetAsync(c->A, 0, (size_t)c->lda * n * es, c->st);
        if (e != cudaSuccess) return bail(lp_cuda_fail(e, "memset A"));
      }
      e = cudaMemcpy2DAsync(c->A, c->lda * es, A_vals, m * es, m * es, n, cudaMemcpyDefault, c->st);
      if (e != cudaSuccess) return bail(lp_cuda_fail(e, "copy A"));
    } else {
      unsigned char* tmp = nullptr;
      if ((st = dalloc(&tmp, (size_t)m * n * es)) != LP_OK) return bail(st);
      e = cudaMemcpyAsync(tmp, A_vals, (size_t)m * n * es, cudaMemcpyDefault, c->st);
      if (e == cudaSuccess)
        e = launch_convert_dense(tmp, a_dtype, true, m, n, c->A, a_dtype, c->lda, c->st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
      dfree(tmp);
      if (e != cudaSuccess) return bail(lp_cuda_fail(e, "row-major A"));
    }
    if ((st = check_finite_dev(c, c->A, a_dtype, (int64_t)c->lda * n, "A")) != LP_OK) return bail(st);
    // streamed copy for the CG products
    lp_dtype sd = p.stream_dtype == LP_F64 ? a_dtype : p.stream_dtype;
    if (sd == LP_F64 && a_dtype == LP_F32) sd = LP_F32;
    c->s_dtype = sd;
    if (sd == a_dtype) {
      c->As = c->A;
      c->lda_s = c->lda;
    } else {
      c->lda_s = round_up(m, (int)(16 / dtype_size(sd)));
      if ((st = dalloc((unsigned char**)&c->As, (size_t)c->lda_s * n * dtype_size(sd))) != LP_OK)
        return bail(st);
      c->own_As = true;
      if (sd == LP_BF16 || sd == LP_F16) {
        // 16-bit copies are stored column-scaled by powers of two (scales folded into D^2)
        if ((st = dalloc(&c->cs2, (size_t)n)) != LP_OK) return bail(st);
        e = launch_convert_colscaled(c->A, a_dtype, c->lda, m, n, c->As, sd, c->lda_s, c->cs2,
                                     c->st);
        c->cs2_on = true;
      } else {
        // convert from the master copy (column-major with leading dim lda): walk as an
        // lda x n matrix, padding rows are zero already.
        e = launch_convert_dense(c->A, a_dtype, false, c->lda, n, c->As, sd, c->lda_s, c->st);
      }
      if (e != cudaSuccess) return bail(lp_cuda_fail(e, "stream copy"));
    }
  } else {
    c->nnz = nnz;
    int64_t* ip = nullptr;
    int32_t* ix = nullptr;
    unsigned char* vv = nullptr;
    int64_t* cur = nullptr;
    if ((st = dalloc(&ip, (size_t)m + 1)) != LP_OK || (st = dalloc(&ix, (size_t)nnz)) != LP_OK ||
        (st = dalloc(&vv, (size_t)nnz * es)) != LP_OK || (st = dalloc(&cur, (size_t)n)) != LP_OK ||
        (st = dalloc(&c->colptr, (size_t)n + 1)) != LP_OK ||
        (st = dalloc(&c->rowidx, (size_t)nnz)) != LP_OK ||
        (st = dalloc((unsigned char**)&c->vals, (size_t)nnz * es)) != LP_OK) {
      dfree(ip); dfree(ix); dfree(vv); dfree(cur);
      return bail(st);
    }
    e = cudaMemcpyAsync(ip, indptr, (m + 1) * sizeof(int64_t), cudaMemcpyDefault, c->st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(ix, indices, nnz * sizeof(int32_t), cudaMemcpyDefault, c->st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(vv, A_vals, nnz * es, cudaMemcpyDefault, c->st);
    // validate the structure on the host copy of indptr (small) and the indices on device
    std::unique_ptr<int64_t[]> hip(new (std::nothrow) int64_t[(size_t)m + 1]);
    if (!hip) {
      dfree(ip); dfree(ix); dfree(vv); dfree(cur);
      return bail(fail(LP_ERR_OOM, "lp_create: host allocation failed"));
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(hip.get(), ip, (m + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost, c->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
    bool ok = (e == cudaSuccess) && hip[0] == 0 && hip[m] == nnz;
    for (int i = 0; ok && i < m; ++i) ok = hip[i] <= hip[i + 1];
    if (ok) {
      // column ids in range: reuse the finiteness flag through a tiny check on host copy
      std::unique_ptr<int32_t[]> hix(new (std::nothrow) int32_t[nnz > 0 ? (size_t)nnz : 1]);
      if (!hix ||
          cudaMemcpyAsync(hix.get(), ix, nnz * sizeof(int32_t), cudaMemcpyDeviceToHost, c->st) !=
              cudaSuccess ||
          cudaStreamSynchronize(c->st) != cudaSuccess)
        ok = false;
      for (int64_t k = 0; ok && k < nnz; ++k) ok = hix[k] >= 0 && hix[k] < n;
    }
    if (ok) e = csr_to_csc(ip, ix, vv, a_dtype, m, n, nnz, c->colptr, cur, c->rowidx, c->vals, c->st);
    if (ok && e == cudaSuccess) e = cudaStreamSynchronize(c->st);
    dfree(ip); dfree(ix); dfree(vv); dfree(cur);
    if (e != cudaSuccess) return bail(lp_cuda_fail(e, "CSR to CSC"));
    if (!ok) return bail(fail(LP_ERR_ARG, "lp_create: malformed CSR (indptr or column ids)"));
    if ((st = check_finite_dev(c, c->vals, a_dtype, nnz, "A")) != LP_OK) return bail(st);
    c->svals = c->vals;
    c->s_dtype = a_dtype;
    if (p.stream_dtype == LP_F32 && a_dtype == LP_F64) {
      // an FP32 copy of the values for the CG products
      if ((st = dalloc((unsigned char**)&c->svals, (size_t)nnz * 4)) != LP_OK) return bail(st);
      c->own_svals = true;
      e = launch_convert_dense(c->vals, LP_F64, false, 1, nnz, c->svals, LP_F32, 1, c->st);
      if (e != cudaSuccess) return bail(lp_cuda_fail(e, "stream values"));
      c->s_dtype = LP_F32;
    }
  }
  c->s_dtype_req = c->s_dtype;
  c->As_req = c->As;
  c->lda_s_req = c->lda_s;
  c->svals_req = c->svals;
  if (!c->sparse) {
    autotune_cgprod(c, c->s_dtype, c->As, c->lda_s);
    if (c->a_dtype != c->s_dtype) autotune_cgprod(c, c->a_dtype, c->A, c->lda);
  }
  // norms of b and c for the stopping rule
  LP_CU(launch_norm2(c->b, m, c->sc, SC_RES2, c->bpart, c->bcnt, c->st));
  if ((st = sync_scalars(c)) != LP_OK) return bail(st);
  c->bnorm = sqrt(c->sc_h[SC_RES2]);
  LP_CU(launch_norm2(c->c, n, c->sc, SC_RES2, c->bpart, c->bcnt, c->st));
  if ((st = sync_scalars(c)) != LP_OK) return bail(st);
  c->cnorm = sqrt(c->sc_h[SC_RES2]);
  *out = c;
  return LP_OK;
}

extern "C" lp_status lp_set_params(lp_ctx* c, const lp_params* prm) {
  if (!c || !prm) return fail(LP_ERR_ARG, "lp_set_params: NULL");
  LP_TRY(check_params(*prm, c->m));
  const int w = prm->sketch_w ? prm->sketch_w : 4 * c->m;
  if (w != c->w || prm->sketch_s != c->ss)
    return fail(LP_ERR_ARG, "lp_set_params: sketch size is fixed at lp_create");
  if (c->sparse && prm->sketch_kind == LP_SKETCH_GAUSSIAN)
    return fail(LP_ERR_ARG, "lp_set_params: the Gaussian sketch needs a dense A");
  lp_dtype sd = prm->stream_dtype == LP_F64 ? c->a_dtype : prm->stream_dtype;
  if (!c->sparse && sd != c->s_dtype && !(sd == LP_F64 && c->a_dtype == LP_F32))
    return fail(LP_ERR_ARG, "lp_set_params: stream dtype is fixed at lp_create");
  c->prm = *prm;
  return LP_OK;
}

// ------------------------------------------------------------------------------------------
// Building blocks
// ------------------------------------------------------------------------------------------

// One pass y = A diag(w) A^T v (w == NULL: identity) with t = A^T v (optional).
// precise: master copy with FP64 accumulation; else the streamed copy.
static lp_status pass_normal(lp_ctx* c, bool precise, const double* v, const double* w, double* t,
                             int red_mode, double* out, const double* p0, int skip_if_done,
                             bool record_mv = false, const double* dz = nullptr,
                             const double* dold = nullptr, double* dnew = nullptr,
                             double* qacc = nullptr, bool weight_in_d2f = false) {
  int nblk;
  bool acc64;
  cudaEvent_t ea = nullptr, eb = nullptr;
  if (record_mv && c->prof_on && (ea = ev_get(c))) cudaEventRecord(ea, c->st);
  if (!c->sparse) {
    ColArgs a{};
    const lp_dtype ta = precise ? c->a_dtype : c->s_dtype;
    a.A = precise ? c->A : c->As;
    a.lda = precise ? c->lda : c->lda_s;
    a.m = c->m;
    a.n = c->n;
    a.v = v;
    a.d2 = w;
    a.d2f = (!precise && (w == c->d2 || weight_in_d2f)) ? c->d2f : nullptr;
    a.d2df = (precise && w == c->d2) ? c->dfc : nullptr;
    a.colout = t;
    a.part = c->part;
    a.fl = c->fl;
    a.sc = c->sc;
    a.skip_if_done = skip_if_done;
    a.dz = dz;
    a.dold = dold;
    a.dnew = dnew;
    acc64 = precise || ta == LP_F64;
    a.flw = c->fl;
    if (qacc && !acc64) {
      a.qacc = qacc;
      a.qsum = out;
      a.cnt = c->bcnt + 1;
      a.scw = c->sc;
    } else {
      qacc = nullptr;
    }
    nblk = -1;
    if (!acc64 && a.d2f && c->use_staged) {
      a.stall_group_p1 = c->stall_group_p1;   // fault injection: next staged product only
      a.wait_ns = c->stall_wait_ns;
      const CgTune& tn = c->tune[(int)ta & 3];
      a.cfg_tc = tn.tc;
      a.cfg_stages = tn.stages;
      a.cfg_ctas = tn.ctas;
      nblk = launch_cgprod(ta, a, c->num_sms, coltile_max_grid(c->num_sms), c->st);
      if (nblk >= 0) {
        c->stall_group_p1 = 0;
        c->stall_wait_ns = 0;
      }
    }
    if (nblk < 0) nblk = launch_coltile(ta, acc64, MODE_NORMAL, a, c->num_sms, c->st);
  } else {
    CscArgs a{};
    const lp_dtype tv = precise ? c->a_dtype : c->s_dtype;
    a.colptr = c->colptr;
    a.rowidx = c->rowidx;
    a.vals = precise ? c->vals : c->svals;
    a.m = c->m;
    a.n = c->n;
    a.v = v;
    a.d2 = w;
    a.colout = t;
    a.part = c->part;
    a.fl = c->fl;
    a.sc = c->sc;
    a.skip_if_done = skip_if_done;
    a.dz = dz;
    a.dold = dold;
    a.dnew = dnew;
    acc64 = precise || tv == LP_F64;
    nblk = launch_csc(tv, acc64, MODE_NORMAL, a, c->num_sms, c->st);
  }
  if (ea) {
    if ((eb = ev_get(c))) cudaEventRecord(eb, c->st);
    c->mv_pending.push_back({-1, ea, eb});
  }
  if (nblk < 0) return fail(LP_ERR_ARG, "unsupported shape for the matrix pass");
  LP_CU(cudaGetLastError());
  if (qacc) return LP_OK;   // reduced by the kernel itself
  RedArgs r{};
  r.mode = red_mode;
  r.part = c->part;
  r.nblk = nblk;
  r.nout = 1;
  r.m = c->m;
  r.acc_f64 = acc64;
  r.out0 = out;
  r.p0 = p0;
  r.dvec = dnew ? dnew : v;
  r.sc = c->sc;
  r.fl = c->fl;
  r.bpart = c->bpart;
  r.bcnt = c->bcnt;
  r.skip_if_done = skip_if_done;
  LP_CU(launch_reduce(r, c->st));
  return LP_OK;
}

// Product with the sketch Q v = G G^T v in FP64, u = G^T v (optional), reduced by red_mode:
// RED_MINUS_P: out = Q v - p0;  RED_PLAIN: out = Q v;  RED_CG_Q: out = q = Q v and d^T q.
static lp_status pass_gram(lp_ctx* c, const double* G, const double* v, double* u, double* out,
                           const double* p0, int red_mode, int skip_if_done,
                           const double* dz = nullptr, const double* dold = nullptr,
                           double* dnew = nullptr) {
  ColArgs a{};
  a.A = G;
  a.lda = c->ldg;
  a.m = c->m;
  a.n = c->w;
  a.v = v;
  a.d2 = nullptr;
  a.colout = u;
  a.part = c->part;
  a.fl = c->fl;
  a.sc = c->sc;
  a.skip_if_done = skip_if_done;
  a.dz = dz;
  a.dold = dold;
  a.dnew = dnew;
  const int nblk = launch_coltile(LP_F64, true, MODE_NORMAL, a, c->num_sms, c->st);
  if (nblk < 0) return fail(LP_ERR_ARG, "unsupported shape for the sketch pass");
  RedArgs r{};
  r.mode = red_mode;
  r.part = c->part;
  r.nblk = nblk;
  r.nout = 1;
  r.m = c->m;
  r.acc_f64 = true;
  r.out0 = out;
  r.p0 = p0;
  r.dvec = dnew ? dnew : v;
  r.sc = c->sc;
  r.fl = c->fl;
  r.bpart = c->bpart;
  r.bcnt = c->bcnt;
  r.skip_if_done = skip_if_done;
  LP_CU(launch_reduce(r, c->st));
  return LP_OK;
}

// Column scales of the streamed copy in use (NULL when it is unscaled).
static const float* stream_cs2(const lp_ctx* c) { return c->cs2_on ? c->cs2 : nullptr; }

// Every solve starts on the stream copy asked for at lp_create.
static void stream_reset(lp_ctx* c) {
  launch_set(nullptr, 0, 0.0, c->fl, FL_TIMEOUT, 0, c->st);
  c->s_dtype = c->s_dtype_req;
  c->As = c->As_req;
  c->lda_s = c->lda_s_req;
  c->svals = c->svals_req;
  c->cs2_on = c->cs2 != nullptr;
  c->switch_iter = -1;
  c->cg_precise = false;
  c->precise_iter = -1;
}

// Stream the master copy instead (FP32 for an FP32 input, FP64 for an FP64 one) for the rest
// of the solve; the FP32 weight of the product is recomputed without the copy's scales.
// Returns false when the master copy is already the one streamed.
static bool stream_switch(lp_ctx* c, int k) {
  if (c->s_dtype == c->a_dtype) return false;
  c->s_dtype = c->a_dtype;
  c->As = c->A;
  c->lda_s = c->lda;
  c->svals = c->vals;
  c->cs2_on = false;
  c->switch_iter = k;
  return launch_d2f(c->d2, nullptr, c->n, c->d2f, c->st) == cudaSuccess;
}

// Alg. 2 step (b): d2, d, mu from (x, s); r_p, r_d, p in one pass; ||r_p||^2, ||r_d||^2.
static lp_status run_residuals(lp_ctx* c, const double* x, const double* y, const double* s,
                               double sigma, double* rp, double* rd, double* p) {
  PhaseScope ps(c, LP_PH_RESIDUALS);
  LP_CU(launch_prep_iterate(x, s, c->n, c->d2, c->d, c->sc, c->bpart, c->bcnt, sigma, c->c, c->st,
                            c->d2f, stream_cs2(c), c->dfc));
  int nblk;
  if (!c->sparse) {
    ColArgs a{};
    a.A = c->A;
    a.lda = c->lda;
    a.m = c->m;
    a.n = c->n;
    a.v = y;
    a.x = x;
    a.s = s;
    a.c = c->c;
    a.sc = c->sc;
    a.colout = rd;
    a.part = c->part;
    a.fl = c->fl;
    a.flw = c->fl;
    if (c->dfc) {
      a.d2df = c->dfc;
      a.xdf = c->dfc + c->n;
      a.isdf = c->dfc + 2 * c->n;
      a.scdf = c->dfc + 3 * c->n;
    }
    nblk = launch_coltile(c->a_dtype, true, MODE_RESID, a, c->num_sms, c->st);
  } else {
    CscArgs a{};
    a.colptr = c->colptr;
    a.rowidx = c->rowidx;
    a.vals = c->vals;
    a.m = c->m;
    a.n = c->n;
    a.v = y;
    a.x = x;
    a.s = s;
    a.c = c->c;
    a.sc = c->sc;
    a.colout = rd;
    a.part = c->part;
    a.fl = c->fl;
    nblk = launch_csc(c->a_dtype, true, MODE_RESID, a, c->num_sms, c->st);
  }
  if (nblk < 0) return fail(LP_ERR_ARG, "unsupported shape for the residual pass");
  LP_CU(cudaGetLastError());
  RedArgs r{};
  r.mode = RED_RESID;
  r.part = c->part;
  r.nblk = nblk;
  r.nout = 2;
  r.m = c->m;
  r.acc_f64 = true;
  r.out0 = rp;
  r.out1 = p;
  r.p0 = c->b;
  r.sc = c->sc;
  r.fl = c->fl;
  r.bpart = c->bpart;
  r.bcnt = c->bcnt;
  LP_CU(launch_reduce(r, c->st));
  LP_CU(launch_norm2(rd, c->n, c->sc, SC_RD2, c->bpart, c->bcnt, c->st));
  return LP_OK;
}

// Alg. 1 step 1 / Alg. 2 step (a): G = A D W(seed, k).
static lp_status run_sketch(lp_ctx* c, const double* d, int k, double* G) {
  PhaseScope ps(c, LP_PH_SKETCH);
  if (c->prm.sketch_kind == LP_SKETCH_GAUSSIAN) {
    if (c->prm.gram_tensor_cores) {
      const size_t need = sketch_tc_work_bytes(c->m, c->n, c->w, c->num_sms);
      if (c->gtc_bytes < need) {
        AllocStream as(c->st);
        dfree(c->gtc);
        c->gtc = nullptr;
        c->gtc_bytes = 0;
        LP_TRY(dalloc((unsigned char**)&c->gtc, need));
        c->gtc_bytes = need;
      }
      LP_CU(launch_sketch_tc(c->a_dtype, c->A, c->lda, c->m, c->n, c->w,
                             gauss_iteration_key(c->prm.seed, k), d, c->gq, G, c->ldg, c->gtc,
                             c->num_sms, c->fl, c->st));
    } else {
      LP_CU(launch_sketch_gauss(c->a_dtype, c->A, c->lda, c->m, c->n, c->w, c->prm.seed, k, c->gq,
                                d, G, c->ldg, c->st));
    }
    return LP_OK;
  }
  LP_CU(cudaMemsetAsync(c->cnt, 0, (c->w + 1) * sizeof(int32_t), c->st));
  LP_CU(launch_sketch_hash(c->prm.seed, k, c->n, c->ss, c->w, c->hb, c->cnt, nullptr, nullptr, c->st));
  LP_CU(launch_sketch_scan(c->cnt, c->w, c->start, c->cursor, c->st));
  LP_CU(launch_sketch_scatter(c->hb, c->n, c->ss, c->w, c->start, c->cursor, c->list, d, c->coef,
                              c->st));
  if (!c->sparse) {
    LP_CU(launch_sketch_gather_dense(c->a_dtype, c->A, c->lda, c->m, c->ss, c->w, c->start,
                                     c->list, d, G, c->ldg, c->st, c->coef));
  } else {
    LP_CU(launch_sketch_gather_csc(c->a_dtype, c->colptr, c->rowidx, c->vals, c->m, c->ss, c->w,
                                   c->start, c->list, d, G, c->ldg, c->st));
  }
  return LP_OK;
}

// Q = G G^T (c->Q, full mp x mp) from the hi / lo float planes of G: on the tensor cores
// (exact digit splitting) or in double-float on the FP32 pipes.
static lp_status run_gram(lp_ctx* c, const float* Gdf) {
  if (c->prm.gram_tensor_cores)
    LP_CU(launch_gram_tc(Gdf, c->ldg, c->m, c->w, c->mp, c->Q, c->gdig, c->gex, c->gpart,
                         c->num_sms, c->fl, c->st));
  else
    LP_CU(launch_gram_df(Gdf, c->ldg, c->m, c->w, c->mp, c->Q, c->Qsplit, c->qsplit, c->st));
  return LP_OK;
}

// Whether M = X^T X can come from the tensor-core Gram product with the context's buffers
// (sized for the m x w sketch; X^T is m x mp).
static bool xtx_on_tensor_cores(const lp_ctx* c) {
  return c->prm.gram_tensor_cores && gram_tc_digit_bytes(c->m, c->mp) <= gram_tc_digit_bytes(c->m, c->w) &&
         gram_tc_part_bytes(c->m, c->mp, c->mp, c->num_sms) <=
             gram_tc_part_bytes(c->m, c->mp, c->w, c->num_sms);
}

// M = X^T X for X = L^{-1} (double-float, row-major mp x mp in c->X; rows and columns past m
// are the identity): the Gram product of the columns of X on the tensor cores -- X's hi and lo
// planes, read column-major with leading dimension mp, are X^T -- into FP64, then split into
// M's double-float planes.
static lp_status form_m_tensor_cores(lp_ctx* c) {
  const size_t mm = (size_t)c->mp * c->mp;
  if (!c->Mf64) {
    AllocStream as(c->st);
    LP_TRY(dalloc(&c->Mf64, mm));
  }
  LP_CU(launch_gram_tc(reinterpret_cast<const float*>(c->X), c->mp, c->m, c->mp, c->mp, c->Mf64,
                       c->gdig, c->gex, c->gpart, c->num_sms, c->fl, c->st));
  LP_CU(launch_split_df(c->Mf64, mm, reinterpret_cast<float*>(c->M), c->st));
  return LP_OK;
}

// Cholesky factor and inverse of (Q + eps diag Q) with M = X^T X (form_m) on the tensor cores
// when the buffers allow, else in the factor's own double-float kernel.
// Task list and counters of the one-launch Cholesky sweep, built on first use (they depend on
// mp only).  False when the sweep keeps the block-step launches.
static lp_status ensure_dag(lp_ctx* c, bool* use) {
  const int nbk = c->mp / kNB;
  *use = c->prm.factor_dag != 0 && nbk <= kDagMaxBlocks;
  if (!*use || c->chtasks) return LP_OK;
  std::vector<uint32_t> t(chol_dag_tasks(nbk, nullptr));
  chol_dag_tasks(nbk, t.data());
  AllocStream as(c->st);
  LP_TRY(dalloc(&c->chtasks, t.size()));
  LP_TRY(dalloc(&c->chsync, chol_dag_sync_words(nbk)));
  LP_CU(cudaMemcpyAsync(c->chtasks, t.data(), t.size() * sizeof(uint32_t), cudaMemcpyHostToDevice,
                        c->st));
  LP_CU(cudaStreamSynchronize(c->st));
  c->chntasks = (int)t.size();
  return LP_OK;
}

static lp_status chol_inverse(lp_ctx* c, double eps, bool form_m) {
  const bool tc = form_m && xtx_on_tensor_cores(c);
  bool dag = false;
  LP_TRY(ensure_dag(c, &dag));
  if (dag)
    LP_CU(launch_chol_dag(c->M, c->X, c->Q, c->mp, c->m, eps, c->chtasks, c->chntasks, c->chsync,
                          c->num_sms, c->fl, c->st, form_m && !tc));
  else
    LP_CU(launch_chol_inverse(c->M, c->X, c->Q, c->mp, c->m, eps, c->fl, c->st, form_m && !tc));
  if (tc) LP_TRY(form_m_tensor_cores(c));
  return LP_OK;
}

// Probe check of a factor stage: ||(Q + eps diag Q)(M 1) - 1|| / sqrt(m) and the pivot flag.
static lp_status factor_check(lp_ctx* c, double eps, double* qerr, bool* brk) {
  // a fixed +-1 probe has a component ~1/sqrt(m) along every eigenvector of Q, so an inverse
  // that is wrong along a few directions of a numerically singular Q (CountSketch) shows; the
  // all-ones vector can miss them
  LP_CU(launch_vec_ops(VOP_SIGNS, c->res, nullptr, nullptr, c->m, nullptr, c->st));
  LP_CU(launch_symv_dot(c->M, c->mp, c->m, c->res, c->tm, c->sc, c->fl, c->bpart, c->bcnt,
                        SYMV_PLAIN, c->st));
  LP_CU(launch_symv_f64(c->Q, c->mp, c->m, c->tm, c->rhs, c->st));
  if (eps > 0.0) LP_CU(launch_add_shift(c->rhs, c->Q, c->mp, c->m, eps, c->tm, c->st));
  LP_CU(launch_vec_ops(VOP_SUB, c->rhs, c->rhs, c->res, c->m, nullptr, c->st));
  LP_CU(launch_norm2(c->rhs, c->m, c->sc, SC_RES2, c->bpart, c->bcnt, c->st));
  LP_TRY(sync_scalars(c));
  *qerr = sqrt(c->sc_h[SC_RES2] / (double)c->m);
  *brk = c->fl_h[FL_BREAK] != 0;
  return LP_OK;
}

// Buffers of the second factor stage, allocated on first use.
static lp_status ensure_stage2(lp_ctx* c) {
  if (c->X1 && c->XF && c->XFT && c->G1df) return LP_OK;
  AllocStream as(c->st);
  const size_t mm = (size_t)c->mp * c->mp;
  if (!c->X1) LP_TRY(dalloc(&c->X1, mm));
  if (!c->XF) LP_TRY(dalloc(&c->XF, mm));
  if (!c->XFT) LP_TRY(dalloc(&c->XFT, mm));
  if (!c->G1df) {
    LP_TRY(dalloc(&c->G1df, (size_t)2 * c->ldg * c->w));
    // rows m..ldg-1 of G1 are never written and must read as zero
    LP_CU(cudaMemsetAsync(c->G1df, 0, (size_t)2 * c->ldg * c->w * sizeof(float), c->st));
  }
  return LP_OK;
}

// Probe error below which a one-stage factor M = Q^{-1} serves as the preconditioner.
constexpr double kDirectQerr = 1e-2;

// Alg. 1 step 2: Q = G G^T, M = Q^{-1} (Eq. pdprecond).  The Gram route squares kappa(G), so
// once Q is numerically singular in double-float (a lost pivot, or a probe error above
// kDirectQerr; CountSketch reaches kappa(Q) ~ 1e17 late in the IPM) the factor takes a second
// stage, in the manner of CholeskyQR2 with a shifted first step:
//   stage 1: (Q + eps1 diag Q) = L1 L1^T, X1 = L1^{-1} (eps1 = 1e-10, raised until no pivot is
//            lost);
//   stage 2: G1 = X1 G, Q2 = G1 G1^T (kappa(Q2) ~ eps1 kappa(Q) instead of kappa(Q)),
//            Q2 = L2 L2^T, X2 = L2^{-1};
// then X = X2 X1 satisfies X G G^T X^T = I up to ~u kappa(G) (u the double-float unit), and
// the preconditioner is applied as X^T (X r): two triangular products whose error grows with
// kappa(G) = kappa(Q)^{1/2}, where the explicit inverse of the one-stage route grows with
// kappa(Q).  Without allow_shift (lp_factor) only the one-stage inverse is formed and a lost
// pivot is an error.  If stage 2 itself loses a pivot, it falls back to a shifted M2 =
// (Q2 + eps diag Q2)^{-1}, eps = 1e-10 ... 1e-4: M is then only a preconditioner, and
// (A D W)^dagger is still applied exactly, by PCG on Q through G.
static lp_status run_factor(lp_ctx* c, const double* G, bool allow_shift) {
  PhaseScope ps(c, LP_PH_FACTOR);
  c->factored = false;
  c->factor_stages = 1;
  LP_CU(launch_split_df(G, (size_t)c->ldg * c->w, c->Gdf, c->st));
  LP_TRY(run_gram(c, c->Gdf));
  double qerr = 0.0;
  bool brk = false;
  LP_CU(launch_set(nullptr, 0, 0.0, c->fl, FL_BREAK, 0, c->st));
  LP_TRY(chol_inverse(c, 0.0, true));
  LP_TRY(factor_check(c, 0.0, &qerr, &brk));
  c->qerr = qerr;
  c->shift = 0.0;
  if (!brk && qerr < (allow_shift ? kDirectQerr : 0.5)) return LP_OK;
  if (!allow_shift)
    return fail(LP_ERR_BREAKDOWN, "sketch A D W is rank deficient (pivot lost in the inverse)");
  LP_TRY(ensure_stage2(c));
  const size_t mm = (size_t)c->mp * c->mp;
  // stage 1: the shifted factor
  double eps1 = 1e-10;
  for (;;) {
    LP_CU(launch_set(nullptr, 0, 0.0, c->fl, FL_BREAK, 0, c->st));
    LP_TRY(chol_inverse(c, eps1, false));   // stage 1 needs X1 = L1^{-1} only
    LP_TRY(sync_scalars(c));
    if (!c->fl_h[FL_BREAK]) break;
    eps1 *= 100.0;
    if (eps1 > 1e-4)
      return fail(LP_ERR_BREAKDOWN, "sketch A D W is rank deficient (shifted first stage lost a pivot)");
  }
  LP_CU(cudaMemcpyAsync(c->X1, c->X, mm * sizeof(double), cudaMemcpyDeviceToDevice, c->st));
  // G1 = X1 G from the hi / lo planes of G that the Gram product left in Gdf
  {
    TrmmArgs t{};
    t.Ah = reinterpret_cast<const float*>(c->X1);
    t.Al = t.Ah + mm;
    t.lda = c->mp;
    t.Bh = c->Gdf;
    t.Bl = c->Gdf + (size_t)c->ldg * c->w;
    t.sbk = 1;
    t.sbj = c->ldg;
    t.M = c->m;
    t.N = c->w;
    t.K = c->m;
    t.b_lower = 0;
    t.Ch = c->G1df;
    t.Cl = c->G1df + (size_t)c->ldg * c->w;
    t.sci = 1;
    t.scj = c->ldg;
    LP_CU(launch_df_trmm(t, c->st));
  }
  LP_TRY(run_gram(c, c->G1df));
  // stage 2
  double eps = 0.0;
  for (;;) {
    LP_CU(launch_set(nullptr, 0, 0.0, c->fl, FL_BREAK, 0, c->st));
    LP_TRY(chol_inverse(c, eps, true));
    LP_TRY(factor_check(c, eps, &qerr, &brk));
    if (!brk && qerr < 0.5) break;
    eps = eps > 0.0 ? eps * 100.0 : 1e-10;
    if (eps > 1e-4)
      return fail(LP_ERR_BREAKDOWN, "sketch A D W is rank deficient (pivot lost in the second stage)");
  }
  // X = X2 X1 (lower triangular) and its transpose, for z = X^T (X r)
  {
    TrmmArgs t{};
    t.Ah = reinterpret_cast<const float*>(c->X);
    t.Al = t.Ah + mm;
    t.lda = c->mp;
    t.Bh = reinterpret_cast<const float*>(c->X1);
    t.Bl = t.Bh + mm;
    t.sbk = c->mp;
    t.sbj = 1;
    t.M = c->mp;
    t.N = c->mp;
    t.K = c->mp;
    t.b_lower = 1;
    t.Ch = reinterpret_cast<float*>(c->XF);
    t.Cl = t.Ch + mm;
    t.sci = c->mp;
    t.scj = 1;
    t.Th = reinterpret_cast<float*>(c->XFT);
    t.Tl = t.Th + mm;
    t.sti = 1;
    t.stj = c->mp;
    LP_CU(launch_df_trmm(t, c->st));
  }
  c->factored = true;
  c->factor_stages = 2;
  c->shift = eps;
  c->qerr = qerr;
  return LP_OK;
}

// Preconditioner apply z = M r with the bookkeeping of `mode` (SYMV_CG_INIT, SYMV_F2,
// SYMV_PLAIN), through the explicit inverse or the two-stage factor.
static lp_status precond_apply(lp_ctx* c, int mode, const double* r, double* z, double rel_tol) {
  if (c->factored)
    LP_CU(launch_precond_factored(c->XF, c->XFT, c->mp, c->m, mode, r, c->ptmp, z, c->sc, c->fl,
                                  c->bpart, c->bcnt, rel_tol, c->st));
  else if (mode == SYMV_CG_INIT)
    LP_CU(launch_symv_init(c->M, c->mp, c->m, r, z, c->sc, c->fl, c->bpart, c->bcnt, rel_tol,
                           c->st));
  else
    LP_CU(launch_symv_dot(c->M, c->mp, c->m, r, z, c->sc, c->fl, c->bpart, c->bcnt, mode, c->st));
  return LP_OK;
}

// CG step r_new = r_old - alpha q, dy += alpha d, z = M r_new, rho and beta.
static lp_status precond_cg_step(lp_ctx* c, const double* rold, const double* q, const double* d,
                                 double* dy, double* rnew, double* z, const double* qf,
                                 double* qzero) {
  if (c->factored)
    LP_CU(launch_precond_factored(c->XF, c->XFT, c->mp, c->m, SYMV_CG_STEP, rnew, c->ptmp, z,
                                  c->sc, c->fl, c->bpart, c->bcnt, 0.0, c->st, rold, q, d, dy,
                                  qf, qzero));
  else
    LP_CU(launch_symv_cg_step(c->M, c->mp, c->m, rold, q, d, dy, rnew, z, c->sc, c->fl, c->bpart,
                              c->bcnt, c->st, qf, qzero));
  return LP_OK;
}

// One CG loop's operands: iteration j forms d_j = z + beta d_{j-1} into d[j & 1], the product
// q = K d_j (into q[j & 1] for the atomically reduced FP32 product) and r_{j+1} into r[(j+1) & 1].
struct CgLoop {
  int op;          // 0: K = A D^2 A^T; 1: K = G G^T (the correction's PCG on Q)
  double* delta;   // the solution accumulates here
  bool atomic_q;
  double* r[2];
  double* d[2];
  double* q[2];
};

static lp_status cg_iteration(lp_ctx* c, const CgLoop& L, int j, bool record_mv) {
  double* dnew = L.d[j & 1];
  const double* dold = L.d[(j + 1) & 1];
  if (L.op == 0)
    LP_TRY(pass_normal(c, c->cg_precise, nullptr, c->d2, nullptr, RED_CG_Q, c->q, nullptr, 1,
                       record_mv, c->z, dold, dnew, L.atomic_q ? L.q[j & 1] : nullptr));
  else
    LP_TRY(pass_gram(c, c->G, nullptr, nullptr, c->q, nullptr, RED_CG_Q, 1, c->z, dold, dnew));
  LP_TRY(precond_cg_step(c, L.r[j & 1], c->q, dnew, L.delta, L.r[(j + 1) & 1], c->z,
                         L.atomic_q ? L.q[j & 1] : nullptr,
                         L.atomic_q ? L.q[(j + 1) & 1] : nullptr));
  return LP_OK;
}

// Everything the captured kernels bake in: the loop's operands and the context state that
// selects kernels and matrices.
struct CgGraphKey {
  int op, atomic_q, precise, factored, use_staged, s_dtype, lda_s, max_trips;
  const void* delta;
  const void* As;
  const void* svals;
};

static void cg_graph_free(lp_ctx::CgGraph& g) {
  if (g.exec) cudaGraphExecDestroy(g.exec);
  if (g.graph) cudaGraphDestroy(g.graph);
  g.exec = nullptr;
  g.graph = nullptr;
}

// Builds the graph of a CG loop: a WHILE node whose body runs iterations 0 and 1 (so the
// buffers' parity is the same at every entry) and then the condition kernel.  The kernels of a
// finished solve return at once, so a solve that stops after an even iteration is exact.
static lp_status cg_graph_build(lp_ctx* c, const CgLoop& L, int max_trips, cudaGraph_t* out) {
  *out = nullptr;
  if (!c->cap_st) LP_CU(cudaStreamCreateWithFlags(&c->cap_st, cudaStreamNonBlocking));
  // the launchers enqueue on c->st: point it at the private stream while recording
  struct StreamSwap {
    lp_ctx* c;
    cudaStream_t saved;
    ~StreamSwap() { c->st = saved; }
  } swap{c, c->st};
  c->st = c->cap_st;
  cudaGraph_t g = nullptr;
  LP_CU(cudaGraphCreate(&g, 0));
  cudaGraphConditionalHandle h;
  cudaError_t e = cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault);
  cudaGraphNodeParams np{};
  np.type = cudaGraphNodeTypeConditional;
  np.conditional.handle = h;
  np.conditional.type = cudaGraphCondTypeWhile;
  np.conditional.size = 1;
  cudaGraphNode_t node;
  if (e == cudaSuccess) e = cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &np);
  if (e == cudaSuccess)
    e = cudaStreamBeginCaptureToGraph(c->st, np.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                      cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) {
    cudaGraphDestroy(g);
    return lp_cuda_fail(e, "CG loop graph");
  }
  lp_status st = cg_iteration(c, L, 0, false);
  if (st == LP_OK) st = cg_iteration(c, L, 1, false);
  if (st == LP_OK) {
    const cudaError_t e2 = launch_cg_cond(h, c->fl, max_trips, c->st);
    if (e2 != cudaSuccess) st = lp_cuda_fail(e2, "CG loop condition");
  }
  cudaGraph_t body = nullptr;
  const cudaError_t e3 = cudaStreamEndCapture(c->st, &body);
  if (st == LP_OK && e3 != cudaSuccess) st = lp_cuda_fail(e3, "CG loop capture");
  if (st != LP_OK) {
    cudaGraphDestroy(g);
    return st;
  }
  *out = g;
  return LP_OK;
}

// Graphs given up: say why once per process (the host-driven loop gives the same results).
static void graph_warn(const lp_ctx* c) {
  static std::atomic<bool> said{false};
  if (!said.exchange(true))
    fprintf(stderr, "lp_gb300: CUDA graphs of the CG loop unavailable (%s); running the "
                    "host-driven loop\n", c->graph_error.c_str());
}

// Runs the CG loop of L as one graph launch (building and caching its graph on first use).
// *ran is false when graphs are unavailable here; the caller then runs the host-driven loop.
static lp_status cg_graph_launch(lp_ctx* c, const CgLoop& L, int max_iter, bool* ran) {
  *ran = false;
  CgGraphKey k{};
  k.op = L.op;
  k.atomic_q = L.atomic_q;
  k.precise = c->cg_precise;
  k.factored = c->factored;
  k.use_staged = c->use_staged;
  k.s_dtype = (int)c->s_dtype;
  k.lda_s = c->lda_s;
  k.max_trips = max_iter / 2 + 2;
  k.delta = L.delta;
  k.As = c->As;
  k.svals = c->svals;
  static_assert(sizeof(CgGraphKey) <= sizeof(lp_ctx::CgGraph::key), "graph key size");
  unsigned char key[sizeof(lp_ctx::CgGraph::key)] = {};
  memcpy(key, &k, sizeof(k));
  cudaGraphExec_t exec = nullptr;
  for (auto& g : c->cg_graphs)
    if (memcmp(g.key, key, sizeof(key)) == 0) exec = g.exec;
  if (!exec) {
    cudaGraph_t g = nullptr;
    if (cg_graph_build(c, L, k.max_trips, &g) != LP_OK) {
      // graphs unavailable (e.g. a driver without conditional nodes): stay eager
      c->graph_error = lp_last_error();
      cudaGetLastError();
      c->use_graphs = false;
      graph_warn(c);
      return LP_OK;
    }
    cudaGraphExec_t ex = nullptr;
    const cudaError_t ei = cudaGraphInstantiate(&ex, g, 0);
    if (ei != cudaSuccess) {
      c->graph_error = std::string("cudaGraphInstantiate: ") + cudaGetErrorString(ei);
      cudaGetLastError();
      cudaGraphDestroy(g);
      c->use_graphs = false;
      graph_warn(c);
      return LP_OK;
    }
    if (c->cg_graphs.size() >= 8) {
      cg_graph_free(c->cg_graphs.front());
      c->cg_graphs.erase(c->cg_graphs.begin());
    }
    lp_ctx::CgGraph cg{};
    memcpy(cg.key, key, sizeof(key));
    cg.graph = g;
    cg.exec = ex;
    c->cg_graphs.push_back(cg);
    exec = ex;
  }
  LP_CU(launch_set(nullptr, 0, 0.0, c->fl, FL_TRIPS, 0, c->st));
  LP_CU(cudaGraphLaunch(exec, c->st));
  ++c->graph_launches;
  *ran = true;
  return LP_OK;
}

// Runs the CG loop of L (op 0, staged FP32-accumulated product) in the serving loop's batch
// engine: the launch descriptors of both iteration parities, exactly those cg_iteration would
// launch, go into a job.  *taken is false when the matrix or the engine cannot take it.
// The CG loop of a dense A streamed below FP64 as one cooperative launch (k_cg_persistent):
// every iteration's product and preconditioner apply in one kernel, with the argument sets of
// the serving engine's jobs.  ran = false when the launch does not cover the shape.
static lp_status cg_persistent_solve(lp_ctx* c, const CgLoop& L, int max_iter, bool* ran) {
  *ran = false;
  CgPersistArgs p{};
  for (int q = 0; q < 2; ++q) {
    ColArgs a{};
    a.A = c->As;
    a.lda = c->lda_s;
    a.m = c->m;
    a.n = c->n;
    a.d2 = c->d2;
    a.d2f = c->d2f;
    a.part = c->part;
    a.fl = c->fl;
    a.sc = c->sc;
    a.skip_if_done = 1;
    a.dz = c->z;
    a.dold = L.d[(q + 1) & 1];
    a.dnew = L.d[q];
    a.flw = c->fl;
    a.qacc = L.q[q];
    a.qsum = c->q;
    a.cnt = c->bcnt + 1;
    a.scw = c->sc;
    p.prod[q] = a;
    p.step1[q] = SymvArgs{c->factored ? c->XF : c->M, c->mp, c->m, L.r[(q + 1) & 1],
                          c->factored ? c->ptmp : c->z, c->sc, c->fl, c->bpart, c->bcnt,
                          SYMV_CG_STEP, 0.0, L.r[q], c->q, L.d[q], L.delta, L.q[q],
                          L.q[(q + 1) & 1], c->factored ? 1 : 0, 0};
    p.step2[q] = SymvArgs{c->XFT, c->mp, c->m, c->ptmp, c->z, c->sc, c->fl, c->bpart, c->bcnt,
                          SYMV_PLAIN, 0.0, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr,
                          0, 1};
  }
  p.factored = c->factored ? 1 : 0;
  p.bar = c->pbar;
  p.fl = c->fl;
  p.wait_ns = 0;
  p.max_trips = max_iter + 4;   // the apply sets the stop flag at max_iter
  LP_CU(cudaMemsetAsync(c->pbar, 0, 32 * sizeof(unsigned), c->st));
  if (launch_cg_persistent(c->s_dtype, p, c->num_sms, c->st) < 0) return LP_OK;
  LP_CU(cudaGetLastError());
  *ran = true;
  ++c->persistent_launches;
  return LP_OK;
}

static lp_status cg_batch_solve(lp_ctx* c, const CgLoop& L, bool* taken) {
  *taken = false;
  int tc = 8, nwarps = 1, S = 3;
  int64_t ngroups = 0;
  size_t smem = 0;
  if (!cgprod_job_shape(c->s_dtype, c->m, c->lda_s, c->n, &tc, &nwarps, &S, &ngroups, &smem))
    return LP_OK;
  if (!c->batch_ready) LP_CU(cudaEventCreateWithFlags(&c->batch_ready, cudaEventDisableTiming));
  CgBatchJob j;
  j.c = c;
  j.ta = c->s_dtype;
  j.tc = tc;
  j.nwarps = nwarps;
  j.prod_smem = smem;
  j.prod_ctas = cg_batch_prod_ctas(c, dtype_size(c->s_dtype), c->num_sms, ngroups);
  j.symv_ctas = (c->m + 7) / 8;
  j.symv_smem = (size_t)((c->m + 3) & ~3) * 2 * sizeof(double);
  j.factored = c->factored;
  j.ready = c->batch_ready;
  for (int p = 0; p < 2; ++p) {
    ColArgs a{};
    a.A = c->As;
    a.lda = c->lda_s;
    a.m = c->m;
    a.n = c->n;
    a.d2 = c->d2;
    a.d2f = c->d2f;
    a.part = c->part;
    a.fl = c->fl;
    a.sc = c->sc;
    a.skip_if_done = 1;
    a.dz = c->z;
    a.dold = L.d[(p + 1) & 1];
    a.dnew = L.d[p];
    a.flw = c->fl;
    a.qacc = L.q[p];
    a.qsum = c->q;
    a.cnt = c->bcnt + 1;
    a.scw = c->sc;
    j.prod[p] = CgProdJob{a, S, 0, 0, ngroups};
    SymvArgs s1{c->factored ? c->XF : c->M, c->mp, c->m, L.r[(p + 1) & 1],
                c->factored ? c->ptmp : c->z, c->sc, c->fl, c->bpart, c->bcnt, SYMV_CG_STEP, 0.0,
                L.r[p], c->q, L.d[p], L.delta, L.q[p], L.q[(p + 1) & 1], c->factored ? 1 : 0, 0};
    SymvArgs s2{c->XFT, c->mp, c->m, c->ptmp, c->z, c->sc, c->fl, c->bpart, c->bcnt, SYMV_PLAIN,
                0.0, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, 0, 1};
    j.step1[p] = s1;
    j.step2[p] = s2;
  }
  lp_status st = LP_OK;
  if (!cg_batcher_run(c->batcher, &j, &st)) return LP_OK;
  *taken = true;
  ++c->batched_solves;
  return st;
}

// PCG from delta = 0 with preconditioner M = Q^{-1} (Alg. 1 step 3), stopping when
// rho_j = r_j^T M r_j <= min(rel^2 rho_0, abs_thr^2) or after max_iter products.
//   op 0: (A D^2 A^T) delta = rhs with A streamed in the context's stream dtype;
//   op 1: (G G^T) delta = rhs in FP64 through the sketch G (for (A D W)^dagger).
static lp_status run_pcg(lp_ctx* c, int op, const double* rhs, double* delta, double rel_tol,
                         double abs_thr, int max_iter, int* iters, double* rho0_out,
                         double* rho_out) {
  PhaseScope ps(c, op == 0 ? LP_PH_PCG : LP_PH_CORRECTION);
  const int m = c->m;
  LP_CU(launch_vec_ops(VOP_ZERO, delta, nullptr, nullptr, m, nullptr, c->st));
  LP_CU(launch_vec_ops(VOP_COPY, c->r, rhs, nullptr, m, nullptr, c->st));
  const double thr2 = isfinite(abs_thr) ? abs_thr * abs_thr : INFINITY;
  LP_CU(launch_set(c->sc, SC_THR2, thr2, c->fl, FL_MAXIT, max_iter, c->st));
  LP_CU(launch_set(nullptr, 0, 0.0, c->fl, FL_NUMERIC, 0, c->st));
  // Richardson's iteration (App. A) replaces CG for the normal equations only; the solve for
  // (A D W)^dagger r~ (op 1) always runs CG
  const bool rich = op == 0 && c->prm.inner_solver == LP_INNER_RICHARDSON;
  LP_CU(launch_set(nullptr, 0, 0.0, c->fl, FL_RICH, rich ? 1 : 0, c->st));
  LP_CU(launch_set(nullptr, 0, 0.0, c->fl, FL_DIVERGED, 0, c->st));
  LP_TRY(precond_apply(c, SYMV_CG_INIT, c->r, c->z, rel_tol));
  // d starts at 0 so that the first fused direction update (beta = 0) gives d = z
  LP_CU(launch_vec_ops(VOP_ZERO, c->d_alt, nullptr, nullptr, m, nullptr, c->st));
  // iteration j: d_j = z + beta d_{j-1} into dbuf[j & 1]; r_{j+1} into rbuf[(j + 1) & 1]
  double* rbuf[2] = {c->r, c->r_alt};
  double* dbuf[2] = {c->dd, c->d_alt};
  // FP32-accumulated dense products reduce themselves into qbuf with atomics
  const bool atomic_q = (op == 0) && !c->sparse && c->s_dtype != LP_F64 && !c->cg_precise;
  double* qbuf[2] = {c->qf, c->qf + (size_t)kQCopies * m};
  if (atomic_q) LP_CU(cudaMemsetAsync(c->qf, 0, (size_t)kQCopies * m * sizeof(double), c->st));
  CgLoop L{op, delta, atomic_q, {rbuf[0], rbuf[1]}, {dbuf[0], dbuf[1]}, {qbuf[0], qbuf[1]}};
  bool finished = false;
  // a context of the serving loop hands the loop to the batch engine (shared launches)
  if (c->batcher && op == 0 && atomic_q && c->use_staged && !c->prof_on &&
      c->stall_group_p1 == 0) {
    bool taken = false;
    LP_TRY(cg_batch_solve(c, L, &taken));
    if (taken) {
      LP_TRY(sync_scalars(c));
      finished = c->fl_h[FL_DONE] != 0;
    }
  }
  // the persistent loop (one cooperative launch per solve), with no profiling events or fault
  // injection to honour
  if (!finished && c->prm.persistent_cg && op == 0 && atomic_q && c->use_staged && !c->prof_on &&
      c->stall_group_p1 == 0) {
    bool ran = false;
    LP_TRY(cg_persistent_solve(c, L, max_iter, &ran));
    if (ran) {
      LP_TRY(sync_scalars(c));
      if (!c->fl_h[FL_DONE])
        return fail(LP_ERR_CUDA, "persistent CG loop ended without its stop flag");
      finished = true;
    }
  }
  // the device-side loop (one graph launch per solve) once this context has run a CG solve
  // eagerly, with no profiling events or fault injection to honour
  if (!finished && c->use_graphs && c->prm.use_graphs && c->cg_solves > 0 && !c->prof_on &&
      c->stall_group_p1 == 0) {
    bool built = false;
    LP_TRY(cg_graph_launch(c, L, max_iter, &built));
    if (built) {
      LP_TRY(sync_scalars(c));
      finished = c->fl_h[FL_DONE] != 0;
    }
  }
  ++c->cg_solves;
  // host-driven loop: cg_batch iterations enqueued per check of the stop flag
  int done_before = 0;
  int j = 0;
  while (!finished) {
    for (int b = 0; b < c->prm.cg_batch; ++b, ++j) LP_TRY(cg_iteration(c, L, j, true));
    LP_TRY(sync_scalars(c));
    if (!c->mv_pending.empty()) prof_harvest_mv(c, c->fl_h[FL_ITERS] - done_before);
    done_before = c->fl_h[FL_ITERS];
    if (c->fl_h[FL_DONE]) break;
  }
  *iters = c->fl_h[FL_ITERS];
  if (rho0_out) *rho0_out = c->sc_h[SC_RHO0];
  if (rho_out) *rho_out = c->sc_h[SC_RHO];
  if (c->fl_h[FL_NUMERIC]) return fail(LP_ERR_NUMERIC, "CG met non-positive curvature or NaN");
  if (c->fl_h[FL_DIVERGED])
    return fail(LP_ERR_NOT_CONVERGED,
                "Richardson iteration diverges: ||I - Q^-1/2 A D^2 A^T Q^-1/2|| >= 1 (widen the sketch)");
  return LP_OK;
}

struct SolveOut {
  int cg_iters = 0;
  int refine = 0;
  double f_norm = 0.0;
  double f_target = 0.0;
};

// Alg. 1 (sketch, factor, PCG with FP64 residual refinement) and the FP64 correction data of
// Eq. compv for the current d2 / d (prepared by launch_prep_iterate).  Results:
//   c->dyacc = dy,  c->rtil = A D^2 A^T dy - p,  c->t = A^T dy,  c->u = (A D W)^dagger r~.
static lp_status run_normal_solve(lp_ctx* c, const double* p, int k, double mu, SolveOut* so) {
  const int m = c->m;
  LP_TRY(run_sketch(c, c->d, k, c->G));
  LP_TRY(run_factor(c, c->G, true));
  double abs_thr = INFINITY;
  if (c->prm.cg_theory_rule)
    abs_thr = c->prm.gamma * c->prm.sigma * sqrt(mu) / (4.0 * sqrt((double)c->n));
  bool lowprec = c->s_dtype != LP_F64 && !c->cg_precise;   // CG products accumulate in FP32
  double rho0 = 0.0, target2 = 0.0, f2_prev = INFINITY, contraction = 0.0;
  int total_it = 0, outer = 0, passes = 0;
  for (;;) {
    int it = 0;
    double r0 = 0.0, rl = 0.0;
    if (outer == 0) {
      LP_TRY(run_pcg(c, 0, p, c->dyacc, c->prm.cg_rel_tol, abs_thr, c->prm.cg_max_iter, &it,
                     &r0, &rl));
      rho0 = r0;
      target2 = std::min(c->prm.cg_rel_tol * c->prm.cg_rel_tol * rho0,
                         isfinite(abs_thr) ? abs_thr * abs_thr : INFINITY);
    } else {
      // refinement: solve (A D^2 A^T) delta = -r~ and add it to dy.  The residual of
      // dy + delta is the residual of this solve, so it stops at the solve's own target, or
      // once its own residual is below what the streamed operator can deliver in one pass
      // (the contraction of the previous pass times the current ||f||): solving the
      // rounded system further would not shrink the true residual.
      LP_CU(launch_vec_ops(VOP_NEG, c->rhs, c->rtil, nullptr, m, nullptr, c->st));
      const double thr = std::max(0.5 * sqrt(target2), 0.5 * contraction * sqrt(f2_prev));
      LP_TRY(run_pcg(c, 0, c->rhs, c->dy, INFINITY, thr, c->prm.cg_max_iter, &it, &r0, &rl));
      LP_CU(launch_vec_ops(VOP_ADD, c->dyacc, c->dyacc, c->dy, m, nullptr, c->st));
    }
    total_it += it;
    // r~ = A D^2 A^T dy - p in FP64 from the input-precision A, with t = A^T dy
    {
      PhaseScope ps(c, LP_PH_RTILDE);
      LP_TRY(pass_normal(c, true, c->dyacc, c->d2, c->t, RED_MINUS_P, c->rtil, p, 0));
    }
    // ||f||^2 = r~^T Q^{-1} r~; qhat = Q^{-1} r~ starts the correction
    LP_TRY(precond_apply(c, SYMV_F2, c->rtil, c->qhat, 0.0));
    LP_TRY(sync_scalars(c));
    const double f2 = c->sc_h[SC_F2];
    if (!isfinite(f2)) return fail(LP_ERR_NUMERIC, "non-finite residual in the normal solve");
    so->f_norm = sqrt(std::max(f2, 0.0));
    so->f_target = sqrt(target2);
    if (!lowprec || f2 <= 4.0 * target2) break;
    // Refinement converges when the streamed operator is close enough to A D^2 A^T in the
    // preconditioned norm; rounding A to 16 bits perturbs it by ~2^-9 relative per entry,
    // which a badly conditioned A D stretches past 1.  A refinement pass that fails to halve
    // ||f|| (or the pass cap) switches the solve to the master copy for the remaining IPM
    // iterations; without a copy to switch to, the cap ends the refinement.
    // contraction of this pass: ||f|| after it over ||f|| before it (pass 0 starts from
    // ||f^(0)|| = sqrt(rho0)); 1/8 or worse after the first solve also means many passes
    contraction = sqrt(f2 / (passes == 0 ? std::max(rho0, 1e-300) : f2_prev));
    const bool stalled = (passes == 0 && contraction > 0.125) || (passes >= 1 && f2 > 0.25 * f2_prev);
    if (stalled || passes >= c->prm.refine_max) {
      if (stream_switch(c, k)) {
        lowprec = c->s_dtype != LP_F64;
      } else {
        // refinement stalls on the master copy itself (FP32 A): the CG products accumulate in
        // FP64-class arithmetic from here on, for the rest of the IPM, and the next pass
        // solves the correction to the target
        c->cg_precise = true;
        c->precise_iter = k;
        lowprec = false;
      }
      passes = 0;
      contraction = 0.0;   // the master copy's passes solve to the target
    }
    f2_prev = f2;
    ++outer;
    ++passes;
  }
  so->cg_iters = total_it;
  // u = (A D W)^dagger r~ = (A D W)^T q with Q q = r~ (Eq. compv, full row rank): PCG on
  // Q = G G^T in FP64 with preconditioner M, then u = G^T q and the residual G u - r~.
  int steps = 0;
  LP_TRY(run_pcg(c, 1, c->rtil, c->qhat, 1e-13, INFINITY, std::max(50, c->prm.refine_max), &steps,
                 nullptr, nullptr));
  {
    PhaseScope ps(c, LP_PH_CORRECTION);
    LP_TRY(pass_gram(c, c->G, c->qhat, c->u, c->res, c->rtil, RED_MINUS_P, 0));
  }
  so->refine = steps + outer;
  return LP_OK;
}

// Alg. 2 steps (d)-(g) with W u gathered from the hashed W (or given).
static lp_status run_step(lp_ctx* c, double* x, double* y, double* s, const double* rd,
                          const double* dy, const double* t, const double* wu_given, double eta,
                          double mu0, double* dx, double* ds) {
  PhaseScope ps(c, LP_PH_UPDATE);
  LP_CU(launch_set(c->sc, SC_ETA, eta, nullptr, 0, 0, c->st));
  LP_CU(launch_set(c->sc, SC_MU0, mu0, nullptr, 0, 0, c->st));
  double* wu = wu_given ? const_cast<double*>(wu_given) : c->wu;
  LP_CU(launch_update_dirs(x, s, c->d2, c->d, rd, t, c->hb, c->ss, c->u, c->n, wu, dx, ds,
                           wu_given ? 1 : 0, c->sc, c->bpart, c->bcnt, c->st));
  LP_CU(launch_step_length(x, s, dx, ds, c->n, c->prm.gamma, c->sc, c->bpart, c->bcnt, c->st));
  LP_CU(launch_apply_step(x, s, y, dx, ds, dy, c->n, c->m, c->sc, c->st));
  return LP_OK;
}

// ------------------------------------------------------------------------------------------
// Entry points
// ------------------------------------------------------------------------------------------

// Algorithm 2 from the start point (resume == nullptr) or continued from a checkpoint.
static lp_status ipm_run(lp_ctx* c, double* x, double* y, double* s, bool start_given,
                         const lp_ipm_state* resume, lp_info* info) {
  stream_reset(c);
  const int m = c->m;
  const int64_t n = c->n;
  lp_info inf{};
  const long long graphs0 = c->graph_launches, pers0 = c->persistent_launches;
  if (resume && resume->stream_switch_iter >= 0) stream_switch(c, resume->stream_switch_iter);
  if (start_given) {
    LP_CU(cudaMemcpyAsync(c->x, x, n * sizeof(double), cudaMemcpyDefault, c->st));
    LP_CU(cudaMemcpyAsync(c->y, y, m * sizeof(double), cudaMemcpyDefault, c->st));
    LP_CU(cudaMemcpyAsync(c->s, s, n * sizeof(double), cudaMemcpyDefault, c->st));
  } else {
    std::unique_ptr<double[]> ones(new (std::nothrow) double[n > 0 ? (size_t)n : 1]);
    if (!ones) return fail(LP_ERR_OOM, "lp_ipm_solve: host allocation failed");
    std::fill(ones.get(), ones.get() + n, 1.0);
    LP_CU(cudaMemcpyAsync(c->x, ones.get(), n * sizeof(double), cudaMemcpyHostToDevice, c->st));
    LP_CU(cudaMemcpyAsync(c->s, ones.get(), n * sizeof(double), cudaMemcpyHostToDevice, c->st));
    LP_CU(cudaMemsetAsync(c->y, 0, m * sizeof(double), c->st));
    LP_CU(cudaStreamSynchronize(c->st));
  }
  const double sigma = c->prm.sigma;
  LP_TRY(run_residuals(c, c->x, c->y, c->s, sigma, c->rp, c->rd, c->p));
  LP_TRY(sync_scalars(c));
  // N(gamma)'s references belong to the start point of the run, not to a resumed iterate
  const double mu0 = resume ? resume->mu0 : c->sc_h[SC_MU];
  const double r0 = resume ? resume->r0 : sqrt(c->sc_h[SC_RP2] + c->sc_h[SC_RD2]);
  lp_status result = LP_ERR_NOT_CONVERGED;
  int k = resume ? resume->k : 0;
  for (;;) {
    const double mu = c->sc_h[SC_MU];
    const double rpn = sqrt(c->sc_h[SC_RP2]), rdn = sqrt(c->sc_h[SC_RD2]);
    const double cx = c->sc_h[SC_CX];
    inf.rp_rel = rpn / (1.0 + c->bnorm);
    inf.rd_rel = rdn / (1.0 + c->cnorm);
    inf.gap_rel = (double)n * mu / (1.0 + fabs(cx));
    inf.mu = mu;
    inf.obj = cx;
    if (!isfinite(mu) || !isfinite(rpn) || !isfinite(rdn)) {
      result = fail(LP_ERR_NUMERIC, "non-finite iterate");
      break;
    }
    if (std::max(inf.rp_rel, std::max(inf.rd_rel, inf.gap_rel)) <= c->prm.tol) {
      result = LP_OK;
      break;
    }
    if (k >= c->prm.ipm_max_iter) {
      result = fail(LP_ERR_NOT_CONVERGED, "IPM iteration cap reached");
      break;
    }
    const double eta = r0 > 0 ? sqrt(rpn * rpn + rdn * rdn) / r0 : 0.0;
    SolveOut so;
    lp_status st = run_normal_solve(c, c->p, k, mu, &so);
    if (st != LP_OK) {
      result = st;
      break;
    }
    inf.cg_iters_total += so.cg_iters;
    inf.cg_iters_last = so.cg_iters;
    if (c->factor_stages == 2) inf.factor_two_stage += 1;
    inf.cg_precise_iter = c->precise_iter;
    inf.refine_steps = so.refine;
    inf.f_norm = so.f_norm;
    inf.f_target = so.f_target;
    const double* wu_given = nullptr;
    if (c->prm.sketch_kind == LP_SKETCH_GAUSSIAN) {
      // the fused update gathers W u from the sparse W's buckets; the Gaussian W needs W u first
      LP_CU(launch_apply_W_gauss(c->prm.seed, k, c->n, c->w, c->gq, c->u, c->wu, c->st));
      wu_given = c->wu;
    }
    st = run_step(c, c->x, c->y, c->s, c->rd, c->dyacc, c->t, wu_given, eta, mu0, c->dx, c->ds);
    if (st != LP_OK) {
      result = st;
      break;
    }
    ++k;
    st = run_residuals(c, c->x, c->y, c->s, sigma, c->rp, c->rd, c->p);
    if (st == LP_OK) st = sync_scalars(c);
    if (st != LP_OK) {
      result = st;
      break;
    }
    inf.alpha_max = c->sc_h[SC_AMAX];
    inf.alpha = c->sc_h[SC_STEP];
    inf.v_norm = sqrt(c->sc_h[SC_V2]);
  }
  inf.ipm_iters = k;
  inf.status = result;
  inf.stream_dtype = c->s_dtype;
  inf.stream_switch_iter = c->switch_iter;
  inf.cg_precise_iter = c->precise_iter;
  inf.cg_graph_solves = (int32_t)(c->graph_launches - graphs0);
  inf.cg_persistent_solves = (int32_t)(c->persistent_launches - pers0);
  c->ipm_state.k = k;
  c->ipm_state.stream_switch_iter = c->switch_iter;
  c->ipm_state.r0 = r0;
  c->ipm_state.mu0 = mu0;
  LP_CU(cudaMemcpyAsync(x, c->x, n * sizeof(double), cudaMemcpyDefault, c->st));
  LP_CU(cudaMemcpyAsync(y, c->y, m * sizeof(double), cudaMemcpyDefault, c->st));
  LP_CU(cudaMemcpyAsync(s, c->s, n * sizeof(double), cudaMemcpyDefault, c->st));
  LP_CU(cudaStreamSynchronize(c->st));
  if (info) *info = inf;
  return result;
}

extern "C" lp_status lp_ipm_solve(lp_ctx* c, double* x, double* y, double* s, int32_t start_given,
                                  lp_info* info) {
  if (!c || !x || !y || !s) return fail(LP_ERR_ARG, "lp_ipm_solve: NULL argument");
  return ipm_run(c, x, y, s, start_given != 0, nullptr, info);
}

extern "C" lp_status lp_ipm_get_state(lp_ctx* c, lp_ipm_state* state) {
  if (!c || !state) return fail(LP_ERR_ARG, "lp_ipm_get_state: NULL argument");
  *state = c->ipm_state;
  return LP_OK;
}

extern "C" lp_status lp_ipm_resume(lp_ctx* c, double* x, double* y, double* s,
                                   const lp_ipm_state* state, lp_info* info) {
  if (!c || !x || !y || !s || !state) return fail(LP_ERR_ARG, "lp_ipm_resume: NULL argument");
  if (state->k < 0 || !(state->r0 >= 0.0) || !isfinite(state->r0) || !(state->mu0 > 0.0) ||
      !isfinite(state->mu0) || state->stream_switch_iter < -1 ||
      state->stream_switch_iter > state->k)
    return fail(LP_ERR_ARG, "lp_ipm_resume: state out of range");
  const lp_ipm_state st = *state;   // the caller may pass the context's own state
  return ipm_run(c, x, y, s, true, &st, info);
}

extern "C" lp_status lp_normal_solve(lp_ctx* c, const double* x, const double* s, const double* p,
                                     int32_t k, double* dy, double* rtil, double* u, double* Wu,
                                     double* Atdy, lp_info* info) {
  if (!c || !x || !s || !p || !dy) return fail(LP_ERR_ARG, "lp_normal_solve: NULL argument");
  if (k < 0) return fail(LP_ERR_ARG, "lp_normal_solve: k < 0");
  stream_reset(c);
  const long long graphs0 = c->graph_launches, pers0 = c->persistent_launches;
  LP_CU(launch_prep_iterate(x, s, c->n, c->d2, c->d, c->sc, c->bpart, c->bcnt, c->prm.sigma,
                            c->c, c->st, c->d2f, stream_cs2(c), c->dfc));
  LP_TRY(sync_scalars(c));
  const double mu = c->sc_h[SC_MU];
  if (!(mu > 0) || !isfinite(mu)) return fail(LP_ERR_ARG, "lp_normal_solve: x, s must be positive");
  LP_CU(cudaMemcpyAsync(c->rhs, p, c->m * sizeof(double), cudaMemcpyDefault, c->st));
  // run_normal_solve uses c->rhs as scratch in refinement: keep p in rp
  LP_CU(cudaMemcpyAsync(c->rp, p, c->m * sizeof(double), cudaMemcpyDefault, c->st));
  SolveOut so;
  LP_TRY(run_normal_solve(c, c->rp, k, mu, &so));
  LP_CU(cudaMemcpyAsync(dy, c->dyacc, c->m * sizeof(double), cudaMemcpyDefault, c->st));
  if (rtil) LP_CU(cudaMemcpyAsync(rtil, c->rtil, c->m * sizeof(double), cudaMemcpyDefault, c->st));
  if (u) LP_CU(cudaMemcpyAsync(u, c->u, c->w * sizeof(double), cudaMemcpyDefault, c->st));
  if (Atdy) LP_CU(cudaMemcpyAsync(Atdy, c->t, c->n * sizeof(double), cudaMemcpyDefault, c->st));
  if (Wu && c->prm.sketch_kind == LP_SKETCH_GAUSSIAN)
    LP_CU(launch_apply_W_gauss(c->prm.seed, k, c->n, c->w, c->gq, c->u, Wu, c->st));
  else if (Wu)
    LP_CU(launch_apply_W(c->hb, c->ss, c->u, c->n, Wu, c->st));
  LP_CU(cudaStreamSynchronize(c->st));
  if (info) {
    lp_info inf{};
    inf.cg_iters_last = so.cg_iters;
    inf.cg_iters_total = so.cg_iters;
    inf.refine_steps = so.refine;
    inf.f_norm = so.f_norm;
    inf.f_target = so.f_target;
    inf.mu = mu;
    inf.stream_dtype = c->s_dtype;
    inf.stream_switch_iter = c->switch_iter;
    inf.factor_two_stage = c->factor_stages == 2 ? 1 : 0;
    inf.cg_precise_iter = c->precise_iter;
    inf.cg_graph_solves = (int32_t)(c->graph_launches - graphs0);
    inf.cg_persistent_solves = (int32_t)(c->persistent_launches - pers0);
    *info = inf;
  }
  return LP_OK;
}

extern "C" lp_status lp_residuals(lp_ctx* c, const double* x, const double* y, const double* s,
                                  double sigma, double* rp, double* rd, double* p, double* mu_out) {
  if (!c || !x || !y || !s || !rp || !rd || !p) return fail(LP_ERR_ARG, "lp_residuals: NULL argument");
  LP_TRY(run_residuals(c, x, y, s, sigma, rp, rd, p));
  LP_TRY(sync_scalars(c));
  if (mu_out) *mu_out = c->sc_h[SC_MU];
  return LP_OK;
}

extern "C" lp_status lp_sketch_indices(uint64_t seed, int32_t k, int64_t n, int32_t s, int32_t w,
                                       int32_t* bucket, int8_t* sign, void* stream) {
  if (n < 0 || s < 1 || w < 1 || w % s != 0 || k < 0)
    return fail(LP_ERR_ARG, "lp_sketch_indices: need n >= 0, s >= 1, w % s == 0, k >= 0");
  if (n == 0) return LP_OK;
  if (!bucket || !sign) return fail(LP_ERR_ARG, "lp_sketch_indices: NULL output");
  LP_CU(launch_sketch_hash(seed, k, n, s, w, nullptr, nullptr, bucket, sign, (cudaStream_t)stream));
  return LP_OK;
}

extern "C" lp_status lp_sketch(lp_ctx* c, const double* d, int32_t k, double* G) {
  if (!c || !d || !G || k < 0) return fail(LP_ERR_ARG, "lp_sketch: bad argument");
  LP_TRY(run_sketch(c, d, k, c->G));
  LP_CU(cudaMemcpy2DAsync(G, c->m * sizeof(double), c->G, c->ldg * sizeof(double),
                          c->m * sizeof(double), c->w, cudaMemcpyDefault, c->st));
  LP_CU(cudaStreamSynchronize(c->st));
  return LP_OK;
}

extern "C" lp_status lp_factor(lp_ctx* c, const double* G, double* Q, double* Minv) {
  if (!c || !G) return fail(LP_ERR_ARG, "lp_factor: NULL argument");
  LP_CU(cudaMemcpy2DAsync(c->G, c->ldg * sizeof(double), G, c->m * sizeof(double),
                          c->m * sizeof(double), c->w, cudaMemcpyDefault, c->st));
  LP_TRY(run_factor(c, c->G, false));
  const size_t row = c->m * sizeof(double), pitch = c->mp * sizeof(double);
  if (Q) LP_CU(cudaMemcpy2DAsync(Q, row, c->Q, pitch, row, c->m, cudaMemcpyDefault, c->st));
  if (Minv) {
    // M is kept as double-float pairs; assemble FP64 entries (device scratch: X)
    LP_CU(launch_df_to_double(c->M, c->mp, c->m, c->X, c->m, c->st));
    LP_CU(cudaMemcpyAsync(Minv, c->X, (size_t)c->m * c->m * sizeof(double), cudaMemcpyDefault,
                          c->st));
  }
  LP_CU(cudaStreamSynchronize(c->st));
  return LP_OK;
}

extern "C" lp_status lp_normal_matvec(lp_ctx* c, const double* d2, const double* v, double* y,
                                      double* t, lp_dtype stream_dtype) {
  if (!c || !d2 || !v || !y) return fail(LP_ERR_ARG, "lp_normal_matvec: NULL argument");
  bool precise;
  stream_reset(c);
  if (stream_dtype == LP_F64) {
    precise = true;
  } else if (stream_dtype == c->s_dtype) {
    precise = false;
  } else {
    return fail(LP_ERR_ARG, "lp_normal_matvec: stream dtype differs from the context's");
  }
  if (!precise && c->s_dtype != LP_F64) {
    // the FP32-accumulated product takes its weight as FP32 (with the copy's column scales)
    LP_CU(launch_d2f(d2, stream_cs2(c), c->n, c->d2f, c->st));
  }
  LP_TRY(pass_normal(c, precise, v, d2, t, RED_PLAIN, y, nullptr, 0, false, nullptr, nullptr,
                     nullptr, nullptr, !precise && c->s_dtype != LP_F64));
  return sync_scalars(c);   // LP_ERR_TIMEOUT if a bounded wait of the product gave up
}

extern "C" lp_status lp_test_stall_copy(lp_ctx* c, int32_t group, uint64_t wait_ns) {
  if (!c || group < 0 || wait_ns == 0 || wait_ns > 1000000000ull)
    return fail(LP_ERR_ARG, "lp_test_stall_copy: need a context, group >= 0, 0 < wait_ns <= 1e9");
  c->stall_group_p1 = (int64_t)group + 1;
  c->stall_wait_ns = wait_ns;
  return LP_OK;
}

extern "C" lp_status lp_step(lp_ctx* c, double* x, double* y, double* s, const double* rd,
                             const double* dy, const double* Atdy, const double* Wu, double mu,
                             double eta, double mu0, double* dx, double* ds, double* out) {
  if (!c || !x || !y || !s || !rd || !dy || !Atdy || !Wu) return fail(LP_ERR_ARG, "lp_step: NULL argument");
  if (!(mu0 > 0)) return fail(LP_ERR_ARG, "lp_step: mu0 must be positive");
  LP_CU(launch_prep_iterate(x, s, c->n, c->d2, c->d, c->sc, c->bpart, c->bcnt, c->prm.sigma,
                            c->c, c->st, c->d2f, stream_cs2(c), c->dfc));
  (void)mu;  // mu is recomputed from x and s on the device
  LP_TRY(run_step(c, x, y, s, rd, dy, Atdy, Wu, eta, mu0, dx ? dx : c->dx, ds ? ds : c->ds));
  LP_TRY(sync_scalars(c));
  if (out) {
    out[0] = c->sc_h[SC_AMAX];
    out[1] = c->sc_h[SC_STEP];
    out[2] = c->sc_h[SC_B];
    out[3] = c->sc_h[SC_C];
  }
  return LP_OK;
}

extern "C" uint64_t lp_footprint_bytes(int32_t m, int64_t n, lp_layout layout, lp_dtype a_dtype,
                                       int64_t nnz, const lp_params* prm, int32_t num_sms) {
  if (m < 1 || n < m) return 0;
  lp_params p;
  if (prm) p = *prm; else lp_params_default(&p);
  if (num_sms <= 0) num_sms = 152;
  const double es = (double)dtype_size(a_dtype);
  const int s = p.sketch_s > 0 ? p.sketch_s : 4;
  const int w = p.sketch_w ? p.sketch_w : 4 * m;
  const int mp = round_up(m, 64);
  const int nt = mp / 64;
  const double dn = (double)n, dm = (double)m;
  double b = 0.0;
  b += 9 * 8 * dn + 4 * dn + 16 * 8 * dm;                                  // n- and m-vectors
  b += (double)std::max(coltile_max_grid(num_sms), csc_max_grid(num_sms)) * 2 * dm * 8;
  b += dn * s * (4 + 4 + 8) + 2.0 * kQCopies * dm * 8 + 3.0 * (w + 1) * 4; // sketch indices, q
  b += (double)round_up(m, 2) * w * 16 + (double)w * 8;                    // G, its split, u
  b += 4.0 * mp * mp * 8;                                                  // Q, M, X, M in FP64
  b += (double)gram_split_cap(m, w, num_sms) * (nt * (nt + 1) / 2) * 64.0 * 64.0 * 8;
  b += (double)gram_tc_digit_bytes(m, w) + 4.0 * gram_tc_rows(m) +
       (double)gram_tc_part_bytes(m, mp, w, num_sms);                      // tensor-core Gram
  b += 3.0 * mp * mp * 8 + (double)round_up(m, 2) * w * 8;               // second factor stage
  if (p.factor_dag && mp / kNB <= kDagMaxBlocks)                           // one-launch sweep
    b += 4.0 * (double)chol_dag_tasks(mp / kNB, nullptr) + 4.0 * chol_dag_sync_words(mp / kNB);
  b += (SC_COUNT + kMaxRedBlocks * 8) * 8.0 + FL_COUNT * 4 + 64;
  b += 8 * dm + 8 * dn;                                                    // b, c
  if (layout != LP_CSR) b += 2.0 * (1 << kGaussBits);                      // Gaussian W table
  if (layout != LP_CSR && p.sketch_kind == LP_SKETCH_GAUSSIAN && p.gram_tensor_cores)
    b += (double)sketch_tc_work_bytes(m, n, w, num_sms);                   // tensor-core sketch
  if (layout != LP_CSR) {
    const int lda = round_up(m, (int)(16 / dtype_size(a_dtype)));
    b += (double)lda * dn * es;
    if (a_dtype == LP_F32) b += 32 * dn;                                   // column scalars
    if (layout == LP_DENSE_ROWMAJOR) b += dm * dn * es;                    // staging copy
    lp_dtype sd = p.stream_dtype == LP_F64 ? a_dtype : p.stream_dtype;
    if (sd == LP_F64 && a_dtype == LP_F32) sd = LP_F32;
    if (sd != a_dtype) {
      const int ldas = round_up(m, (int)(16 / dtype_size(sd)));
      b += (double)ldas * dn * dtype_size(sd);
      if (sd == LP_BF16 || sd == LP_F16) b += 4 * dn;
    }
  } else {
    const double z = (double)std::max<int64_t>(nnz, 0);
    b += 2 * ((dm + 1) * 8 + z * 4 + z * es) + 8 * dn + (dn + 1) * 8;      // CSR staging + CSC
    if (p.stream_dtype == LP_F32 && a_dtype == LP_F64) b += 4 * z;
  }
  b += 60.0 * 512 + 2.0 * (1 << 20);                                       // pool granularity, slack
  return (uint64_t)b;
}

extern "C" lp_status lp_profile_enable(lp_ctx* c, int32_t on) {
  if (!c) return fail(LP_ERR_ARG, "lp_profile_enable: NULL");
  c->prof_on = on != 0;
  return LP_OK;
}

extern "C" lp_status lp_profile_read(lp_ctx* c, lp_profile* out, int32_t reset) {
  if (!c || !out) return fail(LP_ERR_ARG, "lp_profile_read: NULL");
  LP_CU(cudaStreamSynchronize(c->st));
  if (!c->ev_pending.empty()) prof_harvest(c);
  // average over the timed products (the streamed copy may change within a solve)
  c->prof.matvec_bytes = c->prof.matvec_count > 0 ? c->mv_bytes_sum / c->prof.matvec_count
                                                  : matvec_bytes(c);
  c->prof.launches = g_launches.load();
  const CgTune& tn = c->tune[(int)c->s_dtype & 3];
  c->prof.tune_tc = tn.tc;
  c->prof.tune_stages = tn.stages;
  c->prof.tune_ctas = tn.ctas;
  c->prof.tune_us = tn.us;
  c->prof.tune_rule_us = tn.rule_us;
  *out = c->prof;
  if (reset) {
    c->prof = lp_profile{};
    c->mv_bytes_sum = 0.0;
  }
  return LP_OK;
}
