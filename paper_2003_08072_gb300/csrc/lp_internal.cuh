// Internal declarations of the sm_103a LP library: context, scalar slots, kernel launchers.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <string>
#include <vector>

#include "../../include/lp.h"
#include "chol_tasks.h"
#include "gauss_grid.h"

namespace lpk {

// ---- device scalar slots (double sc[SC_COUNT]) ---------------------------------------
enum Scalar {
  SC_MU = 0,      // x^T s / n
  SC_XS,          // x^T s
  SC_SIGMU,       // sigma * mu
  SC_RP2,         // ||r_p||^2
  SC_RD2,         // ||r_d||^2
  SC_CX,          // c^T x
  SC_RHO,         // CG rho_j = r^T Q^{-1} r
  SC_RHO0,        // rho_0 of the current CG solve
  SC_THR2,        // squared CG stop threshold on rho
  SC_ALPHA,       // CG alpha
  SC_BETA,        // CG beta
  SC_DQ,          // d^T q
  SC_B,           // x^T ds + s^T dx
  SC_C,           // dx^T ds
  SC_AMAX,        // alpha_max
  SC_STEP,        // alpha
  SC_V2,          // ||v||^2
  SC_V1,          // 1^T v
  SC_RES2,        // squared norm of a refinement residual
  SC_F2,          // r~^T Q^{-1} r~  (||f^(t)||^2)
  SC_ETA,         // ||r|| / ||r^0||
  SC_MU0,         // mu_0
  SC_AMIN,        // per-element min crossing (internal)
  SC_COUNT = 32
};

enum Flag {
  FL_DONE = 0,   // CG finished (converged or capped)
  FL_ITERS,      // CG iterations of the current solve
  FL_NUMERIC,    // non-finite or non-positive curvature seen
  FL_BREAK,      // non-positive pivot in the factorization
  FL_MAXIT,      // CG iteration cap of the current solve
  FL_TIMEOUT,    // a bounded wait in a kernel gave up
  FL_RICH,       // the running solve is Richardson's iteration (App. A): alpha = 1, beta = 0
  FL_DIVERGED,   // Richardson's residual grew past 1e6 times its start
  FL_TRIPS,      // bodies run by the device-side CG loop of the current graph launch
  FL_COUNT = 16
};

extern std::atomic<long long> g_launches;   // kernel launches issued (lp_api.cu)
inline void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

constexpr int kNB = 32;          // block size of the blocked Cholesky inverse
constexpr int kQCopies = 8;      // copies of the atomically accumulated CG product
constexpr int kMaxRedBlocks = 1024;

// Launch shape of the staged CG product picked by the autotuner, with its measured time and
// the time of the fixed rule on the same matrix.
struct CgTune {
  int tc = 0, stages = 0, ctas = 0;
  float us = 0.f, rule_us = 0.f;
};

}  // namespace lpk

struct CgBatcher;

struct lp_ctx {
  int m = 0;
  int64_t n = 0;
  bool sparse = false;
  lp_params prm{};
  cudaStream_t st = nullptr;
  int dev = 0;
  int num_sms = 0;

  // dense matrix, column-major, 16-byte aligned columns (zero padded rows m..lda-1)
  lp_dtype a_dtype = LP_F64;   // master copy dtype (F64 or F32)
  void* A = nullptr;
  int lda = 0;
  lp_dtype s_dtype = LP_F64;   // streamed copy dtype used by the CG matvec
  void* As = nullptr;          // == A when s_dtype == a_dtype
  int lda_s = 0;
  bool own_As = false;
  float* cs2 = nullptr;        // BF16/F16 copy: per-column 2^(2 e_j) (the copy holds A_j 2^-e_j)
  bool cs2_on = false;         // the streamed copy in use is the scaled one
  // the stream copy asked for at lp_create; a solve whose FP64 refinement stops contracting
  // switches to streaming the master copy (s_dtype = a_dtype) until the next solve starts
  lp_dtype s_dtype_req = LP_F64;
  void* As_req = nullptr;
  int lda_s_req = 0;
  void* svals_req = nullptr;
  int switch_iter = -1;        // IPM iteration of the last switch (-1: none)
  // last resort of the refinement: CG products with FP64-class accumulation over the master
  // copy (double-float for FP32 A) once refinement stalls on the master copy itself
  bool cg_precise = false;
  int precise_iter = -1;       // IPM iteration of that escalation (-1: none)
  lp_ipm_state ipm_state{0, -1, 0.0, 0.0};  // Algorithm 2's state at the end of the last run
  bool use_staged = true;      // CG products through the shared-memory staged pass
  lpk::CgTune tune[4];         // autotuned launch shape of the staged product per stream dtype
  // fault injection for the next staged CG product only (lp_test_stall_copy)
  int64_t stall_group_p1 = 0;
  uint64_t stall_wait_ns = 0;
  double mv_bytes_sum = 0.0;   // algorithmic bytes of the timed CG products

  // CSC (sparse) copy: column pointers, row ids, values
  int64_t nnz = 0;
  int64_t* colptr = nullptr;
  int32_t* rowidx = nullptr;
  void* vals = nullptr;        // a_dtype (F32 or F64)
  void* svals = nullptr;       // stream dtype values (== vals or bf16/f16 copy)
  bool own_svals = false;

  double* b = nullptr;
  double* c = nullptr;
  double bnorm = 0, cnorm = 0;

  // n-vectors
  double *x = nullptr, *y = nullptr, *s = nullptr, *d2 = nullptr, *d = nullptr;
  double *rd = nullptr, *t = nullptr, *wu = nullptr, *dx = nullptr, *ds = nullptr;
  float* d2f = nullptr;        // D^2 rounded to FP32 for the FP32-accumulated CG product
  // dense FP32 A: 4 n double-float pairs D^2, x, 1/s, s - c of the current iterate
  // (written with d2 by launch_prep_iterate) for the FP64-class passes
  float2* dfc = nullptr;
  // m-vectors
  double *rp = nullptr, *p = nullptr, *dy = nullptr, *r = nullptr, *z = nullptr, *dd = nullptr;
  double *q = nullptr, *rtil = nullptr, *qhat = nullptr, *res = nullptr, *tm = nullptr;
  double *dyacc = nullptr, *rhs = nullptr;
  double *r_alt = nullptr, *d_alt = nullptr;   // second buffers of the CG residual / direction
  double* qf = nullptr;        // 2 x kQCopies x m: atomically accumulated CG products (FP32 streams)

  // per-CTA partials of the column-tile kernels
  void* part = nullptr;
  size_t part_bytes = 0;

  // sketch
  int w = 0, ss = 0;
  int32_t* hb = nullptr;       // n*s packed (bucket | sign bit 31)
  int32_t* cnt = nullptr;      // w + 1
  int32_t* start = nullptr;    // w + 1
  int32_t* cursor = nullptr;   // w
  int32_t* list = nullptr;     // n*s entries: column | sign bit 31
  float2* coef = nullptr;      // n*s entries: sign d_i / sqrt(s) as a double-float pair
  double* G = nullptr;         // m x w column-major, leading dimension ldg (even)
  float* Gdf = nullptr;        // G split into hi and lo floats (2 ldg w) for the Gram product
  int ldg = 0;
  double* u = nullptr;         // w

  // factor
  int mp = 0;                  // m rounded up to kNB
  double* Q = nullptr;         // mp x mp row-major (full symmetric)
  double* M = nullptr;         // Q^{-1} as double-float pairs (hi, lo: two mp x mp float matrices)
  double* X = nullptr;         // L^{-1} work buffer of the factor, mp x mp
  double* Qsplit = nullptr;    // split-k partials of the Gram product
  // tensor-core Gram product: digit slices of G, row exponents, double-float partial tiles
  __nv_bfloat16* gdig = nullptr;
  int* gex = nullptr;
  float2* gpart = nullptr;
  int qsplit = 1;
  double shift = 0.0;          // relative diagonal shift used by the last factorization
  // second factor stage (Q numerically singular for the Gram route, e.g. CountSketch late in
  // the IPM): X1 = inverse factor of the shifted first stage, G1 = X1 G as hi / lo planes,
  // XF = X2 X1 and its transpose XFT (double-float planes, mp x mp); allocated on first use
  bool factored = false;       // the preconditioner is applied as XF^T (XF r)
  int factor_stages = 1;       // stages of the last factorization (1 or 2)
  double qerr = 0.0;           // probe error ||Q M 1 - 1|| / sqrt(m) of the last factor stage
  double* Mf64 = nullptr;       // M = X^T X in FP64 from the tensor-core Gram (first use)
  double* X1 = nullptr;
  double* XF = nullptr;
  double* XFT = nullptr;
  float* G1df = nullptr;
  double* ptmp = nullptr;      // m-vector: X r of the factored apply

  // scalars
  double* sc = nullptr;        // device SC_COUNT
  int* fl = nullptr;           // device FL_COUNT
  double* bpart = nullptr;     // last-block reduction partials (kMaxRedBlocks * 8)
  unsigned* bcnt = nullptr;    // last-block counters (16)
  void* pin_blk = nullptr;     // pinned host block holding sc_h and fl_h
  double* sc_h = nullptr;      // pinned host mirror of sc
  int* fl_h = nullptr;         // pinned host mirror of fl

  // CUDA graphs of the CG loop: one WHILE node whose body is two CG iterations and a
  // condition kernel, so a whole CG solve is one graph launch with no host round trip; built
  // per configuration of the loop (operator, copy streamed, preconditioner form, ...)
  struct CgGraph {
    unsigned char key[128];
    cudaGraph_t graph;
    cudaGraphExec_t exec;
  };
  // the serving loop's CG batch engine (lp_batch.cu); its CG solves then share launches
  CgBatcher* batcher = nullptr;
  cudaEvent_t batch_ready = nullptr;
  long long batched_solves = 0;
  bool use_graphs = true;      // lp_params.use_graphs and no failure so far
  cudaStream_t cap_st = nullptr;   // private stream the graphs are recorded on (the context
                                   // stream may be the legacy default stream, which cannot be)
  std::string graph_error;     // why graphs were given up, if they were
  long long cg_solves = 0;     // CG solves run (the first one always runs eagerly)
  std::vector<CgGraph> cg_graphs;
  long long graph_launches = 0;
  long long persistent_launches = 0;
  unsigned* pbar = nullptr;     // grid barrier words of the persistent CG loop (32)
  int16_t* gq = nullptr;        // quantile table of the Gaussian W (dense A)
  void* gtc = nullptr;          // digits and partial tiles of the tensor-core Gaussian sketch
  size_t gtc_bytes = 0;
  uint32_t* chtasks = nullptr;  // task list of the one-launch Cholesky sweep (allocated on first use)
  int chntasks = 0;
  int* chsync = nullptr;        // its claim counter and tile counters

  // profiling (CUDA events on st)
  struct EvPair {
    int phase;                 // LP_PH_* or -1 for a CG product
    cudaEvent_t a, b;
  };
  bool prof_on = false;
  std::vector<cudaEvent_t> ev_pool;
  std::vector<EvPair> ev_pending;
  std::vector<EvPair> mv_pending;   // CG product launches of the current batch
  lp_profile prof{};
};

// ---------------------------------------------------------------------------------------
// error reporting (lp_api.cu)
void lp_set_error(const std::string& msg);
lp_status lp_cuda_fail(cudaError_t e, const char* what);

#define LP_CU(call)                                   \
  do {                                                \
    cudaError_t e__ = (call);                         \
    if (e__ != cudaSuccess) return lp_cuda_fail(e__, #call); \
  } while (0)

// ---------------------------------------------------------------------------------------
// launchers (each enqueues on ctx->st and returns cudaGetLastError())
namespace lpk {

enum ColMode { MODE_NORMAL = 0, MODE_RESID = 1 };

// y-partials of  sum_i a_i * coef_i  over column tiles of a dense column-major matrix.
struct ColArgs {
  const void* A;
  int64_t lda;
  int m;
  int64_t n;
  int64_t ntiles;
  const double* v;     // m-vector for the column dots
  const double* d2;    // NORMAL: per-column weight (NULL = 1)
  const float* d2f;    // NORMAL with FP32 accumulation: the same weight rounded to FP32 (optional)
  const double* x;     // RESID
  const double* s;     // RESID
  const double* c;     // RESID
  const double* sc;    // device scalars (RESID reads SC_SIGMU)
  double* colout;      // NORMAL: t = A^T v (may be NULL); RESID: r_d
  void* part;          // [grid][nout][m] partials (accumulator type)
  const int* fl;       // skip everything when fl[FL_DONE] != 0 and skip_if_done
  int skip_if_done;
  // CG direction update fused into the product: v = dz + beta dold (beta = sc[SC_BETA]); CTA 0
  // stores v into dnew.  Used when dz != NULL.
  const double* dz;
  const double* dold;
  double* dnew;
  // CG with FP32 accumulation: add the row sums into qacc with atomics instead of writing
  // partials; the last CTA forms d^T q (d = dnew) and alpha = rho / d^T q in scw / flw.
  double* qacc;
  double* qsum;        // the last CTA also writes q = sum of the qacc copies here
  unsigned* cnt;
  double* scw;
  int* flw;
  // staged CG product only: limit of each bounded wait (0: 1 s), and a fault-injection hook,
  // 1 + the local column group of CTA 0 whose copy is never issued (0: none, so that a
  // zero-initialised ColArgs injects nothing)
  uint64_t wait_ns;
  int64_t stall_group_p1;
  // staged CG product only: a launch shape chosen by the autotuner (0: the fixed rule)
  int cfg_tc, cfg_stages, cfg_ctas;
  // FP64-class passes over an FP32 A: per-column scalars of the iterate as double-float pairs
  // (written by launch_prep_iterate): NORMAL reads d2df when the weight is D^2; RESID reads
  // x, 1/s and s - c.  NULL: the scalars are split from the FP64 vectors.
  const float2* d2df;
  const float2* xdf;
  const float2* isdf;
  const float2* scdf;
};


// Dense column-tile pass.  acc_f64 selects FP64 accumulation (else FP32).
// Returns the number of CTAs used (partials rows), or -1 on an unsupported shape.
int launch_coltile(lp_dtype ta, bool acc_f64, int mode, ColArgs a, int num_sms, cudaStream_t st);
// CG product (MODE_NORMAL, FP32 accumulation, FP32 weight a.d2f) with A staged through shared
// memory by bulk copies (k_cgprod.cu); -1 when the shape or dtype is not covered.
int launch_cgprod(lp_dtype ta, ColArgs a, int num_sms, int max_grid, cudaStream_t st);
int tune_cgprod(lp_dtype ta, ColArgs a, int num_sms, int max_grid, cudaStream_t st, CgTune* out);

// Sparse (CSC) passes
struct CscArgs {
  const int64_t* colptr;
  const int32_t* rowidx;
  const void* vals;
  int m;
  int64_t n;
  const double* v;
  const double* d2;
  const double* x;
  const double* s;
  const double* c;
  const double* sc;
  double* colout;
  void* part;          // [grid][nout][m]
  const int* fl;
  int skip_if_done;
  const double* dz;    // fused CG direction update, as in ColArgs
  const double* dold;
  double* dnew;
};
int launch_csc(lp_dtype tv, bool acc_f64, int mode, CscArgs a, int num_sms, cudaStream_t st);

// sum partials: out[o][i] = sum_b part[b][o][i]; modes below
enum RedMode { RED_PLAIN = 0, RED_MINUS_P = 1, RED_RESID = 2, RED_CG_Q = 3 };
struct RedArgs {
  int mode;
  const void* part;
  int nblk;
  int nout;
  int m;
  bool acc_f64;
  double* out0;        // PLAIN: y; MINUS_P: y - p0; RESID: r_p = Ax - b; CG_Q: q
  double* out1;        // RESID: p = b - A g
  const double* p0;    // MINUS_P: subtrahend; RESID: b
  const double* dvec;  // CG_Q: d (for d^T q)
  double* sc;
  int* fl;
  double* bpart;
  unsigned* bcnt;
  int skip_if_done;
};
cudaError_t launch_reduce(const RedArgs& a, cudaStream_t st);

// n-vector kernels
cudaError_t launch_prep_iterate(const double* x, const double* s, int64_t n, double* d2, double* d,
                                double* sc, double* bpart, unsigned* bcnt, double sigma,
                                const double* c, cudaStream_t st, float* d2f = nullptr,
                                const float* cs2 = nullptr, float2* dfc = nullptr);
cudaError_t launch_d2f(const double* d2, const float* cs2, int64_t n, float* d2f, cudaStream_t st);
cudaError_t launch_norm2(const double* v, int64_t n, double* sc, int slot, double* bpart,
                         unsigned* bcnt, cudaStream_t st);

// sketch
cudaError_t launch_sketch_hash(uint64_t seed, int k, int64_t n, int s, int w, int32_t* hb,
                               int32_t* cnt, int32_t* bucket_out, int8_t* sign_out, cudaStream_t st);
cudaError_t launch_sketch_scan(const int32_t* cnt, int w, int32_t* start, int32_t* cursor,
                               cudaStream_t st);
// (followed by an order of each bucket's members by column index, so G is reproducible)
cudaError_t launch_sketch_scatter(const int32_t* hb, int64_t n, int s, int w, const int32_t* start,
                                  int32_t* cursor, int32_t* list, const double* d, float2* coef,
                                  cudaStream_t st);
cudaError_t launch_sketch_gather_dense(lp_dtype ta, const void* A, int64_t lda, int m, int s,
                                       int w, const int32_t* start, const int32_t* list,
                                       const double* d, double* G, int ldg, cudaStream_t st,
                                       const float2* coef = nullptr);
cudaError_t launch_sketch_gather_csc(lp_dtype tv, const int64_t* colptr, const int32_t* rowidx,
                                     const void* vals, int m, int s, int w, const int32_t* start,
                                     const int32_t* list, const double* d, double* G, int ldg,
                                     cudaStream_t st);

// factor
// Q = G G^T (double-float, split along w); Gdf: 2 ldg w floats of work space (hi, lo of G)
cudaError_t launch_gram(const double* G, float* Gdf, int ldg, int m, int w, int mp, double* Q,
                        double* Qsplit, int split, cudaStream_t st);
cudaError_t launch_gram_df(const float* Gdf, int ldg, int m, int w, int mp, double* Q,
                           double* Qsplit, int split, cudaStream_t st);
cudaError_t launch_split_df(const double* G, size_t count, float* Gdf, cudaStream_t st);
// Gram product on the tensor cores (k_gram_tc.cu): exact splitting of the hi / lo planes of G
// into 8 BF16 digit slices, tcgen05 products accumulated exactly per chunk in TMEM.
cudaError_t launch_gram_tc(const float* Gdf, int ldg, int m, int w, int mp, double* Q,
                           __nv_bfloat16* digits, int* ex, float2* part, int num_sms, int* fl,
                           cudaStream_t st);
size_t gram_tc_digit_bytes(int m, int w);
size_t gram_tc_part_bytes(int m, int mp, int w, int num_sms);
int gram_tc_rows(int m);
// C = A B in double-float: A lower triangular, row-major planes (Ah, Al) with leading
// dimension lda; B[k][j] = (Bh, Bl)[k sbk + j sbj] (b_lower: zero for k < j); C[i][j] written
// at i sci + j scj, and optionally a second copy T at i sti + j stj.  i < M, j < N, k < K.
struct TrmmArgs {
  const float* Ah;
  const float* Al;
  int64_t lda;
  const float* Bh;
  const float* Bl;
  int64_t sbk, sbj;
  int M, N, K;
  int b_lower;
  float* Ch;
  float* Cl;
  int64_t sci, scj;
  float* Th;
  float* Tl;
  int64_t sti, stj;
};
cudaError_t launch_df_trmm(const TrmmArgs& a, cudaStream_t st);
cudaError_t launch_add_shift(double* out, const double* Q, int mp, int m, double eps,
                             const double* v, cudaStream_t st);
// form_m = false skips M = X^T X (the caller forms it, or needs only X).
cudaError_t launch_chol_inverse(double* M, double* X, const double* Q0, int mp, int m, double eps,
                                int* fl, cudaStream_t st, bool form_m = true);
// The same Cholesky sweep as one launch of tile tasks in dependency order (k_factor.cu):
// tasks from chol_dag_tasks (chol_tasks.h, 4 bytes each), sync = chol_dag_sync_words
// zeroed-per-launch words.
constexpr int kDagCtasPerSm = 2;    // CTAs per SM claiming tasks (126 registers a thread: 2 fit)
constexpr int kDagMaxBlocks = 64;   // nbk above this keeps the block-step launches: there the
                                    // sweep is work-bound and the tasks' claims, waits and
                                    // fences cost more than the launches they save (measured:
                                    // m = 1000 1.36 vs 1.57 ms, 2100 tie, 3000 16.2 vs 14.6 ms)
inline size_t chol_dag_sync_words(int nbk) { return 2 + 2 * (size_t)nbk * nbk; }
cudaError_t launch_chol_dag(double* M, double* X, const double* Q0, int mp, int m, double eps,
                            const uint32_t* tasks, int ntasks, int* sync, int num_sms, int* fl,
                            cudaStream_t st, bool form_m = true);
cudaError_t launch_df_to_double(const double* Mdf, int mp, int m, double* out, int ld,
                                cudaStream_t st);
cudaError_t launch_symv_f64(const double* M, int mp, int m, const double* r, double* z,
                            cudaStream_t st);

// CG / preconditioner
cudaError_t launch_symv_dot(const double* M, int mp, int m, const double* r, double* z,
                            double* sc, int* fl, double* bpart, unsigned* bcnt, int mode,
                            cudaStream_t st);
enum SymvMode { SYMV_PLAIN = 0, SYMV_CG_INIT = 1, SYMV_CG_STEP = 2, SYMV_F2 = 3 };
// Arguments of the preconditioner apply z = M r (k_vec.cu).
struct SymvArgs {
  const double* M;
  int mp, m;
  const double* r;
  double* z;
  double* sc;
  int* fl;
  double* bpart;
  unsigned* bcnt;
  int mode;
  double rel2;     // CG relative tolerance squared (CG_INIT)
  // fused residual update (CG_STEP): r = rold - alpha q; CTA 0 stores r and dy += alpha d
  const double* rold;
  const double* q;
  const double* d;
  double* dy;
  const double* qf;    // the product's atomic q copies (q itself holds their sum)
  double* qzero;       // zeroed by CTA 0 for the next CG product
  // factored preconditioner M = X^T X (X = L^{-1}, lower triangular): the first of its two
  // products, t = X r, forms rho = r^T M r as ||t||^2 (sq); the second, z = X^T t, does no
  // bookkeeping and is skipped once the solve has finished (skip_done)
  int sq;
  int skip_done;
};

// One job of a batched preconditioner apply: one context's rows over CTAs [cta0, cta0 + ncta)
// of the launch (8 rows per CTA).
struct SymvJob {
  SymvArgs a;
  int cta0, ncta;
};
cudaError_t launch_symv_batch(const SymvJob* jobs, int njobs, int total_ctas, size_t smem,
                              cudaStream_t st);

// One job of a batched CG product (k_cgprod.cu): one context's CG product over CTAs
// [cta0, cta0 + ncta) of the launch, with S pipeline stages.
struct CgProdJob {
  ColArgs a;
  int S;
  int cta0, ncta;
  int64_t ngroups;
};
// Shape of one job of a batched CG product: group width tc (8 or 2), warps, stages, dynamic
// shared memory; false when the matrix is not covered by the batched kernels (more than 16
// warps of rows).
bool cgprod_job_shape(lp_dtype ta, int m, int lda, int64_t n, int* tc, int* nwarps, int* S,
                      int64_t* ngroups, size_t* smem);
// Launches the batched product over jobs of one (dtype, tc) group; block = nwarps warps.
cudaError_t launch_cgprod_batch(lp_dtype ta, int tc, const CgProdJob* jobs, int njobs,
                                int total_ctas, int nwarps, size_t smem, cudaStream_t st);
// Persistent CG loop (k_cgprod.cu): one cooperative launch runs CG iterations j = 0, 1, ... until
// the device stop flag, iteration j being the CG product prod[j & 1] and the preconditioner
// apply step1[j & 1] (then step2[j & 1] for the two-stage factor), separated by bounded grid
// barriers (bar: 2 + kBarFan zeroed words, see bulk_util.cuh).  The argument sets are those of the serving engine's jobs.
struct CgPersistArgs {
  ColArgs prod[2];
  SymvArgs step1[2], step2[2];
  int factored;
  unsigned* bar;
  int* fl;
  uint64_t wait_ns;    // limit of each wait (0: 1 s)
  int max_trips;       // iterations at most (the stop flag ends the loop before)
};
// Runs the loop for a dense A streamed in FP32/BF16/FP16 with m <= 4096 (rows of the product in
// at most 8 warps, one row of the apply per warp covered by the grid); -1 when not covered or
// the device cannot launch it cooperatively.  Returns the grid size.
int launch_cg_persistent(lp_dtype ta, CgPersistArgs p, int num_sms, cudaStream_t st);

// CG step with the residual update fused: r_new = r_old - alpha q staged by every CTA, stored by
// CTA 0 with dy += alpha d; then z = M r_new, rho = r_new^T z and the CG bookkeeping.
cudaError_t launch_symv_cg_step(const double* M, int mp, int m, const double* rold,
                                const double* q, const double* d, double* dy, double* rnew,
                                double* z, double* sc, int* fl, double* bpart, unsigned* bcnt,
                                cudaStream_t st, const double* qf = nullptr,
                                double* qzero = nullptr);
cudaError_t launch_symv_init(const double* M, int mp, int m, const double* r, double* z,
                             double* sc, int* fl, double* bpart, unsigned* bcnt, double rel_tol,
                             cudaStream_t st);
// Condition of the device-side CG loop: continue while the solve is unfinished and the body
// has run fewer than max_trips times (a CUDA graph WHILE node's handle).
cudaError_t launch_cg_cond(cudaGraphConditionalHandle h, int* fl, int max_trips, cudaStream_t st);
cudaError_t launch_precond_factored(const double* X, const double* XT, int mp, int m, int mode,
                                    const double* r, double* t, double* z, double* sc, int* fl,
                                    double* bpart, unsigned* bcnt, double rel_tol,
                                    cudaStream_t st, const double* rold = nullptr,
                                    const double* q = nullptr, const double* d = nullptr,
                                    double* dy = nullptr, const double* qf = nullptr,
                                    double* qzero = nullptr);
cudaError_t symv_set_smem(int m);
int coltile_max_grid(int num_sms);
int csc_max_grid(int num_sms);
cudaError_t launch_vec_ops(int op, double* a, const double* b, const double* c, int m,
                           const double* sc, cudaStream_t st);
// VOP_SIGNS: a fixed pseudo-random +-1 vector (the factor's quality probe)
enum VecOp { VOP_COPY = 0, VOP_ZERO = 1, VOP_ADD = 2, VOP_SUB = 3, VOP_NEG = 4, VOP_ONES = 5,
             VOP_SIGNS = 6 };

// IPM update
cudaError_t launch_update_dirs(const double* x, const double* s, const double* d2, const double* d,
                               const double* rd, const double* t, const int32_t* hb, int ss,
                               const double* u, int64_t n, double* wu, double* dx, double* ds,
                               int wu_given, double* sc, double* bpart, unsigned* bcnt,
                               cudaStream_t st);
cudaError_t launch_step_length(const double* x, const double* s, const double* dx,
                               const double* ds, int64_t n, double gamma, double* sc,
                               double* bpart, unsigned* bcnt, cudaStream_t st);
cudaError_t launch_apply_step(double* x, double* s, double* y, const double* dx, const double* ds,
                              const double* dy, int64_t n, int m, const double* sc,
                              cudaStream_t st);

// scalars, sketch application, CSR -> CSC, Gram split
cudaError_t launch_set(double* sc, int slot, double v, int* fl, int fslot, int fv, cudaStream_t st);
cudaError_t launch_apply_W(const int32_t* hb, int ss, const double* u, int64_t n, double* wu,
                           cudaStream_t st);
cudaError_t csr_to_csc(const int64_t* indptr, const int32_t* indices, const void* vals,
                       lp_dtype dt, int m, int64_t n, int64_t nnz, int64_t* colptr,
                       int64_t* cursor, int32_t* rowidx, void* cvals, cudaStream_t st);
int gram_split(int m, int w, int num_sms);
int gram_split_cap(int m, int w, int num_sms);

// conversions
cudaError_t launch_convert_dense(const void* src, lp_dtype sdt, bool rowmajor, int m, int64_t n,
                                 void* dst, lp_dtype ddt, int ldd, cudaStream_t st);
// Gaussian sketch G = A D W (dense A, FP32 or FP64) and W u, W from (seed, k) and the quantile
// table gq of 2^kGaussBits entries (k_gauss.cu: CUDA cores; k_sketch_tc.cu: tensor cores)
uint64_t gauss_iteration_key(uint64_t seed, int k);
cudaError_t launch_sketch_gauss(lp_dtype ta, const void* A, int64_t lda, int m, int64_t n, int w,
                                uint64_t seed, int k, const int16_t* gq, const double* d, double* G,
                                int ldg, cudaStream_t st);
cudaError_t launch_apply_W_gauss(uint64_t seed, int k, int64_t n, int w, const int16_t* gq,
                                 const double* u, double* wu, cudaStream_t st);
// work: sketch_tc_work_bytes(m, n, w, num_sms) bytes of device memory, 256-byte aligned
size_t sketch_tc_work_bytes(int m, int64_t n, int w, int num_sms);
cudaError_t launch_sketch_tc(lp_dtype ta, const void* A, int64_t lda, int m, int64_t n, int w,
                             uint64_t key, const double* d, const int16_t* gq, double* G, int ldg,
                             void* work, int num_sms, int* fl, cudaStream_t st);
int occupancy_cached(const void* func, int threads, size_t smem);
// Raises (never lowers) a kernel's dynamic shared-memory limit to at least `bytes`.
cudaError_t ensure_dyn_smem(const void* func, size_t bytes);
cudaError_t launch_convert_colscaled(const void* src, lp_dtype sdt, int lda, int m, int64_t n,
                                     void* dst, lp_dtype ddt, int ldd, float* cs2,
                                     cudaStream_t st);
cudaError_t launch_check_finite(const void* src, lp_dtype dt, int64_t count, int* flag,
                                cudaStream_t st);

}  // namespace lpk
