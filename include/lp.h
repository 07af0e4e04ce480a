/*
 * lp.h -- C ABI of the GB300 (sm_103a) sketch-preconditioned interior-point LP solver.
 *
 * Method: Chowdhury, London, Avron & Drineas, "Speeding up Linear Programming
 * using Randomized Linear Algebra" (arXiv 2003.08072).  The library solves
 * standard-form LPs  min c^T x  s.t.  A x = b, x >= 0  (Sec. 1, primal and
 * dual problems) with m << n by the infeasible long-step IPM of Algorithm 2,
 * whose normal equations A D^2 A^T dy = p (Eq. normal) are solved by the
 * sketch-preconditioned CG of Algorithm 1 plus the correction vector v of
 * Eq. compv.
 *
 * Conventions for every entry point
 *   - Return value: an lp_status; LP_OK on success.  No entry point aborts or
 *     throws.  lp_last_error() returns a message for the calling thread's
 *     most recent failure.
 *   - Dense matrices are column-major unless the layout says otherwise.
 *     Vectors are float64.  Indices are 0-based.
 *   - "device" pointers must be CUDA device (or managed) memory on the
 *     context's device; "host or device" pointers are classified with
 *     cudaPointerGetAttributes.  The caller owns every buffer it passes and
 *     keeps it alive until the call returns (synchronous entry points) or
 *     until the stream passes the enqueued work (entry points marked
 *     "asynchronous").
 *   - All device work of a context is enqueued on the stream given to
 *     lp_create (NULL = the legacy default stream).  A context must not be
 *     used from two threads at once.
 */
#ifndef LP_GB300_H
#define LP_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lp_ctx lp_ctx;

typedef enum {
  LP_OK = 0,
  LP_ERR_ARG = 1,            /* bad argument: size, NULL, NaN/Inf input, unsupported combination */
  LP_ERR_OOM = 2,            /* device or host allocation failed (or over the serving budget) */
  LP_ERR_CUDA = 3,           /* a CUDA runtime call failed (message in lp_last_error) */
  LP_ERR_BREAKDOWN = 4,      /* factorization of the sketch met a non-positive pivot (rank(ADW) < m) */
  LP_ERR_NOT_CONVERGED = 5,  /* iteration cap reached; outputs hold the last iterate */
  LP_ERR_TIMEOUT = 6,        /* a bounded device-side wait gave up */
  LP_ERR_NUMERIC = 7         /* NaN/Inf appeared in the iteration */
} lp_status;

typedef enum {
  LP_DENSE_COLMAJOR = 0,     /* A_vals is m x n, element (i, j) at i + j*m */
  LP_DENSE_ROWMAJOR = 1,     /* A_vals is m x n, element (i, j) at i*n + j */
  LP_CSR = 2                 /* indptr (m+1, int64), indices (nnz, int32 column ids), A_vals (nnz) */
} lp_layout;

typedef enum { LP_F64 = 0, LP_F32 = 1, LP_BF16 = 2, LP_F16 = 3 } lp_dtype;

typedef enum { LP_INNER_CG = 0, LP_INNER_RICHARDSON = 1 } lp_inner_solver;

typedef enum { LP_SKETCH_SPARSE = 0, LP_SKETCH_GAUSSIAN = 1 } lp_sketch_kind;

/* Parameters of Algorithms 1 and 2.  Defaults from lp_params_default(). */
typedef struct {
  double tol;            /* stop when ||r_p||/(1+||b||), ||r_d||/(1+||c||), n mu/(1+|c^T x|) <= tol (1e-8) */
  double cg_rel_tol;     /* CG stops when ||f^(j)|| <= cg_rel_tol ||f^(0)|| (1e-6), Sec. 6 "tolCG" */
  double sigma;          /* centering parameter in (0, 4/5), Alg. 2 input (0.5, Sec. 6) */
  double gamma;          /* neighbourhood N(gamma) width in (0, 1), Sec. 4 (0.99) */
  int32_t cg_max_iter;   /* CG iteration cap per solve (500) */
  int32_t ipm_max_iter;  /* IPM iteration cap (200) */
  int32_t refine_max;    /* FP64 refinement steps for Q^{-1} r~ and for a low-precision dy (6) */
  int32_t sketch_s;      /* nonzeros per row of W: 1 = CountSketch, 4 = sparse sign (4); unused by the
                            Gaussian sketch */
  int32_t sketch_w;      /* sketch width w; 0 = 4m.  Must be a multiple of sketch_s */
  int32_t cg_theory_rule;/* 1: CG also stops only once ||f|| <= gamma sigma sqrt(mu)/(4 sqrt(n)) (Sec. 4) (1) */
  uint64_t seed;         /* W for IPM iteration k is a function of (seed, k) only (0) */
  lp_dtype stream_dtype; /* dtype A is streamed in by the CG matvec; LP_F64 keeps the input dtype (LP_F64).
                            Dense LP_BF16 / LP_F16 copies hold column j scaled by a power of two 2^-e_j
                            (max |entry| in [0.5, 1)), the scales folded into D^2.  A copy below the
                            input precision is corrected by FP64 refinement; when a refinement pass
                            fails to halve ||f|| (or refine_max passes run) the solve streams the
                            input-precision copy from then on (lp_info.stream_switch_iter). */
  int32_t cg_batch;      /* CG iterations enqueued between host checks of the stop flag (4) */
  int32_t inner_solver;  /* LP_INNER_CG (0): Alg. 1 step 3; LP_INNER_RICHARDSON (1): the preconditioned
                            Richardson iteration of App. A (dy += Q^{-1}(p - A D^2 A^T dy)), same stop
                            rule; it converges only when ||I - Q^{-1/2} A D^2 A^T Q^{-1/2}|| < 1, i.e.
                            for a sketch much wider than 4m, and a diverging run ends the solve with
                            LP_ERR_NOT_CONVERGED (0) */
  int32_t sketch_kind;   /* LP_SKETCH_SPARSE (0): sketch_s nonzeros +-1/sqrt(s) per row of W (Sec. 2);
                            LP_SKETCH_GAUSSIAN (1): W with N(0, 1/w) entries (Sec. 5, the sketch of the
                            experiments, Sec. 6), dense A only: entry (i, b) is q_j / (2^8 sqrt(w)),
                            q_j = round(2^8 Phi^{-1}((j + 1/2) 2^-14)) for the cell j = h >> 50 of the
                            hash h = SplitMix64(key_k ^ (i w + b)) (normal quantiles on a 2^-8 grid);
                            forming A D W costs 2 m n w (tensor cores: gram_tensor_cores) (0) */
  int32_t use_graphs;    /* 1: after a context's first CG solve, each CG solve runs as one CUDA graph
                            launch whose WHILE node repeats the CG iteration on the device until the
                            stop rule holds (no host round trip per cg_batch); 0: every CG iteration
                            is enqueued by the host and the stop flag read every cg_batch
                            iterations.  Profiling (lp_profile_enable) runs the host-driven loop (1) */
  int32_t gram_tensor_cores; /* 1: the Gram product Q = (A D W)(A D W)^T of the factor runs on the tensor
                            cores (tcgen05), made exact by splitting each row of the sketch into nine
                            BF16 digit slices of 6 bits (each entry accurate to ~2^-52 sqrt(w)
                            |G_i| |G_j|, finer than the double-float product), and so does the
                            Gaussian sketch A D W (rows of A D in nine digit slices, W's grid values
                            in two; extra device memory ~(18 m + 4 w) n bytes); 0: double-float
                            products on the FP32 pipes (1) */
  int32_t autotune;      /* 1: lp_create times the CG product's launch shapes (group width, pipeline
                            stages, CTAs per SM) on the matrix itself (A of 64 MB and more; a few ms,
                            kept per shape for the process) and keeps the fastest; 0: fixed rule (1) */
  int32_t shared_cg;     /* serving loop only (read by lp_server_create): 1 = the live instances' CG
                            iterations share launches through the server's batch engine; 0 = each
                            instance runs its own CG loop (one CUDA graph launch per CG solve, the
                            instances overlapping on their own streams) (0) */
  int32_t persistent_cg; /* 1 = the CG loop over a dense A streamed below FP64 (m <= 4096) runs as
                            one cooperative launch per CG solve, products and preconditioner applies
                            separated by bounded grid barriers; 0 = CUDA graph (use_graphs) or host
                            loop.  Measured on GB300 no faster than the graph launches (slower for
                            m <= 300: the kernel holds both phases' registers, so fewer CTAs stream
                            the product).  A serving loop with max_live > 1 sets it to 0 (0) */
  int32_t factor_dag;    /* 1: the blocked Cholesky sweep of the factor (Alg. 1 step 2) runs as one
                            launch whose CTAs claim its 32 x 32 tile products in dependency order,
                            waiting on per-tile counters (bounded waits: LP_ERR_TIMEOUT), so that only
                            the diagonal blocks' pivot chains are sequential; same arithmetic, bitwise
                            the same factor as 0: two launches per block step.  m above 2048 always
                            takes the block-step launches (there the sweep is bound by work, and
                            the launch's task claims and waits cost more than the launches they
                            save), and so does a serving loop with
                            max_live > 1 (its waiting CTAs would hold SMs from the other live
                            instances) (1) */
} lp_params;

/* Per-solve report.  Filled on success and on LP_ERR_NOT_CONVERGED. */
typedef struct {
  int32_t ipm_iters;       /* outer iterations taken */
  int32_t cg_iters_total;  /* products with A D^2 A^T over all CG solves */
  int32_t cg_iters_last;   /* CG iterations of the last normal-equation solve */
  int32_t refine_steps;    /* FP64 refinement steps of the last solve */
  double rp_rel, rd_rel, gap_rel;   /* scaled residuals of the stopping rule at exit */
  double mu;               /* duality measure x^T s / n at exit */
  double obj;              /* c^T x at exit */
  double alpha_max, alpha; /* step-length quantities of the last iteration (Alg. 2 (e), (f)) */
  double f_norm;           /* ||f^(t)|| of the last CG solve (Sec. 3) */
  double v_norm;           /* ||v|| of the last correction vector (Eq. compv) */
  int32_t status;          /* lp_status of the solve */
  double f_target;         /* CG target of the last solve: min(cg_rel_tol ||f^(0)||, gamma sigma sqrt(mu)/(4 sqrt(n))) */
  int32_t stream_dtype;    /* lp_dtype the CG products streamed A in at exit (see lp_params.stream_dtype) */
  int32_t stream_switch_iter; /* IPM iteration at which the solve switched to the master copy; -1 if never */
  int32_t factor_two_stage;   /* normal solves whose factor needed the second stage (Q numerically
                                 singular for the one-stage inverse; see lp_factor) */
  int32_t cg_precise_iter;    /* IPM iteration from which the CG products accumulated in FP64-class
                                 arithmetic over the master copy, because FP64 refinement of FP32
                                 products stopped contracting on the master copy itself; -1 if never */
  int32_t cg_graph_solves;    /* CG solves of this call that ran as one CUDA graph launch each
                                 (lp_params.use_graphs) */
  int32_t cg_persistent_solves; /* CG solves of this call that ran as one persistent cooperative
                                   launch each (lp_params.persistent_cg) */
} lp_info;

/* Fills *prm with the defaults listed above.  LP_ERR_ARG if prm is NULL. */
lp_status lp_params_default(lp_params* prm);

/* Human-readable name of a status code (static string). */
const char* lp_status_str(lp_status st);

/* Message describing the calling thread's most recent error ("" if none). */
const char* lp_last_error(void);

/*
 * lp_create -- copy an LP instance (Eq. primal: A, b, c) to the device.
 *   out      : receives the new context (set to NULL on failure).
 *   m, n     : constraint and variable counts, 1 <= m <= n, m <= 8192.
 *   layout   : LP_DENSE_COLMAJOR / LP_DENSE_ROWMAJOR / LP_CSR.
 *   a_dtype  : element type of A_vals: LP_F64 or LP_F32 (dense); LP_F32 or LP_F64 (CSR).
 *   A_vals   : host or device; dense m*n elements, or nnz CSR values.
 *   indptr   : CSR only (m+1 int64, host or device); NULL for dense.
 *   indices  : CSR only (nnz int32 column ids, host or device); NULL for dense.
 *   nnz      : CSR only; 0 for dense.
 *   b, c     : host or device, m and n float64.
 *   prm      : parameters (copied); NULL = defaults.
 *   stream   : cudaStream_t all work is enqueued on (NULL = legacy default).
 * The context owns all device memory it allocates: the matrix in the layout
 * the kernels stream (column-major with 16-byte aligned columns, or CSC),
 * a low-precision copy when prm->stream_dtype asks for one, and the
 * workspaces (lp_footprint_bytes bounds the total).  The memory comes from the
 * device's default stream-ordered pool (cudaMallocAsync on `stream`); the
 * library raises that pool's release threshold so that memory freed by
 * lp_destroy stays cached in the process for the next context.
 * Errors: LP_ERR_ARG (sizes, NULL, non-finite entries, dtype, the Gaussian
 * sketch with CSR), LP_ERR_OOM, LP_ERR_CUDA.  Synchronous.
 */
lp_status lp_create(lp_ctx** out, int32_t m, int64_t n, lp_layout layout, lp_dtype a_dtype,
                    const void* A_vals, const int64_t* indptr, const int32_t* indices, int64_t nnz,
                    const double* b, const double* c, const lp_params* prm, void* stream);

/* Frees every device buffer of the context.  NULL is a no-op. */
void lp_destroy(lp_ctx* ctx);

/* Replaces the context's parameters (takes effect on the next call). */
lp_status lp_set_params(lp_ctx* ctx, const lp_params* prm);

/*
 * lp_ipm_solve -- Algorithm 2 end to end (Sec. 4).
 *   x, y, s : host or device, n, m, n float64.  On entry the starting point
 *             when start_given != 0, else ignored and the start is x = s = 1,
 *             y = 0 (Sec. 6 starts from all ones).  On exit the last iterate.
 *   info    : may be NULL.
 * Per iteration k: residuals and p (Eq. pdef), W = W(seed, k) (step (a)),
 * Algorithm 1 for dy, v from Eq. compv, ds from Eq. delshat, dx from
 * Eq. delxhat, alpha_max / alpha (steps (e), (f)), update (step (g)).
 * Returns LP_OK when the scaled stopping rule holds, LP_ERR_NOT_CONVERGED at
 * the iteration cap, LP_ERR_BREAKDOWN / LP_ERR_NUMERIC on failure (with the
 * last finite iterate in x, y, s).  Synchronous.
 */
lp_status lp_ipm_solve(lp_ctx* ctx, double* x, double* y, double* s, int32_t start_given,
                       lp_info* info);

/*
 * Checkpoint / resume of Algorithm 2.  Besides the iterate (x, y, s), a run carries its
 * iteration counter k (iteration k draws W = W(seed, k), step (a)) and the references of the
 * neighbourhood N(gamma) fixed at its start point (Sec. 4: ||r^k|| / ||r^0|| <= mu_k / mu_0),
 * plus the iteration at which the CG products switched to the master copy of A.  With these a
 * solve stopped at the iteration cap (LP_ERR_NOT_CONVERGED) or saved to storage continues as
 * if it had not stopped: same W stream, same neighbourhood, same stream dtype.
 */
typedef struct {
  int32_t k;                  /* IPM iterations taken since the start point */
  int32_t stream_switch_iter; /* iteration of the switch to the master copy of A; -1 if none */
  double r0;                  /* ||(r_p, r_d)|| at the start point */
  double mu0;                 /* x^T s / n at the start point */
} lp_ipm_state;

/* State at the end of the last lp_ipm_solve / lp_ipm_resume on ctx (k = 0 and r0 = mu0 = 0
 * before the first).  LP_ERR_ARG for NULL arguments. */
lp_status lp_ipm_get_state(lp_ctx* ctx, lp_ipm_state* state);

/*
 * lp_ipm_resume -- lp_ipm_solve continued from a checkpoint (any context holding the same
 * A, b, c and seed, e.g. a new process).
 *   x, y, s : host or device, n, m, n float64; on entry the iterate saved with *state
 *             (x, s > 0), on exit the last iterate.
 *   state   : from lp_ipm_get_state after the run being continued; k >= 0, r0 >= 0, mu0 > 0.
 * ipm_max_iter caps the total count k, so raise it (lp_set_params) to continue a run that
 * stopped at the cap.  info->ipm_iters is the total count; the CG counts are this call's.
 * Errors as lp_ipm_solve, plus LP_ERR_ARG for a state out of range.  Synchronous.
 */
lp_status lp_ipm_resume(lp_ctx* ctx, double* x, double* y, double* s, const lp_ipm_state* state,
                        lp_info* info);

/*
 * lp_normal_solve -- Algorithm 1 plus the correction of Eq. compv for one iterate.
 *   x, s    : device, n float64, strictly positive; D^2 = X S^{-1} (Sec. 1).
 *   p       : device, m float64 right-hand side.
 *   k       : IPM iteration index selecting W = W(seed, k) (Alg. 2 step (a)).
 *   dy      : device, m float64 output: the CG solution dy-hat = Q^{-1/2} z^t.
 *   rtil    : device, m float64 output or NULL: r~ = A D^2 A^T dy - p (FP64).
 *   u       : device, w float64 output or NULL: u = (A D W)^dagger r~.
 *   Wu      : device, n float64 output or NULL: W u, so that S^{-1} v = D W u.
 *   Atdy    : device, n float64 output or NULL: A^T dy (FP64).
 *   info    : may be NULL; receives cg_iters_last, refine_steps, f_norm.
 * Errors: LP_ERR_ARG, LP_ERR_BREAKDOWN (rank-deficient sketch), LP_ERR_NUMERIC,
 * LP_ERR_CUDA.  Synchronous.
 */
lp_status lp_normal_solve(lp_ctx* ctx, const double* x, const double* s, const double* p,
                          int32_t k, double* dy, double* rtil, double* u, double* Wu,
                          double* Atdy, lp_info* info);

/* ---------------- row-level entry points (one step of the hot path each) ---------------- */

/*
 * lp_residuals -- Alg. 2 step (b) in one pass over A:
 *   r_p = A x - b, r_d = A^T y + s - c, mu = x^T s / n (Eq. update) and
 *   p = -r_p - sigma mu A S^{-1} 1 + A x - A D^2 r_d (Eq. pdef), computed as
 *   p = b - A(sigma mu / s + d^2 r_d).
 *   x, y, s : device (n, m, n).  rp, p: device m outputs.  rd: device n output.
 *   mu_out  : host double output (may be NULL).  Synchronous.
 */
lp_status lp_residuals(lp_ctx* ctx, const double* x, const double* y, const double* s,
                       double sigma, double* rp, double* rd, double* p, double* mu_out);

/*
 * lp_sketch_indices -- the buckets and signs of W for iteration k (Sec. 2, Eq. pdprec):
 *   key = SplitMix64(seed ^ SplitMix64(k)); h = SplitMix64(key ^ (i*s + j));
 *   bucket = j*(w/s) + (((h >> 32) * (w/s)) >> 32); sign = (h & 1) ? -1 : +1.
 *   bucket : device int32 output, n*s (row i, nonzero j at i*s + j).
 *   sign   : device int8 output, n*s (+1 / -1).
 *   stream : cudaStream_t.  Asynchronous.  LP_ERR_ARG if w % s != 0 or sizes invalid.
 */
lp_status lp_sketch_indices(uint64_t seed, int32_t k, int64_t n, int32_t s, int32_t w,
                            int32_t* bucket, int8_t* sign, void* stream);

/*
 * lp_sketch -- A D W (m x w, Eq. pdprecond; Alg. 1 step 1) for W = W(seed, k).
 *   d  : device n float64, the diagonal of D = (X S^{-1})^{1/2}.
 *   G  : device m*w float64 output, column-major (leading dimension m).
 * FP64 accumulation from the input-precision A.  Synchronous.
 */
lp_status lp_sketch(lp_ctx* ctx, const double* d, int32_t k, double* G);

/*
 * lp_factor -- preconditioner of Alg. 1 step 2 from the sketch G = A D W:
 *   Q = G G^T (Eq. pdprecond) and Minv = Q^{-1}, so that PCG with M = Q gives the
 *   iterates of CG on Eq. precond_alt.
 *   G    : device m*w float64, column-major.
 *   Q    : device m*m float64 output or NULL (symmetric).
 *   Minv : device m*m float64 output or NULL (symmetric).
 * LP_ERR_BREAKDOWN if a pivot is not positive (rank(G) < m).  Synchronous.
 * Inside lp_ipm_solve and lp_normal_solve, a Q that is numerically singular for this explicit
 * inverse (a lost pivot, or ||Q Minv z - z|| / sqrt(m) >= 1e-2 for a fixed +-1 probe z; CountSketch reaches
 * kappa(Q) ~ 1e17 late in the IPM) is factored in two stages instead: a shifted Cholesky
 * factor L1 of Q whitens G into G1 = L1^{-1} G, a second Cholesky factor L2 of G1 G1^T
 * follows, and the preconditioner is applied as X^T (X r) with X = L2^{-1} L1^{-1}, whose
 * error grows with kappa(G) rather than kappa(Q) = kappa(G)^2 (lp_info.factor_two_stage).
 */
lp_status lp_factor(lp_ctx* ctx, const double* G, double* Q, double* Minv);

/*
 * lp_normal_matvec -- y = A D^2 A^T v (the operator of Eq. normal), one pass over A.
 *   d2     : device n float64 (D^2).  v: device m float64.  y: device m float64 output.
 *   t      : device n float64 output or NULL: t = A^T v.
 *   stream_dtype : LP_F64 = input precision with FP64 accumulation; LP_F32 /
 *            LP_BF16 / LP_F16 = the context's streamed copy with FP32 accumulation
 *            (must match the context's stream_dtype unless LP_F64).
 * Synchronous.
 */
lp_status lp_normal_matvec(lp_ctx* ctx, const double* d2, const double* v, double* y, double* t,
                           lp_dtype stream_dtype);

/*
 * lp_step -- Alg. 2 steps (d)-(g) for a given dy (fused IPM update, Sec. 4):
 *   ds = -r_d - A^T dy (Eq. delshat); S^{-1} v = D (W u) (Eq. compv);
 *   dx = -x + sigma mu S^{-1} 1 - D^2 ds - S^{-1} v (Eq. delxhat);
 *   alpha_max keeps [0, alpha] inside N(gamma) (step (e)); alpha minimises
 *   mu(alpha) on [0, alpha_max] (step (f)); then x += alpha dx, y += alpha dy,
 *   s += alpha ds (step (g)).
 *   x, y, s : device, updated in place.   rd, Atdy, Wu: device n float64.
 *   dy      : device m.   mu: current x^T s / n.   eta = ||r||/||r^0||.  mu0 = x0^T s0 / n.
 *   dx, ds  : device n float64 outputs or NULL (the directions).
 *   out     : host double[4] output or NULL: {alpha_max, alpha, x^T ds + s^T dx, dx^T ds}.
 * Synchronous.
 */
lp_status lp_step(lp_ctx* ctx, double* x, double* y, double* s, const double* rd,
                  const double* dy, const double* Atdy, const double* Wu, double mu, double eta,
                  double mu0, double* dx, double* ds, double* out);

/*
 * lp_normal_matvec_noalloc -- y = A D^2 A^T v (and t = A^T v) without a context and without
 * allocating any device memory.  The paper has no counterpart: this entry point exists for
 * callers that must not allocate, e.g. code running under a framework that owns every byte
 * of device memory through its own pool, or a latency-critical loop that cannot afford the
 * implicit device synchronisation of cudaMalloc / cudaFree.  The caller passes inputs and
 * outputs; the per-CTA partial sums live in one 4 MiB file-scope __device__ array of the
 * library, which every GPU that loads the library holds until the process exits.
 *   A      : device, column-major m x n with leading dimension lda (lda >= m), 16-byte aligned,
 *            lda * element size a multiple of 16 bytes.  The padding rows m..lda-1 are never
 *            used (they may hold anything, NaN included).
 *   a_dtype: LP_F64 (FP64 accumulation) or LP_F32 / LP_BF16 / LP_F16 (FP32 accumulation).
 *   d2     : device n float64 (D^2).   v: device m float64.   y: device m float64 output.
 *   t      : device n float64 output or NULL.
 *   stream : cudaStream_t the two kernels are enqueued on.  Asynchronous.
 * Limit: m <= min(8192, 4 MiB / (accumulator bytes x SM count)), i.e. m <= 3449 for LP_F64 and
 * m <= 6898 otherwise on a 152-SM GB300; larger m returns LP_ERR_ARG with the limit in
 * lp_last_error().  Each call made outside a stream capture looks up the array's device
 * address (with the device current, so a device reset is harmless); a call during a capture
 * reuses the address of the last call on that device, so make the first call on each device
 * before any stream capture (else LP_ERR_ARG).  All calls share the
 * one array and each overwrites it completely, so calls whose kernels overlap on the GPU (two
 * streams, two threads) race and must be serialised by the caller.
 */
lp_status lp_normal_matvec_noalloc(const void* A, lp_dtype a_dtype, int32_t m, int64_t n,
                                   int64_t lda, const double* d2, const double* v, double* y,
                                   double* t, void* stream);

/* ---------------- measurement (not part of the method) ---------------- */

/* Phases timed by lp_profile_read. */
enum {
  LP_PH_RESIDUALS = 0,   /* Alg. 2 step (b): residual pass and p */
  LP_PH_SKETCH = 1,      /* A D W */
  LP_PH_FACTOR = 2,      /* Q and Q^{-1} */
  LP_PH_PCG = 3,         /* CG iterations on A D^2 A^T (all kernels) */
  LP_PH_RTILDE = 4,      /* FP64 residual passes r~ = A D^2 A^T dy - p */
  LP_PH_CORRECTION = 5,  /* u = (A D W)^dagger r~ */
  LP_PH_UPDATE = 6,      /* directions, step length, update */
  LP_PH_COUNT = 8
};

typedef struct {
  double phase_ms[LP_PH_COUNT];     /* device time per phase: CUDA events on the context stream */
  int64_t phase_calls[LP_PH_COUNT];
  double matvec_ms;                 /* summed duration of the CG product kernels that did work */
  int64_t matvec_count;             /* number of those launches */
  double matvec_bytes;              /* algorithmic bytes of one CG product (read of A, D^2, v) */
  int64_t launches;                 /* kernel launches issued by the library since load (all contexts) */
  int32_t tune_tc, tune_stages, tune_ctas; /* autotuned CG product shape for the copy streamed now
                                              (columns per copy, stages, CTAs per SM); 0: the fixed
                                              rule (not tuned, or no candidate beat it) */
  double tune_us, tune_rule_us;     /* measured time per product of the shape in use and of the
                                       fixed rule (0 when the copy was not tuned) */
} lp_profile;

/*
 * lp_profile_enable -- on != 0 records CUDA events around each phase and around every CG
 * product kernel of this context (adds a few microseconds per event pair); 0 stops recording.
 */
lp_status lp_profile_enable(lp_ctx* ctx, int32_t on);

/* lp_profile_read -- copies the accumulated profile into *out (host); reset != 0 zeroes it. */
lp_status lp_profile_read(lp_ctx* ctx, lp_profile* out, int32_t reset);

/*
 * lp_test_stall_copy -- failure-detection test hook (not part of the method).  The next CG
 * product of this context that stages A through shared memory (a dense context streaming A
 * below FP64) is launched with every bounded device-side wait limited to wait_ns nanoseconds
 * (1 <= wait_ns <= 1e9; the normal limit is 1 s), and its first CTA never issues the bulk copy
 * of its local column group `group` (0-based).  The wait for that copy then runs out, the
 * kernel lets the copies it did issue land, returns without touching memory outside its
 * buffers, and the call that ran the product (lp_normal_matvec, lp_normal_solve,
 * lp_ipm_solve) returns LP_ERR_TIMEOUT with its outputs undefined; the context stays usable
 * and later calls run normally.  No GPU fault is involved.  The hook is consumed by that one
 * product; a group beyond the first CTA's share of columns injects nothing.
 * LP_ERR_ARG for a NULL context, group < 0 or wait_ns outside the range.
 */
lp_status lp_test_stall_copy(lp_ctx* ctx, int32_t group, uint64_t wait_ns);

/* ---------------- memory footprint and the serving loop ---------------- */

/*
 * lp_footprint_bytes -- upper bound on the device bytes lp_create allocates for an instance of
 * this shape (matrix copies, sketch, factor, workspaces), for admission control.  Pure host
 * computation (no device call); num_sms <= 0 means 152.  Returns 0 for invalid sizes.
 */
uint64_t lp_footprint_bytes(int32_t m, int64_t n, lp_layout layout, lp_dtype a_dtype, int64_t nnz,
                            const lp_params* prm, int32_t num_sms);

/*
 * Serving: LP instances submitted one by one are solved with continuous batching.  max_live
 * worker threads each own a CUDA stream; a free worker admits the oldest queued request as soon
 * as its lp_footprint_bytes fits into the part of mem_budget_bytes not held by live requests,
 * solves it with lp_create + lp_ipm_solve (Algorithm 2, parameters prm) and releases the memory.
 * Live instances run concurrently on the GPU.  Admission is first come, first served.
 * With prm->shared_cg and max_live > 1 the CG iterations of the live instances share
 * launches: an instance whose solve reaches a CG loop over a dense A streamed below FP64 hands
 * the loop to the server's batch engine, which advances every such loop by one iteration per
 * round with one batched product launch and one batched preconditioner launch over a
 * per-instance work table (each instance keeps its own scalars and stop rule; results are
 * those of the instance solved alone up to the order of floating-point sums).
 * All buffers passed to the server are HOST memory; submit copies them, so the caller may
 * reuse its buffers as soon as lp_server_submit returns.  One server per device; the device is
 * the calling thread's current one at creation.  A server may be used from several threads.
 */
typedef struct lp_server lp_server;

typedef struct {
  int64_t submitted, completed, failed;   /* counts since creation (failed: status != LP_OK) */
  int64_t queued, live, peak_live;        /* waiting, being solved, most solved at once */
  uint64_t mem_in_use, mem_peak, mem_budget;  /* admitted footprints (bytes) */
  int64_t batched_rounds;    /* rounds of shared CG launches run (one CG iteration of every
                                live instance's CG solve per round) */
  int64_t batched_cg_solves; /* CG solves that ran in shared launches */
} lp_server_stats_t;

/* Errors: LP_ERR_ARG (max_live outside 1..256, zero budget), LP_ERR_CUDA (no device). */
lp_status lp_server_create(lp_server** out, uint64_t mem_budget_bytes, int32_t max_live,
                           const lp_params* prm);

/* Queues one instance (arguments as lp_create, host memory only); *ticket identifies it.
 * Errors: LP_ERR_ARG, LP_ERR_OOM (the instance alone exceeds the budget). */
lp_status lp_server_submit(lp_server* srv, int32_t m, int64_t n, lp_layout layout,
                           lp_dtype a_dtype, const void* A_vals, const int64_t* indptr,
                           const int32_t* indices, int64_t nnz, const double* b, const double* c,
                           int64_t* ticket);

/* Waits up to timeout_ms for a finished request not yet handed out and returns its ticket
 * (completion order).  LP_ERR_TIMEOUT if none finished in time. */
lp_status lp_server_wait_any(lp_server* srv, int32_t timeout_ms, int64_t* ticket);

/* Result of a finished request: x, y, s (host, n / m / n float64, each may be NULL), the
 * lp_info of its solve, and times[3] (may be NULL) = seconds queued, seconds being solved,
 * latency from submission to completion.  Releases the ticket.  Returns the solve's status
 * (its message in lp_last_error), or LP_ERR_ARG for an unknown or unfinished ticket. */
lp_status lp_server_result(lp_server* srv, int64_t ticket, double* x, double* y, double* s,
                           lp_info* info, double* times);

lp_status lp_server_stats(lp_server* srv, lp_server_stats_t* out);

/* Drops queued requests, waits for live ones, frees the server.  NULL is a no-op. */
void lp_server_destroy(lp_server* srv);

#ifdef __cplusplus
}
#endif

#endif /* LP_GB300_H */
