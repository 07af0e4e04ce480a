// Vector kernels: reduction of per-CTA partials, CG scalar steps, preconditioner apply,
// and the fused IPM update (Alg. 2 steps (d)-(g)).  All vectors and scalars are FP64.
#include <math.h>

#include "dev_util.cuh"
#include "symv_body.cuh"

namespace lpk {

// ------------------------------------------------------------------------------------
// Partials [nblk][nout][m] -> m-vectors.  32 rows x 8 block groups per CTA.
// ------------------------------------------------------------------------------------
template <typename ACC>
__global__ void __launch_bounds__(1024) k_reduce(RedArgs a) {
  if (a.skip_if_done && a.fl[FL_DONE]) return;
  // 32 rows x 32 block groups per CTA: each thread sums every 32nd partial of one row
  __shared__ double sh[2][32][33];
  const int rl = threadIdx.x & 31, g = threadIdx.x >> 5;
  const int row = blockIdx.x * 32 + rl;
  const ACC* part = reinterpret_cast<const ACC*>(a.part);
  double s0 = 0.0, s1 = 0.0;
  if (row < a.m) {
    for (int b = g; b < a.nblk; b += 32) {
      s0 += (double)part[((size_t)b * a.nout) * a.m + row];
      if (a.nout > 1) s1 += (double)part[((size_t)b * a.nout + 1) * a.m + row];
    }
  }
  sh[0][g][rl] = s0;
  sh[1][g][rl] = s1;
  __syncthreads();
  double contrib[2] = {0.0, 0.0};
  if (g == 0) {
    double t0 = 0.0, t1 = 0.0;
#pragma unroll 8
    for (int k = 0; k < 32; ++k) {
      t0 += sh[0][k][rl];
      t1 += sh[1][k][rl];
    }
    if (row < a.m) {
      switch (a.mode) {
        case RED_PLAIN: a.out0[row] = t0; break;
        case RED_MINUS_P: a.out0[row] = t0 - a.p0[row]; break;
        case RED_RESID: {
          const double rp = t0 - a.p0[row];
          a.out0[row] = rp;
          a.out1[row] = a.p0[row] - t1;
          contrib[0] = rp * rp;
          break;
        }
        case RED_CG_Q: {
          a.out0[row] = t0;
          contrib[0] = a.dvec[row] * t0;
          break;
        }
      }
    }
  }
  if (a.mode == RED_RESID || a.mode == RED_CG_Q) {
    double v[1] = {contrib[0]};
    if (grid_sum_last<1>(v, a.bpart, a.bcnt) && threadIdx.x == 0) {
      if (a.mode == RED_RESID) {
        a.sc[SC_RP2] = v[0];
      } else {
        set_cg_alpha(v[0], a.sc, a.fl);
      }
    }
  }
}

cudaError_t launch_reduce(const RedArgs& a, cudaStream_t st) {
  const int grid = (a.m + 31) / 32;
  if (a.acc_f64)
    { note_launch(); k_reduce<double><<<grid, 1024, 0, st>>>(a); }
  else
    { note_launch(); k_reduce<float><<<grid, 1024, 0, st>>>(a); }
  return cudaGetLastError();
}

// ------------------------------------------------------------------------------------
// Iterate preparation: d2 = x/s, d = sqrt(d2); x^T s, c^T x -> mu, sigma mu.  With dfc, also
// the double-float pairs of d2, x, 1/s and s - c (four arrays of n) that the FP64-class
// column passes take their per-column scalars from.
// ------------------------------------------------------------------------------------
__global__ void k_prep(const double* __restrict__ x, const double* __restrict__ s, int64_t n,
                       double* __restrict__ d2, double* __restrict__ d, double* sc, double* bpart,
                       unsigned* bcnt, double sigma, const double* __restrict__ c,
                       float* __restrict__ d2f, const float* __restrict__ cs2,
                       float2* __restrict__ dfc) {
  double v[2] = {0.0, 0.0};
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double xi = x[i], si = s[i];
    const double q = xi / si;
    d2[i] = q;
    d[i] = sqrt(q);
    if (d2f) d2f[i] = (float)(cs2 ? q * (double)cs2[i] : q);
    if (dfc) {
      float h, l;
      split_double_bits(q, h, l);
      dfc[i] = make_float2(h, l);
      split_double_bits(xi, h, l);
      dfc[n + i] = make_float2(h, l);
      split_double_bits(1.0 / si, h, l);
      dfc[2 * n + i] = make_float2(h, l);
      split_double_bits(si - c[i], h, l);
      dfc[3 * n + i] = make_float2(h, l);
    }
    v[0] += xi * si;
    v[1] += c[i] * xi;
  }
  if (grid_sum_last<2>(v, bpart, bcnt) && threadIdx.x == 0) {
    sc[SC_XS] = v[0];
    sc[SC_MU] = v[0] / (double)n;
    sc[SC_SIGMU] = sigma * v[0] / (double)n;
    sc[SC_CX] = v[1];
  }
}

static int vec_grid(int64_t n) {
  int64_t g = (n + 255) / 256;
  if (g > 1024) g = 1024;
  if (g < 1) g = 1;
  return (int)g;
}

cudaError_t launch_prep_iterate(const double* x, const double* s, int64_t n, double* d2, double* d,
                                double* sc, double* bpart, unsigned* bcnt, double sigma,
                                const double* c, cudaStream_t st, float* d2f, const float* cs2,
                                float2* dfc) {
  { note_launch(); k_prep<<<vec_grid(n), 256, 0, st>>>(x, s, n, d2, d, sc, bpart, bcnt, sigma, c, d2f, cs2, dfc); }
  return cudaGetLastError();
}

// FP32 weight of the streamed product: d2f = d2 (times the copy's column scales cs2, if any).
__global__ void k_d2f(const double* __restrict__ d2, const float* __restrict__ cs2, int64_t n,
                      float* __restrict__ d2f) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    d2f[i] = (float)(cs2 ? d2[i] * (double)cs2[i] : d2[i]);
}

cudaError_t launch_d2f(const double* d2, const float* cs2, int64_t n, float* d2f, cudaStream_t st) {
  { note_launch(); k_d2f<<<vec_grid(n), 256, 0, st>>>(d2, cs2, n, d2f); }
  return cudaGetLastError();
}

__global__ void k_norm2(const double* __restrict__ v, int64_t n, double* sc, int slot,
                        double* bpart, unsigned* bcnt) {
  double a[1] = {0.0};
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    a[0] += v[i] * v[i];
  if (grid_sum_last<1>(a, bpart, bcnt) && threadIdx.x == 0) sc[slot] = a[0];
}

cudaError_t launch_norm2(const double* v, int64_t n, double* sc, int slot, double* bpart,
                         unsigned* bcnt, cudaStream_t st) {
  { note_launch(); k_norm2<<<vec_grid(n), 256, 0, st>>>(v, n, sc, slot, bpart, bcnt); }
  return cudaGetLastError();
}

// ------------------------------------------------------------------------------------
// Preconditioner apply z = M r (M = Q^{-1}, full symmetric, row-major, leading dim mp),
// warp per row, r staged in shared memory; fused r^T z with CG bookkeeping.
// ------------------------------------------------------------------------------------


template <bool DF>
__global__ void __launch_bounds__(256) k_symv(SymvArgs a) {
  symv_body<DF>(a, blockIdx.x, gridDim.x);
}

__global__ void __launch_bounds__(256) k_symv_batch(const SymvJob* __restrict__ jobs, int njobs) {
  __shared__ int s_job;
  if (threadIdx.x == 0) {
    int lo = 0, hi = njobs - 1;
    while (lo < hi) {   // last job with cta0 <= blockIdx.x
      const int mid = (lo + hi + 1) >> 1;
      if (jobs[mid].cta0 <= (int)blockIdx.x) lo = mid;
      else hi = mid - 1;
    }
    s_job = lo;
  }
  __syncthreads();
  const SymvJob& jb = jobs[s_job];
  symv_body<true>(jb.a, (int)blockIdx.x - jb.cta0, jb.ncta);
}

// Preconditioner apply with M = Q^{-1} stored as DF pairs.
cudaError_t launch_symv_dot(const double* M, int mp, int m, const double* r, double* z,
                            double* sc, int* fl, double* bpart, unsigned* bcnt, int mode,
                            cudaStream_t st) {
  SymvArgs a{M, mp, m, r, z, sc, fl, bpart, bcnt, mode, 0.0, nullptr, nullptr, nullptr, nullptr,
             nullptr, nullptr};
  const size_t smem = (size_t)((m + 3) & ~3) * 2 * sizeof(double);
  { note_launch(); k_symv<true><<<(m + 7) / 8, 256, smem, st>>>(a); }
  return cudaGetLastError();
}

cudaError_t launch_symv_cg_step(const double* M, int mp, int m, const double* rold,
                                const double* q, const double* d, double* dy, double* rnew,
                                double* z, double* sc, int* fl, double* bpart, unsigned* bcnt,
                                cudaStream_t st, const double* qf, double* qzero) {
  SymvArgs a{M, mp, m, rnew, z, sc, fl, bpart, bcnt, SYMV_CG_STEP, 0.0, rold, q, d, dy, qf, qzero};
  const size_t smem = (size_t)((m + 3) & ~3) * 2 * sizeof(double);
  { note_launch(); k_symv<true><<<(m + 7) / 8, 256, smem, st>>>(a); }
  return cudaGetLastError();
}

// Product with an FP64 symmetric matrix (Q in the factor's quality check).
cudaError_t launch_symv_f64(const double* M, int mp, int m, const double* r, double* z,
                            cudaStream_t st) {
  SymvArgs a{M, mp, m, r, z, nullptr, nullptr, nullptr, nullptr, SYMV_PLAIN, 0.0,
             nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  const size_t smem = (size_t)((m + 3) & ~3) * 2 * sizeof(double);
  { note_launch(); k_symv<false><<<(m + 7) / 8, 256, smem, st>>>(a); }
  return cudaGetLastError();
}

cudaError_t launch_symv_init(const double* M, int mp, int m, const double* r, double* z,
                             double* sc, int* fl, double* bpart, unsigned* bcnt, double rel_tol,
                             cudaStream_t st) {
  SymvArgs a{M, mp, m, r, z, sc, fl, bpart, bcnt, SYMV_CG_INIT, rel_tol * rel_tol,
             nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  const size_t smem = (size_t)((m + 3) & ~3) * 2 * sizeof(double);
  { note_launch(); k_symv<true><<<(m + 7) / 8, 256, smem, st>>>(a); }
  return cudaGetLastError();
}

// Factored preconditioner M = X^T X with X = L^{-1} of both factor stages (double-float,
// row-major X and its transpose XT): t = X r carries the CG bookkeeping of `mode` with
// rho = ||t||^2 = r^T M r, then z = X^T t.  For SYMV_CG_STEP the residual update is fused
// into the first product exactly as in launch_symv_cg_step.
cudaError_t launch_precond_factored(const double* X, const double* XT, int mp, int m, int mode,
                                    const double* r, double* t, double* z, double* sc, int* fl,
                                    double* bpart, unsigned* bcnt, double rel_tol,
                                    cudaStream_t st, const double* rold, const double* q,
                                    const double* d, double* dy, const double* qf,
                                    double* qzero) {
  SymvArgs a1{X, mp, m, r, t, sc, fl, bpart, bcnt, mode, rel_tol * rel_tol, rold, q, d, dy, qf,
              qzero, 1, 0};
  const size_t smem = (size_t)((m + 3) & ~3) * 2 * sizeof(double);
  { note_launch(); k_symv<true><<<(m + 7) / 8, 256, smem, st>>>(a1); }
  // the second product finishes an unfinished CG step; for SYMV_F2 / SYMV_PLAIN z is wanted
  const int skip = (mode == SYMV_CG_STEP || mode == SYMV_CG_INIT) ? 1 : 0;
  SymvArgs a2{XT, mp, m, t, z, sc, fl, bpart, bcnt, SYMV_PLAIN, 0.0, nullptr, nullptr, nullptr,
              nullptr, nullptr, nullptr, 0, skip};
  { note_launch(); k_symv<true><<<(m + 7) / 8, 256, smem, st>>>(a2); }
  return cudaGetLastError();
}

__global__ void k_cg_cond(cudaGraphConditionalHandle h, int* fl, int max_trips) {
  const int trips = fl[FL_TRIPS] + 1;
  fl[FL_TRIPS] = trips;
  cudaGraphSetConditional(h, (fl[FL_DONE] == 0 && trips < max_trips) ? 1u : 0u);
}

cudaError_t launch_cg_cond(cudaGraphConditionalHandle h, int* fl, int max_trips, cudaStream_t st) {
  { note_launch(); k_cg_cond<<<1, 1, 0, st>>>(h, fl, max_trips); }
  return cudaGetLastError();
}

cudaError_t launch_symv_batch(const SymvJob* jobs, int njobs, int total_ctas, size_t smem,
                              cudaStream_t st) {
  cudaError_t e = ensure_dyn_smem((const void*)k_symv_batch, smem);
  if (e != cudaSuccess) return e;
  { note_launch(); k_symv_batch<<<total_ctas, 256, smem, st>>>(jobs, njobs); }
  return cudaGetLastError();
}

cudaError_t symv_set_smem(int m) {
  const int bytes = ((m + 3) & ~3) * 2 * (int)sizeof(double);
  cudaError_t e = ensure_dyn_smem((const void*)k_symv<true>, bytes);
  if (e != cudaSuccess) return e;
  return ensure_dyn_smem((const void*)k_symv<false>, bytes);
}

__global__ void k_vec_ops(int op, double* a, const double* b, const double* c, int m) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
    switch (op) {
      case VOP_COPY: a[i] = b[i]; break;
      case VOP_ZERO: a[i] = 0.0; break;
      case VOP_ADD: a[i] = b[i] + c[i]; break;
      case VOP_SUB: a[i] = b[i] - c[i]; break;
      case VOP_NEG: a[i] = -b[i]; break;
      case VOP_ONES: a[i] = 1.0; break;
      case VOP_SIGNS: {   // sign from the top bit of a multiplicative hash of i
        const unsigned h = ((unsigned)i + 1u) * 0x9E3779B1u;
        a[i] = ((h ^ (h >> 15)) & 0x8000u) ? -1.0 : 1.0;
        break;
      }
    }
  }
}

cudaError_t launch_vec_ops(int op, double* a, const double* b, const double* c, int m,
                           const double* sc, cudaStream_t st) {
  (void)sc;
  { note_launch(); k_vec_ops<<<vec_grid(m), 256, 0, st>>>(op, a, b, c, m); }
  return cudaGetLastError();
}

// ------------------------------------------------------------------------------------
// IPM update, Alg. 2 step (d): directions and their inner products.
//   ds = -r_d - A^T dy                            (Eq. delshat)
//   (W u)_i = sum_j sign_ij / sqrt(s) u[bucket_ij] (gather; W from the same hash as the sketch)
//   S^{-1} v = D (W u), v = (X S)^{1/2} W u        (Eq. compv)
//   dx = -x + sigma mu / s - D^2 ds - S^{-1} v     (Eq. delxhat)
// Sums: x^T ds + s^T dx, dx^T ds, ||v||^2, 1^T v.
// ------------------------------------------------------------------------------------
__global__ void k_update_dirs(const double* __restrict__ x, const double* __restrict__ s,
                              const double* __restrict__ d2, const double* __restrict__ d,
                              const double* __restrict__ rd, const double* __restrict__ t,
                              const int32_t* __restrict__ hb, int ss, const double* __restrict__ u,
                              int64_t n, double* wu, double* dx, double* ds, int wu_given,
                              double* sc, double* bpart, unsigned* bcnt) {
  const double sigmu = sc[SC_SIGMU];
  const double inv_sqrt_s = 1.0 / sqrt((double)ss);
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    double w;
    if (wu_given) {
      w = wu[i];
    } else {
      w = 0.0;
      for (int j = 0; j < ss; ++j) {
        const int32_t h = hb[i * ss + j];
        const double uv = u[h & 0x7fffffff];
        w += (h < 0) ? -uv : uv;
      }
      w *= inv_sqrt_s;
      if (wu) wu[i] = w;
    }
    const double xi = x[i], si = s[i];
    const double dsi = -rd[i] - t[i];
    const double dxi = -xi + sigmu / si - d2[i] * dsi - d[i] * w;
    const double vi = sqrt(xi * si) * w;
    dx[i] = dxi;
    ds[i] = dsi;
    acc[0] += xi * dsi + si * dxi;
    acc[1] += dxi * dsi;
    acc[2] += vi * vi;
    acc[3] += vi;
  }
  if (grid_sum_last<4>(acc, bpart, bcnt) && threadIdx.x == 0) {
    sc[SC_B] = acc[0];
    sc[SC_C] = acc[1];
    sc[SC_V2] = acc[2];
    sc[SC_V1] = acc[3];
  }
}

cudaError_t launch_update_dirs(const double* x, const double* s, const double* d2, const double* d,
                               const double* rd, const double* t, const int32_t* hb, int ss,
                               const double* u, int64_t n, double* wu, double* dx, double* ds,
                               int wu_given, double* sc, double* bpart, unsigned* bcnt,
                               cudaStream_t st) {
  { note_launch(); k_update_dirs<<<vec_grid(n), 256, 0, st>>>(x, s, d2, d, rd, t, hb, ss, u, n, wu, dx, ds,
                                             wu_given, sc, bpart, bcnt); }
  return cudaGetLastError();
}

// Smallest a in (0, 1] at which a0 + a1 a + a2 a^2 (a0 >= 0) turns negative; +inf if none.
// Roots from the cancellation-free form of the quadratic formula; a root counts only where
// the polynomial is decreasing.
__device__ double first_crossing(double a0, double a1, double a2) {
  a0 = fmax(a0, 0.0);
  if (a2 == 0.0) return (a1 < 0.0) ? a0 / (-a1) : INFINITY;
  const double disc = a1 * a1 - 4.0 * a2 * a0;
  if (disc < 0.0) return INFINITY;
  const double sq = sqrt(disc);
  const double qq = -0.5 * (a1 + (a1 >= 0.0 ? sq : -sq));
  double best = INFINITY;
  const double r1 = qq / a2;
  const double r2 = (qq != 0.0) ? a0 / qq : INFINITY;
  if (isfinite(r1) && r1 > 0.0 && 2.0 * a2 * r1 + a1 < 0.0) best = fmin(best, r1);
  if (isfinite(r2) && r2 > 0.0 && 2.0 * a2 * r2 + a1 < 0.0) best = fmin(best, r2);
  return best;
}

// Alg. 2 steps (e)-(f).  N(gamma): x_i s_i >= (1-gamma) mu and ||r||/||r0|| <= mu/mu0, with
// mu(a) = (x^T s + a B + a^2 C)/n and r(a) = (1 - a) r (Eq. iip_3).  alpha_max = first
// crossing over all conditions (capped at 1); alpha minimises mu(a) on [0, alpha_max],
// ties to the larger a.
__global__ void k_step_length(const double* __restrict__ x, const double* __restrict__ s,
                              const double* __restrict__ dx, const double* __restrict__ ds,
                              int64_t n, double gamma, double* sc, double* bpart, unsigned* bcnt) {
  const double xs = sc[SC_XS], B = sc[SC_B], C = sc[SC_C];
  const double g1 = 1.0 - gamma;
  const double nn = (double)n;
  const double m0 = g1 * xs / nn, m1 = g1 * B / nn, m2 = g1 * C / nn;
  double best = INFINITY;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double xi = x[i], si = s[i], dxi = dx[i], dsi = ds[i];
    const double a0 = fmax(xi * si - m0, 0.0), a1 = xi * dsi + si * dxi - m1, a2 = dxi * dsi - m2;
    // only crossings in (0, 1] can matter (alpha_max <= 1): a0 + min(a1, 0) + min(a2, 0) is a
    // lower bound of the polynomial on [0, 1], so when it clears its own rounding error the
    // element has no crossing there and the square root and divisions are skipped
    const double lb = a0 + fmin(a1, 0.0) + fmin(a2, 0.0);
    if (lb > 1e-14 * (a0 + fabs(a1) + fabs(a2))) continue;
    best = fmin(best, first_crossing(a0, a1, a2));
  }
  if (grid_min_last(best, bpart, bcnt) && threadIdx.x == 0) {
    const double eta = sc[SC_ETA], mu0 = sc[SC_MU0];
    double amax = fmin(1.0, best);
    const double gr = first_crossing(xs / nn / mu0 - eta, B / nn / mu0 + eta, C / nn / mu0);
    amax = fmin(amax, gr);
    if (!(amax >= 0.0)) amax = 0.0;
    // step (f): minimise f(a) = B a + C a^2 on [0, amax]
    double alpha = amax;
    double fbest = B * amax + C * amax * amax;
    if (fbest > 0.0) {  // f(0) = 0 beats a positive endpoint; a tie keeps the larger a
      alpha = 0.0;
      fbest = 0.0;
    }
    if (C > 0.0) {
      const double vtx = -B / (2.0 * C);
      if (vtx > 0.0 && vtx < amax) {
        const double fv = B * vtx + C * vtx * vtx;
        if (fv < fbest) {
          alpha = vtx;
          fbest = fv;
        }
      }
    }
    sc[SC_AMAX] = amax;
    sc[SC_STEP] = alpha;
  }
}

cudaError_t launch_step_length(const double* x, const double* s, const double* dx,
                               const double* ds, int64_t n, double gamma, double* sc,
                               double* bpart, unsigned* bcnt, cudaStream_t st) {
  { note_launch(); k_step_length<<<vec_grid(n), 256, 0, st>>>(x, s, dx, ds, n, gamma, sc, bpart, bcnt); }
  return cudaGetLastError();
}

// Alg. 2 step (g).
__global__ void k_apply_step(double* x, double* s, double* y, const double* dx, const double* ds,
                             const double* dy, int64_t n, int m, const double* sc) {
  const double al = sc[SC_STEP];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    x[i] = fma(al, dx[i], x[i]);
    s[i] = fma(al, ds[i], s[i]);
    if (i < m) y[i] = fma(al, dy[i], y[i]);
  }
}

cudaError_t launch_apply_step(double* x, double* s, double* y, const double* dx, const double* ds,
                              const double* dy, int64_t n, int m, const double* sc,
                              cudaStream_t st) {
  { note_launch(); k_apply_step<<<vec_grid(n), 256, 0, st>>>(x, s, y, dx, ds, dy, n, m, sc); }
  return cudaGetLastError();
}

}  // namespace lpk
