// Preconditioner factor (Alg. 1 step 2): Q = (A D W)(A D W)^T (Eq. pdprecond) and Q^{-1}.
//
// Alg. 1 obtains Q^{-1/2} from the SVD of A D W.  Preconditioned CG with M = Q visits the same
// iterates dy = Q^{-1/2} z as CG on Eq. precond_alt, so only the operator Q^{-1} is needed.
// It is formed explicitly so that each CG step applies it as one dense symmetric matrix-vector
// product over the whole GPU instead of two sequential triangular solves.
//   1. Gram product G G^T in FP64, lower 64x64 tiles, split along w for parallelism, then
//      summed and mirrored into a full row-major mp x mp matrix (identity on the padding).
//   2. Q^{-1} = L^{-T} L^{-1} from a blocked Cholesky factor Q = L L^T (Q is symmetric positive
//      definite when rank(A D W) = m, Lemma 4.1); a lost pivot flags a numerically singular Q.
#include "dev_util.cuh"

namespace lpk {

constexpr int kGT = 64;   // Gram tile
constexpr int kGK = 16;   // Gram k-chunk

__global__ void __launch_bounds__(256) k_gram_tile(const double* __restrict__ G, int ldg, int m, int w,
                                                   int chunk, double* __restrict__ Qsplit,
                                                   int ntiles) {
  __shared__ __align__(16) double As[kGK][kGT + 2];
  __shared__ __align__(16) double Bs[kGK][kGT + 2];
  int tile = blockIdx.x, ib = 0;
  while ((ib + 1) * (ib + 2) / 2 <= tile) ++ib;
  const int jb = tile - ib * (ib + 1) / 2;
  const int ks = blockIdx.y;
  const int k0 = ks * chunk, k1 = min(w, k0 + chunk);
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  double acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
  for (int k = k0; k < k1; k += kGK) {
#pragma unroll
    for (int l = 0; l < 4; ++l) {
      const int idx = tid + l * 256;
      const int kk = idx >> 6, r = idx & 63;
      const int ra = ib * kGT + r, rb = jb * kGT + r;
      const bool kin = (k + kk) < k1;
      As[kk][r] = (kin && ra < m) ? G[(size_t)(k + kk) * ldg + ra] : 0.0;
      Bs[kk][r] = (kin && rb < m) ? G[(size_t)(k + kk) * ldg + rb] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < kGK; ++kk) {
      double a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty * 4 + i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx * 4 + j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
  double* out = Qsplit + ((size_t)ks * ntiles + tile) * (kGT * kGT);
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) out[(ty * 4 + i) * kGT + tx * 4 + j] = acc[i][j];
}

__global__ void __launch_bounds__(256) k_gram_finish(const double* __restrict__ Qsplit, int split,
                                                     int ntiles, int m, int mp,
                                                     double* __restrict__ Q) {
  const int tile = blockIdx.x;
  int ib = 0;
  while ((ib + 1) * (ib + 2) / 2 <= tile) ++ib;
  const int jb = tile - ib * (ib + 1) / 2;
  for (int e = threadIdx.x; e < kGT * kGT; e += blockDim.x) {
    const int r = e / kGT, cc = e % kGT;
    const int row = ib * kGT + r, col = jb * kGT + cc;
    double v = 0.0;
    for (int ks = 0; ks < split; ++ks) v += Qsplit[((size_t)ks * ntiles + tile) * (kGT * kGT) + e];
    if (row >= m || col >= m) v = (row == col) ? 1.0 : 0.0;
    Q[(size_t)row * mp + col] = v;
    Q[(size_t)col * mp + row] = v;
  }
}

int gram_split(int m, int w, int num_sms) {
  const int nt = (m + kGT - 1) / kGT;
  const int ntiles = nt * (nt + 1) / 2;
  int split = (2 * num_sms + ntiles - 1) / ntiles;
  const int maxsplit = (w + 255) / 256;   // keep >= 256 columns per split
  if (split > maxsplit) split = maxsplit;
  if (split < 1) split = 1;
  return split;
}

cudaError_t launch_gram(const double* G, int ldg, int m, int w, int mp, double* Q, double* Qsplit,
                        int split, cudaStream_t st) {
  const int nt = mp / kGT;
  const int ntiles = nt * (nt + 1) / 2;
  int chunk = (w + split - 1) / split;
  chunk = (chunk + kGK - 1) / kGK * kGK;
  dim3 grid(ntiles, split);
  { note_launch(); k_gram_tile<<<grid, 256, 0, st>>>(G, ldg, m, w, chunk, Qsplit, ntiles); }
  { note_launch(); k_gram_finish<<<ntiles, 256, 0, st>>>(Qsplit, split, ntiles, m, mp, Q); }
  return cudaGetLastError();
}

// ---- Q^{-1} through a blocked Cholesky factor -------------------------------------------
//
// Q = L L^T (right-looking, 32 x 32 blocks) and X = L^{-1} are computed in one left-to-right
// sweep over the block columns k:
//   panel : L_ik = A_ik X_kk^T (i > k)          and  X_kj <- X_kk X_kj (j < k)
//   update: A_ij -= L_ik L_jk^T (k < j <= i)    and  X_ij -= L_ik X_kj (i > k, j <= k)
// and the CTA that finishes the update of the next diagonal block (scheduled first) factors
// it and inverts its triangle in shared memory.  Finally M = X^T X = Q^{-1}, mirrored into
// full storage.  Unlike Gauss-Jordan elimination on Q itself this keeps the error of M near
// kappa(Q) u (backward-stable Cholesky), which matters late in the IPM where kappa(Q) is large.
// A diagonal pivot of the Schur complement below 1e-14 of the original diagonal entry of Q is
// reported as a lost pivot (FL_BREAK).

// Cholesky of a kNB x kNB SPD tile in shared memory (lower triangle, in place), then X = L^{-1}
// (lower triangular, zeros above).  Needs blockDim.x >= kNB.  Returns false on a lost pivot.
__device__ bool chol_inv_tile(double (*P)[kNB + 1], double (*Xs)[kNB + 1], const double* q0) {
  const int tid = threadIdx.x;
  bool ok = true;
  for (int p = 0; p < kNB; ++p) {
    __syncthreads();
    double d = P[p][p];
    if (!(d > 1e-14 * q0[p]) || !isfinite(d)) {
      ok = false;
      d = fmax(fabs(q0[p]), 1e-300);   // keep the arithmetic finite; the flag aborts the solve
    }
    const double l = sqrt(d);
    __syncthreads();
    if (tid == 0) P[p][p] = l;
    if (tid > p && tid < kNB) P[tid][p] /= l;
    __syncthreads();
    for (int e = tid; e < kNB * kNB; e += blockDim.x) {
      const int i = e / kNB, j = e % kNB;
      if (j > p && j <= i) P[i][j] -= P[i][p] * P[j][p];
    }
  }
  __syncthreads();
  if (tid < kNB) {   // column tid of L^{-1} by forward substitution
    const int j = tid;
    for (int i = 0; i < kNB; ++i) {
      if (i < j) {
        Xs[i][j] = 0.0;
        continue;
      }
      double s = (i == j) ? 1.0 : 0.0;
      for (int q = j; q < i; ++q) s -= P[i][q] * Xs[q][j];
      Xs[i][j] = s / P[i][i];
    }
  }
  __syncthreads();
  return ok;
}

__device__ __forceinline__ void tri_decode(int idx, int& i, int& j) {
  i = 0;
  while ((i + 1) * (i + 2) / 2 <= idx) ++i;
  j = idx - i * (i + 1) / 2;
}

__device__ __forceinline__ void load_tile(double (*S)[kNB + 1], const double* src, int ld) {
  for (int e = threadIdx.x; e < kNB * kNB; e += blockDim.x)
    S[e / kNB][e % kNB] = src[(size_t)(e / kNB) * ld + e % kNB];
}

__device__ __forceinline__ void store_tile(double* dst, int ld, double (*S)[kNB + 1]) {
  for (int e = threadIdx.x; e < kNB * kNB; e += blockDim.x)
    dst[(size_t)(e / kNB) * ld + e % kNB] = S[e / kNB][e % kNB];
}

__global__ void __launch_bounds__(256) k_ch_diag0(double* __restrict__ M, double* __restrict__ X,
                                                  const double* __restrict__ Q0, int mp, int* fl) {
  __shared__ double P[kNB][kNB + 1];
  __shared__ double Xs[kNB][kNB + 1];
  __shared__ double q0[kNB];
  if (fl[FL_BREAK]) return;
  load_tile(P, M, mp);
  if (threadIdx.x < kNB) q0[threadIdx.x] = Q0[(size_t)threadIdx.x * mp + threadIdx.x];
  const bool ok = chol_inv_tile(P, Xs, q0);
  if (!ok && threadIdx.x == 0) fl[FL_BREAK] = 1;
  store_tile(M, mp, P);
  store_tile(X, mp, Xs);
}

// grid: (nbk-kb-1) panel CTAs, then kb row-scaling CTAs
__global__ void __launch_bounds__(256) k_ch_panel(double* __restrict__ M, double* __restrict__ X,
                                                  int mp, int nbk, int kb, const int* fl) {
  __shared__ double Ss[kNB][kNB + 1];
  __shared__ double Xk[kNB][kNB + 1];
  if (fl[FL_BREAK]) return;
  const int npan = nbk - kb - 1;
  load_tile(Xk, X + (size_t)(kb * kNB) * mp + kb * kNB, mp);
  double* dst;
  const bool panel = (int)blockIdx.x < npan;
  if (panel) {
    const int i = kb + 1 + blockIdx.x;
    dst = M + (size_t)(i * kNB) * mp + kb * kNB;          // A_ik -> L_ik
  } else {
    const int j = blockIdx.x - npan;
    dst = X + (size_t)(kb * kNB) * mp + j * kNB;          // X_kj
  }
  load_tile(Ss, dst, mp);
  __syncthreads();
  double out[4];
  int cnt = 0;
  for (int e = threadIdx.x; e < kNB * kNB; e += blockDim.x, ++cnt) {
    const int r = e / kNB, cc = e % kNB;
    double acc = 0.0;
    if (panel) {
#pragma unroll 8
      for (int q = 0; q < kNB; ++q) acc = fma(Ss[r][q], Xk[cc][q], acc);   // A_ik X_kk^T
    } else {
#pragma unroll 8
      for (int q = 0; q < kNB; ++q) acc = fma(Xk[r][q], Ss[q][cc], acc);   // X_kk X_kj
    }
    out[cnt] = acc;
  }
  cnt = 0;
  for (int e = threadIdx.x; e < kNB * kNB; e += blockDim.x, ++cnt)
    dst[(size_t)(e / kNB) * mp + e % kNB] = out[cnt];
}

// grid: r(r+1)/2 trailing Cholesky tiles (next diagonal block first), then r(kb+1) inverse
// tiles, r = nbk - kb - 1.
__global__ void __launch_bounds__(256) k_ch_update(double* __restrict__ M, double* __restrict__ X,
                                                   const double* __restrict__ Q0, int mp, int nbk,
                                                   int kb, int* fl) {
  __shared__ double As[kNB][kNB + 1];
  __shared__ double Bs[kNB][kNB + 1];
  __shared__ double Xs[kNB][kNB + 1];
  __shared__ double q0[kNB];
  if (fl[FL_BREAK]) return;
  const int r = nbk - kb - 1;
  const int n1 = r * (r + 1) / 2;
  int b = blockIdx.x;
  double* tile;
  if (b < n1) {
    int ii, jj;
    if (b == 0) {
      ii = jj = 0;
    } else {
      tri_decode(b, ii, jj);   // index 0 is (0, 0), the next diagonal block
    }
    const int i = kb + 1 + ii, j = kb + 1 + jj;
    tile = M + (size_t)(i * kNB) * mp + j * kNB;
    load_tile(As, M + (size_t)(i * kNB) * mp + kb * kNB, mp);   // L_ik
    load_tile(Bs, M + (size_t)(j * kNB) * mp + kb * kNB, mp);   // L_jk
    __syncthreads();
    double upd[4];
    int cnt = 0;
    for (int e = threadIdx.x; e < kNB * kNB; e += blockDim.x, ++cnt) {
      const int rr = e / kNB, cc = e % kNB;
      double acc = 0.0;
#pragma unroll 8
      for (int q = 0; q < kNB; ++q) acc = fma(As[rr][q], Bs[cc][q], acc);
      upd[cnt] = tile[(size_t)rr * mp + cc] - acc;
    }
    if (ii == 0 && jj == 0) {
      __syncthreads();
      cnt = 0;
      for (int e = threadIdx.x; e < kNB * kNB; e += blockDim.x, ++cnt) As[e / kNB][e % kNB] = upd[cnt];
      if (threadIdx.x < kNB) q0[threadIdx.x] = Q0[(size_t)(i * kNB + threadIdx.x) * mp + i * kNB + threadIdx.x];
      const bool ok = chol_inv_tile(As, Xs, q0);
      if (!ok && threadIdx.x == 0) fl[FL_BREAK] = 1;
      store_tile(tile, mp, As);
      store_tile(X + (size_t)(i * kNB) * mp + i * kNB, mp, Xs);
      return;
    }
    cnt = 0;
    for (int e = threadIdx.x; e < kNB * kNB; e += blockDim.x, ++cnt)
      tile[(size_t)(e / kNB) * mp + e % kNB] = upd[cnt];
    return;
  }
  b -= n1;
  const int i = kb + 1 + b / (kb + 1), j = b % (kb + 1);
  tile = X + (size_t)(i * kNB) * mp + j * kNB;
  load_tile(As, M + (size_t)(i * kNB) * mp + kb * kNB, mp);    // L_ik
  load_tile(Bs, X + (size_t)(kb * kNB) * mp + j * kNB, mp);    // X_kj
  __syncthreads();
  double upd[4];
  int cnt = 0;
  for (int e = threadIdx.x; e < kNB * kNB; e += blockDim.x, ++cnt) {
    const int rr = e / kNB, cc = e % kNB;
    double acc = 0.0;
#pragma unroll 8
    for (int q = 0; q < kNB; ++q) acc = fma(As[rr][q], Bs[q][cc], acc);
    upd[cnt] = tile[(size_t)rr * mp + cc] - acc;
  }
  cnt = 0;
  for (int e = threadIdx.x; e < kNB * kNB; e += blockDim.x, ++cnt)
    tile[(size_t)(e / kNB) * mp + e % kNB] = upd[cnt];
}

// M = X^T X for lower tiles (i >= j), sum over block rows q >= i, mirrored into the upper tiles.
__global__ void __launch_bounds__(256) k_ch_xtx(const double* __restrict__ X, double* __restrict__ M,
                                                int mp, int nbk, const int* fl) {
  __shared__ double Xi[kNB][kNB + 1];
  __shared__ double Xj[kNB][kNB + 1];
  if (fl[FL_BREAK]) return;
  int i, j;
  tri_decode(blockIdx.x, i, j);
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  for (int q = i; q < nbk; ++q) {
    __syncthreads();
    load_tile(Xi, X + (size_t)(q * kNB) * mp + i * kNB, mp);
    load_tile(Xj, X + (size_t)(q * kNB) * mp + j * kNB, mp);
    __syncthreads();
    int cnt = 0;
    for (int e = threadIdx.x; e < kNB * kNB; e += blockDim.x, ++cnt) {
      const int rr = e / kNB, cc = e % kNB;
      double a = acc[cnt];
#pragma unroll 8
      for (int t = 0; t < kNB; ++t) a = fma(Xi[t][rr], Xj[t][cc], a);
      acc[cnt] = a;
    }
  }
  int cnt = 0;
  for (int e = threadIdx.x; e < kNB * kNB; e += blockDim.x, ++cnt) {
    const int rr = e / kNB, cc = e % kNB;
    M[(size_t)(i * kNB + rr) * mp + j * kNB + cc] = acc[cnt];
    if (i != j) M[(size_t)(j * kNB + cc) * mp + i * kNB + rr] = acc[cnt];
  }
}

// Relative diagonal shift M_ii *= (1 + eps): keeps the preconditioner positive definite when
// the Gram matrix is numerically singular (e.g. colliding CountSketch buckets late in the IPM).
__global__ void k_shift_diag(double* M, int mp, int m, double eps) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x)
    M[(size_t)i * mp + i] *= (1.0 + eps);
}

cudaError_t launch_shift_diag(double* M, int mp, int m, double eps, cudaStream_t st) {
  { note_launch(); k_shift_diag<<<(m + 255) / 256, 256, 0, st>>>(M, mp, m, eps); }
  return cudaGetLastError();
}

// M (mp x mp, holding Q on entry) becomes Q^{-1}; X is an mp x mp work buffer (L^{-1}).
cudaError_t launch_chol_inverse(double* M, double* X, const double* Q0, int mp, int* fl,
                                cudaStream_t st) {
  const int nbk = mp / kNB;
  cudaError_t e = cudaMemsetAsync(X, 0, (size_t)mp * mp * sizeof(double), st);
  if (e != cudaSuccess) return e;
  { note_launch(); k_ch_diag0<<<1, 256, 0, st>>>(M, X, Q0, mp, fl); }
  for (int kb = 0; kb < nbk; ++kb) {
    const int r = nbk - kb - 1;
    const int npanel = r + kb;
    if (npanel > 0) { note_launch(); k_ch_panel<<<npanel, 256, 0, st>>>(M, X, mp, nbk, kb, fl); }
    const int nupd = r * (r + 1) / 2 + r * (kb + 1);
    if (nupd > 0) { note_launch(); k_ch_update<<<nupd, 256, 0, st>>>(M, X, Q0, mp, nbk, kb, fl); }
  }
  { note_launch(); k_ch_xtx<<<nbk * (nbk + 1) / 2, 256, 0, st>>>(X, M, mp, nbk, fl); }
  return cudaGetLastError();
}

}  // namespace lpk
