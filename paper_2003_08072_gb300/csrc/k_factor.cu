// Preconditioner factor (Alg. 1 step 2): Q = (A D W)(A D W)^T (Eq. pdprecond) and Q^{-1}.
//
// Alg. 1 obtains Q^{-1/2} from the SVD of A D W.  Preconditioned CG with M = Q visits the same
// iterates dy = Q^{-1/2} z as CG on Eq. precond_alt, so only the operator Q^{-1} is needed.
// It is formed explicitly so that each CG step applies it as one dense symmetric matrix-vector
// product over the whole GPU instead of two sequential triangular solves.
//   1. Gram product G G^T in FP64, lower 64x64 tiles, split along w for parallelism, then
//      summed and mirrored into a full row-major mp x mp matrix (identity on the padding).
//   2. In-place blocked Gauss-Jordan inversion with 32 x 32 pivot blocks.  Q is symmetric
//      positive definite when rank(A D W) = m (Lemma 4.1), so every pivot block is SPD and no
//      pivoting is needed; a non-positive pivot flags a rank-deficient sketch.
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

// ---- blocked Gauss-Jordan inversion, pivot block kb --------------------------------------

// A pivot counts as lost when it falls below 1e-12 of the original diagonal entry of Q, i.e.
// when Q is numerically singular (condition number beyond ~1e12).
__global__ void __launch_bounds__(256) k_gj_pivot(const double* __restrict__ M,
                                                  const double* __restrict__ Q0, int mp, int kb,
                                                  double* __restrict__ Pinv, int* fl) {
  __shared__ double P[kNB][kNB + 1];
  __shared__ double f[kNB];
  if (fl[FL_BREAK]) return;
  const int tid = threadIdx.x;
  for (int e = tid; e < kNB * kNB; e += blockDim.x) {
    const int i = e / kNB, j = e % kNB;
    P[i][j] = M[(size_t)(kb * kNB + i) * mp + kb * kNB + j];
  }
  __syncthreads();
  bool bad = false;
  for (int p = 0; p < kNB; ++p) {
    const double piv = P[p][p];
    const double q0 = Q0[(size_t)(kb * kNB + p) * mp + kb * kNB + p];
    if (!(piv > 1e-12 * q0) || !isfinite(piv)) bad = true;
    if (tid < kNB) f[tid] = P[tid][p];
    __syncthreads();
    const double ip = 1.0 / piv;
    if (tid < kNB) P[p][tid] = (tid == p ? 1.0 : P[p][tid]) * ip;
    __syncthreads();
    for (int e = tid; e < kNB * kNB; e += blockDim.x) {
      const int i = e / kNB, j = e % kNB;
      if (i != p) P[i][j] = (j == p ? 0.0 : P[i][j]) - f[i] * P[p][j];
    }
    __syncthreads();
  }
  if (bad && tid == 0) fl[FL_BREAK] = 1;
  for (int e = tid; e < kNB * kNB; e += blockDim.x) Pinv[e] = P[e / kNB][e % kNB];
}

// T[:, jb] = Pinv * M[kb, jb] (row block of the pivot, 32 x mp); C[jb, :] = M[jb, kb].
__global__ void __launch_bounds__(256) k_gj_panel(const double* __restrict__ M, int mp, int kb,
                                                  const double* __restrict__ Pinv,
                                                  double* __restrict__ T, double* __restrict__ C,
                                                  const int* fl) {
  __shared__ double Ps[kNB][kNB + 1];
  __shared__ double Xs[kNB][kNB + 1];
  if (fl[FL_BREAK]) return;
  const int jb = blockIdx.x, tid = threadIdx.x;
  for (int e = tid; e < kNB * kNB; e += blockDim.x) {
    const int i = e / kNB, j = e % kNB;
    Ps[i][j] = Pinv[e];
    Xs[i][j] = M[(size_t)(kb * kNB + i) * mp + jb * kNB + j];
    C[(size_t)(jb * kNB + i) * kNB + j] = M[(size_t)(jb * kNB + i) * mp + kb * kNB + j];
  }
  __syncthreads();
  for (int e = tid; e < kNB * kNB; e += blockDim.x) {
    const int i = e / kNB, j = e % kNB;
    double acc = 0.0;
#pragma unroll 8
    for (int k = 0; k < kNB; ++k) acc = fma(Ps[i][k], Xs[k][j], acc);
    T[(size_t)i * mp + jb * kNB + j] = acc;
  }
}

__global__ void __launch_bounds__(256) k_gj_update(double* __restrict__ M, int mp, int kb,
                                                   const double* __restrict__ Pinv,
                                                   const double* __restrict__ T,
                                                   const double* __restrict__ C, const int* fl) {
  __shared__ double Cs[kNB][kNB + 1];
  __shared__ double Ts[kNB][kNB + 1];
  if (fl[FL_BREAK]) return;
  const int ib = blockIdx.y, jb = blockIdx.x, tid = threadIdx.x;
  if (ib == kb && jb == kb) {
    for (int e = tid; e < kNB * kNB; e += blockDim.x)
      M[(size_t)(kb * kNB + e / kNB) * mp + kb * kNB + e % kNB] = Pinv[e];
    return;
  }
  if (ib == kb) {
    for (int e = tid; e < kNB * kNB; e += blockDim.x) {
      const int i = e / kNB, j = e % kNB;
      M[(size_t)(kb * kNB + i) * mp + jb * kNB + j] = T[(size_t)i * mp + jb * kNB + j];
    }
    return;
  }
  for (int e = tid; e < kNB * kNB; e += blockDim.x) {
    const int i = e / kNB, j = e % kNB;
    Cs[i][j] = C[(size_t)(ib * kNB + i) * kNB + j];
    Ts[i][j] = (jb == kb) ? Pinv[e] : T[(size_t)i * mp + jb * kNB + j];
  }
  __syncthreads();
  for (int e = tid; e < kNB * kNB; e += blockDim.x) {
    const int i = e / kNB, j = e % kNB;
    double acc = 0.0;
#pragma unroll 8
    for (int k = 0; k < kNB; ++k) acc = fma(Cs[i][k], Ts[k][j], acc);
    double* dst = &M[(size_t)(ib * kNB + i) * mp + jb * kNB + j];
    if (jb == kb)
      *dst = -acc;          // column block of the pivot: -C Pinv
    else
      *dst = *dst - acc;    // Schur update
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

cudaError_t launch_gj_inverse(double* M, const double* Q0, int mp, double* Pinv, double* T,
                              double* C, int* fl, cudaStream_t st) {
  const int nb = mp / kNB;
  for (int kb = 0; kb < nb; ++kb) {
    { note_launch(); k_gj_pivot<<<1, 256, 0, st>>>(M, Q0, mp, kb, Pinv, fl); }
    { note_launch(); k_gj_panel<<<nb, 256, 0, st>>>(M, mp, kb, Pinv, T, C, fl); }
    { note_launch(); k_gj_update<<<dim3(nb, nb), 256, 0, st>>>(M, mp, kb, Pinv, T, C, fl); }
  }
  return cudaGetLastError();
}

}  // namespace lpk
