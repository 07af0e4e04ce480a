// Preconditioner factor (Alg. 1 step 2): Q = (A D W)(A D W)^T (Eq. pdprecond) and Q^{-1}.
//
// Alg. 1 obtains Q^{-1/2} from the SVD of A D W.  Preconditioned CG with M = Q visits the same
// iterates dy = Q^{-1/2} z as CG on Eq. precond_alt, so only the operator Q^{-1} is needed.
// It is formed explicitly so that each CG step applies it as one dense symmetric matrix-vector
// product over the whole GPU instead of two sequential triangular solves.
//   1. Gram product G G^T in double-float arithmetic (FP64-class, on the FP32 pipes), lower
//      64x64 tiles, split along w for parallelism, then summed in FP64 and mirrored into a full
//      row-major mp x mp matrix (identity on the padding).
//   2. Q^{-1} = L^{-T} L^{-1} from a blocked Cholesky factor Q = L L^T (Q is symmetric positive
//      definite when rank(A D W) = m, Lemma 4.1); a lost pivot flags a numerically singular Q.
//      The sweep runs either as two launches per block step or as one launch of tile tasks in
//      dependency order (k_ch_dag); both give bitwise the same L and L^{-1}.
#include <algorithm>

#include "bulk_util.cuh"
#include "chol_tasks.h"
#include "dev_util.cuh"

namespace lpk {

constexpr int kGT = 64;   // Gram tile
constexpr int kGK = 16;   // Gram k-chunk

// G (FP64) -> hi + lo floats, once per factorization.  The split costs FP64 conversions, slow
// on this GPU; done inside the tile kernel it was repeated for every tile pair an entry meets
// (m / 64 + 1 times) and bounded the Gram product.
__global__ void k_split_df(const double* __restrict__ G, size_t count, float* __restrict__ Gh,
                           float* __restrict__ Gl) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count;
       i += (size_t)gridDim.x * blockDim.x)
    split_double_bits(G[i], Gh[i], Gl[i]);
}

// One 64 x 64 lower tile of G G^T over a slice of the w columns, in double-float arithmetic on
// the FP32 pipes from the hi + lo split of G; hi*hi products are accumulated with
// TwoProduct/TwoSum, the cross terms plainly.
__global__ void __launch_bounds__(256) k_gram_tile(const float* __restrict__ Gh,
                                                   const float* __restrict__ Gl, int ldg, int m,
                                                   int w, int chunk, double* __restrict__ Qsplit,
                                                   int ntiles) {
  __shared__ __align__(16) float Ah[kGK][kGT + 4];
  __shared__ __align__(16) float Al[kGK][kGT + 4];
  __shared__ __align__(16) float Bh[kGK][kGT + 4];
  __shared__ __align__(16) float Bl[kGK][kGT + 4];
  int tile = blockIdx.x, ib = 0;
  while ((ib + 1) * (ib + 2) / 2 <= tile) ++ib;
  const int jb = tile - ib * (ib + 1) / 2;
  const int ks = blockIdx.y;
  const int k0 = ks * chunk, k1 = min(w, k0 + chunk);
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  float s[4][4], c[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) s[i][j] = c[i][j] = 0.f;
  for (int k = k0; k < k1; k += kGK) {
#pragma unroll
    for (int l = 0; l < 4; ++l) {
      const int idx = tid + l * 256;
      const int kk = idx >> 6, r = idx & 63;
      const int ra = ib * kGT + r, rb = jb * kGT + r;
      const bool kin = (k + kk) < k1;
      const bool va = kin && ra < m, vb = kin && rb < m;
      const size_t ia = (size_t)(k + kk) * ldg + ra, ibb = (size_t)(k + kk) * ldg + rb;
      Ah[kk][r] = va ? Gh[ia] : 0.f;
      Al[kk][r] = va ? Gl[ia] : 0.f;
      Bh[kk][r] = vb ? Gh[ibb] : 0.f;
      Bl[kk][r] = vb ? Gl[ibb] : 0.f;
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < kGK; ++kk) {
      float ah[4], al[4], bh[4], bl[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        ah[i] = Ah[kk][ty * 4 + i];
        al[i] = Al[kk][ty * 4 + i];
        bh[i] = Bh[kk][tx * 4 + i];
        bl[i] = Bl[kk][tx * 4 + i];
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const float p = __fmul_rn(ah[i], bh[j]);
          const float pe = fmaf(ah[i], bh[j], -p);
          float t, e;
          two_sum(s[i][j], p, t, e);
          s[i][j] = t;
          c[i][j] += (e + pe) + fmaf(ah[i], bl[j], al[i] * bh[j]);
        }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) df_renorm(s[i][j], c[i][j]);
    __syncthreads();
  }
  double* out = Qsplit + ((size_t)ks * ntiles + tile) * (kGT * kGT);
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
      out[(ty * 4 + i) * kGT + tx * 4 + j] = (double)s[i][j] + (double)c[i][j];
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

// Largest split of the w columns gram_split may choose: >= 256 columns per split and at most
// about 12 CTAs per SM in total (a host-only bound, also used to size the partial tiles).
int gram_split_cap(int m, int w, int num_sms) {
  const int nt = (m + kGT - 1) / kGT;
  const int ntiles = nt * (nt + 1) / 2;
  int cap = (12 * num_sms + ntiles - 1) / ntiles;
  const int maxsplit = (w + 255) / 256;
  if (cap > maxsplit) cap = maxsplit;
  return cap < 1 ? 1 : cap;
}

// The split of the w columns.  At least enough splits for two CTAs per SM (while the cap
// allows); beyond that, the split with the least estimated time: every CTA has the same work,
// an SM works through its share of the CTAs at a steady rate, so the launch takes about
// ceil(ctas / SMs) x (columns per split + one k-chunk of per-CTA overhead).  At m = 1000,
// w = 4000 on 152 SMs: 10 splits (1360 CTAs, 9 per SM, 400 columns each) against 3 (408
// CTAs, 3 per SM on 104 SMs but 2 on the other 48, 1344 columns each).
int gram_split(int m, int w, int num_sms) {
  const int nt = (m + kGT - 1) / kGT;
  const int ntiles = nt * (nt + 1) / 2;
  const int cap = gram_split_cap(m, w, num_sms);
  int base = (2 * num_sms + ntiles - 1) / ntiles;
  if (base > cap) base = cap;
  if (base < 1) base = 1;
  auto cost = [&](int sp) {
    const int64_t per_sm = ((int64_t)ntiles * sp + num_sms - 1) / num_sms;
    const int64_t chunk = ((w + sp - 1) / sp + kGK - 1) / kGK * kGK;
    return per_sm * (chunk + kGK);
  };
  int best = base;
  for (int sp = base + 1; sp <= cap; ++sp)
    if (cost(sp) < cost(best)) best = sp;
  return best;
}

cudaError_t launch_split_df(const double* G, size_t count, float* Gdf, cudaStream_t st) {
  { note_launch(); k_split_df<<<2048, 256, 0, st>>>(G, count, Gdf, Gdf + count); }
  return cudaGetLastError();
}

cudaError_t launch_gram(const double* G, float* Gdf, int ldg, int m, int w, int mp, double* Q,
                        double* Qsplit, int split, cudaStream_t st) {
  const cudaError_t e = launch_split_df(G, (size_t)ldg * w, Gdf, st);
  if (e != cudaSuccess) return e;
  return launch_gram_df(Gdf, ldg, m, w, mp, Q, Qsplit, split, st);
}

// Gram product of a sketch already held as hi / lo float planes (2 ldg w floats).
cudaError_t launch_gram_df(const float* Gdf, int ldg, int m, int w, int mp, double* Q,
                           double* Qsplit, int split, cudaStream_t st) {
  const int nt = mp / kGT;
  const int ntiles = nt * (nt + 1) / 2;
  int chunk = (w + split - 1) / split;
  chunk = (chunk + kGK - 1) / kGK * kGK;
  const size_t count = (size_t)ldg * w;
  const float* Gh = Gdf;
  const float* Gl = Gdf + count;
  dim3 grid(ntiles, split);
  { note_launch(); k_gram_tile<<<grid, 256, 0, st>>>(Gh, Gl, ldg, m, w, chunk, Qsplit, ntiles); }
  { note_launch(); k_gram_finish<<<ntiles, 256, 0, st>>>(Qsplit, split, ntiles, m, mp, Q); }
  return cudaGetLastError();
}

// ---- products with a triangular double-float factor ---------------------------------------
//
// C = A B with A lower triangular (double-float planes, row-major) and B given by strides,
// in double-float arithmetic on the FP32 pipes: 64 x 64 tiles of C, 16-deep chunks of the
// inner index, the k range cut to where neither factor is structurally zero.  Used by the
// second factor stage below: G1 = X1 G (the sketch whitened by the first stage's inverse
// factor) and X = X2 X1 (the inverse factor of both stages together).
__global__ void __launch_bounds__(256) k_df_trmm(TrmmArgs a) {
  __shared__ __align__(16) float sAh[kGK][kGT + 4];
  __shared__ __align__(16) float sAl[kGK][kGT + 4];
  __shared__ __align__(16) float sBh[kGK][kGT + 4];
  __shared__ __align__(16) float sBl[kGK][kGT + 4];
  const int jb = blockIdx.x, ib = blockIdx.y;
  const int row0 = ib * kGT, col0 = jb * kGT;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  // A[i][k] = 0 for k > i; with b_lower, B[k][j] = 0 for k < j
  const int kend = min(a.K, row0 + kGT);
  const int kbeg = a.b_lower ? col0 : 0;
  const bool b_rowmajor = (a.sbj == 1);
  float s[4][4], c[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) s[i][j] = c[i][j] = 0.f;
  for (int k = kbeg; k < kend; k += kGK) {
#pragma unroll
    for (int l = 0; l < 4; ++l) {
      const int idx = tid + l * 256;
      {
        const int r = idx >> 4, kk = idx & 15;
        const int row = row0 + r, kx = k + kk;
        const bool v = row < a.M && kx < kend;
        const size_t ia = (size_t)row * a.lda + kx;
        sAh[kk][r] = v ? a.Ah[ia] : 0.f;
        sAl[kk][r] = v ? a.Al[ia] : 0.f;
      }
      {
        const int kk = b_rowmajor ? (idx >> 6) : (idx & 15);
        const int cc = b_rowmajor ? (idx & 63) : (idx >> 4);
        const int kx = k + kk, col = col0 + cc;
        const bool v = kx < kend && col < a.N;
        const size_t ibb = (size_t)kx * a.sbk + (size_t)col * a.sbj;
        sBh[kk][cc] = v ? a.Bh[ibb] : 0.f;
        sBl[kk][cc] = v ? a.Bl[ibb] : 0.f;
      }
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < kGK; ++kk) {
      float ah[4], al[4], bh[4], bl[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        ah[i] = sAh[kk][ty * 4 + i];
        al[i] = sAl[kk][ty * 4 + i];
        bh[i] = sBh[kk][tx * 4 + i];
        bl[i] = sBl[kk][tx * 4 + i];
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) df_mac(ah[i], al[i], bh[j], bl[j], s[i][j], c[i][j]);
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) df_renorm(s[i][j], c[i][j]);
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int row = row0 + ty * 4 + i, col = col0 + tx * 4 + j;
      if (row >= a.M || col >= a.N) continue;
      const size_t o = (size_t)row * a.sci + (size_t)col * a.scj;
      a.Ch[o] = s[i][j];
      a.Cl[o] = c[i][j];
      if (a.Th) {
        const size_t o2 = (size_t)row * a.sti + (size_t)col * a.stj;
        a.Th[o2] = s[i][j];
        a.Tl[o2] = c[i][j];
      }
    }
}

cudaError_t launch_df_trmm(const TrmmArgs& a, cudaStream_t st) {
  if (a.M < 1 || a.N < 1) return cudaSuccess;
  dim3 grid((a.N + kGT - 1) / kGT, (a.M + kGT - 1) / kGT);
  if (grid.y > 65535) return cudaErrorInvalidValue;
  { note_launch(); k_df_trmm<<<grid, 256, 0, st>>>(a); }
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

__device__ __forceinline__ void tri_decode(int idx, int& i, int& j) {
  i = 0;
  while ((i + 1) * (i + 2) / 2 <= idx) ++i;
  j = idx - i * (i + 1) / 2;
}

// ---- double-float tiles: the factorization keeps A/L, X = L^{-1} and M = Q^{-1} as pairs of
// float matrices (hi, lo); tile products run on the FP32 pipes (see dev_util.cuh).
struct DFTile {
  float h[kNB][kNB + 1];
  float l[kNB][kNB + 1];
};


__device__ __forceinline__ void load_df(DFTile& T, const float* h, const float* l, size_t off, int ld) {
  for (int e = threadIdx.x; e < kNB * kNB; e += blockDim.x) {
    const size_t a = off + (size_t)(e / kNB) * ld + e % kNB;
    T.h[e / kNB][e % kNB] = h[a];
    T.l[e / kNB][e % kNB] = l[a];
  }
}


// out[k] = sum_q A[r][q] * B(q, c) for the 4 elements e = tid + 256 k (r = e / 32, c = e % 32);
// TRB: B(q, c) = B[c][q] (A B^T), else B[q][c] (A B).  TRA: A(r, q) = A[q][r] (A^T B).
// The four sums are independent dependency chains; they advance together (q outermost) so
// that their latencies overlap.  Each sum still takes its terms in the order q = 0, 1, ...
template <bool TRA, bool TRB>
__device__ __forceinline__ void df_tile_mul(const DFTile& A, const DFTile& B, float (&s)[4],
                                            float (&c)[4]) {
  const int cc = threadIdx.x % kNB, r0 = threadIdx.x / kNB;   // rows r0 + 8 k
#pragma unroll
  for (int k = 0; k < 4; ++k) s[k] = c[k] = 0.f;
#pragma unroll 4
  for (int q = 0; q < kNB; ++q) {
    const float bh = TRB ? B.h[cc][q] : B.h[q][cc];
    const float bl = TRB ? B.l[cc][q] : B.l[q][cc];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int r = r0 + 8 * k;
      const float ah = TRA ? A.h[q][r] : A.h[r][q];
      const float al = TRA ? A.l[q][r] : A.l[r][q];
      df_mac(ah, al, bh, bl, s[k], c[k]);
    }
  }
}

// Factor and invert a diagonal block in double-float arithmetic: T (DF tile, SPD) is replaced
// by its Cholesky factor L (lower triangle) in place, X receives L^{-1}; both are written to
// global DF storage at offset off.  The caller has loaded T and synchronised.  A Schur pivot
// below 1e-14 of the original diagonal entry of Q (q0) counts as lost: returns false.
//
// The block is on the factorization's critical path (one per block step), so its dependency
// chains are kept short and every step does only the work that is live in it.  Pivot p updates
// a_ij -= a_ip a_jp / a_pp on the trailing triangle p < j <= i; enumerated row by row from its
// corner (p+1, p+1), that triangle is a prefix of one fixed enumeration of the kNB-1 sized
// triangle, so each thread keeps the same two slots for the whole sweep and a slot is live
// while its row index is inside the shrinking triangle.  1/a_pp comes from shared memory, and
// the thread of slot 0 (which always owns a_{p+1,p+1}) forms the next reciprocal from the value
// it just computed, before the one barrier of the step.  Column p is never touched after step p,
// so after the sweep the lower triangle holds the unscaled columns; square roots and the scaling
// into L happen afterwards for all columns at once.
// L^{-1} is built by recursive doubling: once the inverses X11, X22 of two neighbouring
// diagonal blocks of size b are known, the block below them is X21 = -X22 (L21 X11), and all
// pairs of one level are formed at once: log2(kNB) levels of two small products each, instead
// of kNB dependent rows.
__device__ bool diag_block(DFTile& T, float* Lh, float* Ll, float* Xh, float* Xl, size_t off, int mp,
                           const double* q0, DFTile& X) {
  static_assert(kNB == 32, "slot and level layout below assume 32 x 32 blocks and 256 threads");
  constexpr int kTri = (kNB - 1) * kNB / 2;   // trailing triangle of pivot 0
  __shared__ float rp_h[kNB], rp_l[kNB];   // 1 / (Schur pivot p)
  __shared__ float inv_h[kNB], inv_l[kNB]; // 1 / l_pp
  __shared__ float w_h[kNB * kNB / 4], w_l[kNB * kNB / 4];   // L21 X11 of one doubling level
  __shared__ int s_ok;
  const int tid = threadIdx.x;
  __shared__ float thr[kNB];                // lost-pivot threshold 1e-14 q0_p (FP32)
  // a lost pivot is replaced by |q0| to keep the arithmetic finite; the flag aborts the solve.
  // The test runs in FP32 (dh carries the pivot to 2^-24, far finer than 1e-14 q0 needs):
  // FP64 latency on this GPU would otherwise sit on every step of the chain.
  auto pivot_recip = [&](int p, float dh, float dl) {
    if (!(dh > thr[p]) || !isfinite(dh)) {
      s_ok = 0;
      dh = fmaxf(thr[p] * 1e14f, 1e-30f);
      dl = 0.f;
      T.h[p][p] = dh;
      T.l[p][p] = dl;
    }
    df_recip(dh, dl, rp_h[p], rp_l[p]);
  };
  if (tid < kNB) thr[tid] = (float)(1e-14 * fabs(q0[tid]));
  __syncthreads();
  if (tid == 0) {
    s_ok = 1;
    pivot_recip(0, T.h[0][0], T.l[0][0]);
  }
  // slot k of this thread: element tid + 256 k of the row-by-row triangle (row ti, column tj)
  int ti[2], tj[2];
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const int e = tid + 256 * k;
    if (e < kTri) {
      tri_decode(e, ti[k], tj[k]);
    } else {
      ti[k] = kNB;   // never live
      tj[k] = 0;
    }
  }
  __syncthreads();
  for (int p = 0; p + 1 < kNB; ++p) {
    const int live = kNB - 1 - p;   // rows of the trailing triangle
    const float rh = rp_h[p], rl = rp_l[p];
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      if (ti[k] < live) {
        const int i = p + 1 + ti[k], j = p + 1 + tj[k];
        float th, tl, h, l;
        df_mul(T.h[i][p], T.l[i][p], T.h[j][p], T.l[j][p], th, tl);
        df_mul(th, tl, rh, rl, h, l);
        float xh = T.h[i][j], xl = T.l[i][j];
        df_add(xh, xl, -h, -l);
        T.h[i][j] = xh;
        T.l[i][j] = xl;
        if (k == 0 && tid == 0) pivot_recip(p + 1, xh, xl);   // slot 0 of thread 0 is (p+1, p+1)
      }
    }
    __syncthreads();
  }
  // l_pp = sqrt(a_pp), 1 / l_pp for every column at once, then l_ip = a_ip / l_pp
  if (tid < kNB) {
    float lh, ll;
    df_sqrt(T.h[tid][tid], T.l[tid][tid], lh, ll);
    df_recip(lh, ll, inv_h[tid], inv_l[tid]);
    T.h[tid][tid] = lh;
    T.l[tid][tid] = ll;
  }
  __syncthreads();
  for (int e = tid; e < kNB * kNB; e += blockDim.x) {
    const int r = e / kNB, cc = e % kNB;
    if (cc < r) {
      float h, l;
      df_mul(T.h[r][cc], T.l[r][cc], inv_h[cc], inv_l[cc], h, l);
      T.h[r][cc] = h;
      T.l[r][cc] = l;
    } else if (cc > r) {
      T.h[r][cc] = 0.f;
      T.l[r][cc] = 0.f;
    }
    X.h[r][cc] = (cc == r) ? inv_h[r] : 0.f;
    X.l[r][cc] = (cc == r) ? inv_l[r] : 0.f;
  }
  __syncthreads();
  // X = L^{-1}: level b joins pairs of b x b diagonal blocks (s0 = 2b * pair); kNB b / 2 <= 256
  // elements per level, one per thread
  for (int b = 1; b < kNB; b <<= 1) {
    const int ne = kNB * b / 2;
    const int pair = tid / (b * b), rr = (tid % (b * b)) / b, cc = tid % b, s0 = 2 * b * pair;
    if (tid < ne) {   // W = L21 X11, X11 lower triangular: q >= cc
      float s = 0.f, c = 0.f;
      for (int q = cc; q < b; ++q)
        df_mac(T.h[s0 + b + rr][s0 + q], T.l[s0 + b + rr][s0 + q], X.h[s0 + q][s0 + cc],
               X.l[s0 + q][s0 + cc], s, c);
      fast_two_sum(s, c, w_h[tid], w_l[tid]);
    }
    __syncthreads();
    if (tid < ne) {   // X21 = -X22 W, X22 lower triangular: q <= rr
      float s = 0.f, c = 0.f;
      for (int q = 0; q <= rr; ++q)
        df_mac(X.h[s0 + b + rr][s0 + b + q], X.l[s0 + b + rr][s0 + b + q],
               w_h[pair * b * b + q * b + cc], w_l[pair * b * b + q * b + cc], s, c);
      float h, l;
      fast_two_sum(s, c, h, l);
      X.h[s0 + b + rr][s0 + cc] = -h;
      X.l[s0 + b + rr][s0 + cc] = -l;
    }
    __syncthreads();
  }
  for (int e = tid; e < kNB * kNB; e += blockDim.x) {
    const int r = e / kNB, cc = e % kNB;
    const size_t a = off + (size_t)r * mp + cc;
    Lh[a] = T.h[r][cc];
    Ll[a] = T.l[r][cc];
    Xh[a] = X.h[r][cc];
    Xl[a] = X.l[r][cc];
  }
  return s_ok != 0;
}

// Q (FP64, full) -> DF pairs of (Q + eps diag(Q)) in the A/L storage.
__global__ void k_q_to_df(const double* __restrict__ Q, int mp, int m, double eps,
                          float* __restrict__ Ah, float* __restrict__ Al) {
  const size_t total = (size_t)mp * mp;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total;
       i += (size_t)gridDim.x * blockDim.x) {
    double v = Q[i];
    const size_t r = i / mp, cc = i % mp;
    if (r == cc && (int)r < m) v *= (1.0 + eps);
    split_double_bits(v, Ah[i], Al[i]);
  }
}

__global__ void __launch_bounds__(256) k_ch_diag0(float* Ah, float* Al, float* Xh, float* Xl,
                                                  const double* __restrict__ Q0, int mp, int* fl) {
  __shared__ DFTile T;
  __shared__ DFTile XT;
  __shared__ double q0[kNB];
  if (fl[FL_BREAK]) return;
  load_df(T, Ah, Al, 0, mp);
  if (threadIdx.x < kNB) q0[threadIdx.x] = Q0[(size_t)threadIdx.x * mp + threadIdx.x];
  __syncthreads();
  const bool ok = diag_block(T, Ah, Al, Xh, Xl, 0, mp, q0, XT);
  if (!ok && threadIdx.x == 0) fl[FL_BREAK] = 1;
}

// grid: (nbk-kb-1) panel CTAs L_ik = A_ik X_kk^T, then kb row-scaling CTAs X_kj <- X_kk X_kj.
__global__ void __launch_bounds__(256) k_ch_panel(float* Ah, float* Al, float* Xh, float* Xl, int mp,
                                                  int nbk, int kb, const int* fl) {
  __shared__ DFTile S;
  __shared__ DFTile XK;
  if (fl[FL_BREAK]) return;
  const int npan = nbk - kb - 1;
  load_df(XK, Xh, Xl, (size_t)(kb * kNB) * mp + kb * kNB, mp);
  const bool panel = (int)blockIdx.x < npan;
  float* dh;
  float* dl;
  size_t off;
  if (panel) {
    off = (size_t)((kb + 1 + blockIdx.x) * kNB) * mp + kb * kNB;
    dh = Ah;
    dl = Al;
  } else {
    off = (size_t)(kb * kNB) * mp + (blockIdx.x - npan) * kNB;
    dh = Xh;
    dl = Xl;
  }
  load_df(S, dh, dl, off, mp);
  __syncthreads();
  float s[4], c[4];
  if (panel)
    df_tile_mul<false, true>(S, XK, s, c);    // A_ik X_kk^T
  else
    df_tile_mul<false, false>(XK, S, s, c);   // X_kk X_kj
  __syncthreads();
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int e = threadIdx.x + 256 * k;
    const size_t a = off + (size_t)(e / kNB) * mp + e % kNB;
    float h, l;
    fast_two_sum(s[k], c[k], h, l);
    dh[a] = h;
    dl[a] = l;
  }
}

// grid: r(r+1)/2 trailing Cholesky tiles (next diagonal block first), then r(kb+1) inverse tiles.
__global__ void __launch_bounds__(256) k_ch_update(float* Ah, float* Al, float* Xh, float* Xl,
                                                   const double* __restrict__ Q0, int mp, int nbk,
                                                   int kb, int* fl) {
  __shared__ DFTile S1;
  __shared__ DFTile S2;
  __shared__ double q0[kNB];
  if (fl[FL_BREAK]) return;
  const int r = nbk - kb - 1;
  const int n1 = r * (r + 1) / 2;
  int b = blockIdx.x;
  float* dh;
  float* dl;
  size_t off;
  float s[4], c[4];
  bool diag = false;
  int i;
  if (b < n1) {
    int ii, jj;
    tri_decode(b, ii, jj);   // index 0 is (0, 0): the next diagonal block first
    i = kb + 1 + ii;
    const int j = kb + 1 + jj;
    diag = (ii == 0 && jj == 0);
    off = (size_t)(i * kNB) * mp + j * kNB;
    dh = Ah;
    dl = Al;
    load_df(S1, Ah, Al, (size_t)(i * kNB) * mp + kb * kNB, mp);   // L_ik
    load_df(S2, Ah, Al, (size_t)(j * kNB) * mp + kb * kNB, mp);   // L_jk
    __syncthreads();
    df_tile_mul<false, true>(S1, S2, s, c);                      // L_ik L_jk^T
  } else {
    b -= n1;
    i = kb + 1 + b / (kb + 1);
    const int j = b % (kb + 1);
    off = (size_t)(i * kNB) * mp + j * kNB;
    dh = Xh;
    dl = Xl;
    load_df(S1, Ah, Al, (size_t)(i * kNB) * mp + kb * kNB, mp);   // L_ik
    load_df(S2, Xh, Xl, (size_t)(kb * kNB) * mp + j * kNB, mp);   // X_kj
    __syncthreads();
    df_tile_mul<false, false>(S1, S2, s, c);                     // L_ik X_kj
  }
  // tile <- tile - (s + c)
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int e = threadIdx.x + 256 * k;
    const size_t a = off + (size_t)(e / kNB) * mp + e % kNB;
    float h = dh[a], l = dl[a];
    df_add(h, l, -s[k], -c[k]);
    s[k] = h;
    c[k] = l;
  }
  if (!diag) {
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int e = threadIdx.x + 256 * k;
      const size_t a = off + (size_t)(e / kNB) * mp + e % kNB;
      dh[a] = s[k];
      dl[a] = c[k];
    }
    return;
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int e = threadIdx.x + 256 * k;
    S1.h[e / kNB][e % kNB] = s[k];
    S1.l[e / kNB][e % kNB] = c[k];
  }
  if (threadIdx.x < kNB) q0[threadIdx.x] = Q0[(size_t)(i * kNB + threadIdx.x) * mp + i * kNB + threadIdx.x];
  __syncthreads();
  const bool ok = diag_block(S1, Ah, Al, Xh, Xl, off, mp, q0, S2);
  if (!ok && threadIdx.x == 0) fl[FL_BREAK] = 1;
}

// ---- the same sweep as one launch of tile tasks ---------------------------------------------
//
// The block-step sweep above is bound by latency, not work: each of its nbk steps is two
// launches, and the update launch lasts as long as the pivot chain of the next diagonal block.
// Here the same tile operations are the tasks of one launch.  The sequential part, per block
// step k
//   L_{k,k-1} = A_{k,k-1} X_{k-1,k-1}^T,  A_kk -= L_{k,k-1} L_{k,k-1}^T,  factor and invert A_kk,
// is one task, F, that runs the whole chain in one CTA with X_{k-1,k-1} kept in shared memory.
// The other CTAs claim the remaining tasks from a counter in a fixed order
//   T(i,k)    L_ik = A_ik X_kk^T, i >= k + 2;
//   XS(k,j)   X_kj <- X_kk X_kj, j < k;
//   U(i,j,k)  A_ij -= L_ik L_jk^T, k < j <= i, except (k+1, k+1) which F does;
//   XU(i,j,k) X_ij -= L_ik X_kj, i > k >= j,
// listed block step after block step (S(0), S(1), ...; within S(k) in the order above, with
// U(k+2,k+1,k) and U(k+2,k+2,k), which F needs next, first).  Every tile has a counter of the
// operations done on it; a task waits (bounded by the global timer) until the counters of its
// inputs reach the values it needs, does its tile product and publishes its own counter.
// Counters (cA for A/L tiles, cX for X tiles, i >= j):
//   cA[i][j] = number of trailing updates applied (k of them before block step k = j), then
//              j + 1 once the tile is final (L_ij, or L_jj and X_jj);
//   cX[i][j] (i > j) = number of updates X_ij -= L_iq X_qj applied (q = j .. i-1), then
//              i - j + 1 once X_ij is final.
// Progress: F is claimed first.  A task of S(k) reads F's results up to step k + 1 and tasks
// listed before it; F's step j reads tasks of S(j - 2) and earlier.  So whenever F waits, the
// first unfinished task of the list has every input ready and is (or will be) claimed by a
// running CTA; whenever that task waits, F can advance.  The launch finishes whatever the
// number of resident CTAs (two or more).  F stays ahead: the two updates it needs at step j
// can start once step j - 1 has published L_{j-1,j-2}, a whole diagonal factor earlier.
// Each tile receives the same operations in the same order as in the block-step sweep, in the
// same arithmetic, so both routes give bitwise the same L and X.  A lost pivot is flagged as
// there; the sweep runs on with the replaced pivot (finite values) and the caller discards the
// result.
__device__ __forceinline__ int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_release(int* p, int v) {
  asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Thread 0: wait until *cnt >= target.  Gives up (false) when another task has flagged a
// timeout, or after limit_ns, flagging FL_TIMEOUT itself.
__device__ bool dag_wait(const int* cnt, int target, int* fl, uint64_t t0, uint64_t limit_ns) {
  for (unsigned spin = 0;; ++spin) {
    if (ld_acquire(cnt) >= target) return true;
    if ((spin & 15u) == 15u) {
      if (*(volatile int*)&fl[FL_TIMEOUT]) return false;
      if (global_ns() - t0 > limit_ns) {
        atomicExch(&fl[FL_TIMEOUT], 1);
        return false;
      }
    }
    if (spin >= 64) __nanosleep(64);
  }
}

// Tile loads through L2 only: a tile read earlier by this SM may have been rewritten since.
__device__ __forceinline__ void load_df_cg(DFTile& T, const float* h, const float* l, size_t off,
                                           int ld) {
  for (int e = threadIdx.x; e < kNB * kNB; e += blockDim.x) {
    const size_t a = off + (size_t)(e / kNB) * ld + e % kNB;
    T.h[e / kNB][e % kNB] = __ldcg(h + a);
    T.l[e / kNB][e % kNB] = __ldcg(l + a);
  }
}

// Makes the CTA's global writes visible, then sets *cnt = v (thread 0).
__device__ __forceinline__ void dag_publish(int* cnt, int v) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    st_release(cnt, v);
  }
}

__global__ void __launch_bounds__(256, 1) k_ch_dag(float* Ah, float* Al, float* Xh, float* Xl,
                                                const double* __restrict__ Q0, int mp, int nbk,
                                                const uint32_t* __restrict__ tasks, int ntasks,
                                                int* sync, int* fl, uint64_t limit_ns) {
  __shared__ DFTile S1;
  __shared__ DFTile S2;
  __shared__ double q0[kNB];
  __shared__ int s_task, s_ok;
  int* cA = sync + 2;
  int* cX = cA + (size_t)nbk * nbk;
  const int tid = threadIdx.x;
  auto tile = [&](int i, int j) { return (size_t)(i * kNB) * mp + j * kNB; };
  for (;;) {
    if (tid == 0) s_task = atomicAdd(&sync[0], 1);
    __syncthreads();
    const int t = s_task;
    if (t >= ntasks) break;
    const uint32_t code = tasks[t];
    const uint32_t kind = code >> 27;
    const int i = (code >> 18) & 511, j = (code >> 9) & 511, k = code & 511;
    if (tid == 0) {
      const uint64_t t0 = global_ns();
      bool ok = true;
      switch (kind) {
        case CT_F:   // waits inside, per block step
          break;
        case CT_T:
          ok = dag_wait(&cA[i * nbk + k], k, fl, t0, limit_ns) &&
               dag_wait(&cA[k * nbk + k], k + 1, fl, t0, limit_ns);
          break;
        case CT_U:
          ok = dag_wait(&cA[i * nbk + k], k + 1, fl, t0, limit_ns) &&
               dag_wait(&cA[j * nbk + k], k + 1, fl, t0, limit_ns) &&
               dag_wait(&cA[i * nbk + j], k, fl, t0, limit_ns);
          break;
        case CT_XS:
          ok = dag_wait(&cA[k * nbk + k], k + 1, fl, t0, limit_ns) &&
               dag_wait(&cX[k * nbk + j], k - j, fl, t0, limit_ns);
          break;
        default:   // CT_XU
          ok = dag_wait(&cA[i * nbk + k], k + 1, fl, t0, limit_ns) &&
               (j == k ? dag_wait(&cA[k * nbk + k], k + 1, fl, t0, limit_ns)
                       : dag_wait(&cX[k * nbk + j], k - j + 1, fl, t0, limit_ns)) &&
               dag_wait(&cX[i * nbk + j], k - j, fl, t0, limit_ns);
          break;
      }
      if (ok) __threadfence();
      s_ok = ok ? 1 : 0;
    }
    __syncthreads();
    if (!s_ok) break;   // a timeout: every other task gives up at its next wait
    float s[4], c[4];
    if (kind == CT_F) {
      // The critical chain, block step after block step in this CTA; X_{k-1,k-1} stays in S2.
      bool ok = true;
      for (int k = 0; k < nbk; ++k) {
        if (k > 0) {
          // the trailing updates of A_{k,k-1} and A_kk by steps 0 .. k-2 (other CTAs)
          if (tid == 0) {
            const uint64_t t0 = global_ns();
            const bool w = dag_wait(&cA[k * nbk + k - 1], k - 1, fl, t0, limit_ns) &&
                           dag_wait(&cA[k * nbk + k], k - 1, fl, t0, limit_ns);
            if (w) __threadfence();
            s_ok = w ? 1 : 0;
          }
          __syncthreads();
          if (!s_ok) {
            ok = false;
            break;
          }
          // L_{k,k-1} = A_{k,k-1} X_{k-1,k-1}^T, published before the diagonal work
          load_df_cg(S1, Ah, Al, tile(k, k - 1), mp);
          __syncthreads();
          df_tile_mul<false, true>(S1, S2, s, c);
          __syncthreads();
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const int e = tid + 256 * q;
            const size_t a = tile(k, k - 1) + (size_t)(e / kNB) * mp + e % kNB;
            float h, l;
            fast_two_sum(s[q], c[q], h, l);
            Ah[a] = h;
            Al[a] = l;
            S1.h[e / kNB][e % kNB] = h;
            S1.l[e / kNB][e % kNB] = l;
          }
          dag_publish(&cA[k * nbk + k - 1], k);
          df_tile_mul<false, true>(S1, S1, s, c);   // L L^T
          __syncthreads();
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const int e = tid + 256 * q;
            const size_t a = tile(k, k) + (size_t)(e / kNB) * mp + e % kNB;
            float h = __ldcg(Ah + a), l = __ldcg(Al + a);
            df_add(h, l, -s[q], -c[q]);
            S1.h[e / kNB][e % kNB] = h;
            S1.l[e / kNB][e % kNB] = l;
          }
        } else {
          load_df_cg(S1, Ah, Al, 0, mp);
        }
        if (tid < kNB) q0[tid] = Q0[(size_t)(k * kNB + tid) * mp + k * kNB + tid];
        __syncthreads();
        if (!diag_block(S1, Ah, Al, Xh, Xl, tile(k, k), mp, q0, S2) && tid == 0)
          atomicExch(&fl[FL_BREAK], 1);
        dag_publish(&cA[k * nbk + k], k + 1);
      }
      if (!ok) break;
      continue;
    }
    float* dh;
    float* dl;
    size_t off;
    bool acc;   // tile -= product, else tile = product
    int* cnt;
    int val;
    switch (kind) {
      case CT_T:   // L_ik = A_ik X_kk^T
        off = tile(i, k);
        load_df_cg(S1, Ah, Al, off, mp);
        load_df_cg(S2, Xh, Xl, tile(k, k), mp);
        __syncthreads();
        df_tile_mul<false, true>(S1, S2, s, c);
        dh = Ah, dl = Al, acc = false, cnt = &cA[i * nbk + k], val = k + 1;
        break;
      case CT_U:   // A_ij -= L_ik L_jk^T
        off = tile(i, j);
        load_df_cg(S1, Ah, Al, tile(i, k), mp);
        load_df_cg(S2, Ah, Al, tile(j, k), mp);
        __syncthreads();
        df_tile_mul<false, true>(S1, S2, s, c);
        dh = Ah, dl = Al, acc = true, cnt = &cA[i * nbk + j], val = k + 1;
        break;
      case CT_XS:   // X_kj <- X_kk X_kj
        off = tile(k, j);
        load_df_cg(S1, Xh, Xl, tile(k, k), mp);
        load_df_cg(S2, Xh, Xl, off, mp);
        __syncthreads();
        df_tile_mul<false, false>(S1, S2, s, c);
        dh = Xh, dl = Xl, acc = false, cnt = &cX[k * nbk + j], val = k - j + 1;
        break;
      default:   // CT_XU: X_ij -= L_ik X_kj
        off = tile(i, j);
        load_df_cg(S1, Ah, Al, tile(i, k), mp);
        load_df_cg(S2, Xh, Xl, tile(k, j), mp);
        __syncthreads();
        df_tile_mul<false, false>(S1, S2, s, c);
        dh = Xh, dl = Xl, acc = true, cnt = &cX[i * nbk + j], val = k - j + 1;
        break;
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int e = tid + 256 * q;
      const size_t a = off + (size_t)(e / kNB) * mp + e % kNB;
      float h, l;
      if (acc) {
        h = __ldcg(dh + a);
        l = __ldcg(dl + a);
        df_add(h, l, -s[q], -c[q]);
      } else {
        fast_two_sum(s[q], c[q], h, l);
      }
      dh[a] = h;
      dl[a] = l;
    }
    dag_publish(cnt, val);
  }
}

// M = X^T X (lower tiles, summed over block rows q >= i) stored as DF pairs (Mh, Ml), mirrored.
__global__ void __launch_bounds__(256) k_ch_xtx(const float* Xh, const float* Xl, float* Mh,
                                                float* Ml, int mp, int nbk, const int* fl) {
  __shared__ DFTile Xi;
  __shared__ DFTile Xj;
  if (fl[FL_BREAK]) return;
  int i, j;
  tri_decode(blockIdx.x, i, j);
  float s[4] = {0.f, 0.f, 0.f, 0.f}, c[4] = {0.f, 0.f, 0.f, 0.f};
  for (int q = i; q < nbk; ++q) {
    __syncthreads();
    load_df(Xi, Xh, Xl, (size_t)(q * kNB) * mp + i * kNB, mp);
    load_df(Xj, Xh, Xl, (size_t)(q * kNB) * mp + j * kNB, mp);
    __syncthreads();
    float s2[4], c2[4];
    df_tile_mul<true, false>(Xi, Xj, s2, c2);   // X_qi^T X_qj
#pragma unroll
    for (int k = 0; k < 4; ++k) df_add(s[k], c[k], s2[k], c2[k]);
  }
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int e = threadIdx.x + 256 * k, rr = e / kNB, cc = e % kNB;
    const size_t a = (size_t)(i * kNB + rr) * mp + j * kNB + cc;
    const size_t bsym = (size_t)(j * kNB + cc) * mp + i * kNB + rr;
    Mh[a] = s[k];
    Ml[a] = c[k];
    if (i != j) {
      Mh[bsym] = s[k];
      Ml[bsym] = c[k];
    }
  }
}

// (Mh + Ml) -> double, m x m with leading dimension ld (for lp_factor's output).
__global__ void k_df_to_double(const float* Mh, const float* Ml, int mp, int m, double* out, int ld) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < (size_t)m * m;
       i += (size_t)gridDim.x * blockDim.x) {
    const size_t r = i / m, cc = i % m;
    out[r * ld + cc] = (double)Mh[r * mp + cc] + (double)Ml[r * mp + cc];
  }
}

cudaError_t launch_df_to_double(const double* Mdf, int mp, int m, double* out, int ld,
                                cudaStream_t st) {
  const float* Mh = reinterpret_cast<const float*>(Mdf);
  { note_launch(); k_df_to_double<<<1024, 256, 0, st>>>(Mh, Mh + (size_t)mp * mp, mp, m, out, ld); }
  return cudaGetLastError();
}

// out_i += eps Q_ii v_i: turns Q v into (Q + eps diag Q) v for the factor's quality check.
__global__ void k_add_shift(double* out, const double* Q, int mp, int m, double eps, const double* v) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x)
    out[i] += eps * Q[(size_t)i * mp + i] * v[i];
}

cudaError_t launch_add_shift(double* out, const double* Q, int mp, int m, double eps,
                             const double* v, cudaStream_t st) {
  { note_launch(); k_add_shift<<<(m + 255) / 256, 256, 0, st>>>(out, Q, mp, m, eps, v); }
  return cudaGetLastError();
}

// Q (FP64, mp x mp) -> M = (Q + eps diag Q)^{-1} as DF pairs in M's storage (Mh = (float*)M,
// Ml = Mh + mp^2); X (same size) is work space for L^{-1}.
cudaError_t launch_chol_inverse(double* M, double* X, const double* Q0, int mp, int m, double eps,
                                int* fl, cudaStream_t st, bool form_m) {
  const int nbk = mp / kNB;
  const size_t mm = (size_t)mp * mp;
  float* Ah = reinterpret_cast<float*>(M);
  float* Al = Ah + mm;
  float* Xh = reinterpret_cast<float*>(X);
  float* Xl = Xh + mm;
  cudaError_t e = cudaMemsetAsync(X, 0, mm * sizeof(double), st);
  if (e != cudaSuccess) return e;
  { note_launch(); k_q_to_df<<<1024, 256, 0, st>>>(Q0, mp, m, eps, Ah, Al); }
  { note_launch(); k_ch_diag0<<<1, 256, 0, st>>>(Ah, Al, Xh, Xl, Q0, mp, fl); }
  for (int kb = 0; kb < nbk; ++kb) {
    const int r = nbk - kb - 1;
    const int npanel = r + kb;
    if (npanel > 0) { note_launch(); k_ch_panel<<<npanel, 256, 0, st>>>(Ah, Al, Xh, Xl, mp, nbk, kb, fl); }
    const int nupd = r * (r + 1) / 2 + r * (kb + 1);
    if (nupd > 0) { note_launch(); k_ch_update<<<nupd, 256, 0, st>>>(Ah, Al, Xh, Xl, Q0, mp, nbk, kb, fl); }
  }
  if (form_m) { note_launch(); k_ch_xtx<<<nbk * (nbk + 1) / 2, 256, 0, st>>>(Xh, Xl, Ah, Al, mp, nbk, fl); }
  return cudaGetLastError();
}

cudaError_t launch_chol_dag(double* M, double* X, const double* Q0, int mp, int m, double eps,
                            const uint32_t* tasks, int ntasks, int* sync, int num_sms, int* fl,
                            cudaStream_t st, bool form_m) {
  const int nbk = mp / kNB;
  const size_t mm = (size_t)mp * mp;
  float* Ah = reinterpret_cast<float*>(M);
  float* Al = Ah + mm;
  float* Xh = reinterpret_cast<float*>(X);
  float* Xl = Xh + mm;
  cudaError_t e = cudaMemsetAsync(X, 0, mm * sizeof(double), st);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(sync, 0, chol_dag_sync_words(nbk) * sizeof(int), st);
  if (e != cudaSuccess) return e;
  { note_launch(); k_q_to_df<<<1024, 256, 0, st>>>(Q0, mp, m, eps, Ah, Al); }
  const int grid = std::max(1, std::min(ntasks, num_sms * kDagCtasPerSm));
  { note_launch(); k_ch_dag<<<grid, 256, 0, st>>>(Ah, Al, Xh, Xl, Q0, mp, nbk, tasks, ntasks, sync, fl, kWaitLimitNs); }
  if (form_m) { note_launch(); k_ch_xtx<<<nbk * (nbk + 1) / 2, 256, 0, st>>>(Xh, Xl, Ah, Al, mp, nbk, fl); }
  return cudaGetLastError();
}

}  // namespace lpk
