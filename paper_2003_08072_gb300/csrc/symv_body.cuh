// Preconditioner apply z = M r (M = Q^{-1}, full symmetric, row-major, leading dim mp),
// warp per row, r staged in shared memory; fused r^T z with CG bookkeeping.  Shared by the
// single launch (k_symv), the serving engine's batched launch and the persistent CG loop.
#pragma once

#include "dev_util.cuh"

namespace lpk {

// DF: M holds double-float pairs (Mh = (float*)M, Ml = Mh + mp^2) and the row sums run on the
// FP32 pipes; otherwise M is FP64.
// The body runs as block bid of a grid of nblk blocks (one row per warp: rows W bid .. W bid +
// W - 1 for W warps per block, 8 in the single and batched launches): the whole
// launch (k_symv) or one job's share of a batched launch (k_symv_batch).
template <bool DF>
__device__ __forceinline__ void symv_body(const SymvArgs& a, int bid, int nblk) {
  if ((a.mode == SYMV_CG_STEP || a.skip_done) && a.fl[FL_DONE]) return;
  extern __shared__ double rs[];
  const int m4 = (a.m + 3) & ~3;                      // rows of M are padded (mp >= m4)
  float* rh = reinterpret_cast<float*>(rs + m4);      // DF: r split into hi / lo floats
  float* rl = rh + m4;
  const double al = a.rold ? a.sc[SC_ALPHA] : 0.0;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int row = bid * (int)(blockDim.x >> 5) + warp;
  const int n4 = m4 >> 2;
  // DF: the first kPre chunks of this warp's row of M do not depend on the CG step, so they are
  // loaded before r is staged and their latency hides behind it
  constexpr int kPre = 8;
  float4 pmh[DF ? kPre : 1], pml[DF ? kPre : 1];
  const float4* Mh = nullptr;
  const float4* Ml = nullptr;
  if constexpr (DF) {
    Mh = reinterpret_cast<const float4*>(reinterpret_cast<const float*>(a.M) + (size_t)row * a.mp);
    Ml = reinterpret_cast<const float4*>(reinterpret_cast<const float*>(a.M) +
                                         (size_t)a.mp * a.mp + (size_t)row * a.mp);
#pragma unroll
    for (int k = 0; k < kPre; ++k) {
      const int j = lane + 32 * k;
      if (row < a.m && j < n4) {
        pmh[k] = __ldcg(Mh + j);
        pml[k] = __ldcg(Ml + j);
      } else {
        pmh[k] = make_float4(0.f, 0.f, 0.f, 0.f);
        pml[k] = pmh[k];
      }
    }
  }
  // a thread's loads of q and r_old are all issued before any of its stores
  constexpr int kU = 4;
  for (int base = threadIdx.x; base < m4; base += kU * blockDim.x) {
    double qv[kU], rv[kU];
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const int i = base + u * blockDim.x;
      qv[u] = 0.0;
      rv[u] = 0.0;
      if (i < a.m) {
        if (a.rold) {
          // with atomic copies the product's last CTA has already summed them into q
          qv[u] = a.q[i];
          rv[u] = a.rold[i];
        } else {
          rv[u] = a.r[i];
        }
      }
    }
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const int i = base + u * blockDim.x;
      if (i >= m4) continue;
      double v = rv[u];
      if (a.rold && i < a.m) {
        v = fma(-al, qv[u], rv[u]);
        if (bid == 0) {
          const_cast<double*>(a.r)[i] = v;
          a.dy[i] = fma(al, a.d[i], a.dy[i]);
          if (a.qzero)
#pragma unroll
            for (int k = 0; k < kQCopies; ++k) a.qzero[(size_t)k * a.m + i] = 0.0;
        }
      }
      rs[i] = v;
      if (DF) split_double_bits(v, rh[i], rl[i]);
    }
  }
  __syncthreads();
  double dotc = 0.0;
  if (row < a.m) {
    double acc;
    if constexpr (DF) {
      const float4* rh4 = reinterpret_cast<const float4*>(rh);
      const float4* rl4 = reinterpret_cast<const float4*>(rl);
      float s = 0.f, c = 0.f;
#pragma unroll
      for (int k = 0; k < kPre; ++k) {
        const int j = lane + 32 * k;
        if (j < n4) {
          const float4 mh = pmh[k], ml = pml[k];
          const float4 xh = rh4[j], xl = rl4[j];
          df_mac(mh.x, ml.x, xh.x, xl.x, s, c);
          df_mac(mh.y, ml.y, xh.y, xl.y, s, c);
          df_mac(mh.z, ml.z, xh.z, xl.z, s, c);
          df_mac(mh.w, ml.w, xh.w, xl.w, s, c);
        }
      }
#pragma unroll 8
      for (int j = lane + 32 * kPre; j < n4; j += 32) {
        const float4 mh = __ldcg(Mh + j), ml = __ldcg(Ml + j);
        const float4 xh = rh4[j], xl = rl4[j];
        df_mac(mh.x, ml.x, xh.x, xl.x, s, c);
        df_mac(mh.y, ml.y, xh.y, xl.y, s, c);
        df_mac(mh.z, ml.z, xh.z, xl.z, s, c);
        df_mac(mh.w, ml.w, xh.w, xl.w, s, c);
      }
#pragma unroll
      for (int off = 16; off >= 1; off >>= 1)
        df_add(s, c, __shfl_xor_sync(kFull, s, off), __shfl_xor_sync(kFull, c, off));
      acc = (double)s + (double)c;
    } else {
      const double* Mr = a.M + (size_t)row * a.mp;
      acc = 0.0;
      for (int j = lane; j < a.m; j += 32) acc = fma(Mr[j], rs[j], acc);
      acc = warp_sum(acc);
    }
    if (lane == 0) {
      a.z[row] = acc;
      dotc = a.sq ? acc * acc : acc * rs[row];
    }
  }
  if (a.mode == SYMV_PLAIN) return;
  double v[1] = {dotc};
  if (!grid_sum_last_b<1>(v, a.bpart, a.bcnt, bid, nblk) || threadIdx.x != 0) return;
  const double rho = v[0];
  if (a.mode == SYMV_F2) {
    a.sc[SC_F2] = rho;
    return;
  }
  if (!isfinite(rho)) {
    a.fl[FL_NUMERIC] = 1;
    a.fl[FL_DONE] = 1;
    return;
  }
  if (a.mode == SYMV_CG_INIT) {
    a.sc[SC_RHO] = rho;
    a.sc[SC_RHO0] = rho;
    const double rel = a.rel2 * rho;
    const double thr = a.sc[SC_THR2] < rel ? a.sc[SC_THR2] : rel;
    a.sc[SC_THR2] = thr;
    a.sc[SC_BETA] = 0.0;
    a.fl[FL_ITERS] = 0;
    a.fl[FL_DONE] = (rho <= thr || rho <= 0.0) ? 1 : 0;
  } else {
    const int it = a.fl[FL_ITERS] + 1;
    a.fl[FL_ITERS] = it;
    const bool rich = a.fl[FL_RICH] != 0;
    a.sc[SC_BETA] = rich ? 0.0 : rho / a.sc[SC_RHO];
    a.sc[SC_RHO] = rho;
    if (rho <= a.sc[SC_THR2] || it >= a.fl[FL_MAXIT]) a.fl[FL_DONE] = 1;
    if (rich && rho > 1e12 * a.sc[SC_RHO0]) {   // ||f|| grew 1e6-fold: the iteration diverges
      a.fl[FL_DIVERGED] = 1;
      a.fl[FL_DONE] = 1;
    }
  }
}

}  // namespace lpk
