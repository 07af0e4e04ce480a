// Column-tile passes over an FP32 column-major A with double-float accumulation: the FP64-class
// products of Alg. 2 step (b) (residuals and p) and of r~ = A D^2 A^T dy - p (Eq. addl)
// without FP64 arithmetic units, which are ~64x slower than FP32 ones on this GPU.
// Same structure as k_coltile.cu (warps own row slices, column tiles, transposing shuffle
// reduction, one barrier per tile); every sum is an unnormalised double-float pair.
#include <algorithm>

#include "dev_util.cuh"

namespace lpk {

template <int TILE>
__device__ __forceinline__ void df_transpose_reduce(float (&h)[TILE], float (&l)[TILE], int lane,
                                                    float& rh, float& rl) {
#pragma unroll
  for (int off = TILE / 2; off >= 1; off >>= 1) {
    const bool upper = (lane & off) != 0;
#pragma unroll
    for (int i = 0; i < off; ++i) {
      const float sh = upper ? h[i] : h[i + off];
      const float sl = upper ? l[i] : l[i + off];
      float kh = upper ? h[i + off] : h[i];
      float kl = upper ? l[i + off] : l[i];
      df_add(kh, kl, __shfl_xor_sync(kFull, sh, off), __shfl_xor_sync(kFull, sl, off));
      h[i] = kh;
      l[i] = kl;
    }
  }
  rh = h[0];
  rl = l[0];
#pragma unroll
  for (int off = TILE; off < 32; off <<= 1)
    df_add(rh, rl, __shfl_xor_sync(kFull, rh, off), __shfl_xor_sync(kFull, rl, off));
}

template <int SPW, int TILE, int MODE>
__global__ void __launch_bounds__(512) k_coltile_df(ColArgs a) {
  constexpr int VEC = 4;
  constexpr int NOUT = (MODE == MODE_RESID) ? 2 : 1;
  if (a.skip_if_done && a.fl[FL_DONE]) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  __shared__ float red_h[2][16][TILE];
  __shared__ float red_l[2][16][TILE];
  __shared__ float coef_h[NOUT][TILE];
  __shared__ float coef_l[NOUT][TILE];

  float vh[SPW][VEC], vl[SPW][VEC];
  float ys[NOUT][SPW][VEC], yc[NOUT][SPW][VEC];
  int rowb[SPW];
  bool rok[SPW];
#pragma unroll
  for (int sl = 0; sl < SPW; ++sl) {
    rowb[sl] = ((warp * SPW + sl) * 32 + lane) * VEC;
    rok[sl] = rowb[sl] < a.m;
#pragma unroll
    for (int e = 0; e < VEC; ++e) {
      const int row = rowb[sl] + e;
      double x = 0.0;
      if (rok[sl] && row < a.m) {
        if (a.dz) {   // fused CG direction update d = z + beta d_old
          x = fma(a.sc[SC_BETA], a.dold[row], a.dz[row]);
          if (blockIdx.x == 0) a.dnew[row] = x;
        } else {
          x = a.v[row];
        }
      }
      split_double(x, vh[sl][e], vl[sl][e]);
#pragma unroll
      for (int o = 0; o < NOUT; ++o) ys[o][sl][e] = yc[o][sl][e] = 0.f;
    }
  }
  double sigmu = 0.0;
  if constexpr (MODE == MODE_RESID) sigmu = a.sc[SC_SIGMU];

  const float* A = reinterpret_cast<const float*>(a.A);
  const int cl = lane % TILE;
  int it = 0;
  // software pipeline: the next tile's columns are loaded while the current one is computed
  uint4 an[TILE][SPW];
  auto load_tile = [&](int64_t tl, uint4 (&dst)[TILE][SPW]) {
#pragma unroll
    for (int c = 0; c < TILE; ++c) {
      const int64_t col = tl * TILE + c;
#pragma unroll
      for (int sl = 0; sl < SPW; ++sl)
        dst[c][sl] = (tl < a.ntiles && col < a.n && rok[sl]) ? ld_stream(A + col * a.lda + rowb[sl])
                                                             : make_uint4(0u, 0u, 0u, 0u);
    }
  };
  load_tile(blockIdx.x, an);
  for (int64_t tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x, ++it) {
    const int64_t col0 = tile * TILE;
    uint4 ar[TILE][SPW];
#pragma unroll
    for (int c = 0; c < TILE; ++c)
#pragma unroll
      for (int sl = 0; sl < SPW; ++sl) ar[c][sl] = an[c][sl];
    load_tile(tile + gridDim.x, an);
    const int64_t mycol = col0 + cl;
    const bool cok = mycol < a.n;
    double pc0 = 0.0, pc1 = 1.0, pc2 = 0.0;
    if (cok) {
      if constexpr (MODE == MODE_NORMAL) {
        pc0 = a.d2 ? a.d2[mycol] : 1.0;
      } else {
        pc0 = a.x[mycol];
        pc1 = a.s[mycol];
        pc2 = a.c[mycol];
      }
    }
    float dh[TILE], dl[TILE];
#pragma unroll
    for (int c = 0; c < TILE; ++c) {
      float s = 0.f, cc = 0.f;
#pragma unroll
      for (int sl = 0; sl < SPW; ++sl) {
        float av[VEC];
        unpack<float, float>(ar[c][sl], av);
#pragma unroll
        for (int e = 0; e < VEC; ++e) df_fma(av[e], vh[sl][e], vl[sl][e], s, cc);
      }
      dh[c] = s;
      dl[c] = cc;
    }
    float wh, wl;
    df_transpose_reduce<TILE>(dh, dl, lane, wh, wl);
    if (lane < TILE) {
      red_h[it & 1][warp][lane] = wh;
      red_l[it & 1][warp][lane] = wl;
    }
    __syncthreads();
    // per-column scalar work once per column, one column per warp: sum over warps, coefficients
    for (int cc = warp; cc < TILE; cc += nwarps) {
      float h = lane < nwarps ? red_h[it & 1][lane][cc] : 0.f;
      float l = lane < nwarps ? red_l[it & 1][lane][cc] : 0.f;
#pragma unroll
      for (int off = 16; off >= 1; off >>= 1)
        df_add(h, l, __shfl_xor_sync(kFull, h, off), __shfl_xor_sync(kFull, l, off));
      const double q0 = __shfl_sync(kFull, pc0, cc);
      const double q1 = __shfl_sync(kFull, pc1, cc);
      const double q2 = __shfl_sync(kFull, pc2, cc);
      if (lane == 0) {
        const int64_t col = col0 + cc;
        const bool ok = col < a.n;
        const double dot = (double)h + (double)l;
        double cf[NOUT];
        if constexpr (MODE == MODE_NORMAL) {
          cf[0] = ok ? q0 * dot : 0.0;
          if (a.colout && ok) a.colout[col] = dot;
        } else {
          const double rdv = dot + q1 - q2;
          cf[0] = ok ? q0 : 0.0;
          cf[1] = ok ? (sigmu + q0 * rdv) / q1 : 0.0;
          if (ok) a.colout[col] = rdv;
        }
#pragma unroll
        for (int o = 0; o < NOUT; ++o) split_double(cf[o], coef_h[o][cc], coef_l[o][cc]);
      }
    }
    __syncthreads();
    float ch[NOUT], cfl[NOUT];
#pragma unroll
    for (int o = 0; o < NOUT; ++o) {
      ch[o] = coef_h[o][cl];
      cfl[o] = coef_l[o][cl];
    }
#pragma unroll
    for (int c = 0; c < TILE; ++c) {
      float bh[NOUT], bl[NOUT];
#pragma unroll
      for (int o = 0; o < NOUT; ++o) {
        bh[o] = __shfl_sync(kFull, ch[o], c);
        bl[o] = __shfl_sync(kFull, cfl[o], c);
      }
#pragma unroll
      for (int sl = 0; sl < SPW; ++sl) {
        float av[VEC];
        unpack<float, float>(ar[c][sl], av);
#pragma unroll
        for (int o = 0; o < NOUT; ++o)
#pragma unroll
          for (int e = 0; e < VEC; ++e) df_fma(av[e], bh[o], bl[o], ys[o][sl][e], yc[o][sl][e]);
      }
    }
    // keep the compensation small relative to the running sum
#pragma unroll
    for (int o = 0; o < NOUT; ++o)
#pragma unroll
      for (int sl = 0; sl < SPW; ++sl)
#pragma unroll
        for (int e = 0; e < VEC; ++e) df_renorm(ys[o][sl][e], yc[o][sl][e]);
  }
  double* part = reinterpret_cast<double*>(a.part);
#pragma unroll
  for (int o = 0; o < NOUT; ++o)
#pragma unroll
    for (int sl = 0; sl < SPW; ++sl)
#pragma unroll
      for (int e = 0; e < VEC; ++e) {
        const int row = rowb[sl] + e;
        if (rok[sl] && row < a.m)
          part[((size_t)blockIdx.x * NOUT + o) * a.m + row] =
              (double)ys[o][sl][e] + (double)yc[o][sl][e];
      }
}

template <int MODE>
int launch_df_t(ColArgs a, int num_sms, cudaStream_t st) {
  constexpr int VEC = 4;
  const int nslices = (a.m + 32 * VEC - 1) / (32 * VEC);
  int spw = 1;
  while ((nslices + spw - 1) / spw > 16) spw *= 2;
  if (spw > 4) return -1;
  const int threads = ((nslices + spw - 1) / spw) * 32;
  const int tile = std::max(2, 8 / spw);
  a.ntiles = (a.n + tile - 1) / tile;
  void (*kern)(ColArgs) = nullptr;
  switch (spw) {
    case 1: kern = k_coltile_df<1, 8, MODE>; break;
    case 2: kern = k_coltile_df<2, 4, MODE>; break;
    default: kern = k_coltile_df<4, 2, MODE>; break;
  }
  int per_sm = occupancy_cached((const void*)kern, threads, 0);
  if (per_sm > 8) per_sm = 8;
  int64_t grid = (int64_t)num_sms * per_sm;
  if (grid > a.ntiles) grid = a.ntiles;
  if (grid < 1) grid = 1;
  { note_launch(); kern<<<(unsigned)grid, threads, 0, st>>>(a); }
  return (int)grid;
}

// FP32 A, FP64-class (double-float) accumulation; partials are doubles.  -1 if m is too large.
int launch_coltile_df(int mode, ColArgs a, int num_sms, cudaStream_t st) {
  return mode == MODE_RESID ? launch_df_t<MODE_RESID>(a, num_sms, st)
                            : launch_df_t<MODE_NORMAL>(a, num_sms, st);
}

}  // namespace lpk
