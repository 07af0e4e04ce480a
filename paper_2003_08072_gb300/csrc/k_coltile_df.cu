// Column-tile passes over an FP32 column-major A with double-float accumulation: the FP64-class
// products of Alg. 2 step (b) (residuals and p) and of r~ = A D^2 A^T dy - p (Eq. addl)
// without FP64 arithmetic units, which are ~64x slower than FP32 ones on this GPU.
// Same structure as k_coltile.cu (warps own row slices, column tiles, transposing shuffle
// reduction, one barrier per tile); every sum is an unnormalised double-float pair.
#include <algorithm>

#include "bulk_util.cuh"
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
      split_double_bits(x, vh[sl][e], vl[sl][e]);
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

// ---- one warp per column (m <= 1024) -------------------------------------------------------
// A warp owns whole columns: lane l holds rows 128 k + 4 l + e (k < NV, e < 4), so its dot with
// v is one butterfly of double-float sums inside the warp (every lane ends with the same total;
// no block barrier) and its share of the row sums touches only the lane's own accumulators.
// Each warp streams its columns (gw, gw + W, ... over the W warps of the grid) through a ring
// of S column slots in shared memory: lane 0 issues one bulk copy per column, S columns ahead,
// completing on the slot's mbarrier, and refills a slot once the whole warp is past its second
// read.  v sits in shared memory once per CTA as double-float pairs and the per-column scalars
// arrive as prepared double-float pairs, so the column loop runs on the FP32 pipes alone (the
// FP64 units of this GPU are ~64x slower).  At the end the warps of a CTA sum their row sums
// through shared memory (over the rings) and the CTA writes one partial, as the tiled kernel
// above does.  Every wait is bounded: a warp whose wait gives up sets FL_TIMEOUT, stops, and
// waits (bounded) for the copies it still has in flight before the CTA goes on.
template <int NV, int MODE, int NW, int S>
__global__ void __launch_bounds__(NW * 32, 1) k_colwarp_df(ColArgs a) {
  constexpr int NOUT = (MODE == MODE_RESID) ? 2 : 1;
  constexpr int R = 128 * NV;   // row slots of one column
  constexpr int C4 = R / 4;     // float4 per column slot
  static_assert(NOUT * 2 <= S, "the row-sum exchange reuses each warp's ring");
  if (a.skip_if_done && a.fl[FL_DONE]) return;
  extern __shared__ __align__(128) float4 dsm[];
  __shared__ uint64_t bars[NW * S];
  __shared__ int s_timeout;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  float4* svh = dsm;                                  // v, hi parts
  float4* svl = dsm + C4;                             // v, lo parts
  float4* ring = dsm + 2 * C4 + (size_t)warp * S * C4;
  const float* A = reinterpret_cast<const float*>(a.A);
  const int64_t gw = (int64_t)blockIdx.x * NW + warp;
  const int64_t W = (int64_t)gridDim.x * NW;
  const int my_cols = gw < a.n ? (int)((a.n - 1 - gw) / W) + 1 : 0;
  const unsigned bytes = (unsigned)(((a.m + 3) & ~3) * sizeof(float));   // lda >= m rounded to 4
  const uint64_t wait_ns = a.wait_ns ? a.wait_ns : kWaitLimitNs;
  auto issue = [&](int i) {   // lane 0: copy local column i into slot i % S
    uint64_t* bar = &bars[warp * S + i % S];
    mbar_arrive_expect_tx(bar, bytes);
    bulk_g2s(ring + (size_t)(i % S) * C4, A + (gw + (int64_t)i * W) * a.lda, bytes, bar);
  };
  if (tid == 0) {
    for (int i = 0; i < NW * S; ++i) mbar_init(&bars[i], 1);
    s_timeout = 0;
    fence_mbarrier_init();
  }
  {
    float* vh = reinterpret_cast<float*>(svh);
    float* vl = reinterpret_cast<float*>(svl);
    const double beta = a.dz ? a.sc[SC_BETA] : 0.0;
    for (int r = tid; r < R; r += blockDim.x) {
      double x = 0.0;
      if (r < a.m) {
        if (a.dz) {   // fused CG direction update d = z + beta d_old
          x = fma(beta, a.dold[r], a.dz[r]);
          if (blockIdx.x == 0) a.dnew[r] = x;
        } else {
          x = a.v[r];
        }
      }
      split_double_bits(x, vh[r], vl[r]);
    }
  }
  float smh = 0.f, sml = 0.f;   // RESID: sigma mu
  if constexpr (MODE == MODE_RESID) split_double(a.sc[SC_SIGMU], smh, sml);
  // the ring starts zeroed: a copy fills the first m rounded up to 4 rows of its slot (the
  // library's copy of A has zero padding rows), so every row slot a lane reads is A or zero
  for (int q = lane; q < S * C4; q += 32) ring[q] = make_float4(0.f, 0.f, 0.f, 0.f);
  __syncthreads();   // v staged, barriers initialised, rings zeroed
  if (lane == 0) {
    fence_proxy_async_smem();
    for (int i = 0; i < S && i < my_cols; ++i) issue(i);
  }

  float yh[NOUT][NV][4], yl[NOUT][NV][4];
#pragma unroll
  for (int o = 0; o < NOUT; ++o)
#pragma unroll
    for (int k = 0; k < NV; ++k)
#pragma unroll
      for (int e = 0; e < 4; ++e) yh[o][k][e] = yl[o][k][e] = 0.f;
  // float4 k of this lane: rows 128 k + 4 lane .. + 3 of the column (zero past the matrix)
  auto col4 = [&](const float4* slot, int k) -> float4 { return slot[32 * k + lane]; };
  auto renorm = [&]() {
#pragma unroll
    for (int o = 0; o < NOUT; ++o)
#pragma unroll
      for (int k = 0; k < NV; ++k)
#pragma unroll
        for (int e = 0; e < 4; ++e) df_renorm(yh[o][k][e], yl[o][k][e]);
  };
  int timeout_i = -1;
  for (int i = 0; i < my_cols; ++i) {
    const int slot_i = i % S;
    const bool ok = mbar_wait_bounded(&bars[warp * S + slot_i], (unsigned)((i / S) & 1), wait_ns);
    if (!__all_sync(kFull, ok)) {
      timeout_i = i;
      break;
    }
    const float4* slot = ring + (size_t)slot_i * C4;
    const int64_t col = gw + (int64_t)i * W;
    // t_j = a_j^T v: two interleaved double-float sums per lane, then the warp butterfly
    float s0 = 0.f, c0 = 0.f, s1 = 0.f, c1 = 0.f;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      const float4 av = col4(slot, k);
      const float4 xh = svh[32 * k + lane], xl = svl[32 * k + lane];
      df_fma(av.x, xh.x, xl.x, s0, c0);
      df_fma(av.y, xh.y, xl.y, s1, c1);
      df_fma(av.z, xh.z, xl.z, s0, c0);
      df_fma(av.w, xh.w, xl.w, s1, c1);
    }
    df_add(s0, c0, s1, c1);
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1)
      df_add(s0, c0, __shfl_xor_sync(kFull, s0, off), __shfl_xor_sync(kFull, c0, off));
    // coefficients of the column in the row sums
    float ch[NOUT], cl[NOUT];
    if constexpr (MODE == MODE_NORMAL) {
      if (a.d2df) {
        const float2 w = a.d2df[col];
        df_mul(s0, c0, w.x, w.y, ch[0], cl[0]);
      } else if (a.d2) {
        float wh, wl;
        split_double(a.d2[col], wh, wl);
        df_mul(s0, c0, wh, wl, ch[0], cl[0]);
      } else {
        fast_two_sum(s0, c0, ch[0], cl[0]);
      }
      if (a.colout && lane == 0) a.colout[col] = (double)s0 + (double)c0;
    } else {
      // (r_d)_j = t_j + (s_j - c_j) once, written out exactly (a normalised double-float pair
      // is a double), and the coefficient (sigma mu + x_j (r_d)_j) (1 / s_j) from that same
      // value: the right-hand side stays consistent with the r_d the step uses, whatever the
      // size of d2 (no division in the column loop)
      const float2 xv = a.xdf[col], is = a.isdf[col], scv = a.scdf[col];
      ch[0] = xv.x;
      cl[0] = xv.y;
      df_add(s0, c0, scv.x, scv.y);
      if (lane == 0) a.colout[col] = (double)s0 + (double)c0;
      float th, tl;
      df_mul(xv.x, xv.y, s0, c0, th, tl);
      df_add(th, tl, smh, sml);
      df_mul(th, tl, is.x, is.y, ch[1], cl[1]);
    }
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      const float4 av4 = col4(slot, k);
      const float av[4] = {av4.x, av4.y, av4.z, av4.w};
#pragma unroll
      for (int o = 0; o < NOUT; ++o)
#pragma unroll
        for (int e = 0; e < 4; ++e) df_fma(av[e], ch[o], cl[o], yh[o][k][e], yl[o][k][e]);
    }
    if ((i & 7) == 7) renorm();
    __syncwarp();   // the whole warp is past its reads of the slot
    if (lane == 0 && i + S < my_cols) {
      fence_proxy_async_smem();
      issue(i + S);
    }
  }
  renorm();
  if (timeout_i >= 0) {
    // columns timeout_i .. timeout_i + S - 1 were issued and not all waited for; nothing
    // after them was issued.  Let them land before the ring is reused or the CTA exits.
    if (lane == 0) {
      const int last = min(timeout_i + S - 1, my_cols - 1);
      for (int i = timeout_i; i <= last; ++i)
        mbar_wait_bounded(&bars[warp * S + i % S], (unsigned)((i / S) & 1), wait_ns);
      s_timeout = 1;
    }
    __syncwarp();
  }
  __syncthreads();   // every ring is idle
  if (s_timeout && tid == 0 && a.flw) a.flw[FL_TIMEOUT] = 1;
  // row sums of each warp into its own ring, then the CTA sum per row
  float4* rw = ring;
#pragma unroll
  for (int o = 0; o < NOUT; ++o)
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      rw[(2 * o) * C4 + 32 * k + lane] =
          make_float4(yh[o][k][0], yh[o][k][1], yh[o][k][2], yh[o][k][3]);
      rw[(2 * o + 1) * C4 + 32 * k + lane] =
          make_float4(yl[o][k][0], yl[o][k][1], yl[o][k][2], yl[o][k][3]);
    }
  __syncthreads();
  const float* rf = reinterpret_cast<const float*>(dsm + 2 * C4);
  double* part = reinterpret_cast<double*>(a.part);
  for (int idx = tid; idx < NOUT * R; idx += blockDim.x) {
    const int o = idx / R, r = idx % R;
    if (r >= a.m) continue;
    float h = 0.f, l = 0.f;
#pragma unroll 4
    for (int w = 0; w < NW; ++w) {
      const size_t base = ((size_t)w * S + 2 * o) * R;
      df_add(h, l, rf[base + r], rf[base + R + r]);
    }
    part[((size_t)blockIdx.x * NOUT + o) * a.m + r] = (double)h + (double)l;
  }
}

template <int NV, int MODE, int NW, int S>
int launch_colwarp(ColArgs a, int num_sms, cudaStream_t st) {
  const size_t smem = (size_t)(2 + NW * S) * 128 * NV * sizeof(float);
  void (*kern)(ColArgs) = k_colwarp_df<NV, MODE, NW, S>;
  if (ensure_dyn_smem((const void*)kern, smem) != cudaSuccess) return -1;
  int64_t grid = num_sms;   // one CTA per SM
  const int64_t need = (a.n + NW - 1) / NW;
  if (grid > need) grid = need;
  if (grid < 1) grid = 1;
  { note_launch(); kern<<<(unsigned)grid, NW * 32, smem, st>>>(a); }
  return (int)grid;
}

// Warp-per-column pass for m <= 1024 over an FP32 A whose leading dimension keeps columns
// 16-byte aligned (RESID needs the prepared column scalars); -1 otherwise.
template <int MODE>
int launch_colwarp_df(ColArgs a, int num_sms, cudaStream_t st) {
  if (a.m > 1024 || (a.lda & 3) != 0 || ((uintptr_t)a.A & 15) != 0) return -1;
  if (MODE == MODE_RESID && !(a.xdf && a.isdf && a.scdf)) return -1;
  // RESID keeps two sets of row sums (about 224 registers a thread at m <= 1024): 8 warps
  constexpr int NW = (MODE == MODE_RESID) ? 8 : 16;
  constexpr int S = (MODE == MODE_RESID) ? 4 : 3;
  if (a.m <= 256) return launch_colwarp<2, MODE, NW, S>(a, num_sms, st);
  if (a.m <= 512) return launch_colwarp<4, MODE, NW, S>(a, num_sms, st);
  return launch_colwarp<8, MODE, NW, S>(a, num_sms, st);
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
  const int g = mode == MODE_RESID ? launch_colwarp_df<MODE_RESID>(a, num_sms, st)
                                   : launch_colwarp_df<MODE_NORMAL>(a, num_sms, st);
  if (g >= 0) return g;
  return mode == MODE_RESID ? launch_df_t<MODE_RESID>(a, num_sms, st)
                            : launch_df_t<MODE_NORMAL>(a, num_sms, st);
}

}  // namespace lpk
