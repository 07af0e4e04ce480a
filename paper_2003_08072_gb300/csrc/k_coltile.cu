// Dense column-tile passes over a column-major A (m x n, m << n).
//
// One pass streams A exactly once and, per column a_i, forms the dot a_i^T v and then
// accumulates a_i * coef_i into per-CTA row accumulators:
//   MODE_NORMAL : coef_i = d2_i (a_i^T v)       -> y = A D^2 A^T v  (Eq. normal; CG product
//                 of Alg. 1), optional t = A^T v (needed for ds, Eq. delshat)
//   MODE_RESID  : r_d,i = a_i^T y + s_i - c_i,  coef0_i = x_i, coef1_i = sigma mu/s_i + d2_i r_d,i
//                 -> A x and A g in the same pass, giving r_p = A x - b and
//                 p = b - A g (Alg. 2 step (b), Eq. update, Eq. pdef)
//
// Layout: A column-major with leading dimension lda (a multiple of 16 bytes), rows m..lda-1
// zero.  A warp owns SPW "slices" of 32 lanes x 16 bytes of rows; the CTA has enough warps to
// cover all m rows, so v and the row accumulators live in registers and every load of A is
// a coalesced 128-bit streaming load.  A CTA walks column tiles of TILE columns; the TILE
// partial dots of a warp are combined by a transposing shuffle reduction, then across warps
// through a double-buffered shared array (one __syncthreads per tile).
//
// Used for FP64 A (FP64 accumulation), the FP64 residual pass, the allocation-free entry point,
// and any shape the shared-memory staged CG product (k_cgprod.cu) does not cover; FP32 A with
// FP64-class accumulation goes to the double-float pass (k_coltile_df.cu).
#include <algorithm>

#include "dev_util.cuh"

namespace lpk {

template <typename TA, typename ACC, int SPW, int TILE, int MODE>
__global__ void __launch_bounds__(512) k_coltile(ColArgs a) {
  constexpr int VEC = VecN<TA>::N;
  constexpr int NOUT = (MODE == MODE_RESID) ? 2 : 1;
  if (a.skip_if_done && a.fl[FL_DONE]) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  __shared__ ACC red[2][16][TILE];

  ACC vr[SPW][VEC];
  ACC yr[NOUT][SPW][VEC];
  int rowb[SPW];
  bool rok[SPW];
  int tailv[SPW];   // rows of the slice's vector below m (VEC unless it straddles row m)
#pragma unroll
  for (int sl = 0; sl < SPW; ++sl) {
    rowb[sl] = ((warp * SPW + sl) * 32 + lane) * VEC;
    rok[sl] = rowb[sl] < a.m;
    tailv[sl] = min(VEC, a.m - rowb[sl]);
#pragma unroll
    for (int e = 0; e < VEC; ++e) {
      const int row = rowb[sl] + e;
      double vv = 0.0;
      if (rok[sl] && row < a.m) {
        if (a.dz) {   // fused CG direction update d = z + beta d_old
          vv = fma(a.sc[SC_BETA], a.dold[row], a.dz[row]);
          if (blockIdx.x == 0) a.dnew[row] = vv;
        } else {
          vv = a.v[row];
        }
      }
      vr[sl][e] = (ACC)vv;
#pragma unroll
      for (int o = 0; o < NOUT; ++o) yr[o][sl][e] = (ACC)0;
    }
  }
  double sigmu = 0.0;
  if constexpr (MODE == MODE_RESID) sigmu = a.sc[SC_SIGMU];

  const TA* A = reinterpret_cast<const TA*>(a.A);
  const int cl = lane % TILE;
  int it = 0;
  for (int64_t tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x, ++it) {
    const int64_t col0 = tile * TILE;
    uint4 ar[TILE][SPW];
#pragma unroll
    for (int c = 0; c < TILE; ++c) {
      const int64_t col = col0 + c;
#pragma unroll
      for (int sl = 0; sl < SPW; ++sl) {
        if (col < a.n && rok[sl]) {
          const uint4 r = ld_stream(A + col * a.lda + rowb[sl]);
          // the padding rows m..lda-1 of a caller's matrix may hold anything
          ar[c][sl] = tailv[sl] < VEC ? mask_tail<TA>(r, tailv[sl]) : r;
        } else {
          ar[c][sl] = make_uint4(0u, 0u, 0u, 0u);
        }
      }
    }
    // per-column operands for column col0 + (lane % TILE)
    const int64_t mycol = col0 + cl;
    const bool cok = mycol < a.n;
    double pc0 = 0.0, pc1 = 1.0, pc2 = 0.0;
    float pcf = 0.f;
    if (cok) {
      if constexpr (MODE == MODE_NORMAL) {
        if (std::is_same<ACC, float>::value && a.d2f)
          pcf = a.d2f[mycol];
        else
          pc0 = a.d2 ? a.d2[mycol] : 1.0;
      } else {
        pc0 = a.x[mycol];
        pc1 = a.s[mycol];
        pc2 = a.c[mycol];
      }
    }
    // column dots
    ACC pd[TILE];
#pragma unroll
    for (int c = 0; c < TILE; ++c) {
      ACC acc = (ACC)0;
#pragma unroll
      for (int sl = 0; sl < SPW; ++sl) {
        ACC av[VEC];
        unpack<TA, ACC>(ar[c][sl], av);
#pragma unroll
        for (int e = 0; e < VEC; ++e) acc = fma(av[e], vr[sl][e], acc);
      }
      pd[c] = acc;
    }
    const ACC wsum = warp_transpose_reduce<TILE, ACC>(pd, lane);
    if (lane < TILE) red[it & 1][warp][lane] = wsum;
    __syncthreads();
    ACC dot = (ACC)0;
    for (int wi = 0; wi < nwarps; ++wi) dot += red[it & 1][wi][cl];

    ACC cf[NOUT];
    if constexpr (MODE == MODE_NORMAL) {
      if (std::is_same<ACC, float>::value && a.d2f)
        cf[0] = cok ? (ACC)(pcf * (float)dot) : (ACC)0;   // FP32 weight: no FP64 work per column
      else
        cf[0] = cok ? (ACC)(pc0 * (double)dot) : (ACC)0;
      if (a.colout && warp == 0 && lane < TILE && cok) a.colout[mycol] = (double)dot;
    } else {
      const double rdv = (double)dot + pc1 - pc2;   // (A^T y + s - c)_i
      const double d2v = pc0 / pc1;                  // x_i / s_i
      cf[0] = cok ? (ACC)pc0 : (ACC)0;
      cf[1] = cok ? (ACC)(sigmu / pc1 + d2v * rdv) : (ACC)0;
      if (warp == 0 && lane < TILE && cok) a.colout[mycol] = rdv;
    }
    // row accumulation y += a_c * coef_c
#pragma unroll
    for (int c = 0; c < TILE; ++c) {
      ACC cc[NOUT];
#pragma unroll
      for (int o = 0; o < NOUT; ++o) cc[o] = __shfl_sync(kFull, cf[o], c);
#pragma unroll
      for (int sl = 0; sl < SPW; ++sl) {
        ACC av[VEC];
        unpack<TA, ACC>(ar[c][sl], av);
#pragma unroll
        for (int o = 0; o < NOUT; ++o)
#pragma unroll
          for (int e = 0; e < VEC; ++e) yr[o][sl][e] = fma(cc[o], av[e], yr[o][sl][e]);
      }
    }
  }
  if constexpr (MODE == MODE_NORMAL && std::is_same<ACC, float>::value) {
    if (a.qacc) {
      // kQCopies copies of q spread the atomic traffic over more L2 lines
      double* qc = a.qacc + (size_t)(blockIdx.x % kQCopies) * a.m;
#pragma unroll
      for (int sl = 0; sl < SPW; ++sl)
#pragma unroll
        for (int e = 0; e < VEC; ++e) {
          const int row = rowb[sl] + e;
          if (rok[sl] && row < a.m) atomicAdd(&qc[row], (double)yr[0][sl][e]);
        }
      // last CTA: d^T q and alpha (no waiting: the last CTA to arrive does the work)
      __shared__ bool s_last;
      __threadfence();
      __syncthreads();
      if (threadIdx.x == 0) s_last = (atomicAdd(a.cnt, 1u) == gridDim.x - 1);
      __syncthreads();
      if (!s_last) return;
      __threadfence();
      double dq[1] = {0.0};
      for (int i = threadIdx.x; i < a.m; i += blockDim.x) {
        double qi = 0.0;
#pragma unroll
        for (int k = 0; k < kQCopies; ++k) qi += __ldcg(&a.qacc[(size_t)k * a.m + i]);
        a.qsum[i] = qi;
        dq[0] += a.dnew[i] * qi;
      }
      block_sum<1>(dq);
      if (threadIdx.x == 0) {
        *a.cnt = 0u;
        set_cg_alpha(dq[0], a.scw, a.flw);
      }
      return;
    }
  }
  ACC* part = reinterpret_cast<ACC*>(a.part);
#pragma unroll
  for (int o = 0; o < NOUT; ++o)
#pragma unroll
    for (int sl = 0; sl < SPW; ++sl)
#pragma unroll
      for (int e = 0; e < VEC; ++e) {
        const int row = rowb[sl] + e;
        if (rok[sl] && row < a.m) part[((size_t)blockIdx.x * NOUT + o) * a.m + row] = yr[o][sl][e];
      }
}

namespace {

template <typename TA, typename ACC, int MODE>
int launch_t(ColArgs a, int num_sms, cudaStream_t st) {
  constexpr int VEC = VecN<TA>::N;
  const int nslices = (a.m + 32 * VEC - 1) / (32 * VEC);
  int spw = 1;
  while ((nslices + spw - 1) / spw > 16) spw *= 2;
  if (spw > 8) return -1;
  const int nwarps = (nslices + spw - 1) / spw;
  const int threads = nwarps * 32;
  // Registers: TILE x SPW 16-byte vectors of A plus 2 x SPW x VEC accumulators.  Types whose
  // unpacked vector is 32 bytes (bf16/f16 -> f32, f32 -> f64) get half the tile width.
  constexpr bool wide = VEC * sizeof(ACC) > 16;
  const int tile = std::max(2, (wide ? 8 : 16) / spw);
  a.ntiles = (a.n + tile - 1) / tile;
  void (*kern)(ColArgs) = nullptr;
  if constexpr (wide) {
    switch (spw) {
      case 1: kern = k_coltile<TA, ACC, 1, 8, MODE>; break;
      case 2: kern = k_coltile<TA, ACC, 2, 4, MODE>; break;
      case 4: kern = k_coltile<TA, ACC, 4, 2, MODE>; break;
      default: kern = k_coltile<TA, ACC, 8, 2, MODE>; break;
    }
  } else {
    switch (spw) {
      case 1: kern = k_coltile<TA, ACC, 1, 16, MODE>; break;
      case 2: kern = k_coltile<TA, ACC, 2, 8, MODE>; break;
      case 4: kern = k_coltile<TA, ACC, 4, 4, MODE>; break;
      default: kern = k_coltile<TA, ACC, 8, 2, MODE>; break;
    }
  }
  int per_sm = occupancy_cached((const void*)kern, threads, 0);
  if (per_sm > 8) per_sm = 8;
  int64_t grid = (int64_t)num_sms * per_sm;
  if (grid > a.ntiles) grid = a.ntiles;
  if (grid < 1) grid = 1;
  { note_launch(); kern<<<(unsigned)grid, threads, 0, st>>>(a); }
  return (int)grid;
}

}  // namespace

// Largest number of CTAs a column-tile pass may use (sizes the partial buffer).
int coltile_max_grid(int num_sms) { return num_sms * 8; }

int launch_coltile_df(int mode, ColArgs a, int num_sms, cudaStream_t st);   // k_coltile_df.cu

int launch_coltile(lp_dtype ta, bool acc_f64, int mode, ColArgs a, int num_sms, cudaStream_t st) {
  // FP32 A with FP64-class accumulation runs on the FP32 pipes in double-float arithmetic
  // (k_coltile_df.cu); the FP64-unit kernel remains for shapes beyond its register budget.
  if (ta == LP_F32 && acc_f64) {
    const int g = launch_coltile_df(mode, a, num_sms, st);
    if (g >= 0) return g;
  }
  if (mode == MODE_NORMAL) {
    switch (ta) {
      case LP_F64: return launch_t<double, double, MODE_NORMAL>(a, num_sms, st);
      case LP_F32:
        return acc_f64 ? launch_t<float, double, MODE_NORMAL>(a, num_sms, st)
                       : launch_t<float, float, MODE_NORMAL>(a, num_sms, st);
      case LP_BF16: return launch_t<__nv_bfloat16, float, MODE_NORMAL>(a, num_sms, st);
      case LP_F16: return launch_t<__half, float, MODE_NORMAL>(a, num_sms, st);
    }
  } else {
    switch (ta) {
      case LP_F64: return launch_t<double, double, MODE_RESID>(a, num_sms, st);
      case LP_F32: return launch_t<float, double, MODE_RESID>(a, num_sms, st);
      default: return -1;
    }
  }
  return -1;
}

}  // namespace lpk

namespace lpk {

// Same kernel selection as launch_coltile (MODE_NORMAL, accumulator of the streamed type) with
// the grid limited to max_grid CTAs, for callers whose partial buffer has a fixed capacity.
namespace {
template <typename TA, typename ACC>
int launch_capped_t(ColArgs a, int num_sms, int max_grid, cudaStream_t st) {
  constexpr int VEC = VecN<TA>::N;
  const int nslices = (a.m + 32 * VEC - 1) / (32 * VEC);
  int spw = 1;
  while ((nslices + spw - 1) / spw > 16) spw *= 2;
  if (spw > 8) return -1;
  const int threads = ((nslices + spw - 1) / spw) * 32;
  constexpr bool wide = VEC * sizeof(ACC) > 16;
  const int tile = std::max(2, (wide ? 8 : 16) / spw);
  a.ntiles = (a.n + tile - 1) / tile;
  void (*kern)(ColArgs) = nullptr;
  if constexpr (wide) {
    switch (spw) {
      case 1: kern = k_coltile<TA, ACC, 1, 8, MODE_NORMAL>; break;
      case 2: kern = k_coltile<TA, ACC, 2, 4, MODE_NORMAL>; break;
      case 4: kern = k_coltile<TA, ACC, 4, 2, MODE_NORMAL>; break;
      default: kern = k_coltile<TA, ACC, 8, 2, MODE_NORMAL>; break;
    }
  } else {
    switch (spw) {
      case 1: kern = k_coltile<TA, ACC, 1, 16, MODE_NORMAL>; break;
      case 2: kern = k_coltile<TA, ACC, 2, 8, MODE_NORMAL>; break;
      case 4: kern = k_coltile<TA, ACC, 4, 4, MODE_NORMAL>; break;
      default: kern = k_coltile<TA, ACC, 8, 2, MODE_NORMAL>; break;
    }
  }
  int per_sm = occupancy_cached((const void*)kern, threads, 0);
  if (per_sm > 8) per_sm = 8;
  int64_t grid = (int64_t)num_sms * per_sm;
  if (grid > max_grid) grid = max_grid;
  if (grid > a.ntiles) grid = a.ntiles;
  if (grid < 1) grid = 1;
  { note_launch(); kern<<<(unsigned)grid, threads, 0, st>>>(a); }
  return (int)grid;
}
}  // namespace

int launch_coltile_capped(lp_dtype ta, ColArgs a, int num_sms, int max_grid, cudaStream_t st) {
  switch (ta) {
    case LP_F64: return launch_capped_t<double, double>(a, num_sms, max_grid, st);
    case LP_F32: return launch_capped_t<float, float>(a, num_sms, max_grid, st);
    case LP_BF16: return launch_capped_t<__nv_bfloat16, float>(a, num_sms, max_grid, st);
    case LP_F16: return launch_capped_t<__half, float>(a, num_sms, max_grid, st);
  }
  return -1;
}

}  // namespace lpk
