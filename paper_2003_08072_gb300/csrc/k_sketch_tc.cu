// Gaussian sketch G = A D W (Sec. 5; the sketch of the paper's experiments, Sec. 6) on the
// tensor cores, exact to the double-float accuracy of the entries of A D.
//
// The entries of W are integers over a common scale, W_kc = q_kc / (2^8 sqrt(w)) with
// |q_kc| <= 1026 (the quantile grid of gauss_grid.h), so q splits exactly into two signed 6-bit
// digits, q = 64 E_0 + E_1 (|E_0| <= 16, |E_1| <= 32).  Row i of A D is scaled by 2^-e_i
// (max_k |A_ik d_k| < 2^e_i) and each scaled entry x = A_ik d_k 2^-e_i in (-1, 1), formed in
// double-float, is written as nine signed 6-bit digits, x = sum_{s<9} D_s 2^(-6(s+1)) + r,
// |D_0| <= 64, |D_s| <= 33, |r| <= 2^-55 (the split of the tensor-core Gram product, after
// Ozaki, Ogita, Oishi & Rump 2012).  Then
//     G_ic = 2^(e_i - 8) / sqrt(w) sum_{l<9} 2^(-6 l) L_l[c][i],
//     L_l = sum_{s+t=l} E_t D_s^T   (t < 2, s < 9; the pair s = 8, t = 1, of weight 2^-54, is
// dropped).  Each L_l is a sum of integer products, at most 64 * 32 + 33 * 16 = 2576 per
// column of A and level, so over a chunk of 4096 columns of A every partial sum stays below
// 2^24 and FP32 accumulation in the tensor core is exact.  The level sums of a chunk are folded
// into double-float per thread.
//
// Layout.  Both digit arrays are written tile by tile in the order the tensor core reads them:
// W as [I][kb][slice][16 row groups][2][8][8], A D as [J][kb][slice][4 row groups][2][8][8]
// (I, J the tiles of 128 sketch columns and of 32 rows of A, kb the blocks of 16 columns of A,
// an 8-row group's two core matrices of 8 rows x 16 bytes), so the digits of one tile for
// four consecutive k blocks are one contiguous range: a pipeline stage is two bulk copies
// (32 KB of W, 36 KB of A D).  The tensor core's M side is W (a tile of 128 sketch columns c,
// two slices), its N side A D (a tile of 32 rows i, nine
// slices one after another), so one MMA of W slice t with the D slices s0 .. s1 writes the
// level accumulators t + s0 .. t + s1, which lie side by side in tensor memory (level l at
// columns 32 l).  Per k block: E_0 x D_0..7 (levels 0-7, N = 256), E_0 x D_8 (level 8, N = 32),
// E_1 x D_0..7 (levels 1-8, N = 256); the first two of a chunk's first k block overwrite, every
// other product accumulates.
//
// k_sketch_tc: one CTA per (128 x 32 tile of G^T, range of column chunks), 160 threads, one CTA
// per SM (204 KB of shared memory in 3 stages, 512 tensor-memory columns).  Warp 4 (lane 0) issues the
// bulk copies of each stage (completing on its full mbarrier); warp 0 (lane 0) issues the
// products and commits them to the stage's empty mbarrier; at the end of each chunk warps 0-3
// read the accumulators back (thread t owns sketch column 128 I + t) and add them into
// double-float registers.  Every mbarrier wait is bounded by the global timer (1 s); a wait
// that gives up sets FL_TIMEOUT, the copies already issued are waited for (again bounded) and
// the CTA still frees its tensor memory.  G^T tile rows are G's columns, so the partial tiles
// are stored, and G written, column-major as the rest of the solver keeps it.
#include <algorithm>

#include "dev_util.cuh"
#include "tc_util.cuh"

namespace lpk {

namespace {

constexpr int kTM = 128;                          // sketch columns per tile (TMEM lanes)
constexpr int kTI = 32;                           // rows of A per tile
constexpr int kKB = 16;                           // columns of A per k block (one MMA K step)
constexpr int kSA = 9;                            // digit slices of A D
constexpr int kSW = 2;                            // digit slices of W
constexpr int kKC = 4096;                         // columns of A per exactly accumulated chunk
constexpr int kSK = 4;                            // k blocks per pipeline stage
constexpr int kNS = 3;                            // pipeline stages
constexpr int kWSlice = (kTM / 8) * tc::kCore;    // 4 KB: one slice of the W tile
constexpr int kASlice = (kTI / 8) * tc::kCore;    // 1 KB: one slice of the A D tile
constexpr int kWBytes = kSW * kWSlice;            // 8 KB
constexpr int kABytes = kSA * kASlice;            // 9 KB
constexpr int kStageW = kSK * kWBytes;            // 32 KB: the stage's W digits
constexpr int kStage = kStageW + kSK * kABytes;   // 68 KB: then its A D digits
constexpr int kSmemBytes = kNS * kStage + 256;    // stages, mbarriers, TMEM address
constexpr int kRowAlign = kTI;                    // rows of the A D digits: whole tiles

__device__ __forceinline__ uint64_t sm64(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
  const __nv_bfloat16 x = __float2bfloat16_rn(a), y = __float2bfloat16_rn(b);
  return (uint32_t)__bfloat16_as_ushort(x) | ((uint32_t)__bfloat16_as_ushort(y) << 16);
}

}  // namespace

// ---- digits of W ---------------------------------------------------------------------------
// Item (kb, row group g, half hk, row r8) writes the 8 digit pairs of sketch column c = 8 g +
// r8 at columns k = 16 kb + 8 hk .. + 7 of A, as one 16-byte store per slice; consecutive
// threads take consecutive r8, then hk, so a warp writes 512 contiguous bytes per slice.
// Entry (k, c) of W is q[h >> 50] with h = SplitMix64(key ^ (k w + c)), as in k_gauss.cu.
__global__ void __launch_bounds__(256) k_w_digits(uint64_t key, int64_t n, int w, int ngw,
                                                  int64_t nkb, const int16_t* __restrict__ gq,
                                                  __nv_bfloat16* __restrict__ Wd) {
  const int64_t per_kb = (int64_t)ngw * 16;
  const int64_t total = nkb * per_kb;
  for (int64_t it = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; it < total;
       it += (int64_t)gridDim.x * blockDim.x) {
    const int64_t kb = it / per_kb;
    const int rem = (int)(it - kb * per_kb);
    const int r8 = rem & 7, hk = (rem >> 3) & 1, g = rem >> 4;
    const int c = g * 8 + r8;
    const int64_t k0 = kb * kKB + hk * 8;
    float e0[8], e1[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const int64_t k = k0 + e;
      int q = 0;
      if (c < w && k < n) q = __ldg(gq + (sm64(key ^ ((uint64_t)k * (uint64_t)w + (uint64_t)c)) >> 50));
      const int d0 = (q + 32) >> 6;   // floor((q + 32) / 64): q = 64 d0 + d1, -32 <= d1 < 32
      e0[e] = (float)d0;
      e1[e] = (float)(q - 64 * d0);
    }
    const size_t base =
        ((((size_t)(g >> 4) * nkb + kb) * kSW * 16 + (g & 15)) * 2 + hk) * 64 + r8 * 8;
    const size_t sstep = 16 * 128;   // elements of one slice of a tile's k block
    uint4 v0, v1;
    v0.x = pack_bf16(e0[0], e0[1]);
    v0.y = pack_bf16(e0[2], e0[3]);
    v0.z = pack_bf16(e0[4], e0[5]);
    v0.w = pack_bf16(e0[6], e0[7]);
    v1.x = pack_bf16(e1[0], e1[1]);
    v1.y = pack_bf16(e1[2], e1[3]);
    v1.z = pack_bf16(e1[4], e1[5]);
    v1.w = pack_bf16(e1[6], e1[7]);
    *reinterpret_cast<uint4*>(Wd + base) = v0;
    *reinterpret_cast<uint4*>(Wd + base + sstep) = v1;
  }
}

// ---- row exponents of A D ------------------------------------------------------------------
// ex[i] (zeroed before) <- max_k |A_ik d_k| as float bits (an integer atomic max orders
// non-negative floats like their values); columns spread over blockIdx.y.  The product is
// taken in FP32: an exponent one too small leaves |x| below 1 + 2^-22, whose leading digit is
// still at most 64.
template <typename TA>
__global__ void k_ad_row_max(const TA* __restrict__ A, int64_t lda, int m, int64_t n,
                             const double* __restrict__ d, int* __restrict__ ex) {
  __shared__ float red[8][33];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int row = blockIdx.x * 32 + tx;
  const int64_t per = (n + gridDim.y - 1) / gridDim.y;
  const int64_t k0 = blockIdx.y * per, k1 = min(n, k0 + per);
  float mx = 0.f;
  if (row < m)
    for (int64_t k = k0 + ty; k < k1; k += 8)
      mx = fmaxf(mx, fabsf((float)A[k * lda + row] * (float)d[k]));
  red[ty][tx] = mx;
  __syncthreads();
  if (ty == 0 && row < m) {
#pragma unroll
    for (int j = 1; j < 8; ++j) mx = fmaxf(mx, red[j][tx]);
    if (mx > 0.f) atomicMax(&ex[row], __float_as_int(mx));
  }
}

// ex[i] <- e_i with max_k |A_ik d_k| < 2^e_i (0 for a zero row and for padding rows)
__global__ void k_ad_row_exp(int m, int rows_p, int* __restrict__ ex) {
  const int row = blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= rows_p) return;
  const float mx = __int_as_float(ex[row]);
  int e = 0;
  if (row < m && mx > 0.f) frexpf(mx, &e);
  ex[row] = row < m ? max(e, -125) : 0;   // 2^-e stays a normal float
}

// ---- digits of A D -------------------------------------------------------------------------
// Item (kb, row group g, half hk, row r8): row i = 8 g + r8 at columns k = 16 kb + 8 hk .. + 7,
// nine 16-byte stores (one per slice), zero outside m x n.  x = A_ik d_k 2^-e_i in double-float
// (FP32 A: the product with the split of d_k, exact to 2^-48; FP64 A: the FP64 product, then
// split), then D_s = rint(64 x_s), x_{s+1} = 64 x_s - D_s.
template <typename TA>
__global__ void __launch_bounds__(256) k_ad_digits(const TA* __restrict__ A, int64_t lda, int m,
                                                   int64_t n, const double* __restrict__ d,
                                                   const int* __restrict__ ex, int ngm, int64_t nkb,
                                                   __nv_bfloat16* __restrict__ Dd) {
  const int64_t per_kb = (int64_t)ngm * 16;
  const int64_t total = nkb * per_kb;
  for (int64_t it = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; it < total;
       it += (int64_t)gridDim.x * blockDim.x) {
    const int64_t kb = it / per_kb;
    const int rem = (int)(it - kb * per_kb);
    const int r8 = rem & 7, hk = (rem >> 3) & 1, g = rem >> 4;
    const int i = g * 8 + r8;
    const int64_t k0 = kb * kKB + hk * 8;
    float rh[8], rl[8];
    const float sc = (i < m) ? __int_as_float((127 - ex[i]) << 23) : 0.f;   // 2^-e_i
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const int64_t k = k0 + e;
      float h = 0.f, l = 0.f;
      if (i < m && k < n) {
        if constexpr (sizeof(TA) == 4) {
          const float a = (float)A[k * lda + i];
          float dh, dl;
          split_double_bits(d[k], dh, dl);
          const float p = __fmul_rn(a, dh);
          const float pe = fmaf(a, dh, -p);
          fast_two_sum(p, pe + a * dl, h, l);
        } else {
          split_double_bits((double)A[k * lda + i] * d[k], h, l);
        }
      }
      rh[e] = h * sc;   // exact scalings by a power of two
      rl[e] = l * sc;
    }
    const size_t base =
        ((((size_t)(g >> 2) * nkb + kb) * kSA * 4 + (g & 3)) * 2 + hk) * 64 + r8 * 8;
    const size_t sstep = 4 * 128;   // elements of one slice of a tile's k block
#pragma unroll
    for (int s = 0; s < kSA; ++s) {
      float dg[8];
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const float th = rh[e] * 64.f, tl = rl[e] * 64.f;   // exact scalings
        dg[e] = rintf(th + tl);
        rh[e] = th - dg[e];                                // exact: |th - d| < 1 + |tl|
        rl[e] = tl;
      }
      uint4 v;
      v.x = pack_bf16(dg[0], dg[1]);
      v.y = pack_bf16(dg[2], dg[3]);
      v.z = pack_bf16(dg[4], dg[5]);
      v.w = pack_bf16(dg[6], dg[7]);
      *reinterpret_cast<uint4*>(Dd + base + s * sstep) = v;
    }
  }
}

// ---- the product ---------------------------------------------------------------------------
struct SketchTcArgs {
  const __nv_bfloat16* Wd;   // W digits, [I][kb][2][16][2][8][8]
  const __nv_bfloat16* Dd;   // A D digits, [J][kb][9][4][2][8][8]
  int64_t nkb;               // k blocks of 16 columns of A (a multiple of kSK)
  int NJ;                    // tiles along the rows of A (tile = I NJ + J)
  int ntile;
  int chunks_per_cta;        // chunks of kKC columns per CTA (blockIdx.y selects the range)
  float2* part;              // [gridDim.y][ntile][128][32] double-float partial tiles of G^T
  int* fl;
};

__device__ __forceinline__ void fold_sync() {   // warps 0-3 only (the TMEM lanes' owners)
  asm volatile("bar.sync 1, 128;" ::: "memory");
}

__global__ void __launch_bounds__(160, 1) k_sketch_tc(SketchTcArgs a) {
  extern __shared__ __align__(1024) unsigned char smem[];
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + kNS * kStage);
  uint64_t* empty = full + kNS;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + kNS * kStage + 192);
  // s_pfail: the producer gave up; s_gfail: a thread of warps 0-3 gave up (read by them only
  // after a barrier of theirs, so that all four take the same branch)
  __shared__ int s_pfail, s_gfail, s_issued, s_consumed;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int tile = blockIdx.x, I = tile / a.NJ, J = tile % a.NJ;
  constexpr int kb_per_chunk = kKC / kKB;
  const int64_t kb0 = (int64_t)blockIdx.y * a.chunks_per_cta * kb_per_chunk;
  const int64_t kb1 = min(a.nkb, kb0 + (int64_t)a.chunks_per_cta * kb_per_chunk);
  float2* out = a.part + (((size_t)blockIdx.y * a.ntile + tile) * kTM + tid) * kTI;
  if (kb0 >= kb1) {   // an empty column range: its partial tile is zero
    if (tid < kTM)
      for (int c = 0; c < kTI; ++c) out[c] = make_float2(0.f, 0.f);
    return;
  }
  if (warp == 0) tc::alloc(tmem_slot, 512);
  if (tid == 0) {
    for (int i = 0; i < kNS; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], 1);
    }
    fence_mbarrier_init();
    s_pfail = 0;
    s_gfail = 0;
    s_issued = 0;
    s_consumed = 0;
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = *tmem_slot;
  const uint32_t sbase = smem_u32(smem);
  const int nst = (int)((kb1 - kb0) / kSK);   // stages of this CTA (kb0, kb1 multiples of kSK)
  constexpr int st_per_chunk = kb_per_chunk / kSK;

  if (warp == 4) {
    // producer: stage q (k blocks kb0 + kSK q ..) into buffer q % kNS once the products of
    // stage q - kNS, the buffer's last reader, are done
    if (lane == 0) {
      const unsigned char* gW = reinterpret_cast<const unsigned char*>(a.Wd);
      const unsigned char* gD = reinterpret_cast<const unsigned char*>(a.Dd);
      for (int q = 0; q < nst; ++q) {
        const int st = q % kNS;
        if (q >= kNS && !mbar_wait_bounded(&empty[st], ((q / kNS) - 1) & 1, kWaitLimitNs)) {
          s_pfail = 1;
          break;
        }
        if (*(volatile int*)&s_gfail) break;
        const size_t kb = (size_t)(kb0 + (int64_t)q * kSK);
        unsigned char* dst = smem + st * kStage;
        mbar_arrive_expect_tx(&full[st], (unsigned)kStage);
        bulk_g2s(dst, gW + ((size_t)I * a.nkb + kb) * kWBytes, (unsigned)kStageW, &full[st]);
        bulk_g2s(dst + kStageW, gD + ((size_t)J * a.nkb + kb) * kABytes,
                 (unsigned)(kStage - kStageW), &full[st]);
        s_issued = q + 1;
      }
    }
    __syncwarp();
  } else {
    const uint64_t desc0 = tc::sdesc(sbase);
    const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);
    float rh[kTI], rl[kTI];   // this thread's row of the partial tile, double-float
#pragma unroll
    for (int c = 0; c < kTI; ++c) rh[c] = rl[c] = 0.f;
    for (int c0 = 0; c0 < nst; c0 += st_per_chunk) {
      const int c1 = min(nst, c0 + st_per_chunk);
      if (tid == 0) {
        for (int q = c0; q < c1; ++q) {
          const int st = q % kNS;
          if (*(volatile int*)&s_pfail || !mbar_wait_bounded(&full[st], (q / kNS) & 1, kWaitLimitNs)) {
            s_gfail = 1;
            break;
          }
          tc::fence_after();
#pragma unroll
          for (int j = 0; j < kSK; ++j) {
            const uint32_t first_acc = (q == c0 && j == 0) ? 0u : 1u;
            const uint64_t w0 = desc0 + ((uint32_t)(st * kStage + j * kWBytes) >> 4);
            const uint64_t w1 = w0 + (uint32_t)(kWSlice >> 4);
            const uint64_t d0 = desc0 + ((uint32_t)(st * kStage + kStageW + j * kABytes) >> 4);
            const uint64_t d8 = d0 + (uint32_t)((8 * kASlice) >> 4);
            tc::mma(tmem, w0, d0, tc::idesc(kTM, 8 * kTI), first_acc);        // levels 0-7
            tc::mma(tmem + 8 * kTI, w0, d8, tc::idesc(kTM, kTI), first_acc);  // level 8
            tc::mma(tmem + kTI, w1, d0, tc::idesc(kTM, 8 * kTI), 1u);         // levels 1-8
          }
          tc::commit(&empty[st]);
          s_consumed = q + 1;
        }
      }
      __syncwarp();
      fold_sync();
      // all products of the chunk are done once the last stage's empty barrier has fired
      if (tid == 0 && !*(volatile int*)&s_gfail) {
        const int ql = c1 - 1;
        if (!mbar_wait_bounded(&empty[ql % kNS], (ql / kNS) & 1, kWaitLimitNs)) s_gfail = 1;
      }
      fold_sync();
      if (*(volatile int*)&s_gfail) break;
      tc::fence_after();
#pragma unroll
      for (int cg = 0; cg < kTI / 16; ++cg) {
        float hs[16], ls[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) hs[j] = ls[j] = 0.f;
#pragma unroll
        for (int l = 0; l < kSA; ++l) {
          uint32_t v[16];
          tc::ld16(lane_base + (uint32_t)(l * kTI + cg * 16), v);
          const float sc = __int_as_float((127 - 6 * l) << 23);   // 2^(-6 l), exact
#pragma unroll
          for (int j = 0; j < 16; ++j) df_add(hs[j], ls[j], __uint_as_float(v[j]) * sc, 0.f);
        }
#pragma unroll
        for (int j = 0; j < 16; ++j) df_add(rh[cg * 16 + j], rl[cg * 16 + j], hs[j], ls[j]);
      }
      tc::fence_before();
      fold_sync();
    }
    if (!*(volatile int*)&s_gfail) {
      float4* o = reinterpret_cast<float4*>(out);
#pragma unroll
      for (int j = 0; j < kTI / 2; ++j)
        o[j] = make_float4(rh[2 * j], rl[2 * j], rh[2 * j + 1], rl[2 * j + 1]);
    }
  }
  __syncthreads();
  if (s_pfail || s_gfail) {
    // let copies and products already issued finish (bounded) before the memory goes away
    if (tid == 0) {
      if (a.fl) a.fl[FL_TIMEOUT] = 1;
      for (int q = s_consumed; q < s_issued; ++q)
        mbar_wait_bounded(&full[q % kNS], (q / kNS) & 1, kWaitLimitNs);
      if (s_consumed > 0)
        mbar_wait_bounded(&empty[(s_consumed - 1) % kNS], ((s_consumed - 1) / kNS) & 1,
                          kWaitLimitNs);
    }
    __syncthreads();
  }
  tc::fence_before();
  __syncthreads();
  if (warp == 0) tc::dealloc(tmem, 512);
}

// G (column-major, ldg x w) from the partial tiles: G_ic = 2^(e_i - 8) rsw sum over the splits,
// zero on the padding rows m <= i < ldg.  The splits are summed in double-float on the FP32
// pipes (each partial is a double-float pair already; FP64 adds run at a small fraction of
// the FP32 rate on this GPU), then converted once.
__global__ void k_sketch_tc_finish(const float2* __restrict__ part, int nsplit, int ntile, int NJ,
                                   const int* __restrict__ ex, int m, int ldg, int w, double rsw,
                                   double* __restrict__ G) {
  const int64_t total = (int64_t)ldg * w;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(idx / ldg), i = (int)(idx - (int64_t)c * ldg);
    double v = 0.0;
    if (i < m) {
      const int tile = (c / kTM) * NJ + i / kTI;
      const size_t off = ((size_t)tile * kTM + (c % kTM)) * kTI + (i % kTI);
      float sh = 0.f, sl = 0.f;
      for (int sp = 0; sp < nsplit; ++sp) {
        const float2 p = part[(size_t)sp * ntile * kTM * kTI + off];
        df_add(sh, sl, p.x, p.y);
      }
      v = ldexp((double)sh + (double)sl, ex[i] - 8) * rsw;
    }
    G[idx] = v;
  }
}

// ---- host side -------------------------------------------------------------------------

namespace {

struct SketchTcShape {
  int64_t nkb;        // k blocks of 16 columns of A, padded to a multiple of kSK
  int ngw, ngm;       // 8-row groups of the W and A D digits
  int NI, NJ, ntile;  // tiles (128 sketch columns x 32 rows of A)
  int nchunks, split, per_cta;
  size_t wd_bytes, dd_bytes, part_bytes, ex_bytes;
};

size_t align256(size_t b) { return (b + 255) / 256 * 256; }

// Splits of the column chunks over CTAs.  One CTA per SM at a time, so a launch takes about
// (waves of CTAs) x (chunks per CTA) chunk times; the smallest split reaching the least such
// product is taken (fewer partial tiles to write and sum).
SketchTcShape sketch_tc_shape(int m, int64_t n, int w, int num_sms) {
  SketchTcShape s{};
  s.nkb = ((n + kKB - 1) / kKB + kSK - 1) / kSK * kSK;
  const int wp = (w + kTM - 1) / kTM * kTM, mp = (m + kRowAlign - 1) / kRowAlign * kRowAlign;
  s.ngw = wp / 8;
  s.ngm = mp / 8;
  s.NI = wp / kTM;
  s.NJ = mp / kTI;
  s.ntile = s.NI * s.NJ;
  s.nchunks = (int)((s.nkb * kKB + kKC - 1) / kKC);
  s.split = 1;
  int64_t best = -1;
  for (int sp = 1; sp <= s.nchunks; ++sp) {
    const int per = (s.nchunks + sp - 1) / sp;
    if ((s.nchunks + per - 1) / per != sp) continue;   // no CTA without columns
    const int64_t waves = ((int64_t)s.ntile * sp + num_sms - 1) / num_sms;
    if (best < 0 || waves * per < best) {
      best = waves * per;
      s.split = sp;
    }
  }
  s.per_cta = (s.nchunks + s.split - 1) / s.split;
  s.wd_bytes = align256((size_t)s.nkb * kSW * s.ngw * tc::kCore);
  s.dd_bytes = align256((size_t)s.nkb * kSA * s.ngm * tc::kCore);
  s.part_bytes = align256((size_t)s.split * s.ntile * kTM * kTI * sizeof(float2));
  s.ex_bytes = align256((size_t)mp * sizeof(int));
  return s;
}

}  // namespace

size_t sketch_tc_work_bytes(int m, int64_t n, int w, int num_sms) {
  const SketchTcShape s = sketch_tc_shape(m, n, w, num_sms);
  return s.wd_bytes + s.dd_bytes + s.part_bytes + s.ex_bytes;
}

cudaError_t launch_sketch_tc(lp_dtype ta, const void* A, int64_t lda, int m, int64_t n, int w,
                             uint64_t key, const double* d, const int16_t* gq, double* G, int ldg,
                             void* work, int num_sms, int* fl, cudaStream_t st) {
  if (ta != LP_F32 && ta != LP_F64) return cudaErrorInvalidValue;
  if (m < 1 || n < 1 || w < 1 || ldg < m) return cudaErrorInvalidValue;
  const SketchTcShape s = sketch_tc_shape(m, n, w, num_sms);
  unsigned char* p = static_cast<unsigned char*>(work);
  __nv_bfloat16* Wd = reinterpret_cast<__nv_bfloat16*>(p);
  __nv_bfloat16* Dd = reinterpret_cast<__nv_bfloat16*>(p + s.wd_bytes);
  float2* part = reinterpret_cast<float2*>(p + s.wd_bytes + s.dd_bytes);
  int* ex = reinterpret_cast<int*>(p + s.wd_bytes + s.dd_bytes + s.part_bytes);
  const int rows_p = s.ngm * 8;
  cudaError_t e = cudaMemsetAsync(ex, 0, (size_t)rows_p * sizeof(int), st);
  if (e != cudaSuccess) return e;
  // columns of A over blockIdx.y, ~512 per CTA, so that the row maxima spread over the GPU
  const int ysplit = (int)std::max<int64_t>(1, std::min<int64_t>(4096, n / 512));
  const int64_t cap = (int64_t)num_sms * 16;
  const int64_t items_d = s.nkb * s.ngm * 16, items_w = s.nkb * s.ngw * 16;
  const unsigned grid_d = (unsigned)std::max<int64_t>(1, std::min<int64_t>(cap, (items_d + 255) / 256));
  const unsigned grid_w = (unsigned)std::max<int64_t>(1, std::min<int64_t>(cap, (items_w + 255) / 256));
  if (ta == LP_F32) {
    note_launch();
    k_ad_row_max<float><<<dim3((rows_p + 31) / 32, ysplit), 256, 0, st>>>((const float*)A, lda, m, n, d, ex);
    note_launch();
    k_ad_row_exp<<<(rows_p + 255) / 256, 256, 0, st>>>(m, rows_p, ex);
    note_launch();
    k_ad_digits<float><<<grid_d, 256, 0, st>>>((const float*)A, lda, m, n, d, ex, s.ngm, s.nkb, Dd);
  } else {
    note_launch();
    k_ad_row_max<double><<<dim3((rows_p + 31) / 32, ysplit), 256, 0, st>>>((const double*)A, lda, m, n, d, ex);
    note_launch();
    k_ad_row_exp<<<(rows_p + 255) / 256, 256, 0, st>>>(m, rows_p, ex);
    note_launch();
    k_ad_digits<double><<<grid_d, 256, 0, st>>>((const double*)A, lda, m, n, d, ex, s.ngm, s.nkb, Dd);
  }
  note_launch();
  k_w_digits<<<grid_w, 256, 0, st>>>(key, n, w, s.ngw, s.nkb, gq, Wd);
  e = ensure_dyn_smem((const void*)k_sketch_tc, kSmemBytes);
  if (e != cudaSuccess) return e;
  SketchTcArgs a{};
  a.Wd = Wd;
  a.Dd = Dd;
  a.nkb = s.nkb;
  a.NJ = s.NJ;
  a.ntile = s.ntile;
  a.chunks_per_cta = s.per_cta;
  a.part = part;
  a.fl = fl;
  note_launch();
  k_sketch_tc<<<dim3(s.ntile, s.split), 160, kSmemBytes, st>>>(a);
  const int64_t total = (int64_t)ldg * w;
  const unsigned grid_f = (unsigned)std::max<int64_t>(1, std::min<int64_t>(4096, (total + 255) / 256));
  note_launch();
  k_sketch_tc_finish<<<grid_f, 256, 0, st>>>(part, s.split, s.ntile, s.NJ, ex, m, ldg, w,
                                             1.0 / sqrt((double)w), G);
  return cudaGetLastError();
}

}  // namespace lpk
