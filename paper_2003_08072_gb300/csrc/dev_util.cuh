// Device helpers: vector unpacking, warp reductions, last-block grid reductions.
#pragma once

#include "lp_internal.cuh"

namespace lpk {

constexpr unsigned kFull = 0xffffffffu;

template <typename T> struct VecN;
template <> struct VecN<double> { static constexpr int N = 2; };
template <> struct VecN<float> { static constexpr int N = 4; };
template <> struct VecN<__nv_bfloat16> { static constexpr int N = 8; };
template <> struct VecN<__half> { static constexpr int N = 8; };

// 16 bytes of TA -> N values of ACC
template <typename TA, typename ACC>
__device__ __forceinline__ void unpack(const uint4& r, ACC (&o)[VecN<TA>::N]) {
  if constexpr (sizeof(TA) == 8) {
    o[0] = (ACC)__hiloint2double((int)r.y, (int)r.x);
    o[1] = (ACC)__hiloint2double((int)r.w, (int)r.z);
  } else if constexpr (sizeof(TA) == 4) {
    o[0] = (ACC)__uint_as_float(r.x);
    o[1] = (ACC)__uint_as_float(r.y);
    o[2] = (ACC)__uint_as_float(r.z);
    o[3] = (ACC)__uint_as_float(r.w);
  } else {
    const unsigned w[4] = {r.x, r.y, r.z, r.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      if constexpr (std::is_same<TA, __nv_bfloat16>::value) {
        // a bf16 is the upper half of a float32
        o[2 * i] = (ACC)__uint_as_float(w[i] << 16);
        o[2 * i + 1] = (ACC)__uint_as_float(w[i] & 0xffff0000u);
      } else {
        __half2 h = *reinterpret_cast<const __half2*>(&w[i]);
        float2 f = __half22float2(h);
        o[2 * i] = (ACC)f.x;
        o[2 * i + 1] = (ACC)f.y;
      }
    }
  }
}

// Zeroes the elements of a 16-byte vector from element `valid` on (1 <= valid): the rows at or
// past m of a column whose leading dimension is padded, so that whatever the padding holds
// (NaN or Inf included) cannot reach a sum.
template <typename TA>
__device__ __forceinline__ uint4 mask_tail(uint4 r, int valid) {
  const int keep_bits = valid * (int)(sizeof(TA) * 8);
  uint32_t w[4] = {r.x, r.y, r.z, r.w};
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int lo = 32 * i;
    if (keep_bits <= lo) w[i] = 0u;
    else if (keep_bits < lo + 32) w[i] &= (1u << (keep_bits - lo)) - 1u;
  }
  return make_uint4(w[0], w[1], w[2], w[3]);
}

// Streaming 16-byte load (read once per pass: evict-first in L1 and L2).
__device__ __forceinline__ uint4 ld_stream(const void* p) {
  return __ldcs(reinterpret_cast<const uint4*>(p));
}

// Reduce TILE per-lane values over the 32 lanes of a warp: afterwards lane l holds the
// full sum of value (l % TILE).  TILE-1 + log2(32/TILE) shuffles instead of TILE*5.
template <int TILE, typename T>
__device__ __forceinline__ T warp_transpose_reduce(T (&v)[TILE], int lane) {
#pragma unroll
  for (int off = TILE / 2; off >= 1; off >>= 1) {
    const bool upper = (lane & off) != 0;
#pragma unroll
    for (int i = 0; i < off; ++i) {
      T send = upper ? v[i] : v[i + off];
      T keep = upper ? v[i + off] : v[i];
      v[i] = keep + __shfl_xor_sync(kFull, send, off);
    }
  }
  T r = v[0];
#pragma unroll
  for (int off = TILE; off < 32; off <<= 1) r += __shfl_xor_sync(kFull, r, off);
  return r;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int off = 16; off >= 1; off >>= 1) v += __shfl_xor_sync(kFull, v, off);
  return v;
}

__device__ __forceinline__ double warp_min(double v) {
#pragma unroll
  for (int off = 16; off >= 1; off >>= 1) v = fmin(v, __shfl_xor_sync(kFull, v, off));
  return v;
}

// Block-wide sum of NV doubles (result valid in thread 0).  blockDim.x <= 1024.
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV]) {
  __shared__ double sh[NV][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k) v[k] = warp_sum(v[k]);
  __syncthreads();
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < NV; ++k) sh[k][warp] = v[k];
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      double t = lane < nw ? sh[k][lane] : 0.0;
      v[k] = warp_sum(t);
    }
  }
}

// Grid-wide sum with the "last block finishes" pattern (no spin wait): each block
// writes its NV partials, the last block to arrive sums all partials in block order
// (deterministic) and returns true in all of its threads with v holding the totals.
// The same over a virtual grid of nblk blocks (bid = this block's index in it): a batched
// launch runs several such grids, one per job of its work table.
template <int NV>
__device__ __forceinline__ bool grid_sum_last_b(double (&v)[NV], double* bpart, unsigned* counter,
                                                unsigned bid, unsigned nblk) {
  __shared__ bool s_last;
  block_sum<NV>(v);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) bpart[bid * NV + k] = v[k];
    __threadfence();
    unsigned ticket = atomicAdd(counter, 1u);
    s_last = (ticket == nblk - 1);
  }
  __syncthreads();
  if (!s_last) return false;
  __threadfence();
  // sum partials in fixed block order, NV values spread over threads
  double tot[NV];
#pragma unroll
  for (int k = 0; k < NV; ++k) tot[k] = 0.0;
  for (unsigned b = threadIdx.x; b < nblk; b += blockDim.x)
#pragma unroll
    for (int k = 0; k < NV; ++k) tot[k] += __ldcg(&bpart[b * NV + k]);
  block_sum<NV>(tot);
  __shared__ double s_tot[NV];
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) s_tot[k] = tot[k];
    *counter = 0u;
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < NV; ++k) v[k] = s_tot[k];
  return true;
}

template <int NV>
__device__ __forceinline__ bool grid_sum_last(double (&v)[NV], double* bpart, unsigned* counter) {
  return grid_sum_last_b<NV>(v, bpart, counter, blockIdx.x, gridDim.x);
}

// Grid-wide minimum, same pattern.
__device__ __forceinline__ bool grid_min_last(double& v, double* bpart, unsigned* counter) {
  __shared__ double sh[32];
  __shared__ bool s_last;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  v = warp_min(v);
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double b = sh[0];
    for (int i = 1; i < nw; ++i) b = fmin(b, sh[i]);
    bpart[blockIdx.x] = b;
    __threadfence();
    unsigned ticket = atomicAdd(counter, 1u);
    s_last = (ticket == gridDim.x - 1);
  }
  __syncthreads();
  if (!s_last) return false;
  __threadfence();
  if (threadIdx.x == 0) {
    double b = __ldcg(&bpart[0]);
    for (unsigned i = 1; i < gridDim.x; ++i) b = fmin(b, __ldcg(&bpart[i]));
    sh[0] = b;
    *counter = 0u;
  }
  __syncthreads();
  v = sh[0];
  return true;
}

// Step length of one iteration from d^T q: CG's alpha = rho / d^T q (Alg. 1 step 3), or the
// unit step of Richardson's iteration (App. A), whose update dy += M (p - K dy) is the same
// iteration with alpha = 1 and beta = 0.  A non-positive or non-finite d^T q stops the solve.
__device__ __forceinline__ void set_cg_alpha(double dq, double* sc, int* fl) {
  sc[SC_DQ] = dq;
  if (!(dq > 0.0) || !isfinite(dq)) {
    fl[FL_NUMERIC] = 1;
    fl[FL_DONE] = 1;
    sc[SC_ALPHA] = 0.0;
  } else {
    sc[SC_ALPHA] = fl[FL_RICH] ? 1.0 : sc[SC_RHO] / dq;
  }
}

}  // namespace lpk

namespace lpk {

// ---- double-float arithmetic on FP32 pipes -------------------------------------------------
// Error-free transformations: TwoSum (Knuth, TAOCP vol. 2) gives s + e = a + b exactly;
// TwoProduct with a fused multiply-add (as in Ogita, Rump & Oishi, "Accurate sum and dot
// product", SIAM J. Sci. Comput. 2005) gives p + e = a * b exactly.  A value is carried as an
// unnormalised pair (s, c) whose sum is the result; FP32 numbers times a double coefficient
// split into two floats give products accurate to ~2^-48 relative.

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {  // |a| >= |b|
  s = __fadd_rn(a, b);
  e = __fsub_rn(b, __fsub_rn(s, a));
}

__device__ __forceinline__ void split_double(double x, float& hi, float& lo) {
  hi = (float)x;
  lo = (float)(x - (double)hi);
}

// The same split from the bits of x, on the integer and FP32 pipes (the FP64 conversions of
// split_double run on this GPU's slow FP64 units): hi is x rounded to 24 significant bits by
// adding half a unit of the 29 dropped mantissa bits to the bit pattern and clearing them (a
// carry into the exponent field is the correct rounding), lo the signed remainder
// (|lo| <= 2^28 units of 2^(e-1075), rounded to FP32), so hi + lo is within 2^-49 of x, as
// with split_double.  Inputs outside 2^-70 < |x| < 2^100 (and zero) take split_double.
__device__ __forceinline__ void split_double_bits(double x, float& hi, float& lo) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int e = (int)((b >> 52) & 0x7ff);   // biased exponent
  if (e < 1023 - 70 || e > 1023 + 100) {
    split_double(x, hi, lo);
    return;
  }
  const unsigned long long bh = (b + (1ull << 28)) & ~((1ull << 29) - 1ull);
  const int eh = (int)((bh >> 52) & 0x7ff);
  const unsigned sign = (unsigned)(b >> 63) << 31;
  hi = __uint_as_float(sign | ((unsigned)(eh - 1023 + 127) << 23) |
                       (unsigned)((bh >> 29) & 0x7fffffu));
  const float rem = __int2float_rn((int)(long long)(b - bh));   // |b - bh| <= 2^28
  // 2^(e-1075) is a normal float for e >= 950
  const float scaled = rem * __uint_as_float((unsigned)(e - 1075 + 127) << 23);
  lo = sign ? -scaled : scaled;
}

// (s, c) += a * (bh + bl).  The leading product is rounded on its own (__fmul_rn is never
// contracted into an FMA), so that p + pe == a * bh exactly and TwoSum sees the rounded p.
__device__ __forceinline__ void df_fma(float a, float bh, float bl, float& s, float& c) {
  const float p = __fmul_rn(a, bh);
  const float pe = fmaf(a, bh, -p);
  float t, e;
  two_sum(s, p, t, e);
  s = t;
  c += (e + pe) + a * bl;
}

// (s, c) += (ah + al) * (bh + bl)
__device__ __forceinline__ void df_mac(float ah, float al, float bh, float bl, float& s, float& c) {
  const float p = __fmul_rn(ah, bh);
  const float pe = fmaf(ah, bh, -p);
  float t, e;
  two_sum(s, p, t, e);
  s = t;
  c += (e + pe) + fmaf(ah, bl, al * bh);
}

// (s1, c1) += (s2, c2), renormalised
__device__ __forceinline__ void df_add(float& s1, float& c1, float s2, float c2) {
  float t, e;
  two_sum(s1, s2, t, e);
  e += c1 + c2;
  fast_two_sum(t, e, s1, c1);
}

// (h, l) = (ah + al) * (bh + bl)
__device__ __forceinline__ void df_mul(float ah, float al, float bh, float bl, float& h, float& l) {
  const float p = __fmul_rn(ah, bh);
  const float pe = fmaf(ah, bh, -p);
  fast_two_sum(p, pe + fmaf(ah, bl, al * bh), h, l);
}

// Square root and reciprocal of a double-float: the FP32 result refined by one Newton step
// evaluated with an exact product (Dekker 1971; Hida, Li & Bailey, "Algorithms for quad-double
// precision floating point arithmetic", 2001).  Inputs positive and normal.
__device__ __forceinline__ void df_sqrt(float ah, float al, float& h, float& l) {
  const float x = sqrtf(ah);
  const float p = __fmul_rn(x, x);
  const float pe = fmaf(x, x, -p);
  const float r = (((ah - p) - pe) + al) / (2.f * x);
  fast_two_sum(x, r, h, l);
}

__device__ __forceinline__ void df_recip(float bh, float bl, float& h, float& l) {
  // seed: the hardware's approximate reciprocal (PTX rcp.approx, about 1 ulp); the Newton
  // step below squares its relative error, as it would that of a correctly rounded seed
  float y;
  asm("rcp.approx.f32 %0, %1;" : "=f"(y) : "f"(bh));
  const float p = __fmul_rn(bh, y);
  const float pe = fmaf(bh, y, -p);
  const float e = ((1.0f - p) - pe) - bl * y;   // 1 - (bh + bl) y
  fast_two_sum(y, y * e, h, l);
}

__device__ __forceinline__ void df_renorm(float& s, float& c) {
  float t, e;
  fast_two_sum(s, c, t, e);
  s = t;
  c = e;
}

}  // namespace lpk
