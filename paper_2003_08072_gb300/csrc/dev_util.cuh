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
template <int NV>
__device__ __forceinline__ bool grid_sum_last(double (&v)[NV], double* bpart, unsigned* counter) {
  __shared__ bool s_last;
  block_sum<NV>(v);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) bpart[blockIdx.x * NV + k] = v[k];
    __threadfence();
    unsigned ticket = atomicAdd(counter, 1u);
    s_last = (ticket == gridDim.x - 1);
  }
  __syncthreads();
  if (!s_last) return false;
  __threadfence();
  // sum partials in fixed block order, NV values spread over threads
  double tot[NV];
#pragma unroll
  for (int k = 0; k < NV; ++k) tot[k] = 0.0;
  for (unsigned b = threadIdx.x; b < gridDim.x; b += blockDim.x)
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

}  // namespace lpk
