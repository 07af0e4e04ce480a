// Gaussian sketch A D W (Sec. 5; the sketch of the paper's experiments, Sec. 6) and W u.
//
// W (n x w) has entries N(0, 1/w), drawn by inversion of the normal CDF from the iteration key
// of the sparse sketch: for entry (i, b), t = i w + b,
//   h = SplitMix64(key ^ t),  j = h >> 50  (one of 2^14 equiprobable cells),
//   W[i, b] = q_j / (2^8 sqrt(w)),  q_j = round(2^8 Phi^{-1}((j + 1/2) 2^-14)),
// Phi the standard normal CDF.  The table q (|q_j| <= 1026) is computed once per process on the
// host (gauss_grid.h) and kept in each context's device memory.  Every use of W (the sketch on
// either path and W u) reads the same table, so the sketch and the correction vector see the
// same W and A S^-1 v = (A D W) u holds to the accuracy of G; the integer grid is what lets
// the tensor-core sketch (k_sketch_tc.cu) form A D W exactly.
//
// This file's G = A D W is the product on the CUDA cores in double-float, of cost 2 m n w
// (the tensor-core path is the default): a CTA owns 256 rows, 8 sketch columns and a slice of
// the n columns of A (slices spread the work over the GPU when m and w are small), walks its
// slice in chunks, generates the chunk's 8 columns of D W into shared memory as double-float
// coefficients, accumulates in double-float and adds its partial sums into G with FP64
// atomics; W u takes one thread per row of W with FP64 accumulation.
#include "dev_util.cuh"

namespace lpk {

namespace {

__device__ __forceinline__ uint64_t sm64(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// q of entry (i, b): W[i, b] = q / (2^8 sqrt(w))
__device__ __forceinline__ int gauss_q(uint64_t key, int64_t i, int b, int w,
                                       const int16_t* __restrict__ gq) {
  const uint64_t t = (uint64_t)i * (uint64_t)w + (uint64_t)b;
  return __ldg(gq + (sm64(key ^ t) >> 50));
}

constexpr int kGB = 8;     // sketch columns per CTA
constexpr int kGC = 128;   // columns of A per chunk

}  // namespace

template <typename TA>
__global__ void __launch_bounds__(256) k_sketch_gauss(const TA* __restrict__ A, int64_t lda, int m,
                                                      int64_t n, int w, uint64_t key, double rsw,
                                                      const int16_t* __restrict__ gq,
                                                      const double* __restrict__ d,
                                                      double* __restrict__ G, int ldg,
                                                      int64_t slice) {
  __shared__ float ch[kGC][kGB], cl[kGC][kGB];
  const int b0 = blockIdx.x * kGB;
  const int r = blockIdx.y * 256 + threadIdx.x;
  float s[kGB], c[kGB];
#pragma unroll
  for (int q = 0; q < kGB; ++q) s[q] = c[q] = 0.f;
  const int64_t ibeg = blockIdx.z * slice;
  const int64_t iend = min(n, ibeg + slice);
  for (int64_t i0 = ibeg; i0 < iend; i0 += kGC) {
    __syncthreads();
    for (int e = threadIdx.x; e < kGC * kGB; e += blockDim.x) {
      const int ii = e / kGB, bb = e % kGB;
      const int64_t i = i0 + ii;
      double cf = 0.0;
      if (i < iend && b0 + bb < w) cf = d[i] * ((double)gauss_q(key, i, b0 + bb, w, gq) * rsw);
      split_double(cf, ch[ii][bb], cl[ii][bb]);
    }
    __syncthreads();
    if (r < m) {
      const int cnt = (int)((iend - i0) < kGC ? (iend - i0) : kGC);
      for (int ii = 0; ii < cnt; ++ii) {
        const TA av = A[(i0 + ii) * lda + r];
        if constexpr (sizeof(TA) == 4) {
#pragma unroll
          for (int q = 0; q < kGB; ++q) df_fma((float)av, ch[ii][q], cl[ii][q], s[q], c[q]);
        } else {
          float ah, al;
          split_double((double)av, ah, al);
#pragma unroll
          for (int q = 0; q < kGB; ++q) df_mac(ah, al, ch[ii][q], cl[ii][q], s[q], c[q]);
        }
      }
    }
  }
  if (r < m)
#pragma unroll
    for (int q = 0; q < kGB; ++q)
      if (b0 + q < w) atomicAdd(&G[(size_t)(b0 + q) * ldg + r], (double)s[q] + (double)c[q]);
}

__global__ void k_apply_W_gauss(uint64_t key, int64_t n, int w, double rsw,
                                const int16_t* __restrict__ gq, const double* __restrict__ u,
                                double* __restrict__ wu) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int b = 0; b < w; ++b) acc = fma((double)gauss_q(key, i, b, w, gq), u[b], acc);
    wu[i] = acc * rsw;
  }
}

uint64_t gauss_iteration_key(uint64_t seed, int k) {
  auto h = [](uint64_t x) {
    uint64_t z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
  };
  return h(seed ^ h((uint64_t)(int64_t)k));
}

cudaError_t launch_sketch_gauss(lp_dtype ta, const void* A, int64_t lda, int m, int64_t n, int w,
                                uint64_t seed, int k, const int16_t* gq, const double* d, double* G,
                                int ldg, cudaStream_t st) {
  const uint64_t key = gauss_iteration_key(seed, k);
  const double rsw = 1.0 / (256.0 * sqrt((double)w));
  if (ta != LP_F32 && ta != LP_F64) return cudaErrorInvalidValue;
  // slices of the n columns so that about 4 CTAs per SM have work
  int dev = 0, sms = 152;
  if (cudaGetDevice(&dev) == cudaSuccess)
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t tiles = (int64_t)((w + kGB - 1) / kGB) * ((m + 255) / 256);
  int64_t nsl = (4 * (int64_t)sms + tiles - 1) / tiles;
  const int64_t max_sl = (n + kGC - 1) / kGC;
  if (nsl > max_sl) nsl = max_sl;
  if (nsl > 65535) nsl = 65535;
  if (nsl < 1) nsl = 1;
  int64_t slice = (n + nsl - 1) / nsl;
  slice = (slice + kGC - 1) / kGC * kGC;
  nsl = (n + slice - 1) / slice;
  cudaError_t e = cudaMemsetAsync(G, 0, (size_t)ldg * w * sizeof(double), st);
  if (e != cudaSuccess) return e;
  dim3 grid((unsigned)((w + kGB - 1) / kGB), (unsigned)((m + 255) / 256), (unsigned)nsl);
  if (ta == LP_F32) {
    note_launch();
    k_sketch_gauss<float><<<grid, 256, 0, st>>>((const float*)A, lda, m, n, w, key, rsw, gq, d, G,
                                                 ldg, slice);
  } else {
    note_launch();
    k_sketch_gauss<double><<<grid, 256, 0, st>>>((const double*)A, lda, m, n, w, key, rsw, gq, d,
                                                  G, ldg, slice);
  }
  return cudaGetLastError();
}

cudaError_t launch_apply_W_gauss(uint64_t seed, int k, int64_t n, int w, const int16_t* gq,
                                 const double* u, double* wu, cudaStream_t st) {
  int64_t g = (n + 255) / 256;
  if (g > 4096) g = 4096;
  if (g < 1) g = 1;
  note_launch();
  k_apply_W_gauss<<<(unsigned)g, 256, 0, st>>>(gauss_iteration_key(seed, k), n, w,
                                               1.0 / (256.0 * sqrt((double)w)), gq, u, wu);
  return cudaGetLastError();
}

}  // namespace lpk
