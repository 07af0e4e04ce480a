// Sparse sketch A D W (Sec. 2 Eq. pdprec; Alg. 1 step 1; Alg. 2 step (a)).
//
// W (n x w) has s nonzeros +-1/sqrt(s) per row, generated on the fly from a counter hash:
//   key    = SplitMix64(seed ^ SplitMix64(k))           (one W per IPM iteration k)
//   h      = SplitMix64(key ^ (i*s + j))                 (row i, nonzero j)
//   bucket = j*(w/s) + (((h >> 32) * (w/s)) >> 32)       (Lemire multiply-shift, block j)
//   sign   = (h & 1) ? -1 : +1
// SplitMix64: Steele, Lea & Flood (OOPSLA 2014); range reduction: Lemire (ACM TOMS 2019).
//
// Instead of scatter-adding every column of A D into its bucket with atomics, the columns
// are bucket-sorted (histogram, scan, scatter of column ids) and each bucket column of the
// sketch is then formed by one CTA that gathers its member columns of A and accumulates in
// FP64 registers: every column of A is read once per nonzero of W and every column of the
// sketch is written once.
#include "dev_util.cuh"

namespace lpk {

__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__global__ void k_sketch_hash(uint64_t seed, int k, int64_t n, int s, int w, int32_t* hb,
                              int32_t* cnt, int32_t* bucket_out, int8_t* sign_out) {
  const uint64_t key = splitmix64(seed ^ splitmix64((uint64_t)(int64_t)k));
  const uint64_t width = (uint64_t)(w / s);
  const int64_t total = n * (int64_t)s;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t h = splitmix64(key ^ (uint64_t)idx);
    const int j = (int)(idx % s);
    const int32_t bucket = (int32_t)((uint64_t)j * width + (((h >> 32) * width) >> 32));
    const bool neg = (h & 1ull) != 0;
    if (hb) hb[idx] = bucket | (neg ? (int32_t)0x80000000 : 0);
    if (cnt) atomicAdd(&cnt[bucket], 1);
    if (bucket_out) bucket_out[idx] = bucket;
    if (sign_out) sign_out[idx] = neg ? (int8_t)-1 : (int8_t)1;
  }
}

cudaError_t launch_sketch_hash(uint64_t seed, int k, int64_t n, int s, int w, int32_t* hb,
                               int32_t* cnt, int32_t* bucket_out, int8_t* sign_out, cudaStream_t st) {
  const int64_t total = n * (int64_t)s;
  int64_t grid = (total + 255) / 256;
  if (grid > 4096) grid = 4096;
  if (grid < 1) grid = 1;
  { note_launch(); k_sketch_hash<<<(unsigned)grid, 256, 0, st>>>(seed, k, n, s, w, hb, cnt, bucket_out, sign_out); }
  return cudaGetLastError();
}

// Exclusive scan of cnt[0..w) into start[0..w], start[w] = total; cursor zeroed.  One CTA.
__global__ void __launch_bounds__(1024) k_scan(const int32_t* cnt, int w, int32_t* start,
                                               int32_t* cursor) {
  __shared__ int32_t sums[1024];
  const int t = threadIdx.x;
  const int per = (w + 1023) / 1024;
  const int b0 = t * per, b1 = min(w, b0 + per);
  int32_t local = 0;
  for (int i = b0; i < b1; ++i) local += cnt[i];
  sums[t] = local;
  __syncthreads();
  for (int off = 1; off < 1024; off <<= 1) {   // Hillis-Steele inclusive scan
    int32_t v = (t >= off) ? sums[t - off] : 0;
    __syncthreads();
    sums[t] += v;
    __syncthreads();
  }
  int32_t run = sums[t] - local;
  for (int i = b0; i < b1; ++i) {
    start[i] = run;
    run += cnt[i];
    cursor[i] = 0;
  }
  if (t == 1023) start[w] = sums[1023];
}

cudaError_t launch_sketch_scan(const int32_t* cnt, int w, int32_t* start, int32_t* cursor,
                               cudaStream_t st) {
  { note_launch(); k_scan<<<1, 1024, 0, st>>>(cnt, w, start, cursor); }
  return cudaGetLastError();
}

// Bucket scatter of the nonzeros of W.  With d given, each entry also gets its coefficient
// sign * d_i / sqrt(s) as a double-float pair (computed once per nonzero, not per gather thread).
__global__ void k_scatter(const int32_t* hb, int64_t n, int s, const int32_t* start,
                          int32_t* cursor, int32_t* list, const double* d, float2* coef) {
  const int64_t total = n * (int64_t)s;
  const double inv_sqrt_s = 1.0 / sqrt((double)s);
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int32_t h = hb[idx];
    const int32_t b = h & 0x7fffffff;
    const int32_t pos = start[b] + atomicAdd(&cursor[b], 1);
    const int64_t col = idx / s;
    list[pos] = (int32_t)col | (h & (int32_t)0x80000000);
    if (coef) {
      const double v = (h < 0 ? -d[col] : d[col]) * inv_sqrt_s;
      float ch, cl;
      split_double_bits(v, ch, cl);
      coef[pos] = make_float2(ch, cl);
    }
  }
}

// Members of each bucket in column order.  The scatter places them through an atomic cursor, so
// their order -- and with it the rounding of each bucket's sum in the gather -- would change from
// run to run.  One CTA per bucket ranks its members by column index (distinct within a bucket:
// the s nonzeros of a column lie in s different buckets) and writes them back in that order.
// A bucket of more than kSortCap members (far beyond n s / w on any sketch used here) keeps the
// scatter's order.
constexpr int kSortCap = 2048;

__global__ void __launch_bounds__(256) k_sort_buckets(const int32_t* __restrict__ start,
                                                      int32_t* __restrict__ list,
                                                      float2* __restrict__ coef) {
  __shared__ int32_t key[kSortCap];
  __shared__ float2 cf[kSortCap];
  const int b = blockIdx.x;
  const int32_t s0 = start[b], len = start[b + 1] - s0;
  if (len <= 1 || len > kSortCap) return;
  for (int i = threadIdx.x; i < len; i += blockDim.x) {
    key[i] = list[s0 + i];
    if (coef) cf[i] = coef[s0 + i];
  }
  __syncthreads();
  for (int i = threadIdx.x; i < len; i += blockDim.x) {
    const int32_t ki = key[i] & 0x7fffffff;
    int r = 0;
    for (int j = 0; j < len; ++j) r += (key[j] & 0x7fffffff) < ki;
    list[s0 + r] = key[i];
    if (coef) coef[s0 + r] = cf[i];
  }
}

cudaError_t launch_sketch_scatter(const int32_t* hb, int64_t n, int s, int w, const int32_t* start,
                                  int32_t* cursor, int32_t* list, const double* d, float2* coef,
                                  cudaStream_t st) {
  const int64_t total = n * (int64_t)s;
  int64_t grid = (total + 255) / 256;
  if (grid > 4096) grid = 4096;
  if (grid < 1) grid = 1;
  { note_launch(); k_scatter<<<(unsigned)grid, 256, 0, st>>>(hb, n, s, start, cursor, list, d, coef); }
  { note_launch(); k_sort_buckets<<<(unsigned)w, 256, 0, st>>>(start, list, coef); }
  return cudaGetLastError();
}

// One CTA per bucket b: G[:, b] = sum over member (column i, sign) of sign/sqrt(s) d_i A[:, i].
// Warps cover the rows (SPW slices of 32 lanes x 16 bytes each); FP64 accumulation.
template <typename TA, int SPW>
__global__ void __launch_bounds__(512) k_gather_dense(const TA* __restrict__ A, int64_t lda, int m,
                                                      int s, const int32_t* __restrict__ start,
                                                      const int32_t* __restrict__ list,
                                                      const double* __restrict__ d,
                                                      double* __restrict__ G, int ldg) {
  constexpr int VEC = VecN<TA>::N;
  constexpr int UNR = 4;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int b = blockIdx.x;
  const double inv_sqrt_s = 1.0 / sqrt((double)s);
  double acc[SPW][VEC];
  int rowb[SPW];
  bool rok[SPW];
#pragma unroll
  for (int sl = 0; sl < SPW; ++sl) {
    rowb[sl] = ((warp * SPW + sl) * 32 + lane) * VEC;
    rok[sl] = rowb[sl] < m;
#pragma unroll
    for (int e = 0; e < VEC; ++e) acc[sl][e] = 0.0;
  }
  const int e0 = start[b], e1 = start[b + 1];
  for (int e = e0; e < e1; e += UNR) {
    uint4 ar[UNR][SPW];
    double cf[UNR];
#pragma unroll
    for (int u = 0; u < UNR; ++u) {
      cf[u] = 0.0;
      if (e + u < e1) {
        const int32_t ent = list[e + u];
        const int64_t col = ent & 0x7fffffff;
        const double dv = d[col] * inv_sqrt_s;
        cf[u] = (ent < 0) ? -dv : dv;
#pragma unroll
        for (int sl = 0; sl < SPW; ++sl)
          ar[u][sl] = rok[sl] ? __ldg(reinterpret_cast<const uint4*>(A + col * lda + rowb[sl]))
                              : make_uint4(0u, 0u, 0u, 0u);
      } else {
#pragma unroll
        for (int sl = 0; sl < SPW; ++sl) ar[u][sl] = make_uint4(0u, 0u, 0u, 0u);
      }
    }
#pragma unroll
    for (int u = 0; u < UNR; ++u)
#pragma unroll
      for (int sl = 0; sl < SPW; ++sl) {
        double av[VEC];
        unpack<TA, double>(ar[u][sl], av);
#pragma unroll
        for (int q = 0; q < VEC; ++q) acc[sl][q] = fma(cf[u], av[q], acc[sl][q]);
      }
  }
#pragma unroll
  for (int sl = 0; sl < SPW; ++sl)
#pragma unroll
    for (int q = 0; q < VEC; ++q) {
      const int row = rowb[sl] + q;
      if (rok[sl] && row < m) G[(size_t)b * ldg + row] = acc[sl][q];
    }
}

// FP32 A: the same gather with double-float accumulation on the FP32 pipes.
template <int SPW>
__global__ void __launch_bounds__(512) k_gather_dense_df(const float* __restrict__ A, int64_t lda,
                                                         int m, const int32_t* __restrict__ start,
                                                         const int32_t* __restrict__ list,
                                                         const float2* __restrict__ coef,
                                                         double* __restrict__ G, int ldg) {
  constexpr int VEC = 4;
  constexpr int UNR = 4;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int b = blockIdx.x;
  float as[SPW][VEC], ac[SPW][VEC];
  int rowb[SPW];
  bool rok[SPW];
#pragma unroll
  for (int sl = 0; sl < SPW; ++sl) {
    rowb[sl] = ((warp * SPW + sl) * 32 + lane) * VEC;
    rok[sl] = rowb[sl] < m;
#pragma unroll
    for (int e = 0; e < VEC; ++e) as[sl][e] = ac[sl][e] = 0.f;
  }
  const int e0 = start[b], e1 = start[b + 1];
  for (int e = e0; e < e1; e += UNR) {
    uint4 ar[UNR][SPW];
    float2 cf[UNR];
#pragma unroll
    for (int u = 0; u < UNR; ++u) {
      if (e + u < e1) {
        const int64_t col = list[e + u] & 0x7fffffff;
        cf[u] = coef[e + u];
#pragma unroll
        for (int sl = 0; sl < SPW; ++sl)
          ar[u][sl] = rok[sl] ? ld_stream(A + col * lda + rowb[sl]) : make_uint4(0u, 0u, 0u, 0u);
      } else {
        cf[u] = make_float2(0.f, 0.f);
#pragma unroll
        for (int sl = 0; sl < SPW; ++sl) ar[u][sl] = make_uint4(0u, 0u, 0u, 0u);
      }
    }
#pragma unroll
    for (int u = 0; u < UNR; ++u)
#pragma unroll
      for (int sl = 0; sl < SPW; ++sl) {
        float av[VEC];
        unpack<float, float>(ar[u][sl], av);
#pragma unroll
        for (int q = 0; q < VEC; ++q) df_fma(av[q], cf[u].x, cf[u].y, as[sl][q], ac[sl][q]);
      }
#pragma unroll
    for (int sl = 0; sl < SPW; ++sl)
#pragma unroll
      for (int q = 0; q < VEC; ++q) df_renorm(as[sl][q], ac[sl][q]);
  }
#pragma unroll
  for (int sl = 0; sl < SPW; ++sl)
#pragma unroll
    for (int q = 0; q < VEC; ++q) {
      const int row = rowb[sl] + q;
      if (rok[sl] && row < m) G[(size_t)b * ldg + row] = (double)as[sl][q] + (double)ac[sl][q];
    }
}

template <typename TA>
static cudaError_t gather_dense_t(const void* A, int64_t lda, int m, int s, int w,
                                  const int32_t* start, const int32_t* list, const double* d,
                                  double* G, int ldg, cudaStream_t st) {
  constexpr int VEC = VecN<TA>::N;
  const int nslices = (m + 32 * VEC - 1) / (32 * VEC);
  int spw = 1;
  while ((nslices + spw - 1) / spw > 16) spw *= 2;
  const int threads = ((nslices + spw - 1) / spw) * 32;
  const TA* Ap = reinterpret_cast<const TA*>(A);
  switch (spw) {
    case 1: { note_launch(); k_gather_dense<TA, 1><<<w, threads, 0, st>>>(Ap, lda, m, s, start, list, d, G, ldg); } break;
    case 2: { note_launch(); k_gather_dense<TA, 2><<<w, threads, 0, st>>>(Ap, lda, m, s, start, list, d, G, ldg); } break;
    case 4: { note_launch(); k_gather_dense<TA, 4><<<w, threads, 0, st>>>(Ap, lda, m, s, start, list, d, G, ldg); } break;
    default: { note_launch(); k_gather_dense<TA, 8><<<w, threads, 0, st>>>(Ap, lda, m, s, start, list, d, G, ldg); } break;
  }
  return cudaGetLastError();
}

cudaError_t launch_sketch_gather_dense(lp_dtype ta, const void* A, int64_t lda, int m, int s,
                                       int w, const int32_t* start, const int32_t* list,
                                       const double* d, double* G, int ldg, cudaStream_t st,
                                       const float2* coef) {
  if (ta == LP_F64) return gather_dense_t<double>(A, lda, m, s, w, start, list, d, G, ldg, st);
  if (ta == LP_F32 && coef) {
    const int nslices = (m + 127) / 128;
    int spw = 1;
    while ((nslices + spw - 1) / spw > 16) spw *= 2;
    const int threads = ((nslices + spw - 1) / spw) * 32;
    const float* Af = reinterpret_cast<const float*>(A);
    if (spw == 1) {
      { note_launch(); k_gather_dense_df<1><<<w, threads, 0, st>>>(Af, lda, m, start, list, coef, G, ldg); }
      return cudaGetLastError();
    }
    if (spw == 2) {
      { note_launch(); k_gather_dense_df<2><<<w, threads, 0, st>>>(Af, lda, m, start, list, coef, G, ldg); }
      return cudaGetLastError();
    }
  }
  if (ta == LP_F32) return gather_dense_t<float>(A, lda, m, s, w, start, list, d, G, ldg, st);
  return cudaErrorInvalidValue;
}

// CSC gather: one CTA per bucket accumulates its member columns into a shared FP64 column
// of length m (shared-memory atomics), then writes it.  Warp per member column, lanes over
// the column's nonzeros.
template <typename TV>
__global__ void __launch_bounds__(256) k_gather_csc(const int64_t* __restrict__ colptr,
                                                    const int32_t* __restrict__ rowidx,
                                                    const TV* __restrict__ vals, int m, int s,
                                                    const int32_t* __restrict__ start,
                                                    const int32_t* __restrict__ list,
                                                    const double* __restrict__ d,
                                                    double* __restrict__ G, int ldg) {
  extern __shared__ double acc[];
  const int b = blockIdx.x;
  for (int i = threadIdx.x; i < m; i += blockDim.x) acc[i] = 0.0;
  __syncthreads();
  const double inv_sqrt_s = 1.0 / sqrt((double)s);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int e0 = start[b], e1 = start[b + 1];
  for (int e = e0 + warp; e < e1; e += nw) {
    const int32_t ent = list[e];
    const int64_t col = ent & 0x7fffffff;
    const double dv = d[col] * inv_sqrt_s;
    const double cf = (ent < 0) ? -dv : dv;
    for (int64_t k = colptr[col] + lane; k < colptr[col + 1]; k += 32)
      atomicAdd(&acc[rowidx[k]], cf * (double)vals[k]);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < m; i += blockDim.x) G[(size_t)b * ldg + i] = acc[i];
}

cudaError_t launch_sketch_gather_csc(lp_dtype tv, const int64_t* colptr, const int32_t* rowidx,
                                     const void* vals, int m, int s, int w, const int32_t* start,
                                     const int32_t* list, const double* d, double* G, int ldg,
                                     cudaStream_t st) {
  const size_t smem = (size_t)m * sizeof(double);
  if (tv == LP_F32) {
    if (cudaError_t e = ensure_dyn_smem((const void*)k_gather_csc<float>, smem)) return e;
    { note_launch(); k_gather_csc<float><<<w, 256, smem, st>>>(colptr, rowidx, (const float*)vals, m, s, start,
                                              list, d, G, ldg); }
  } else if (tv == LP_F64) {
    if (cudaError_t e = ensure_dyn_smem((const void*)k_gather_csc<double>, smem)) return e;
    { note_launch(); k_gather_csc<double><<<w, 256, smem, st>>>(colptr, rowidx, (const double*)vals, m, s, start,
                                               list, d, G, ldg); }
  } else {
    return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace lpk
