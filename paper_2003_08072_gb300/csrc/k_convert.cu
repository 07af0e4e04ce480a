// Layout and precision conversion of the input matrix, finiteness checks, scalar setters.
#include <map>
#include <mutex>
#include <tuple>
#include <unordered_map>

#include "dev_util.cuh"

namespace lpk {

template <typename TD>
__device__ __forceinline__ TD to_dt(double v);
template <> __device__ __forceinline__ double to_dt<double>(double v) { return v; }
template <> __device__ __forceinline__ float to_dt<float>(double v) { return (float)v; }
template <> __device__ __forceinline__ __nv_bfloat16 to_dt<__nv_bfloat16>(double v) {
  return __double2bfloat16(v);
}
template <> __device__ __forceinline__ __half to_dt<__half>(double v) { return __double2half(v); }

template <typename TS>
__device__ __forceinline__ double from_src(const void* src, size_t idx) {
  return (double)reinterpret_cast<const TS*>(src)[idx];
}

// Column-major source (leading dim m) -> column-major dest (leading dim ldd), zero padding.
template <typename TS, typename TD>
__global__ void k_conv_colmajor(const void* src, int m, int64_t n, TD* dst, int ldd) {
  const int64_t total = (int64_t)ldd * n;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t col = idx / ldd;
    const int row = (int)(idx - col * ldd);
    const double v = row < m ? from_src<TS>(src, (size_t)col * m + row) : 0.0;
    dst[idx] = to_dt<TD>(v);
  }
}

// Row-major source (m x n, leading dim n) -> column-major dest, 32 x 32 tiles through shared.
template <typename TS, typename TD>
__global__ void k_conv_rowmajor(const void* src, int m, int64_t n, TD* dst, int ldd) {
  __shared__ double tile[32][33];
  const int64_t c0 = (int64_t)blockIdx.x * 32;
  const int r0 = blockIdx.y * 32;
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int r = r0 + i;
    const int64_t c = c0 + threadIdx.x;
    tile[i][threadIdx.x] = (r < m && c < n) ? from_src<TS>(src, (size_t)r * n + c) : 0.0;
  }
  __syncthreads();
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int64_t c = c0 + i;
    const int r = r0 + threadIdx.x;
    if (c < n && r < ldd) dst[(size_t)c * ldd + r] = to_dt<TD>(r < m ? tile[threadIdx.x][i] : 0.0);
  }
}

template <typename TS, typename TD>
static cudaError_t conv_t(const void* src, bool rowmajor, int m, int64_t n, void* dst, int ldd,
                          cudaStream_t st) {
  if (rowmajor) {
    dim3 grid((unsigned)((n + 31) / 32), (unsigned)((ldd + 31) / 32));
    { note_launch(); k_conv_rowmajor<TS, TD><<<grid, dim3(32, 8), 0, st>>>(src, m, n, (TD*)dst, ldd); }
  } else {
    int64_t total = (int64_t)ldd * n;
    int64_t g = (total + 255) / 256;
    if (g > 65535) g = 65535;
    { note_launch(); k_conv_colmajor<TS, TD><<<(unsigned)g, 256, 0, st>>>(src, m, n, (TD*)dst, ldd); }
  }
  return cudaGetLastError();
}

template <typename TS>
static cudaError_t conv_s(const void* src, bool rowmajor, int m, int64_t n, void* dst,
                          lp_dtype ddt, int ldd, cudaStream_t st) {
  switch (ddt) {
    case LP_F64: return conv_t<TS, double>(src, rowmajor, m, n, dst, ldd, st);
    case LP_F32: return conv_t<TS, float>(src, rowmajor, m, n, dst, ldd, st);
    case LP_BF16: return conv_t<TS, __nv_bfloat16>(src, rowmajor, m, n, dst, ldd, st);
    case LP_F16: return conv_t<TS, __half>(src, rowmajor, m, n, dst, ldd, st);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_convert_dense(const void* src, lp_dtype sdt, bool rowmajor, int m, int64_t n,
                                 void* dst, lp_dtype ddt, int ldd, cudaStream_t st) {
  if (sdt == LP_F64) return conv_s<double>(src, rowmajor, m, n, dst, ddt, ldd, st);
  if (sdt == LP_F32) return conv_s<float>(src, rowmajor, m, n, dst, ddt, ldd, st);
  if (sdt == LP_BF16) return conv_s<__nv_bfloat16>(src, rowmajor, m, n, dst, ddt, ldd, st);
  if (sdt == LP_F16) return conv_s<__half>(src, rowmajor, m, n, dst, ddt, ldd, st);
  return cudaErrorInvalidValue;
}

// Column-scaled low-precision copy: column j of the master matrix (column-major, leading dim
// lda, m rows) is multiplied by 2^-e_j, with e_j chosen so that max_i |a_ij| 2^-e_j lies in
// [0.5, 1), and rounded to TD; cs2[j] = 2^(2 e_j).  A power of two is exact in every format, so
// A D^2 A^T = A_s (S^2 D^2) A_s^T with A_s the stored copy and S = diag(2^e_j): the scales move
// into the FP32 weight of the product and the copy keeps the format's full relative precision
// whatever the column norms (FP16 would otherwise overflow or go subnormal).  One warp per
// column.
template <typename TS, typename TD>
__global__ void k_conv_colscaled(const TS* __restrict__ src, int lda, int m, int64_t n,
                                 TD* __restrict__ dst, int ldd, float* __restrict__ cs2) {
  const int lane = threadIdx.x & 31;
  const int64_t wid = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t col = wid; col < n; col += nw) {
    const TS* a = src + col * (int64_t)lda;
    double mx = 0.0;
    for (int r = lane; r < m; r += 32) mx = fmax(mx, fabs((double)a[r]));
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) mx = fmax(mx, __shfl_xor_sync(kFull, mx, off));
    int e = mx > 0.0 ? ilogb(mx) + 1 : 0;
    e = e < -60 ? -60 : (e > 60 ? 60 : e);
    if (lane == 0) cs2[col] = ldexpf(1.0f, 2 * e);
    TD* o = dst + col * (int64_t)ldd;
    for (int r = lane; r < ldd; r += 32) o[r] = to_dt<TD>(r < m ? ldexp((double)a[r], -e) : 0.0);
  }
}

template <typename TS, typename TD>
static cudaError_t conv_scaled_t(const void* src, int lda, int m, int64_t n, void* dst, int ldd,
                                 float* cs2, cudaStream_t st) {
  int64_t g = (n * 32 + 255) / 256;
  if (g > 8192) g = 8192;
  { note_launch(); k_conv_colscaled<TS, TD><<<(unsigned)g, 256, 0, st>>>((const TS*)src, lda, m, n, (TD*)dst, ldd, cs2); }
  return cudaGetLastError();
}

cudaError_t launch_convert_colscaled(const void* src, lp_dtype sdt, int lda, int m, int64_t n,
                                     void* dst, lp_dtype ddt, int ldd, float* cs2,
                                     cudaStream_t st) {
  if (sdt == LP_F32 && ddt == LP_BF16)
    return conv_scaled_t<float, __nv_bfloat16>(src, lda, m, n, dst, ldd, cs2, st);
  if (sdt == LP_F32 && ddt == LP_F16)
    return conv_scaled_t<float, __half>(src, lda, m, n, dst, ldd, cs2, st);
  if (sdt == LP_F64 && ddt == LP_BF16)
    return conv_scaled_t<double, __nv_bfloat16>(src, lda, m, n, dst, ldd, cs2, st);
  if (sdt == LP_F64 && ddt == LP_F16)
    return conv_scaled_t<double, __half>(src, lda, m, n, dst, ldd, cs2, st);
  return cudaErrorInvalidValue;
}

template <typename T>
__global__ void k_check_finite(const T* src, int64_t count, int* flag) {
  int bad = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x)
    if (!isfinite((double)src[i])) bad = 1;
  if (__any_sync(kFull, bad) && (threadIdx.x & 31) == 0) atomicOr(flag, 1);
}

cudaError_t launch_check_finite(const void* src, lp_dtype dt, int64_t count, int* flag,
                                cudaStream_t st) {
  int64_t g = (count + 255) / 256;
  if (g > 4096) g = 4096;
  if (g < 1) g = 1;
  if (dt == LP_F64)
    { note_launch(); k_check_finite<double><<<(unsigned)g, 256, 0, st>>>((const double*)src, count, flag); }
  else if (dt == LP_F32)
    { note_launch(); k_check_finite<float><<<(unsigned)g, 256, 0, st>>>((const float*)src, count, flag); }
  else
    return cudaErrorInvalidValue;
  return cudaGetLastError();
}

__global__ void k_set_scalars(double* sc, int slot, double v, int* fl, int fslot, int fv) {
  if (sc) sc[slot] = v;
  if (fl) fl[fslot] = fv;
}

cudaError_t launch_set(double* sc, int slot, double v, int* fl, int fslot, int fv,
                       cudaStream_t st) {
  { note_launch(); k_set_scalars<<<1, 1, 0, st>>>(sc, slot, v, fl, fslot, fv); }
  return cudaGetLastError();
}

// (W u)_i = sum_j sign_ij/sqrt(s) u[bucket_ij]
__global__ void k_apply_W(const int32_t* hb, int ss, const double* u, int64_t n, double* wu) {
  const double inv = 1.0 / sqrt((double)ss);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    double w = 0.0;
    for (int j = 0; j < ss; ++j) {
      const int32_t h = hb[i * ss + j];
      const double uv = u[h & 0x7fffffff];
      w += (h < 0) ? -uv : uv;
    }
    wu[i] = w * inv;
  }
}

cudaError_t launch_apply_W(const int32_t* hb, int ss, const double* u, int64_t n, double* wu,
                           cudaStream_t st) {
  int64_t g = (n + 255) / 256;
  if (g > 4096) g = 4096;
  if (g < 1) g = 1;
  { note_launch(); k_apply_W<<<(unsigned)g, 256, 0, st>>>(hb, ss, u, n, wu); }
  return cudaGetLastError();
}

// Dynamic shared-memory limits only ever go up: contexts on other threads may launch the same
// kernel concurrently with a larger need, and lowering the limit between their attribute call
// and their launch would make that launch fail.  The limit is raised for any size (not only
// above 48 KB): the 48 KB default covers static plus dynamic shared memory together.
// Resident CTAs per SM of a kernel at a block size and dynamic shared memory, queried once
// per (kernel, threads, smem) and cached: the launchers are also recorded into CUDA graphs,
// where nothing but the launches themselves should reach the runtime.
int occupancy_cached(const void* func, int threads, size_t smem) {
  static std::mutex mu;
  static std::map<std::tuple<const void*, int, size_t>, int> cache;
  std::lock_guard<std::mutex> lk(mu);
  const auto key = std::make_tuple(func, threads, smem);
  auto it = cache.find(key);
  if (it != cache.end()) return it->second;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, func, threads, smem) != cudaSuccess) {
    cudaGetLastError();
    per_sm = 0;
  }
  if (per_sm < 1) per_sm = 1;
  cache[key] = per_sm;
  return per_sm;
}

cudaError_t ensure_dyn_smem(const void* func, size_t bytes) {
  static std::mutex mu;
  static std::unordered_map<const void*, size_t> set;
  std::lock_guard<std::mutex> lk(mu);
  size_t& cur = set[func];
  if (bytes <= cur) return cudaSuccess;
  const cudaError_t e =
      cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess) cur = bytes;
  return e;
}

}  // namespace lpk
