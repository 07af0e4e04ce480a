// Sparse (CSC) passes over A: the same two column operations as the dense column-tile
// kernels (see k_coltile.cu), for a matrix stored by columns (column pointers, row ids,
// values).  Eight lanes share a column: they gather v[row] from shared memory for the
// column dot, reduce with three shuffles, and scatter a_i * coef_i into per-CTA row
// accumulators in shared memory.  Each CTA writes its accumulators once as partials.
#include "dev_util.cuh"

namespace lpk {

template <typename TV, typename ACC, int MODE>
__global__ void __launch_bounds__(512) k_csc(CscArgs a) {
  constexpr int NOUT = (MODE == MODE_RESID) ? 2 : 1;
  if (a.skip_if_done && a.fl[FL_DONE]) return;
  extern __shared__ __align__(16) unsigned char smraw[];
  ACC* vs = reinterpret_cast<ACC*>(smraw);
  ACC* ys = vs + a.m;
  const TV* vals = reinterpret_cast<const TV*>(a.vals);
  for (int i = threadIdx.x; i < a.m; i += blockDim.x) {
    double vv;
    if (a.dz) {   // fused CG direction update d = z + beta d_old
      vv = fma(a.sc[SC_BETA], a.dold[i], a.dz[i]);
      if (blockIdx.x == 0) a.dnew[i] = vv;
    } else {
      vv = a.v[i];
    }
    vs[i] = (ACC)vv;
#pragma unroll
    for (int o = 0; o < NOUT; ++o) ys[o * a.m + i] = (ACC)0;
  }
  __syncthreads();
  double sigmu = 0.0;
  if constexpr (MODE == MODE_RESID) sigmu = a.sc[SC_SIGMU];
  const int lane = threadIdx.x & 31, grp = lane >> 3, gl = lane & 7;
  const int nwarps = blockDim.x >> 5;
  int64_t gw = (int64_t)blockIdx.x * nwarps + (threadIdx.x >> 5);
  const int64_t tw = (int64_t)gridDim.x * nwarps;
  // Columns are short (a few nonzeros each), so a group's work is one round trip to memory
  // per column: the next column's pointers are loaded while the current one is processed,
  // the lane's first nonzero (value, row) stays in registers from the dot to the scatter,
  // and the column's scalars are loaded together with its nonzeros.
  int64_t col = gw * 4 + grp;
  int64_t k0 = 0, k1 = 0;
  if (col < a.n) {
    k0 = a.colptr[col];
    k1 = a.colptr[col + 1];
  }
  for (; gw * 4 < a.n; gw += tw, col += tw * 4) {
    const bool valid = col < a.n;
    const int64_t ncol = col + tw * 4;
    int64_t nk0 = 0, nk1 = 0;
    if (ncol < a.n) {
      nk0 = a.colptr[ncol];
      nk1 = a.colptr[ncol + 1];
    }
    const bool has0 = valid && k0 + gl < k1;
    const ACC v0 = has0 ? (ACC)vals[k0 + gl] : (ACC)0;
    const int r0 = has0 ? a.rowidx[k0 + gl] : 0;
    double w = 1.0, xi = 0.0, si = 1.0, ci = 0.0;
    if (valid) {
      if constexpr (MODE == MODE_NORMAL) {
        if (a.d2) w = a.d2[col];
      } else {
        xi = a.x[col];
        si = a.s[col];
        ci = a.c[col];
      }
    }
    ACC dot = has0 ? v0 * vs[r0] : (ACC)0;
    for (int64_t k = k0 + gl + 8; k < k1; k += 8) dot = fma((ACC)vals[k], vs[a.rowidx[k]], dot);
    dot += __shfl_xor_sync(kFull, dot, 4);
    dot += __shfl_xor_sync(kFull, dot, 2);
    dot += __shfl_xor_sync(kFull, dot, 1);
    if (valid) {
      ACC cf[NOUT];
      if constexpr (MODE == MODE_NORMAL) {
        cf[0] = (ACC)(w * (double)dot);
        if (a.colout && gl == 0) a.colout[col] = (double)dot;
      } else {
        const double rdv = (double)dot + si - ci;
        cf[0] = (ACC)xi;
        cf[1] = (ACC)(sigmu / si + (xi / si) * rdv);
        if (gl == 0) a.colout[col] = rdv;
      }
      if (has0) {
#pragma unroll
        for (int o = 0; o < NOUT; ++o) atomicAdd(&ys[o * a.m + r0], cf[o] * v0);
      }
      for (int64_t k = k0 + gl + 8; k < k1; k += 8) {
        const int r = a.rowidx[k];
        const ACC av = (ACC)vals[k];
#pragma unroll
        for (int o = 0; o < NOUT; ++o) atomicAdd(&ys[o * a.m + r], cf[o] * av);
      }
    }
    k0 = nk0;
    k1 = nk1;
  }
  __syncthreads();
  ACC* part = reinterpret_cast<ACC*>(a.part);
  for (int i = threadIdx.x; i < a.m; i += blockDim.x)
#pragma unroll
    for (int o = 0; o < NOUT; ++o)
      part[((size_t)blockIdx.x * NOUT + o) * a.m + i] = ys[o * a.m + i];
}

int csc_max_grid(int num_sms) { return num_sms * 4; }

template <typename TV, typename ACC, int MODE>
static int launch_csc_t(CscArgs a, int num_sms, cudaStream_t st) {
  constexpr int NOUT = (MODE == MODE_RESID) ? 2 : 1;
  const size_t smem = (size_t)a.m * sizeof(ACC) * (1 + NOUT);
  if (smem > 220 * 1024) return -1;
  auto kern = k_csc<TV, ACC, MODE>;
  if (ensure_dyn_smem((const void*)kern, smem) != cudaSuccess) return -1;
  int per_sm = occupancy_cached((const void*)kern, 512, smem);
  if (per_sm > 4) per_sm = 4;   // the partials buffer holds csc_max_grid rows
  int64_t grid = (int64_t)num_sms * per_sm;
  const int64_t need = (a.n + 63) / 64;
  if (grid > need) grid = need;
  if (grid < 1) grid = 1;
  { note_launch(); kern<<<(unsigned)grid, 512, smem, st>>>(a); }
  return (int)grid;
}

int launch_csc(lp_dtype tv, bool acc_f64, int mode, CscArgs a, int num_sms, cudaStream_t st) {
  if (mode == MODE_NORMAL) {
    if (tv == LP_F64) return launch_csc_t<double, double, MODE_NORMAL>(a, num_sms, st);
    if (tv == LP_F32)
      return acc_f64 ? launch_csc_t<float, double, MODE_NORMAL>(a, num_sms, st)
                     : launch_csc_t<float, float, MODE_NORMAL>(a, num_sms, st);
    return -1;
  }
  if (tv == LP_F64) return launch_csc_t<double, double, MODE_RESID>(a, num_sms, st);
  if (tv == LP_F32) return launch_csc_t<float, double, MODE_RESID>(a, num_sms, st);
  return -1;
}

// CSR -> CSC on the device: count per column, scan (host-provided offsets), scatter, then
// sort each column's entries by row so the layout is deterministic.
__global__ void k_csr_count(const int64_t* indptr, const int32_t* indices, int m, int64_t nnz,
                            int64_t* colcnt) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nnz;
       k += (int64_t)gridDim.x * blockDim.x)
    atomicAdd(reinterpret_cast<unsigned long long*>(&colcnt[indices[k] + 1]), 1ull);
}

template <typename TV>
__global__ void k_csr_scatter(const int64_t* indptr, const int32_t* indices, const TV* vals, int m,
                              const int64_t* colptr, int64_t* cursor, int32_t* rowidx,
                              TV* cvals) {
  for (int row = blockIdx.x; row < m; row += gridDim.x) {
    for (int64_t k = indptr[row] + threadIdx.x; k < indptr[row + 1]; k += blockDim.x) {
      const int32_t col = indices[k];
      const int64_t pos = colptr[col] + (int64_t)atomicAdd(
                                            reinterpret_cast<unsigned long long*>(&cursor[col]), 1ull);
      rowidx[pos] = row;
      cvals[pos] = vals[k];
    }
  }
}

template <typename TV>
__global__ void k_csc_sortcols(const int64_t* colptr, int64_t n, int32_t* rowidx, TV* cvals) {
  for (int64_t col = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; col < n;
       col += (int64_t)gridDim.x * blockDim.x) {
    const int64_t k0 = colptr[col], k1 = colptr[col + 1];
    for (int64_t i = k0 + 1; i < k1; ++i) {   // insertion sort (columns are short)
      const int32_t r = rowidx[i];
      const TV v = cvals[i];
      int64_t j = i - 1;
      while (j >= k0 && rowidx[j] > r) {
        rowidx[j + 1] = rowidx[j];
        cvals[j + 1] = cvals[j];
        --j;
      }
      rowidx[j + 1] = r;
      cvals[j + 1] = v;
    }
  }
}

__global__ void k_inclusive_scan_i64(int64_t* a, int64_t len) {
  // single-CTA chunked scan (len = n + 1)
  __shared__ int64_t sums[1024];
  const int t = threadIdx.x;
  const int64_t per = (len + 1023) / 1024;
  const int64_t b0 = t * per, b1 = min(len, b0 + per);
  int64_t local = 0;
  for (int64_t i = b0; i < b1; ++i) local += a[i];
  sums[t] = local;
  __syncthreads();
  for (int off = 1; off < 1024; off <<= 1) {
    int64_t v = (t >= off) ? sums[t - off] : 0;
    __syncthreads();
    sums[t] += v;
    __syncthreads();
  }
  int64_t run = sums[t] - local;
  for (int64_t i = b0; i < b1; ++i) {
    run += a[i];
    a[i] = run;
  }
}

cudaError_t csr_to_csc(const int64_t* indptr, const int32_t* indices, const void* vals,
                       lp_dtype dt, int m, int64_t n, int64_t nnz, int64_t* colptr,
                       int64_t* cursor, int32_t* rowidx, void* cvals, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(colptr, 0, (n + 1) * sizeof(int64_t), st);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(cursor, 0, n * sizeof(int64_t), st);
  if (e != cudaSuccess) return e;
  int64_t g = (nnz + 255) / 256;
  if (g > 8192) g = 8192;
  if (g < 1) g = 1;
  { note_launch(); k_csr_count<<<(unsigned)g, 256, 0, st>>>(indptr, indices, m, nnz, colptr); }
  { note_launch(); k_inclusive_scan_i64<<<1, 1024, 0, st>>>(colptr, n + 1); }
  const int rg = m < 8192 ? m : 8192;
  int64_t sg = (n + 255) / 256;
  if (sg > 8192) sg = 8192;
  if (sg < 1) sg = 1;
  if (dt == LP_F32) {
    { note_launch(); k_csr_scatter<float><<<rg, 256, 0, st>>>(indptr, indices, (const float*)vals, m, colptr,
                                             cursor, rowidx, (float*)cvals); }
    { note_launch(); k_csc_sortcols<float><<<(unsigned)sg, 256, 0, st>>>(colptr, n, rowidx, (float*)cvals); }
  } else {
    { note_launch(); k_csr_scatter<double><<<rg, 256, 0, st>>>(indptr, indices, (const double*)vals, m, colptr,
                                              cursor, rowidx, (double*)cvals); }
    { note_launch(); k_csc_sortcols<double><<<(unsigned)sg, 256, 0, st>>>(colptr, n, rowidx, (double*)cvals); }
  }
  return cudaGetLastError();
}

}  // namespace lpk
