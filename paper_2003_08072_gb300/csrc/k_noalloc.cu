// Allocation-free product y = A D^2 A^T v (and t = A^T v) for callers that cannot allocate
// device memory.  The per-CTA partial sums live in one file-scope __device__ array instead of
// a context workspace, so this entry point needs no lp_ctx and calls no allocator.
#include <mutex>
#include <string>

#include "dev_util.cuh"

namespace lpk {
int launch_coltile_capped(lp_dtype ta, ColArgs a, int num_sms, int max_grid, cudaStream_t st);
}

using namespace lpk;

namespace {

// 4 MiB of partial sums, held by every GPU that loads the library until the process exits.
constexpr size_t kScratchBytes = size_t(4) << 20;
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

// In host code g_scratch is only a host-side stand-in for the device symbol; its device
// address is looked up with the device current.  The lookup is repeated on every call made
// outside a stream capture (the address changes if the context is torn down and re-created,
// e.g. after cudaDeviceReset); during a capture the address cached by the last such call is
// used, so the first call on a device must come before any capture.
constexpr int kMaxDevices = 64;
void* g_scratch_dev[kMaxDevices] = {};
int g_num_sms[kMaxDevices] = {};
std::mutex g_setup_mu;

lp_status setup_device(int dev, cudaStream_t stream) {
  std::lock_guard<std::mutex> lock(g_setup_mu);
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(stream, &cap) != cudaSuccess) {
    cudaGetLastError();
    cap = cudaStreamCaptureStatusActive;   // unknown: do not touch the cache
  }
  if (cap != cudaStreamCaptureStatusNone) {
    if (g_scratch_dev[dev]) return LP_OK;
    lp_set_error("lp_normal_matvec_noalloc: the first call on a device must precede stream capture");
    return LP_ERR_ARG;
  }
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
  if (e != cudaSuccess || !p) return lp_cuda_fail(e, "cudaGetSymbolAddress(scratch)");
  if (!g_num_sms[dev]) {
    int sms = 0;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return lp_cuda_fail(e, "cudaDeviceGetAttribute");
    g_num_sms[dev] = sms;
  }
  g_scratch_dev[dev] = p;
  return LP_OK;
}

size_t dt_size(lp_dtype t) { return t == LP_F64 ? 8 : (t == LP_F32 ? 4 : 2); }

}  // namespace

extern "C" lp_status lp_normal_matvec_noalloc(const void* A, lp_dtype a_dtype, int32_t m, int64_t n,
                                              int64_t lda, const double* d2, const double* v,
                                              double* y, double* t, void* stream) {
  if (!A || !d2 || !v || !y) {
    lp_set_error("lp_normal_matvec_noalloc: NULL A, d2, v or y");
    return LP_ERR_ARG;
  }
  if (a_dtype != LP_F64 && a_dtype != LP_F32 && a_dtype != LP_BF16 && a_dtype != LP_F16) {
    lp_set_error("lp_normal_matvec_noalloc: unknown dtype");
    return LP_ERR_ARG;
  }
  const size_t es = dt_size(a_dtype);
  if (m < 1 || n < 1 || lda < m || (lda * (int64_t)es) % 16 != 0 ||
      reinterpret_cast<uintptr_t>(A) % 16 != 0) {
    lp_set_error("lp_normal_matvec_noalloc: need m >= 1, n >= 1, lda >= m, 16-byte aligned A and "
                 "columns (lda * element size a multiple of 16)");
    return LP_ERR_ARG;
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return lp_cuda_fail(e, "cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices) {
    lp_set_error("lp_normal_matvec_noalloc: device ordinal beyond 63");
    return LP_ERR_ARG;
  }
  lp_status st = setup_device(dev, (cudaStream_t)stream);
  if (st != LP_OK) return st;
  // Each CTA writes m partial sums of the accumulator type; the grid must fit the scratch.
  const size_t acc = (a_dtype == LP_F64) ? 8 : 4;
  const int64_t max_grid = (int64_t)(kScratchBytes / (acc * (size_t)m));
  const int sms = g_num_sms[dev];
  if (max_grid < sms || m > 8192) {
    lp_set_error("lp_normal_matvec_noalloc: m = " + std::to_string(m) +
                 " exceeds the 4 MiB scratch limit of " +
                 std::to_string(std::min<int64_t>(8192, kScratchBytes / (acc * (size_t)sms))) +
                 " rows for this dtype on this device");
    return LP_ERR_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  ColArgs a{};
  a.A = A;
  a.lda = lda;
  a.m = m;
  a.n = n;
  a.v = v;
  a.d2 = d2;
  a.colout = t;
  a.part = g_scratch_dev[dev];
  a.fl = nullptr;
  a.skip_if_done = 0;
  const int nblk = launch_coltile_capped(a_dtype, a, sms, (int)max_grid, s);
  if (nblk < 0) {
    lp_set_error("lp_normal_matvec_noalloc: unsupported shape");
    return LP_ERR_ARG;
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return lp_cuda_fail(e, "lp_normal_matvec_noalloc launch");
  RedArgs r{};
  r.mode = RED_PLAIN;
  r.part = g_scratch_dev[dev];
  r.nblk = nblk;
  r.nout = 1;
  r.m = m;
  r.acc_f64 = (a_dtype == LP_F64);
  r.out0 = y;
  e = launch_reduce(r, s);
  if (e != cudaSuccess) return lp_cuda_fail(e, "lp_normal_matvec_noalloc reduce");
  return LP_OK;
}
