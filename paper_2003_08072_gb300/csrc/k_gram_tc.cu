// Gram product Q = G G^T of the sketch (Alg. 1 step 2, Eq. pdprecond) on the tensor cores.
//
// Q must be accurate to far below 1/kappa(Q) (kappa(Q) reaches ~1e10 late in the IPM), so a
// single 16-bit product is useless; the product is made exact instead, by an error-free split
// of G into small integers (the splitting idea of Ozaki, Ogita, Oishi & Rump, "Error-free
// transformations of matrix multiplication by using fast routines of matrix multiplication and
// its applications", Numer. Algorithms 2012).  Row i of G is scaled by 2^-e_i (max |G_ik| <
// 2^e_i) and each scaled entry x = G_ik 2^-e_i in (-1, 1) is written as
//     x = sum_{s<9} d_s 2^(-6(s+1)) + r,   |d_0| <= 64, |d_s| <= 33 (s > 0), |r| <= 2^-55,
// with integer digits d_s (exact in BF16).  Then
//     Q_ij = 2^(e_i + e_j - 12) sum_{l<9} 2^(-6 l) L_l[i][j],   L_l = sum_{s+t=l} D_s D_t^T,
// dropping the products with s + t >= 9 (each below 2^-52.5 of 2^(e_i + e_j), so an entry of
// Q errs by ~2^-52.5 sqrt(w) |G_i| |G_j|, finer than the double-float product this replaces).
// Each L_l is a sum of integer products; over a chunk of 1024 columns of G every partial sum
// stays below 2^24 (at most 2 products of 64 x 33 and 7 of 33 x 33 per column and level,
// 4096 for level 0), so FP32 accumulation in the tensor core is exact.  The level sums of a
// chunk are folded into double-float per thread.
//
// Layout.  The digits are written in the order the tensor core reads them: for each block of
// 16 columns of G and each slice, the row groups' 8 x 16 core-matrix pairs (8 rows x 16 bytes
// each) are contiguous, [kb][slice][row group][2][8][8].  A tile's operands for one k block
// are then one contiguous range per slice (A: 128 rows = 4 KB, B: 32 rows = 1 KB), fetched by
// cp.async.bulk into a 4-stage shared-memory ring; the no-swizzle K-major matrix descriptor
// addresses a slice with leading byte offset 128 (the next 8 columns) and stride byte offset
// 256 (the next 8 rows).  Because B's slices lie one after another, the products of A slice s
// with all B slices t <= 8 - s are one MMA of N = 32 (9 - s) whose output columns are exactly
// the level accumulators s .. 8: ten MMAs per k block instead of 45, each reading A once.
//
// k_gram_tc: one CTA per (128 x 32 tile of the lower triangle of Q, range of column chunks),
// 128 threads, one CTA per SM (180 KB of shared memory).  Thread 0 issues the bulk copies
// (completing on a full mbarrier per stage) and the tcgen05.mma (kind::f16, BF16 x BF16 ->
// FP32, M = 128, N = 32 (9 - s) <= 256, K = 16) into nine level accumulators in tensor memory
// (9 x 32 of its 512 columns); tcgen05.commit arrives on the stage's empty mbarrier when its
// products are done.  At the end of each chunk all four warps read the accumulators back with tcgen05.ld
// (thread t owns row t of the tile) and add them into the CTA's double-float partial tile.
// Every mbarrier wait is bounded by the global timer (1 s); a wait that gives up sets
// FL_TIMEOUT, the copies already issued are waited for (again bounded) and the CTA still
// frees its tensor memory.
#include <algorithm>

#include "dev_util.cuh"

namespace lpk {

namespace {

constexpr int kTM = 128;      // rows of a tile (TMEM lanes)
constexpr int kTN = 32;       // columns of a tile
constexpr int kKB = 16;       // columns of G per pipeline stage (one MMA K step)
constexpr int kSl = 9;        // digit slices (and level accumulators)
constexpr int kKC = 1024;     // columns of G per exactly accumulated chunk
constexpr int kNS = 4;        // pipeline stages
constexpr int kCore = 256;    // bytes of one row group's two core matrices (8 rows x 16 cols)
constexpr int kASlice = (kTM / 8) * kCore;      // 4 KB: one slice of the A tile
constexpr int kBSlice = (kTN / 8) * kCore;      // 1 KB: one slice of the B tile
constexpr int kABytes = kSl * kASlice;          // 36 KB
constexpr int kBBytes = kSl * kBSlice;          // 9 KB
constexpr int kStage = kABytes + kBBytes;       // 45 KB
constexpr int kSmemBytes = kNS * kStage + 256;  // stages, mbarriers, TMEM address
constexpr uint64_t kWaitNs = 1000000000ull;

// Instruction descriptor of tcgen05.mma kind::f16: FP32 accumulator (bits 4-5 = 1), BF16 A
// and B (bits 7-9, 10-12 = 1), both K-major (bits 15, 16 = 0), N >> 3 in bits 17-22 and
// M >> 4 in bits 24-28.
__host__ __device__ constexpr uint32_t idesc(int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) |
         ((uint32_t)(kTM >> 4) << 24);
}

__device__ __forceinline__ uint32_t su32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// Shared-memory matrix descriptor, no swizzle, K-major: core matrices of 8 rows x 16 bytes
// (128 B contiguous), adjacent along K 128 B apart (leading byte offset), adjacent 8-row groups
// 256 B apart (stride byte offset); bits 46-47 hold the descriptor version 1.  The start
// address is bits 0-13 (address >> 4), so later slices and stages add (offset >> 4) to it.
__device__ __forceinline__ uint64_t sdesc(uint32_t addr) {
  return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)(128u >> 4) << 16) |
         ((uint64_t)((uint32_t)kCore >> 4) << 32) | (1ull << 46);
}

__device__ __forceinline__ void mbar_arrive_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(bar)),
               "r"(bytes)
               : "memory");
}

// global -> shared bulk copy completing on an mbarrier (16-byte aligned, size multiple of 16)
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes,
                                         uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          dst),
      "l"(src), "r"(bytes), "r"(su32(bar))
      : "memory");
}

__device__ __forceinline__ void mbar_init(uint64_t* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try(uint64_t* bar, unsigned parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(su32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ uint64_t gtimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Bounded wait for the phase of `bar` with the given parity; false after kWaitNs.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity) {
  if (mbar_try(bar, parity)) return true;
  const uint64_t t0 = gtimer();
  for (unsigned spin = 1;; ++spin) {
    if (mbar_try(bar, parity)) return true;
    if ((spin & 255u) == 0 && gtimer() - t0 > kWaitNs) return false;
  }
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tc_mma(uint32_t dtmem, uint64_t adesc, uint64_t bdesc,
                                       uint32_t id, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(dtmem),
      "l"(adesc), "l"(bdesc), "r"(id), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void tc_commit(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          su32(bar))
      : "memory");
}

// 16 consecutive 32-bit columns of this warp's 32 TMEM lanes (thread = lane)
__device__ __forceinline__ void tc_ld16(uint32_t taddr, uint32_t (&v)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
      "%11, %12, %13, %14, %15}, [%16];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
        "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
        "=r"(v[14]), "=r"(v[15])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Tiles of the lower triangle of Q: row block I (128 rows), column blocks J = 0..min(4I+3, NT-1).
__host__ __device__ __forceinline__ int tiles_in_row(int I, int NT) {
  return 4 * I + 4 < NT ? 4 * I + 4 : NT;
}

}  // namespace

struct GramTcArgs {
  const __nv_bfloat16* D;   // digits in tile order [kb][slice][row group][2][8][8]
  int ngroups;              // row groups of 8 (rows_p / 8)
  int nkb;                  // k blocks of 16 columns (wp / 16)
  int NT;                   // column blocks of 32 (mp / 32)
  int ntile;                // tiles in the lower triangle
  int chunks_per_cta;       // chunks of kKC columns per CTA (blockIdx.y selects the range)
  float2* part;             // [gridDim.y][ntile][128][32] double-float partial tiles
  int* fl;
};

__device__ __forceinline__ void fold_barrier() {   // warps 0-3 only (the TMEM lanes' owners)
  asm volatile("bar.sync 1, 128;" ::: "memory");
}

// Warp roles: warp 4 (lane 0) issues the bulk copies; warp 0 (lane 0) issues the products;
// warps 0-3 read the accumulators back (warp w owns TMEM lanes 32w .. 32w + 31).
__global__ void __launch_bounds__(160, 1) k_gram_tc(GramTcArgs a) {
  extern __shared__ __align__(1024) unsigned char smem[];
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + kNS * kStage);
  uint64_t* empty = full + kNS;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + kNS * kStage + 128);
  // s_pfail: the producer gave up; s_gfail: a thread of warps 0-3 gave up (read by them only
  // after a barrier of theirs, so that all four take the same branch)
  __shared__ int s_pfail, s_gfail, s_issued, s_consumed;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  int tile = blockIdx.x, I = 0;
  while (tile >= tiles_in_row(I, a.NT)) {
    tile -= tiles_in_row(I, a.NT);
    ++I;
  }
  const int J = tile;
  const int kb_per_chunk = kKC / kKB;
  const int kb0 = blockIdx.y * a.chunks_per_cta * kb_per_chunk;
  const int kb1 = min(a.nkb, kb0 + a.chunks_per_cta * kb_per_chunk);
  float2* out = a.part + (((size_t)blockIdx.y * a.ntile + blockIdx.x) * kTM + tid) * kTN;
  if (kb0 >= kb1) {   // an empty column range: its partial tile is zero
    if (tid < kTM)
      for (int c = 0; c < kTN; ++c) out[c] = make_float2(0.f, 0.f);
    return;
  }

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(
                     su32(tmem_slot))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    for (int i = 0; i < kNS; ++i) {
      mbar_init(&full[i]);
      mbar_init(&empty[i]);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    s_pfail = 0;
    s_gfail = 0;
    s_issued = 0;
    s_consumed = 0;
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const uint32_t sbase = su32(smem);
  const int nkb = kb1 - kb0;

  if (warp == 4) {
    // producer: block q of this CTA into stage q % kNS once the products of block q - kNS,
    // the stage's last reader, are done
    if (lane == 0) {
      const unsigned char* gD = reinterpret_cast<const unsigned char*>(a.D);
      const size_t slice_bytes = (size_t)a.ngroups * kCore;
      const size_t kb_bytes = kSl * slice_bytes;
      const size_t a_off = (size_t)(I * (kTM / 8)) * kCore;
      const size_t b_off = (size_t)(J * (kTN / 8)) * kCore;
      for (int q = 0; q < nkb; ++q) {
        const int st = q % kNS;
        if (q >= kNS && !mbar_wait(&empty[st], ((q / kNS) - 1) & 1)) {
          s_pfail = 1;
          break;
        }
        if (*(volatile int*)&s_gfail) break;
        const unsigned char* src = gD + (size_t)(kb0 + q) * kb_bytes;
        const uint32_t dst = sbase + st * kStage;
        mbar_arrive_tx(&full[st], (uint32_t)kStage);
#pragma unroll
        for (int sl = 0; sl < kSl; ++sl) {
          bulk_g2s(dst + sl * kASlice, src + sl * slice_bytes + a_off, (uint32_t)kASlice,
                   &full[st]);
          bulk_g2s(dst + kABytes + sl * kBSlice, src + sl * slice_bytes + b_off,
                   (uint32_t)kBSlice, &full[st]);
        }
        s_issued = q + 1;
      }
    }
    __syncwarp();
  } else {
    const uint64_t adesc0 = sdesc(sbase), bdesc0 = sdesc(sbase + kABytes);
    // The level sums of a finished chunk, scaled by 2^(-6 l) and summed in double-float, are
    // added into this CTA's partial tile (row tid, 32 columns), which only this CTA touches.
    const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);
    auto fold = [&](bool first) {
#pragma unroll 1
      for (int cg = 0; cg < kTN / 16; ++cg) {
        float hs[16], ls[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) hs[j] = ls[j] = 0.f;
#pragma unroll
        for (int l = 0; l < kSl; ++l) {
          uint32_t v[16];
          tc_ld16(lane_base + (uint32_t)(l * kTN + cg * 16), v);
          const float sc = __int_as_float((127 - 6 * l) << 23);   // 2^(-6 l), exact
#pragma unroll
          for (int j = 0; j < 16; ++j) df_add(hs[j], ls[j], __uint_as_float(v[j]) * sc, 0.f);
        }
        float4* o = reinterpret_cast<float4*>(out + cg * 16);
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          float h0 = hs[2 * j], l0 = ls[2 * j], h1 = hs[2 * j + 1], l1 = ls[2 * j + 1];
          if (!first) {
            const float4 p = o[j];
            df_add(h0, l0, p.x, p.y);
            df_add(h1, l1, p.z, p.w);
          }
          o[j] = make_float4(h0, l0, h1, l1);
        }
      }
    };
    bool first_chunk = true;
    for (int c0 = 0; c0 < nkb; c0 += kb_per_chunk) {
      const int c1 = min(nkb, c0 + kb_per_chunk);
      if (tid == 0) {
        for (int q = c0; q < c1; ++q) {
          const int st = q % kNS;
          if (*(volatile int*)&s_pfail || !mbar_wait(&full[st], (q / kNS) & 1)) {
            s_gfail = 1;
            break;
          }
          tc_fence_after();
          // A slice s times B slices 0 .. 8 - s (levels s .. 8, adjacent accumulators); slice 0
          // writes every level, so its products are the chunk's first and overwrite
          const uint32_t first_acc = (q == c0) ? 0u : 1u;
          const uint32_t soff = (uint32_t)(st * kStage) >> 4;
          tc_mma(tmem, adesc0 + soff, bdesc0 + soff, idesc(256), first_acc);
          tc_mma(tmem + 8 * kTN, adesc0 + soff, bdesc0 + soff + (uint32_t)(8 * kBSlice >> 4),
                 idesc(kTN), first_acc);
#pragma unroll
          for (int s = 1; s < kSl; ++s)
            tc_mma(tmem + (uint32_t)(s * kTN), adesc0 + soff + (uint32_t)(s * kASlice >> 4),
                   bdesc0 + soff, idesc((kSl - s) * kTN), 1u);
          tc_commit(&empty[st]);
          s_consumed = q + 1;
        }
      }
      __syncwarp();
      fold_barrier();
      // all products of the chunk are done once the last block's empty barrier has fired
      if (!*(volatile int*)&s_gfail) {
        const int ql = c1 - 1;
        if (!mbar_wait(&empty[ql % kNS], (ql / kNS) & 1)) s_gfail = 1;
      }
      fold_barrier();
      if (*(volatile int*)&s_gfail) break;
      tc_fence_after();
      fold(first_chunk);
      first_chunk = false;
      tc_fence_before();
      fold_barrier();
    }
  }
  __syncthreads();
  if (s_pfail || s_gfail) {
    // let copies and products already issued finish (bounded) before the memory goes away
    if (tid == 0) {
      if (a.fl) a.fl[FL_TIMEOUT] = 1;
      for (int q = s_consumed; q < s_issued; ++q) mbar_wait(&full[q % kNS], (q / kNS) & 1);
      if (s_consumed > 0)
        mbar_wait(&empty[(s_consumed - 1) % kNS], ((s_consumed - 1) / kNS) & 1);
    }
    __syncthreads();
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem) : "memory");
}

// Row exponents: e_i with max_k |G_ik| < 2^e_i (from the hi part of the double-float split;
// 0 for an all-zero or padding row).  k_row_max spreads the columns over blockIdx.y and
// combines the blocks' row maxima with an integer atomic max on the float bits (non-negative
// floats order like their bit patterns) in ex, zeroed before; k_row_exp turns them into
// exponents in place.
__global__ void k_row_max(const float* __restrict__ Gh, int ldg, int m, int w, int* __restrict__ ex) {
  __shared__ float red[8][33];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int row = blockIdx.x * 32 + tx;
  const int per = (w + gridDim.y - 1) / gridDim.y;
  const int k0 = blockIdx.y * per, k1 = min(w, k0 + per);
  float mx = 0.f;
  if (row < m)
    for (int k = k0 + ty; k < k1; k += 8) mx = fmaxf(mx, fabsf(Gh[(size_t)k * ldg + row]));
  red[ty][tx] = mx;
  __syncthreads();
  if (ty == 0 && row < m) {
#pragma unroll
    for (int j = 1; j < 8; ++j) mx = fmaxf(mx, red[j][tx]);
    if (mx > 0.f) atomicMax(&ex[row], __float_as_int(mx));
  }
}

__global__ void k_row_exp(int m, int rows_p, int* __restrict__ ex) {
  const int row = blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= rows_p) return;
  const float mx = __int_as_float(ex[row]);
  int e = 0;
  if (row < m && mx > 0.f) frexpf(mx, &e);
  ex[row] = row < m ? e : 0;
}

// Digits of the scaled rows, written in tile order [kb][slice][row group][2][8][8] (k block of
// 16 columns, slice, 8-row group, 8-column half, row in the group, column in the half) for
// rows < rows_p and columns < wp, zero outside m x w.  A 32-row x 64-column block is staged
// through shared memory so that G is read along its columns.
__global__ void __launch_bounds__(256) k_ozaki_digits(const float* __restrict__ Gh,
                                                      const float* __restrict__ Gl, int ldg, int m,
                                                      int w, int ngroups,
                                                      const int* __restrict__ ex,
                                                      __nv_bfloat16* __restrict__ D) {
  __shared__ float sh[64][33], sl[64][33];
  const int r0 = blockIdx.y * 32, k0 = blockIdx.x * 64;
  for (int e = threadIdx.x; e < 32 * 64; e += 256) {
    const int r = e & 31, kk = e >> 5, row = r0 + r, k = k0 + kk;
    const bool in = row < m && k < w;
    sh[kk][r] = in ? Gh[(size_t)k * ldg + row] : 0.f;
    sl[kk][r] = in ? Gl[(size_t)k * ldg + row] : 0.f;
  }
  __syncthreads();
  // thread -> (row in group, column in half); loop over the 4 groups x 8 halves of the block,
  // so a warp writes 4 rows x 8 columns = 64 contiguous bytes per slice
  const int e8 = threadIdx.x & 7, r8 = (threadIdx.x >> 3) & 7, part = threadIdx.x >> 6;
  for (int it = part; it < 4 * 8; it += 4) {
    const int gl = it >> 3, half = it & 7;   // group within the block, 8-column half
    const int r = gl * 8 + r8, kk = half * 8 + e8;
    const int row = r0 + r, k = k0 + kk;
    const float sc = __int_as_float((127 - ex[row]) << 23);   // 2^(-e_i), |e_i| < 127
    float rh = sh[kk][r] * sc, rl = sl[kk][r] * sc;            // x = rh + rl, |x| < 1
    const int kb = k >> 4, hk = (k >> 3) & 1, g = row >> 3;
    __nv_bfloat16* dst =
        D + (((size_t)kb * kSl * ngroups + g) * 2 + hk) * 64 + r8 * 8 + e8;
    const size_t sstep = (size_t)ngroups * 128;   // elements of one slice of a k block
#pragma unroll
    for (int s = 0; s < kSl; ++s) {
      const float th = rh * 64.f, tl = rl * 64.f;   // exact scalings
      const float d = rintf(th + tl);
      rh = th - d;                                  // exact: |th - d| < 1 + |tl|
      rl = tl;
      dst[s * sstep] = __float2bfloat16_rn(d);      // |d| <= 64: exact in BF16
    }
  }
}

// Q (row-major mp x mp, full symmetric, identity on the padding) from the partial tiles.
__global__ void k_gram_tc_finish(const float2* __restrict__ part, int nsplit, int ntile, int NT,
                                 const int* __restrict__ ex, int m, int mp,
                                 double* __restrict__ Q) {
  const int64_t total = (int64_t)mp * (mp + 1) / 2;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    int row = (int)((sqrt(8.0 * (double)idx + 1.0) - 1.0) * 0.5);
    while ((int64_t)row * (row + 1) / 2 > idx) --row;
    while ((int64_t)(row + 1) * (row + 2) / 2 <= idx) ++row;
    const int col = (int)(idx - (int64_t)row * (row + 1) / 2);
    double v;
    if (row >= m || col >= m) {
      v = (row == col) ? 1.0 : 0.0;
    } else {
      const int I = row / kTM, J = col / kTN;
      int t = J;
      for (int i = 0; i < I; ++i) t += tiles_in_row(i, NT);
      const size_t off = ((size_t)t * kTM + (row % kTM)) * kTN + (col % kTN);
      double sh = 0.0, slo = 0.0;
      for (int sp = 0; sp < nsplit; ++sp) {
        const float2 p = part[(size_t)sp * ntile * kTM * kTN + off];
        sh += (double)p.x;
        slo += (double)p.y;
      }
      v = ldexp(sh + slo, ex[row] + ex[col] - 12);
    }
    Q[(size_t)row * mp + col] = v;
    Q[(size_t)col * mp + row] = v;
  }
}

// ---- host side -------------------------------------------------------------------------

int gram_tc_rows(int m) { return (m + kTM - 1) / kTM * kTM; }
int gram_tc_pitch(int w) { return (w + 63) / 64 * 64; }

static int gram_tc_ntile(int m, int mp) {
  const int MT = gram_tc_rows(m) / kTM, NT = mp / kTN;
  int n = 0;
  for (int I = 0; I < MT; ++I) n += tiles_in_row(I, NT);
  return n;
}

// Splits of the column chunks over CTAs: about two CTAs per SM in total.
// Splits of the column chunks over CTAs.  One CTA per SM at a time, so a launch takes about
// (waves of CTAs) x (chunks per CTA) chunk times; the smallest split reaching the least such
// product is taken (fewer partial tiles to write and sum).
int gram_tc_split(int m, int mp, int w, int num_sms) {
  const int nchunks = (gram_tc_pitch(w) + kKC - 1) / kKC;
  const int64_t ntile = gram_tc_ntile(m, mp);
  int best = 1;
  int64_t best_cost = -1;
  for (int split = 1; split <= nchunks; ++split) {
    const int per_cta = (nchunks + split - 1) / split;
    if ((nchunks + per_cta - 1) / per_cta != split) continue;   // no CTA without columns
    const int64_t waves = (ntile * split + num_sms - 1) / num_sms;
    const int64_t cost = waves * per_cta;
    if (best_cost < 0 || cost < best_cost) {
      best = split;
      best_cost = cost;
    }
  }
  return best;
}

size_t gram_tc_digit_bytes(int m, int w) {
  return (size_t)kSl * gram_tc_rows(m) * gram_tc_pitch(w) * sizeof(__nv_bfloat16);
}
size_t gram_tc_part_bytes(int m, int mp, int w, int num_sms) {
  return (size_t)gram_tc_split(m, mp, w, num_sms) * gram_tc_ntile(m, mp) * kTM * kTN *
         sizeof(float2);
}

cudaError_t launch_gram_tc(const float* Gdf, int ldg, int m, int w, int mp, double* Q,
                           __nv_bfloat16* digits, int* ex, float2* part, int num_sms, int* fl,
                           cudaStream_t st) {
  const int rows_p = gram_tc_rows(m), wp = gram_tc_pitch(w);
  const float* Gh = Gdf;
  const float* Gl = Gdf + (size_t)ldg * w;
  {
    cudaError_t e0 = cudaMemsetAsync(ex, 0, (size_t)rows_p * sizeof(int), st);
    if (e0 != cudaSuccess) return e0;
    const int ysplit = std::max(1, std::min(16, w / 256));
    note_launch();
    k_row_max<<<dim3(rows_p / 32, ysplit), 256, 0, st>>>(Gh, ldg, m, w, ex);
    note_launch();
    k_row_exp<<<(rows_p + 255) / 256, 256, 0, st>>>(m, rows_p, ex);
  }
  {
    dim3 grid(wp / 64, rows_p / 32);
    note_launch();
    k_ozaki_digits<<<grid, 256, 0, st>>>(Gh, Gl, ldg, m, w, rows_p / 8, ex, digits);
  }
  GramTcArgs a{};
  a.D = digits;
  a.ngroups = rows_p / 8;
  a.nkb = wp / kKB;
  a.NT = mp / kTN;
  a.ntile = gram_tc_ntile(m, mp);
  const int nchunks = (wp + kKC - 1) / kKC;
  const int split = gram_tc_split(m, mp, w, num_sms);
  a.chunks_per_cta = (nchunks + split - 1) / split;
  a.part = part;
  a.fl = fl;
  cudaError_t e = ensure_dyn_smem((const void*)k_gram_tc, kSmemBytes);
  if (e != cudaSuccess) return e;
  {
    dim3 grid(a.ntile, split);
    note_launch();
    k_gram_tc<<<grid, 160, kSmemBytes, st>>>(a);
  }
  {
    const int64_t total = (int64_t)mp * (mp + 1) / 2;
    const int grid = (int)std::min<int64_t>(4096, (total + 255) / 256);
    note_launch();
    k_gram_tc_finish<<<grid, 256, 0, st>>>(part, split, a.ntile, a.NT, ex, m, mp, Q);
  }
  return cudaGetLastError();
}

}  // namespace lpk
