// CG product y = A D^2 A^T v (Alg. 1 step 3) over a column-major A streamed below FP64,
// with FP32 accumulation, A staged through shared memory by bulk asynchronous copies.
//
// The register-tiled pass (k_coltile.cu) keeps the column tile it works on in registers, so a
// CTA cannot load tile t+1 while it reduces tile t, and at large m (or 16-bit types, whose
// unpacked tile is twice as wide) it runs one CTA per SM with idle gaps between tiles.  Here
// the CTA is a pipeline: one thread issues cp.async.bulk copies of whole column groups (a group
// of TC consecutive columns is one contiguous range of TC * lda elements) into a ring of S
// shared-memory stages, each completing on its own mbarrier, S - 1 groups ahead of the warps
// that consume them.  A stage is refilled once every warp is past the __syncthreads of the
// following group, which comes after the last read of the stage.
//
// Per group the warps form the TC column dots a_i^T v (rows split across warps as slices of
// 32 lanes x 16 bytes, v in registers), reduce them across the CTA through shared memory,
// weight them with D^2 (FP32, times the column scales of a scaled 16-bit copy), and add
// a_i * coef_i into per-thread row accumulators.  With one row slice per warp, 16-bit groups
// stay unpacked in registers between the two phases instead of being read and unpacked twice.
// For FP32 copies the products of four groups (32 columns) are summed first and added to the
// accumulator with an error-free TwoSum (the error term kept in a second accumulator), so a row
// sum over the ~n/grid columns a CTA sees loses no more than a few FP32 units; the CTA sums go
// to q with FP64 atomics.  Keeping the FP32-accumulated product near FP32 accuracy keeps CG's residual
// recurrence close to the true residual, which spares most FP64 refinement rounds.  The last
// CTA forms d^T q and alpha; without a q buffer the sums go to per-CTA partials.
//
// Every wait on an mbarrier is bounded by the global timer; a wait that gives up sets
// FL_TIMEOUT and the CTA carries on without the data (the host turns the flag into
// LP_ERR_TIMEOUT), so no thread leaves early and no copy is left writing into the CTA's
// shared memory after it exits.
#include <algorithm>

#include "bulk_util.cuh"
#include "dev_util.cuh"
#include "symv_body.cuh"

namespace lpk {


// Shared memory: S stages of TC * lda elements, then S mbarriers.  The body runs as block bid
// of a grid of nblk blocks: the whole launch (k_cgprod) or one job's share of a batched launch
// (k_cgprod_batch).
// inval: end the stage mbarriers' lives before returning (the persistent CG loop reuses their
// shared memory for the preconditioner apply and initialises them again next iteration).
template <typename TA, int SPW, int TC, bool KEEP>
__device__ __forceinline__ void cgprod_body(const ColArgs& a, int S, int64_t ngroups, int bid,
                                            int nblk, bool inval = false) {
  constexpr int VEC = VecN<TA>::N;
  constexpr bool COMP = sizeof(TA) == 4;   // compensated row sums for FP32 copies
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ float red[2][16][TC];
  __shared__ int s_timeout;
  if (a.skip_if_done && a.fl[FL_DONE]) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const size_t stage_elems = (size_t)TC * a.lda;
  TA* stages = reinterpret_cast<TA*>(smem);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + (size_t)S * stage_elems * sizeof(TA));
  const TA* A = reinterpret_cast<const TA*>(a.A);

  // groups of this CTA: bid, bid + nblk, ...
  const int my_groups = bid < ngroups ? (int)((ngroups - 1 - bid) / nblk) + 1 : 0;
  const int64_t col_step = (int64_t)nblk * TC;
  const uint64_t wait_ns = a.wait_ns ? a.wait_ns : kWaitLimitNs;
  auto issue = [&](int i, int stage) {   // thread 0: copy local group i into a stage
    // fault-injection hook: CTA 0 never issues the copy of its group stall_group, so the
    // wait for it runs out (its stage keeps stale data; nothing is written out of bounds)
    if (bid == 0 && (int64_t)i + 1 == a.stall_group_p1) return;
    const int64_t col0 = ((int64_t)bid + (int64_t)i * nblk) * TC;
    const int ncols = (int)std::min<int64_t>(TC, a.n - col0);
    const unsigned bytes = (unsigned)((size_t)ncols * a.lda * sizeof(TA));
    uint64_t* bar = &bars[stage];
    mbar_arrive_expect_tx(bar, bytes);
    bulk_g2s(stages + (size_t)stage * stage_elems, A + col0 * a.lda, bytes, bar);
  };
  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) mbar_init(&bars[s], 1);
    s_timeout = 0;
    fence_mbarrier_init();
    fence_proxy_async_smem();
    for (int i = 0; i < std::min(S - 1, my_groups); ++i) issue(i, i);
  }

  // v and the row accumulators (g: partial sums of the last groups, yc: TwoSum error terms of
  // the compensated sums)
  constexpr int kFlush = 4;
  float vr[SPW][VEC], yr[SPW][VEC], yc[COMP ? SPW : 1][VEC], g[COMP ? SPW : 1][VEC];
  int rowb[SPW];
  bool rok[SPW];
#pragma unroll
  for (int sl = 0; sl < SPW; ++sl) {
    rowb[sl] = ((warp * SPW + sl) * 32 + lane) * VEC;
    rok[sl] = rowb[sl] < a.m;
#pragma unroll
    for (int e = 0; e < VEC; ++e) {
      const int row = rowb[sl] + e;
      double x = 0.0;
      if (rok[sl] && row < a.m) {
        if (a.dz) {   // fused CG direction update d = z + beta d_old
          x = fma(a.sc[SC_BETA], a.dold[row], a.dz[row]);
          if (bid == 0) a.dnew[row] = x;
        } else {
          x = a.v[row];
        }
      }
      vr[sl][e] = (float)x;
      yr[sl][e] = 0.f;
      if constexpr (COMP) {
        yc[sl][e] = 0.f;
        g[sl][e] = 0.f;
      }
    }
  }
  __syncthreads();   // barriers initialised before anyone waits on them

  const int cl = lane % TC;
  bool timed_out = false;
  int timeout_group = -1;   // the local group whose wait gave up (thread 0 issues the copies)
  // stage of group i is i % S and its phase parity (i / S) & 1, both kept as running counters
  int stage = 0, prev_stage = S - 1;
  unsigned parity = 0;
  int64_t col0 = (int64_t)bid * TC;
  for (int i = 0; i < my_groups; ++i, col0 += col_step) {
    const TA* st = stages + (size_t)stage * stage_elems;
    // after one wait has given up, the rest are skipped (and no further copies issued)
    if (!timed_out && !mbar_wait_bounded(&bars[stage], parity, wait_ns)) {
      timed_out = true;
      timeout_group = i;
    }
    const int ncols = (int)std::min<int64_t>(TC, a.n - col0);
    const int64_t mycol = col0 + cl;
    const bool cok = mycol < a.n;
    const float w = cok ? a.d2f[mycol] : 0.f;
    // column dots from the staged group; with KEEP the unpacked group stays in registers for
    // the accumulation below instead of being read and unpacked a second time
    float kept[KEEP ? TC : 1][KEEP ? SPW : 1][VEC];
    float pd[TC];
#pragma unroll
    for (int c = 0; c < TC; ++c) {
      float acc = 0.f;
      if (c < ncols) {
#pragma unroll
        for (int sl = 0; sl < SPW; ++sl) {
          if (!rok[sl]) continue;
          const uint4 r = *reinterpret_cast<const uint4*>(st + (size_t)c * a.lda + rowb[sl]);
          float av[VEC];
          unpack<TA, float>(r, av);
#pragma unroll
          for (int e = 0; e < VEC; ++e) {
            if constexpr (KEEP) kept[c][sl][e] = av[e];
            acc = fmaf(av[e], vr[sl][e], acc);
          }
        }
      }
      pd[c] = acc;
    }
    const float wsum = warp_transpose_reduce<TC, float>(pd, lane);
    if (lane < TC) red[i & 1][warp][lane] = wsum;
    __syncthreads();
    // every warp is past group i-1: its stage may be refilled with group i + S - 1
    if (threadIdx.x == 0 && !timed_out && i + S - 1 < my_groups) {
      fence_proxy_async_smem();
      issue(i + S - 1, prev_stage);
    }
    float dot = 0.f;
    for (int wi = 0; wi < nwarps; ++wi) dot += red[i & 1][wi][cl];
    const float cf = cok ? w * dot : 0.f;
    if (a.colout && warp == 0 && lane < TC && cok) a.colout[mycol] = (double)dot;
#pragma unroll
    for (int c = 0; c < TC; ++c) {
      const float cc = __shfl_sync(kFull, cf, c);
      if (c >= ncols) continue;
#pragma unroll
      for (int sl = 0; sl < SPW; ++sl) {
        if (!rok[sl]) continue;
        float av[VEC];
        if constexpr (KEEP) {
#pragma unroll
          for (int e = 0; e < VEC; ++e) av[e] = kept[c][sl][e];
        } else {
          const uint4 r = *reinterpret_cast<const uint4*>(st + (size_t)c * a.lda + rowb[sl]);
          unpack<TA, float>(r, av);
        }
#pragma unroll
        for (int e = 0; e < VEC; ++e) {
          if constexpr (COMP) g[sl][e] = fmaf(cc, av[e], g[sl][e]);
          else yr[sl][e] = fmaf(cc, av[e], yr[sl][e]);
        }
      }
    }
    if constexpr (COMP) {
      // every kFlush groups (and after the last) the partial sum joins the accumulator
      if ((i + 1) % kFlush == 0 || i + 1 == my_groups) {
#pragma unroll
        for (int sl = 0; sl < SPW; ++sl)
#pragma unroll
          for (int e = 0; e < VEC; ++e) {
            float t, err;
            two_sum(yr[sl][e], g[sl][e], t, err);
            yr[sl][e] = t;
            yc[sl][e] += err;
            g[sl][e] = 0.f;
          }
      }
    }
    prev_stage = stage;
    if (++stage == S) {
      stage = 0;
      parity ^= 1u;
    }
  }
  if (timed_out) s_timeout = 1;
  __syncthreads();
  if (s_timeout) {
    if (threadIdx.x == 0) {
      if (a.flw) a.flw[FL_TIMEOUT] = 1;
      // let copies still in flight land before the CTA's shared memory goes away.  Thread 0
      // issues every copy and waits for every group before it refills that group's stage, so
      // if its own wait for group g gave up, groups g .. g + S - 2 were issued and not yet
      // waited for, and nothing after them was issued; if thread 0 never gave up, it has
      // already seen every copy land.
      if (timeout_group >= 0) {
        const int last = std::min(timeout_group + S - 2, my_groups - 1);
        for (int i = timeout_group; i <= last; ++i)
          mbar_wait_bounded(&bars[i % S], (unsigned)((i / S) & 1), wait_ns);
      }
    }
    __syncthreads();
  }
  if (inval) {
    __syncthreads();   // every wait on the stage barriers is over
    if (threadIdx.x == 0)
      for (int s = 0; s < S; ++s) mbar_inval(&bars[s]);
  }
  auto row_sum = [&](int sl, int e) -> double {
    if constexpr (COMP) return (double)yr[sl][e] + (double)yc[sl][e];
    else return (double)yr[sl][e];
  };

  if (a.qacc) {
    // kQCopies copies of q spread the atomic traffic over more L2 lines
    double* qc = a.qacc + (size_t)(bid % kQCopies) * a.m;
#pragma unroll
    for (int sl = 0; sl < SPW; ++sl)
#pragma unroll
      for (int e = 0; e < VEC; ++e) {
        const int row = rowb[sl] + e;
        if (rok[sl] && row < a.m) atomicAdd(&qc[row], row_sum(sl, e));
      }
    // last CTA: d^T q and alpha (no waiting: the last CTA to arrive does the work)
    __shared__ bool s_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = (atomicAdd(a.cnt, 1u) == (unsigned)nblk - 1);
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
  float* part = reinterpret_cast<float*>(a.part);
#pragma unroll
  for (int sl = 0; sl < SPW; ++sl)
#pragma unroll
    for (int e = 0; e < VEC; ++e) {
      const int row = rowb[sl] + e;
      if (rok[sl] && row < a.m) part[(size_t)bid * a.m + row] = (float)row_sum(sl, e);
    }
}

template <typename TA, int SPW, int TC, bool KEEP>
__global__ void __launch_bounds__(512) k_cgprod(ColArgs a, int S, int64_t ngroups) {
  cgprod_body<TA, SPW, TC, KEEP>(a, S, ngroups, blockIdx.x, gridDim.x);
}

// Batched CG product: every CTA finds its job in the work table (sorted by cta0) and runs that
// job's product as block (blockIdx.x - cta0) of a grid of ncta blocks.
template <typename TA, int SPW, int TC, bool KEEP>
__global__ void __launch_bounds__(512) k_cgprod_batch(const CgProdJob* __restrict__ jobs,
                                                      int njobs) {
  __shared__ int s_job;
  if (threadIdx.x == 0) {
    int lo = 0, hi = njobs - 1;
    while (lo < hi) {   // last job with cta0 <= blockIdx.x
      const int mid = (lo + hi + 1) >> 1;
      if (jobs[mid].cta0 <= (int)blockIdx.x) lo = mid;
      else hi = mid - 1;
    }
    s_job = lo;
  }
  __syncthreads();
  const CgProdJob& jb = jobs[s_job];
  cgprod_body<TA, SPW, TC, KEEP>(jb.a, jb.S, jb.ngroups, (int)blockIdx.x - jb.cta0, jb.ncta);
}

namespace {

constexpr size_t kSmemBudget = 200 * 1024;   // dynamic shared memory per SM used by the pass

// 16-bit groups are kept unpacked in registers between the two phases (KEEP).  Measured on
// GB300 (m = 1000 and 2000, n = 200000 and 500000): keeping the group is 15-20% faster for
// 16-bit types and slower for FP32 (whose registers go to the compensated sums instead);
// paired FP32 FMAs (fma.rn.f32x2) and groups of 16 columns were slower.
template <typename TA>
constexpr bool keep_default() {
  return sizeof(TA) == 2;
}

constexpr size_t kSmemTuneLimit = 220 * 1024;   // what a tuned shape may use per SM

template <typename TA, int SPW, int TC>
int launch_cgprod_t(ColArgs a, int nwarps, int num_sms, int max_grid, cudaStream_t st) {
  const size_t col_bytes = (size_t)a.lda * sizeof(TA);
  const size_t stage = (size_t)TC * col_bytes;
  int ctas = 0, S = 0;
  if (a.cfg_ctas > 0 && a.cfg_stages >= 2 &&
      (size_t)a.cfg_ctas * a.cfg_stages * (stage + 8) <= kSmemTuneLimit &&
      a.cfg_ctas * nwarps * 32 <= 2048) {
    // the shape the autotuner measured fastest for this matrix
    ctas = a.cfg_ctas;
    S = a.cfg_stages;
  } else {
    // rule: enough warps per SM to hide shared-memory latency, up to 4 CTAs of few warps
    ctas = std::max(1, std::min(4, 16 / nwarps));
    for (; ctas >= 1; --ctas) {
      S = (int)std::min<size_t>(6, (kSmemBudget / ctas) / (stage + 8));
      if (S >= 3) break;
    }
    if (ctas < 1) {
      ctas = 1;
      S = (int)std::min<size_t>(6, kSmemBudget / (stage + 8));
    }
  }
  if (S < 2) return -1;
  const size_t smem = (size_t)S * stage + (size_t)S * 8;
  auto kern = k_cgprod<TA, SPW, TC, keep_default<TA>() && SPW == 1>;
  if (ensure_dyn_smem((const void*)kern, smem) != cudaSuccess) {
    cudaGetLastError();
    return -1;
  }
  const int64_t ngroups = (a.n + TC - 1) / TC;
  int64_t grid = (int64_t)num_sms * ctas;
  if (grid > max_grid) grid = max_grid;
  if (grid > ngroups) grid = ngroups;
  if (grid < 1) grid = 1;
  { note_launch(); kern<<<(unsigned)grid, nwarps * 32, smem, st>>>(a, S, ngroups); }
  return (int)grid;
}

template <typename TA>
int launch_cgprod_dt(ColArgs a, int num_sms, int max_grid, cudaStream_t st) {
  constexpr int VEC = VecN<TA>::N;
  const int nslices = (a.m + 32 * VEC - 1) / (32 * VEC);
  int spw = 1;
  while ((nslices + spw - 1) / spw > 16) spw *= 2;
  if (spw > 4) return -1;
  const int nwarps = (nslices + spw - 1) / spw;
  // groups of 8 columns while a stage stays within 64 KB, else of 2 (or the tuned width)
  bool wide_cols = (size_t)8 * a.lda * sizeof(TA) > 64 * 1024;
  if (a.cfg_tc == 2) wide_cols = true;
  if (a.cfg_tc == 8 && (size_t)8 * a.lda * sizeof(TA) * 2 <= kSmemTuneLimit) wide_cols = false;
  switch (spw) {
    case 1:
      return wide_cols ? launch_cgprod_t<TA, 1, 2>(a, nwarps, num_sms, max_grid, st)
                       : launch_cgprod_t<TA, 1, 8>(a, nwarps, num_sms, max_grid, st);
    case 2:
      return wide_cols ? launch_cgprod_t<TA, 2, 2>(a, nwarps, num_sms, max_grid, st)
                       : launch_cgprod_t<TA, 2, 8>(a, nwarps, num_sms, max_grid, st);
    default:
      return wide_cols ? launch_cgprod_t<TA, 4, 2>(a, nwarps, num_sms, max_grid, st)
                       : launch_cgprod_t<TA, 4, 8>(a, nwarps, num_sms, max_grid, st);
  }
}

}  // namespace

// Autotuner of the launch shape: group width TC (columns per bulk copy), pipeline stages S
// and CTAs per SM, timed with CUDA events on the matrix itself (a few launches per candidate,
// writing per-CTA partial sums only).  The fastest candidate is returned together with the
// time of the fixed rule, so the choice can be reported.
int tune_cgprod(lp_dtype ta, ColArgs a, int num_sms, int max_grid, cudaStream_t st,
                CgTune* out) {
  const size_t es = ta == LP_F32 ? 4 : 2;
  if (ta != LP_F32 && ta != LP_BF16 && ta != LP_F16) return -1;
  const int vec = (int)(16 / es);
  const int nslices = (a.m + 32 * vec - 1) / (32 * vec);
  int spw = 1;
  while ((nslices + spw - 1) / spw > 16) spw *= 2;
  if (spw > 4) return -1;
  const int nwarps = (nslices + spw - 1) / spw;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    cudaGetLastError();
    if (e0) cudaEventDestroy(e0);
    return -1;
  }
  auto time_it = [&](ColArgs b) -> float {
    if (launch_cgprod(ta, b, num_sms, max_grid, st) < 0) return -1.f;   // warm-up
    cudaEventRecord(e0, st);
    constexpr int kReps = 3;
    for (int r = 0; r < kReps; ++r)
      if (launch_cgprod(ta, b, num_sms, max_grid, st) < 0) return -1.f;
    cudaEventRecord(e1, st);
    float ms = 0.f;
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
      cudaGetLastError();
      return -1.f;
    }
    return 1000.f * ms / kReps;
  };
  a.qacc = nullptr;   // partial sums only: nothing of the CG state is touched
  a.skip_if_done = 0;
  a.dz = nullptr;
  a.cfg_tc = a.cfg_stages = a.cfg_ctas = 0;
  CgTune best{};
  best.rule_us = time_it(a);
  best.us = best.rule_us;
  for (int tc : {8, 2}) {
    const size_t stage = (size_t)tc * a.lda * es;
    if (tc == 8 && 2 * stage > kSmemTuneLimit) continue;
    for (int ctas = 1; ctas <= 4; ++ctas) {
      if (ctas * nwarps * 32 > 2048) continue;
      for (int S = 2; S <= 6; ++S) {
        if ((size_t)ctas * S * (stage + 8) > kSmemTuneLimit) continue;
        ColArgs b = a;
        b.cfg_tc = tc;
        b.cfg_stages = S;
        b.cfg_ctas = ctas;
        const float us = time_it(b);
        if (us > 0.f && (best.us <= 0.f || us < best.us)) {
          best.us = us;
          best.tc = tc;
          best.stages = S;
          best.ctas = ctas;
        }
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  *out = best;   // ctas == 0: no candidate beat the fixed rule, which stays in use
  return best.rule_us > 0.f ? 0 : -1;
}

// ---- batched CG products (the serving loop's shared launches) --------------------------

// ---- persistent CG loop ----------------------------------------------------------------
// One CTA (the product's warps, one row slice each) runs, per iteration, its share of the CG
// product (cgprod_body as block b of the whole grid) and, for the first ceil(m / warps) CTAs,
// one row per warp of the preconditioner apply (symv_body); grid barriers order the product's q and alpha before the apply, and the apply's
// r, z, rho and beta before the next product.  After each iteration every CTA reads the stop
// flag (set by the apply's last CTA: converged, iteration cap, non-finite) and the timeout flag.
// The two bodies share the dynamic shared memory; the product ends its mbarriers' lives first.
template <typename TA, int SPW, int TC, bool KEEP>
__global__ void __launch_bounds__(256) k_cg_persistent(CgPersistArgs p, int S, int64_t ngroups,
                                                        int nblk_symv) {
  const uint64_t lim = p.wait_ns ? p.wait_ns : kWaitLimitNs;
  for (int j = 0; j < p.max_trips; ++j) {
    const int par = j & 1;
    cgprod_body<TA, SPW, TC, KEEP>(p.prod[par], S, ngroups, blockIdx.x, gridDim.x, true);
    bool ok = grid_sync_bounded(p.bar, lim);
    if (ok) {
      if ((int)blockIdx.x < nblk_symv) symv_body<true>(p.step1[par], blockIdx.x, nblk_symv);
      if (p.factored) {
        ok = grid_sync_bounded(p.bar, lim);
        if (ok && (int)blockIdx.x < nblk_symv) symv_body<true>(p.step2[par], blockIdx.x, nblk_symv);
      }
    }
    if (ok) ok = grid_sync_bounded(p.bar, lim);
    if (!ok) {
      if (threadIdx.x == 0) p.fl[FL_TIMEOUT] = 1;
      return;
    }
    const int done = *reinterpret_cast<volatile int*>(&p.fl[FL_DONE]);
    const int to = *reinterpret_cast<volatile int*>(&p.fl[FL_TIMEOUT]);
    if (done || to) return;
  }
}

namespace {

template <typename TA, int SPW, int TC>
int launch_cg_persistent_t(CgPersistArgs p, int nwarps, int num_sms, cudaStream_t st) {
  constexpr bool KEEP = keep_default<TA>() && SPW == 1;
  const ColArgs& a = p.prod[0];
  const size_t stage = (size_t)TC * a.lda * sizeof(TA);
  const size_t symv_bytes = (size_t)((a.m + 3) & ~3) * 2 * sizeof(double);
  const int threads = 32 * nwarps;
  const int nblk_symv = (a.m + nwarps - 1) / nwarps;   // one row of the apply per warp
  const int64_t ngroups = (a.n + TC - 1) / TC;
  auto kern = k_cg_persistent<TA, SPW, TC, KEEP>;
  // as many CTAs per SM (up to 8) as registers and shared memory allow, with 3-4 stages where
  // that still gives every row of the apply a warp, else with 2
  int per_sm = 0, S = 0;
  size_t smem = 0;
  for (int min_s = 3; min_s >= 2 && !per_sm; --min_s) {
    for (int k = 8; k >= 1; --k) {
      const int s_k = (int)std::min<size_t>(4, (kSmemBudget / k) / (stage + 8));
      if (s_k < min_s) continue;
      const size_t sm_k = std::max((size_t)s_k * stage + (size_t)s_k * 8, symv_bytes);
      if (ensure_dyn_smem((const void*)kern, sm_k) != cudaSuccess) {
        cudaGetLastError();
        return -1;
      }
      int occ = 0;
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, threads, sm_k) != cudaSuccess) {
        cudaGetLastError();
        return -1;
      }
      if (occ < k || (int64_t)num_sms * k < nblk_symv) continue;
      per_sm = k;
      S = s_k;
      smem = sm_k;
      break;
    }
  }
  if (!per_sm) return -1;   // the apply's rows cannot all be co-resident
  {
    int64_t grid = (int64_t)num_sms * per_sm;
    if (grid > ngroups) grid = std::max<int64_t>(ngroups, nblk_symv);
    int Si = S;
    int64_t ng = ngroups;
    int nb = nblk_symv;
    void* args[] = {&p, &Si, &ng, &nb};
    note_launch();
    const cudaError_t e = cudaLaunchCooperativeKernel((const void*)kern, dim3((unsigned)grid),
                                                      dim3(threads), args, smem, st);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return -1;
    }
    return (int)grid;
  }
}

template <typename TA>
int launch_cg_persistent_dt(CgPersistArgs p, int num_sms, cudaStream_t st) {
  constexpr int VEC = VecN<TA>::N;
  const ColArgs& a = p.prod[0];
  const int nslices = (a.m + 32 * VEC - 1) / (32 * VEC);
  const bool wide = (size_t)8 * a.lda * sizeof(TA) > 64 * 1024;
  // the product's own warps (one row slice each, up to 8): the block size of both phases
  if (nslices <= 8)
    return wide ? launch_cg_persistent_t<TA, 1, 2>(p, nslices, num_sms, st)
                : launch_cg_persistent_t<TA, 1, 8>(p, nslices, num_sms, st);
  if (nslices <= 16)
    return wide ? launch_cg_persistent_t<TA, 2, 2>(p, (nslices + 1) / 2, num_sms, st)
                : launch_cg_persistent_t<TA, 2, 8>(p, (nslices + 1) / 2, num_sms, st);
  if (nslices <= 32)
    return wide ? launch_cg_persistent_t<TA, 4, 2>(p, (nslices + 3) / 4, num_sms, st)
                : launch_cg_persistent_t<TA, 4, 8>(p, (nslices + 3) / 4, num_sms, st);
  return -1;
}

}  // namespace

int launch_cg_persistent(lp_dtype ta, CgPersistArgs p, int num_sms, cudaStream_t st) {
  static int coop = -1;   // device attribute, read once per process
  if (coop < 0) {
    int dev = 0, v = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&v, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess) {
      cudaGetLastError();
      v = 0;
    }
    coop = v;
  }
  if (!coop || p.prod[0].m > 4096) return -1;
  switch (ta) {
    case LP_F32: return launch_cg_persistent_dt<float>(p, num_sms, st);
    case LP_BF16: return launch_cg_persistent_dt<__nv_bfloat16>(p, num_sms, st);
    case LP_F16: return launch_cg_persistent_dt<__half>(p, num_sms, st);
    default: return -1;
  }
}

bool cgprod_job_shape(lp_dtype ta, int m, int lda, int64_t n, int* tc, int* nwarps, int* S,
                      int64_t* ngroups, size_t* smem) {
  if (ta != LP_F32 && ta != LP_BF16 && ta != LP_F16) return false;
  const size_t es = ta == LP_F32 ? 4 : 2;
  const int vec = (int)(16 / es);
  const int nslices = (m + 32 * vec - 1) / (32 * vec);
  if (nslices > 16) return false;   // one row slice per warp (SPW = 1) only
  *nwarps = nslices;
  *tc = ((size_t)8 * lda * es > 64 * 1024) ? 2 : 8;
  const size_t stage = (size_t)(*tc) * lda * es;
  *S = 3;
  *ngroups = (n + *tc - 1) / *tc;
  *smem = (size_t)(*S) * stage + (size_t)(*S) * 8;
  return true;
}

template <typename TA, int TC>
cudaError_t launch_cgprod_batch_t(const CgProdJob* jobs, int njobs, int total_ctas, int nwarps,
                                  size_t smem, cudaStream_t st) {
  auto kern = k_cgprod_batch<TA, 1, TC, keep_default<TA>()>;
  cudaError_t e = ensure_dyn_smem((const void*)kern, smem);
  if (e != cudaSuccess) return e;
  { note_launch(); kern<<<total_ctas, nwarps * 32, smem, st>>>(jobs, njobs); }
  return cudaGetLastError();
}

cudaError_t launch_cgprod_batch(lp_dtype ta, int tc, const CgProdJob* jobs, int njobs,
                                int total_ctas, int nwarps, size_t smem, cudaStream_t st) {
  switch (ta) {
    case LP_F32:
      return tc == 2 ? launch_cgprod_batch_t<float, 2>(jobs, njobs, total_ctas, nwarps, smem, st)
                     : launch_cgprod_batch_t<float, 8>(jobs, njobs, total_ctas, nwarps, smem, st);
    case LP_BF16:
      return tc == 2
                 ? launch_cgprod_batch_t<__nv_bfloat16, 2>(jobs, njobs, total_ctas, nwarps, smem, st)
                 : launch_cgprod_batch_t<__nv_bfloat16, 8>(jobs, njobs, total_ctas, nwarps, smem, st);
    case LP_F16:
      return tc == 2 ? launch_cgprod_batch_t<__half, 2>(jobs, njobs, total_ctas, nwarps, smem, st)
                     : launch_cgprod_batch_t<__half, 8>(jobs, njobs, total_ctas, nwarps, smem, st);
    default:
      return cudaErrorInvalidValue;
  }
}

// Returns the number of CTAs (partial rows) or -1 when the shape is not covered (the caller
// then uses the register-tiled pass).  Needs a.d2f (the FP32 weight).
int launch_cgprod(lp_dtype ta, ColArgs a, int num_sms, int max_grid, cudaStream_t st) {
  if (!a.d2f) return -1;
  switch (ta) {
    case LP_F32: return launch_cgprod_dt<float>(a, num_sms, max_grid, st);
    case LP_BF16: return launch_cgprod_dt<__nv_bfloat16>(a, num_sms, max_grid, st);
    case LP_F16: return launch_cgprod_dt<__half>(a, num_sms, max_grid, st);
    default: return -1;
  }
}

}  // namespace lpk
