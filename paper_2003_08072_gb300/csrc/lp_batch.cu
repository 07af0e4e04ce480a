// CG batch engine of the serving loop: the preconditioned CG iterations of all live instances
// advance in shared launches.
//
// A serving worker whose context reaches a CG solve on the normal equations (Alg. 1 step 3)
// prepares the solve on its own stream as usual (start residual, first preconditioner apply,
// zeroed accumulators), then hands the loop to the engine as a job and waits.  The engine
// thread keeps a work table of the live jobs and runs rounds on its own stream: one round is
// one CG iteration of every job, i.e. one batched launch of the CG product (k_cgprod_batch:
// each job gets a share of the CTAs proportional to its matrix and runs the product of its
// own iteration) and one batched preconditioner apply with the fused CG step (k_symv_batch;
// a second one for jobs whose preconditioner is the two-stage factor).  Every job keeps its
// own scalars, flags and reduction counters, so jobs at different iterations, of different
// sizes and stream dtypes, share a launch; a finished job's kernels return at once.  Rounds
// are issued without waiting on the host (a few in flight); after each round a small kernel
// copies the jobs' stop flags into host-visible memory, and once the round's event has passed
// its finished jobs go back to their workers.  Jobs that arrive join at the next round, after
// an event that orders their set-up on their own stream before it.
#include <algorithm>
#include <condition_variable>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "lp_batch.cuh"

using namespace lpk;

namespace {

constexpr int kRing = 4;            // rounds in flight at most
constexpr int kMaxJobs = 256;
constexpr size_t kBytesPerCta = 32 * 1024;    // matrix bytes per CTA of a job's product

}  // namespace

struct CgBatcher {
  int dev = 0;
  int num_sms = 0;
  cudaStream_t st = nullptr;
  std::thread th;
  std::mutex mu;
  std::condition_variable cv;
  bool stop = false;
  std::vector<CgBatchJob*> pending;
  std::vector<CgBatchJob*> active;
  std::vector<CgBatchJob*> draining;   // done, waiting for their last round to finish
  // per slot of the ring: the round's work table (pinned host, device), the stop flags of its
  // jobs (host memory the GPU writes), the jobs it ran, and an event marking its end
  unsigned char* h_tab = nullptr;
  unsigned char* d_tab = nullptr;
  int* h_done = nullptr;
  int* d_done = nullptr;            // device alias of h_done
  const int** h_flags = nullptr;    // per slot: the jobs' flag arrays (pinned host)
  const int** d_flags = nullptr;
  cudaEvent_t ev[kRing] = {};
  std::vector<CgBatchJob*> ran[kRing];
  long long rounds = 0;
  long long jobs_run = 0;
  bool broken = false;
};

CgBatchJob::CgBatchJob() = default;

// Stop flags of a round's jobs, gathered after the round into host-visible memory.
__global__ void k_gather_done(const int* const* flags, int nj, int* out) {
  for (int i = threadIdx.x; i < nj; i += blockDim.x) out[i] = flags[i][FL_DONE];
}

namespace {

// Bytes of one round's table at most: product jobs, then the two apply lists, packed.
size_t round_bytes() {
  return (size_t)kMaxJobs * (sizeof(CgProdJob) + 2 * sizeof(SymvJob));
}

// Enqueues one round (one CG iteration of every active job) into ring slot k.
bool launch_round(CgBatcher* b, int k) {
  const int nj = (int)b->active.size();
  unsigned char* h = b->h_tab + (size_t)k * round_bytes();
  unsigned char* d = b->d_tab + (size_t)k * round_bytes();
  // packed table: nj product jobs, nj first applies, the second applies of factored jobs
  CgProdJob* hp = reinterpret_cast<CgProdJob*>(h);
  SymvJob* hs1 = reinterpret_cast<SymvJob*>(h + (size_t)nj * sizeof(CgProdJob));
  SymvJob* hs2 = hs1 + nj;
  // products grouped by kernel instance (dtype, group width): jobs of a group are contiguous
  int np = 0;
  struct Group {
    lp_dtype ta;
    int tc, first, count, ctas, nwarps;
    size_t smem;
  };
  Group groups[6];
  int ngroups = 0;
  for (lp_dtype ta : {LP_F32, LP_BF16, LP_F16}) {
    for (int tc : {8, 2}) {
      Group g{ta, tc, np, 0, 0, 1, 0};
      for (CgBatchJob* j : b->active) {
        if (j->ta != ta || j->tc != tc) continue;
        const int parity = (int)((b->rounds - j->round0) & 1);
        CgProdJob pj = j->prod[parity];
        pj.cta0 = g.ctas;
        pj.ncta = j->prod_ctas;
        hp[np++] = pj;
        g.count += 1;
        g.ctas += j->prod_ctas;
        g.nwarps = std::max(g.nwarps, j->nwarps);
        g.smem = std::max(g.smem, j->prod_smem);
      }
      if (g.count) groups[ngroups++] = g;
    }
  }
  int n1 = 0, n2 = 0, c1 = 0, c2 = 0;
  size_t sm1 = 0, sm2 = 0;
  for (int i = 0; i < nj; ++i) {
    CgBatchJob* j = b->active[i];
    const int parity = (int)((b->rounds - j->round0) & 1);
    hs1[n1++] = SymvJob{j->step1[parity], c1, j->symv_ctas};
    c1 += j->symv_ctas;
    sm1 = std::max(sm1, j->symv_smem);
    if (j->factored) {
      hs2[n2++] = SymvJob{j->step2[parity], c2, j->symv_ctas};
      c2 += j->symv_ctas;
      sm2 = std::max(sm2, j->symv_smem);
    }
    b->h_flags[k * kMaxJobs + i] = j->c->fl;
  }
  const size_t used = (size_t)nj * sizeof(CgProdJob) + (size_t)(nj + n2) * sizeof(SymvJob);
  if (cudaMemcpyAsync(d, h, used, cudaMemcpyHostToDevice, b->st) != cudaSuccess) return false;
  if (cudaMemcpyAsync(b->d_flags + k * kMaxJobs, b->h_flags + k * kMaxJobs,
                      nj * sizeof(const int*), cudaMemcpyHostToDevice, b->st) != cudaSuccess)
    return false;
  const CgProdJob* dp = reinterpret_cast<const CgProdJob*>(d);
  const SymvJob* ds1 = reinterpret_cast<const SymvJob*>(d + (size_t)nj * sizeof(CgProdJob));
  const SymvJob* ds2 = ds1 + nj;
  for (int g = 0; g < ngroups; ++g)
    if (launch_cgprod_batch(groups[g].ta, groups[g].tc, dp + groups[g].first, groups[g].count,
                            groups[g].ctas, groups[g].nwarps, groups[g].smem,
                            b->st) != cudaSuccess)
      return false;
  if (launch_symv_batch(ds1, n1, c1, sm1, b->st) != cudaSuccess) return false;
  if (n2 && launch_symv_batch(ds2, n2, c2, sm2, b->st) != cudaSuccess) return false;
  note_launch();
  k_gather_done<<<1, 256, 0, b->st>>>(b->d_flags + k * kMaxJobs, nj, b->d_done + k * kMaxJobs);
  if (cudaGetLastError() != cudaSuccess) return false;
  if (cudaEventRecord(b->ev[k], b->st) != cudaSuccess) return false;
  b->ran[k] = b->active;
  for (CgBatchJob* j : b->active) j->last_round = b->rounds;
  ++b->rounds;
  return true;
}

// Rounds are issued without waiting, up to kRing in flight.  Before a slot is reused its
// round has finished: its jobs whose flag says done (set by their own kernels, so nothing of
// theirs runs after that round) go back to their workers.  New jobs join at every round.
void engine_main(CgBatcher* b) {
  cudaSetDevice(b->dev);
  long long retired = 0;   // rounds whose flags have been read
  for (;;) {
    {
      std::unique_lock<std::mutex> lk(b->mu);
      b->cv.wait(lk, [&] {
        return b->stop || !b->pending.empty() || !b->active.empty() || retired < b->rounds;
      });
      if (b->stop && b->pending.empty() && b->active.empty() && b->draining.empty() &&
          retired == b->rounds)
        break;
      for (CgBatchJob* j : b->pending) {
        if (b->broken || cudaStreamWaitEvent(b->st, j->ready, 0) != cudaSuccess) {
          cudaGetLastError();
          j->status = LP_ERR_CUDA;
          j->finished = true;
          continue;
        }
        j->round0 = b->rounds;
        b->active.push_back(j);
        ++b->jobs_run;
      }
      b->pending.clear();
      b->cv.notify_all();
    }
    // the slot of the next round must be free: retire the oldest round first when the ring is
    // full, or when no job is left to run a round for
    const bool need_slot = b->rounds - retired >= kRing;
    if ((need_slot || b->active.empty()) && retired < b->rounds) {
      const int k = (int)(retired % kRing);
      const bool ok = cudaEventSynchronize(b->ev[k]) == cudaSuccess;
      std::lock_guard<std::mutex> lk(b->mu);
      if (!ok) {
        cudaGetLastError();
        b->broken = true;
      }
      // a job whose flag says done leaves the active list at once (no new round includes it)
      // but goes back to its worker only when the last round it was part of has finished:
      // rounds still in flight read its flags and buffers
      std::vector<CgBatchJob*> still;
      for (CgBatchJob* j : b->active) {
        bool done = !ok;
        for (size_t i = 0; i < b->ran[k].size(); ++i)
          if (b->ran[k][i] == j && b->h_done[k * kMaxJobs + i]) done = true;
        if (done) {
          j->status = ok ? LP_OK : LP_ERR_CUDA;
          b->draining.push_back(j);
        } else {
          still.push_back(j);
        }
      }
      b->active.swap(still);
      ++retired;
      std::vector<CgBatchJob*> left;
      for (CgBatchJob* j : b->draining) {
        if (j->last_round < retired) j->finished = true;
        else left.push_back(j);
      }
      b->draining.swap(left);
      b->cv.notify_all();
      continue;
    }
    if (b->active.empty()) continue;
    if (b->broken || !launch_round(b, (int)(b->rounds % kRing))) {
      cudaGetLastError();
      cudaStreamSynchronize(b->st);   // nothing of the engine runs after the jobs return
      cudaGetLastError();
      std::lock_guard<std::mutex> lk(b->mu);
      b->broken = true;
      for (CgBatchJob* j : b->active) {
        j->status = LP_ERR_CUDA;
        j->finished = true;
      }
      for (CgBatchJob* j : b->draining) j->finished = true;
      b->active.clear();
      b->draining.clear();
      retired = b->rounds;
      b->cv.notify_all();
    }
  }
}

}  // namespace

namespace lpk {

CgBatcher* cg_batcher_create(int dev, int num_sms) {
  CgBatcher* b = new (std::nothrow) CgBatcher();
  if (!b) return nullptr;
  b->dev = dev;
  b->num_sms = num_sms;
  bool ok = cudaStreamCreateWithFlags(&b->st, cudaStreamNonBlocking) == cudaSuccess &&
            cudaMallocHost(&b->h_tab, kRing * round_bytes()) == cudaSuccess &&
            cudaMalloc(&b->d_tab, kRing * round_bytes()) == cudaSuccess &&
            cudaHostAlloc(&b->h_done, kRing * kMaxJobs * sizeof(int), cudaHostAllocMapped) ==
                cudaSuccess &&
            cudaHostGetDevicePointer((void**)&b->d_done, b->h_done, 0) == cudaSuccess &&
            cudaMallocHost(&b->h_flags, kRing * kMaxJobs * sizeof(int*)) == cudaSuccess &&
            cudaMalloc(&b->d_flags, kRing * kMaxJobs * sizeof(int*)) == cudaSuccess;
  for (int k = 0; ok && k < kRing; ++k)
    ok = cudaEventCreateWithFlags(&b->ev[k], cudaEventDisableTiming) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    cg_batcher_destroy(b);
    return nullptr;
  }
  try {
    b->th = std::thread(engine_main, b);
  } catch (const std::exception&) {
    cg_batcher_destroy(b);
    return nullptr;
  }
  return b;
}

void cg_batcher_destroy(CgBatcher* b) {
  if (!b) return;
  if (b->th.joinable()) {
    {
      std::lock_guard<std::mutex> lk(b->mu);
      b->stop = true;
    }
    b->cv.notify_all();
    b->th.join();
  }
  if (b->st) cudaStreamSynchronize(b->st);
  if (b->h_tab) cudaFreeHost(b->h_tab);
  if (b->d_tab) cudaFree(b->d_tab);
  if (b->h_done) cudaFreeHost(b->h_done);
  if (b->h_flags) cudaFreeHost(b->h_flags);
  if (b->d_flags) cudaFree(b->d_flags);
  for (int k = 0; k < kRing; ++k)
    if (b->ev[k]) cudaEventDestroy(b->ev[k]);
  if (b->st) cudaStreamDestroy(b->st);
  cudaGetLastError();
  delete b;
}

void cg_batcher_stats(CgBatcher* b, long long* rounds, long long* jobs) {
  std::lock_guard<std::mutex> lk(b->mu);
  *rounds = b->rounds;
  *jobs = b->jobs_run;
}

// Queues the job and waits until the engine has run its CG solve to its stop rule.
bool cg_batcher_run(CgBatcher* b, CgBatchJob* j, lp_status* st) {
  if (cudaEventRecord(j->ready, j->c->st) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  std::unique_lock<std::mutex> lk(b->mu);
  if (b->broken || b->stop || (int)(b->active.size() + b->pending.size()) >= kMaxJobs)
    return false;
  j->finished = false;
  b->pending.push_back(j);
  b->cv.notify_all();
  b->cv.wait(lk, [&] { return j->finished; });
  *st = j->status;
  return true;
}

// CTAs of a job's product: about kBytesPerCta of its matrix each (measured on GB300 with the
// serving stream: 32 KB beat 8 KB and 256 KB), at least one, at most eight per SM.
int cg_batch_prod_ctas(const lp_ctx* c, size_t elem_bytes, int num_sms, int64_t ngroups) {
  const double bytes = (double)c->lda_s * (double)c->n * (double)elem_bytes;
  int64_t k = (int64_t)(bytes / kBytesPerCta) + 1;
  k = std::min<int64_t>(k, 8 * (int64_t)num_sms);
  k = std::min<int64_t>(k, ngroups);
  return (int)std::max<int64_t>(k, 1);
}

}  // namespace lpk
