// CG batch engine of the serving loop (lp_batch.cu): shared launches of the CG iterations of
// all live instances.
#pragma once

#include "lp_internal.cuh"

struct CgBatcher;

// One context's CG solve handed to the engine: the launch descriptors of its two iteration
// parities (buffers alternate between iterations j and j + 1) and its share of the launches.
struct CgBatchJob {
  CgBatchJob();
  lp_ctx* c = nullptr;
  lp_dtype ta = LP_F32;
  int tc = 8, nwarps = 1, prod_ctas = 1, symv_ctas = 1;
  size_t prod_smem = 0, symv_smem = 0;
  bool factored = false;
  lpk::CgProdJob prod[2];
  lpk::SymvArgs step1[2];   // r <- r - alpha q, dy <- dy + alpha d, z = M r (or t = X r)
  lpk::SymvArgs step2[2];   // z = X^T t (two-stage factor only)
  cudaEvent_t ready = nullptr;   // recorded on the context's stream after the solve's set-up
  long long round0 = 0;      // engine round of the job's first iteration
  long long last_round = -1; // last engine round that included the job
  lp_status status = LP_OK;
  bool finished = false;
};

namespace lpk {

CgBatcher* cg_batcher_create(int dev, int num_sms);
void cg_batcher_destroy(CgBatcher* b);
void cg_batcher_stats(CgBatcher* b, long long* rounds, long long* jobs);
// Runs the job's CG loop in the engine; false when the engine did not take it (the caller
// then runs the loop itself), else *st is the outcome.
bool cg_batcher_run(CgBatcher* b, CgBatchJob* j, lp_status* st);
int cg_batch_prod_ctas(const lp_ctx* c, size_t elem_bytes, int num_sms, int64_t ngroups);

}  // namespace lpk
