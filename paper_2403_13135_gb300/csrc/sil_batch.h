// sil_batch.h -- internal interface of the persistent batch kernel, shared by
// the batched entry point and the server.
#pragma once
#include <cuda_runtime.h>

#include "sil_common.h"

namespace sil {

struct BatchLaunch {
  const Req* reqs;          // device array of n request descriptors
  const int64_t* prefix;    // device int64[n+1]: first global chip of each request
  int n;
  int dt;
  DevParams dp;
  int chip;
  unsigned long long* head;  // device work-queue head (zeroed by the prologue)
  int grid;
  int schedule;             // kSched*: how CTAs get their chips
  int threads = kThreadsNarrow;  // threads per CTA: kThreadsNarrow or kThreadsWide
};

enum { kSchedStride = 0, kSchedQueue = 1, kSchedPerChip = 2 };

// Enqueues the prologue (zero counts, reset head) and the persistent kernel.
// batch_max_ctas_per_sm() must have been called once for the same (dt, H/S,
// chip) class first (it sets the kernel's shared-memory limit).
cudaError_t launch_batch(const BatchLaunch& b, cudaStream_t s);
int batch_max_ctas_per_sm(int dt, bool hs, int chip, int threads = kThreadsNarrow);

}  // namespace sil
