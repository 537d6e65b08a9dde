// sil_batch_kernel.cuh -- the persistent batch kernel (internal).  Each
// (dtype, H/S) class of it is compiled in a translation unit of its own
// (sil_batch_k_*.cu: the four instances of resident or not x 256 or 320
// threads per CTA), so the library builds in parallel.
#pragma once
#include <cuda_runtime.h>

#include "sil.h"
#include "sil_batch.h"
#include "sil_chip.cuh"
#include "sil_common.h"
#include "sil_generic.cuh"

namespace sil {

// Tile holding global chip k: largest t with prefix[t] <= k.
__device__ __forceinline__ int find_tile(const int64_t* prefix, int n, int64_t k) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (prefix[mid] <= k)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

// Schedules of the batch kernel (chosen by the autotuner):
//   kSchedStride  persistent CTAs, CTA c labels global chips c, c + grid, ...
//   kSchedQueue   persistent CTAs taking the next chip from the queue head
//   kSchedPerChip one CTA per chip (grid = total chips): the hardware block
//                 scheduler hands chips to slots as they free up
template <int DT, bool HS, bool RESIDENT, int NT>
__global__ void __launch_bounds__(NT, RESIDENT ? ResidentCtas<DT, HS, NT>::k : ((DT == SIL_U8) ? 2 : 1))
    k_label_batch(const Req* __restrict__ reqs, const int64_t* __restrict__ prefix,
                  int n, DevParams dp, int chip, unsigned long long* head,
                  int schedule) {
  extern __shared__ __align__(128) uint8_t smem_raw[];
  __shared__ uint8_t lut[256];
  __shared__ long long s_next;
  __shared__ __align__(16) ChipStat st_generic;
  const int64_t total = prefix[n];
  constexpr uint32_t kCols = PlaneCols<NT>::kCols;
  ChipSmem<DT, HS>& sm = *reinterpret_cast<ChipSmem<DT, HS>*>(smem_raw);
  if (RESIDENT && !ChipSmem<DT, HS>::kSmemPlane) plane_alloc(&sm.st.tmem, kCols);
  int64_t k = blockIdx.x;
  if (schedule == kSchedQueue) {
    if (threadIdx.x == 0) s_next = (long long)atomicAdd(head, 1ull);
    __syncthreads();
    k = s_next;
  }
  while (k < total) {
    const int t = find_tile(prefix, n, k);
    const Req& r = reqs[t];
    const int64_t local = k - prefix[t];
    const int64_t cy = local / r.gx, cx = local - cy * r.gx;
    if (RESIDENT) {
      label_chip<DT, HS>(r, dp, chip, cy, cx, sm, lut, lut);  // (batches have no V' output)
    } else {
      label_chip_generic<DT, HS>(r, dp, chip, cy, cx, st_generic, lut);
    }
    if (schedule == kSchedQueue) {
      __syncthreads();  // everyone has read s_next
      if (threadIdx.x == 0) s_next = (long long)atomicAdd(head, 1ull);
      __syncthreads();
      k = s_next;
    } else if (schedule == kSchedStride) {
      k += gridDim.x;
    } else {
      break;
    }
  }
  if (RESIDENT && !ChipSmem<DT, HS>::kSmemPlane) plane_free(sm.st.tmem, kCols);
}

// The kernel instances of one (dtype, H/S) class.
template <int DT, bool HS>
struct BatchKernels {
  // Enqueues the kernel of b (resident when b.chip fits, b.threads per CTA).
  static cudaError_t launch(const BatchLaunch& b, cudaStream_t s);
  // The kernel instance, for attribute and occupancy queries.
  static const void* fn(bool resident, int threads);
};

template <int DT, bool HS>
cudaError_t BatchKernels<DT, HS>::launch(const BatchLaunch& b, cudaStream_t s) {
  const bool res = b.chip <= kResidentChip;
  const size_t smem = res ? resident_smem_bytes(DT, HS, b.threads) : 0;
  if (res) {
    if (b.threads == kThreadsWide)
      k_label_batch<DT, HS, true, kThreadsWide><<<b.grid, kThreadsWide, smem, s>>>(
          b.reqs, b.prefix, b.n, b.dp, b.chip, b.head, b.schedule);
    else
      k_label_batch<DT, HS, true, kThreadsNarrow><<<b.grid, kThreadsNarrow, smem, s>>>(
          b.reqs, b.prefix, b.n, b.dp, b.chip, b.head, b.schedule);
  } else {
    if (b.threads == kThreadsWide)
      k_label_batch<DT, HS, false, kThreadsWide><<<b.grid, kThreadsWide, 0, s>>>(
          b.reqs, b.prefix, b.n, b.dp, b.chip, b.head, b.schedule);
    else
      k_label_batch<DT, HS, false, kThreadsNarrow><<<b.grid, kThreadsNarrow, 0, s>>>(
          b.reqs, b.prefix, b.n, b.dp, b.chip, b.head, b.schedule);
  }
  return cudaGetLastError();
}

template <int DT, bool HS>
const void* BatchKernels<DT, HS>::fn(bool resident, int threads) {
  if (resident)
    return threads == kThreadsWide
               ? reinterpret_cast<const void*>(k_label_batch<DT, HS, true, kThreadsWide>)
               : reinterpret_cast<const void*>(k_label_batch<DT, HS, true, kThreadsNarrow>);
  return threads == kThreadsWide
             ? reinterpret_cast<const void*>(k_label_batch<DT, HS, false, kThreadsWide>)
             : reinterpret_cast<const void*>(k_label_batch<DT, HS, false, kThreadsNarrow>);
}

extern template struct BatchKernels<SIL_U8, false>;
extern template struct BatchKernels<SIL_U8, true>;
extern template struct BatchKernels<SIL_U16, false>;
extern template struct BatchKernels<SIL_U16, true>;

}  // namespace sil
