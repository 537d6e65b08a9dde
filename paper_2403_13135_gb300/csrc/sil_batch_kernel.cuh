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
  __shared__ __align__(16) ChipStat st_generic;
  __shared__ __align__(16) Req s_req;
  __shared__ long long s_k, s_cy, s_cx;
  constexpr uint32_t kCols = PlaneCols<NT>::kCols;
  ChipSmem<DT, HS>& sm = *reinterpret_cast<ChipSmem<DT, HS>*>(smem_raw);
  if (RESIDENT && !ChipSmem<DT, HS>::kSmemPlane) plane_alloc(&sm.st.tmem, kCols);
  if (threadIdx.x == 0) s_k = schedule == kSchedQueue ? (long long)atomicAdd(head, 1ull) : (long long)blockIdx.x;
  __syncthreads();
  while (true) {
    // the chip's request and position through shared memory, so that no
    // loop state stays in registers across the chip
    if (threadIdx.x == 0) {
      const long long k = s_k;
      if (k < prefix[n]) {
        const int t = find_tile(prefix, n, k);
        s_req = reqs[t];
        const int64_t local = k - prefix[t];
        s_cy = local / s_req.gx;
        s_cx = local - s_cy * s_req.gx;
      } else {
        s_cy = -1;
      }
    }
    __syncthreads();
    if (s_cy < 0) break;
    if (RESIDENT) {
      label_chip<DT, HS>(s_req, dp, chip, s_cy, s_cx, sm, lut, lut);  // (batches have no V' output)
    } else {
      label_chip_generic<DT, HS>(s_req, dp, chip, s_cy, s_cx, st_generic, lut);
    }
    if (schedule == kSchedPerChip) break;
    __syncthreads();  // every thread is done with s_req and s_k
    if (threadIdx.x == 0) s_k = schedule == kSchedQueue ? (long long)atomicAdd(head, 1ull) : s_k + gridDim.x;
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
