// sil_label_kernel.cuh -- the single-request labelling kernels (internal).
// Each (dtype, H/S) class is compiled in a translation unit of its own
// (sil_label_k_*.cu), so the library builds in parallel.
#pragma once
#include <cuda_runtime.h>

#include <mutex>

#include "sil.h"
#include "sil_chip.cuh"
#include "sil_common.h"
#include "sil_generic.cuh"

namespace sil {

int device_sm_count();

// Work item k -> chip (cy, cx).  When the grid's last column is narrower
// than the chip, those chips (the slowest: their last half-warp lanes take a
// separate path) come first and the rest follow row by row, so that the
// last wave of the launch holds the bottom row's chips, the cheapest (often
// shorter than the chip).
__device__ __forceinline__ void chip_of(int64_t k, const Req& r, int chip, int64_t& cy,
                                        int64_t& cx) {
  const bool narrow_last = r.gx > 1 && (r.W % chip) != 0;
  if (!narrow_last) {
    cy = k / r.gx;
    cx = k - cy * r.gx;
  } else if (k < r.gy) {
    cy = k;
    cx = r.gx - 1;
  } else {
    const int64_t j = k - r.gy, g = r.gx - 1;
    cy = j / g;
    cx = j - cy * g;
  }
}

// Chip blockIdx.x of the request's grid (in chip_of order): one CTA per
// chip, so the hardware block scheduler hands the next chip to whichever
// slot frees first (and no chip loop keeps registers live across a chip).
template <int DT, bool HS>
__global__ void __launch_bounds__(kThreadsNarrow, (ResidentCtas<DT, HS>::k))
    k_label(Req r, DevParams dp, int chip) {
  extern __shared__ __align__(128) uint8_t smem_raw[];
  __shared__ uint8_t lut[256];
  __shared__ uint8_t vlut[256];
  ChipSmem<DT, HS>& sm = *reinterpret_cast<ChipSmem<DT, HS>*>(smem_raw);
  constexpr uint32_t kCols = PlaneCols<kThreadsNarrow>::kCols;
  if (!ChipSmem<DT, HS>::kSmemPlane) plane_alloc(&sm.st.tmem, kCols);
  int64_t cy, cx;
  chip_of(blockIdx.x, r, chip, cy, cx);
  label_chip<DT, HS>(r, dp, chip, cy, cx, sm, lut, vlut);
  if (!ChipSmem<DT, HS>::kSmemPlane) plane_free(sm.st.tmem, kCols);
}

// Chip kbeg + blockIdx.x / kSplitChip, labelled by a cluster of kSplitChip
// CTAs (one row slice each).  Used when a request has so few chips that
// kSplitChip CTAs per chip still fit in one wave: a chip then takes about
// 0.6 of the time one CTA needs (the statistics and table phases do not
// shrink with the slice).
constexpr int kSplitChip = 4;
template <int DT>
__global__ void __cluster_dims__(kSplitChip, 1, 1)
    __launch_bounds__(kThreadsNarrow, (ResidentCtas<SIL_U8, false>::k))
    k_label_split(Req r, DevParams dp, int chip, int64_t kbeg) {
  static_assert(DT == SIL_U8, "the split kernel serves u8 requests");
  extern __shared__ __align__(128) uint8_t smem_raw[];
  __shared__ uint8_t lut[256];
  __shared__ uint8_t vlut[256];
  ChipSmem<SIL_U8, false>& sm = *reinterpret_cast<ChipSmem<SIL_U8, false>*>(smem_raw);
  constexpr uint32_t kCols = PlaneCols<kThreadsNarrow>::kCols;
  if (!ChipSmem<SIL_U8, false>::kSmemPlane) plane_alloc(&sm.st.tmem, kCols);
  const int64_t k = kbeg + blockIdx.x / kSplitChip;
  const int64_t cy = k / r.gx, cx = k - cy * r.gx;
  label_chip<SIL_U8, false, kSplitChip>(r, dp, chip, cy, cx, sm, lut, vlut);
  if (!ChipSmem<SIL_U8, false>::kSmemPlane) plane_free(sm.st.tmem, kCols);
}

template <int DT, bool HS>
__global__ void __launch_bounds__(kThreadsNarrow, 2)
    k_label_generic(Req r, DevParams dp, int chip) {
  __shared__ __align__(16) ChipStat st;
  __shared__ uint8_t lut[256];
  const int64_t nchips = int64_t(r.gx) * r.gy;
  for (int64_t k = blockIdx.x; k < nchips; k += gridDim.x) {
    const int64_t cy = k / r.gx, cx = k - cy * r.gx;
    label_chip_generic<DT, HS>(r, dp, chip, cy, cx, st, lut);
  }
}

// Whether a grid of n chips goes to the split kernel: when kSplitChip CTAs
// per chip fit in one wave of resident CTAs.  (Splitting the chips of a
// last, partly filled wave of a larger grid was measured too: it does not
// shorten the launch, because the split chips can only start once the full
// waves end and still take 0.6 of a chip's time.)
inline bool split_all_chips(int64_t n, int64_t slots) {
  return slots > 0 && n > 0 && n * kSplitChip <= slots;
}

// The kernels of one (dtype, H/S) class.
template <int DT, bool HS>
struct LabelKernels {
  // Enqueues the labelling of request r (grid CTAs; the resident kernel when
  // the chip fits in shared memory).
  static cudaError_t launch(const Req& r, const DevParams& dp, int chip, int grid, cudaStream_t s);
  // Resident CTAs of the resident kernel on the device (SMs x CTAs per SM).
  static int64_t slots(size_t smem);
};

template <int DT, bool HS>
int64_t LabelKernels<DT, HS>::slots(size_t smem) {
  static std::once_flag once;
  static int64_t n = 0;
  std::call_once(once, [&] {
    const int per_sm = resident_ctas_per_sm(reinterpret_cast<const void*>(k_label<DT, HS>),
                                            kThreadsNarrow, smem, tmem_plane(DT, HS) ? plane_cols(kThreadsNarrow) : 0);
    n = int64_t(per_sm) * device_sm_count();
  });
  return n;
}

template <int DT, bool HS>
cudaError_t LabelKernels<DT, HS>::launch(const Req& r, const DevParams& dp, int chip, int grid,
                                         cudaStream_t s) {
  if (chip <= kResidentChip) {
    static std::once_flag once;
    static cudaError_t attr_err = cudaSuccess;
    const size_t smem = resident_smem_bytes(DT, HS, kThreadsNarrow);
    std::call_once(once, [&] {
      attr_err = set_resident_attrs(reinterpret_cast<const void*>(k_label<DT, HS>), smem);
      if constexpr (DT == SIL_U8 && !HS) {
        if (attr_err == cudaSuccess)
          attr_err = set_resident_attrs(reinterpret_cast<const void*>(k_label_split<SIL_U8>), smem);
      }
    });
    if (attr_err != cudaSuccess) return attr_err;
    // One CTA of 256 threads per chip (grid = the chip count, whatever the
    // caller's grid): the hardware block scheduler hands the next chip to
    // whichever slot frees first, which balances chips of uneven cost
    // (narrow edge chips, chips of one label) better than a fixed
    // persistent stride (measured 143 vs 162 us on the 10980^2 scene);
    // 320-thread CTAs were slower at every request size measured (a 512^2
    // tile to the 10980^2 scene).
    const int64_t nchips = int64_t(r.gx) * r.gy;
    if (nchips > int64_t(0x7fffffff)) return cudaErrorInvalidConfiguration;
    if constexpr (DT == SIL_U8 && !HS) {
      if (split_all_chips(nchips, slots(smem))) {
        k_label_split<SIL_U8><<<int(nchips * kSplitChip), kThreadsNarrow, smem, s>>>(r, dp, chip, 0);
        return cudaGetLastError();
      }
    }
    k_label<DT, HS><<<int(nchips), kThreadsNarrow, smem, s>>>(r, dp, chip);
    return cudaGetLastError();
  } else {
    k_label_generic<DT, HS><<<grid, kThreadsNarrow, 0, s>>>(r, dp, chip);
  }
  return cudaGetLastError();
}

extern template struct LabelKernels<SIL_U8, false>;
extern template struct LabelKernels<SIL_U8, true>;
extern template struct LabelKernels<SIL_U16, false>;
extern template struct LabelKernels<SIL_U16, true>;

}  // namespace sil
