// sil_common.h -- host/device shared definitions of libsil (not part of the
// public ABI; the public header is include/sil.h).
#pragma once
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

#include "sil.h"

namespace sil {

// Parameters as the kernels see them (derived once on the host per call).
struct DevParams {
  uint8_t lo[3][3];  // [class][H, S, V]
  uint8_t hi[3][3];
  int32_t filter, median, mm_min_range, frac_den, v_trunc, max_shift;
  int32_t bgr;
  int32_t need_hs;        // 1 if some class range narrows H or S
  uint64_t u16_mul;       // ceil(2^40 / u16_scale): n / s == (n * mul) >> 40
  uint32_t u16_half;      // u16_scale / 2
  // -1 and 2^8, 2^16, 2^24, read from the kernel parameters so that the
  // median's subtractions, byte extractions and byte packing stay integer
  // multiply-adds, which issue on a different pipe than min/max and permutes.
  uint32_t neg1;
  uint32_t sh8, sh16, sh24;
};

// One labelling request (a tile or a whole scene) as the kernels see it.
struct Req {
  const uint8_t* img;
  int64_t H, W, pitch;
  uint8_t* labels;        // may be null
  int64_t lpitch;
  unsigned long long* counts;  // uint64[4], accumulated with atomics
  uint32_t* chip_counts;  // may be null
  int32_t gx, gy;         // chip grid
  int64_t chip_begin;     // index of this request's first chip in a batch
  uint8_t* vprime = nullptr;  // optional: the filter's corrected value V' per pixel
  int64_t vpitch = 0;
};

// Largest chip side handled with the chip resident in shared memory.
constexpr int kResidentChip = 256;
// Threads per CTA of the chip kernels: one half-warp row band per 16
// threads.  256 (16 bands of 16 rows on a 256-row chip) everywhere except
// where the batch autotuner picks 320 (20 bands of 12-13 rows); shared
// memory is laid out for the larger.  Each band also decodes the two rows
// beyond its ends for the median, so fewer, taller bands decode fewer rows
// twice (16 bands: 12.5 % extra, 20 bands: 15.6 %); 256 was faster than
// 320 at every request size measured.  At least 256: one thread per
// histogram bin in the statistics.
constexpr int kThreadsNarrow = 256;
constexpr int kThreadsWide = 320;
constexpr int kMaxThreads = kThreadsWide;

// Dynamic shared memory of a resident chip kernel of `threads` threads
// (the layout up to the row ring plus threads / 16 ring bands), raised where
// needed so that no more CTAs fit an SM than its tensor memory holds planes
// for: the block scheduler does not count tensor memory, and an allocation
// beyond an SM's 512 columns would wait for another CTA to finish.
size_t resident_smem_bytes(int dt, bool hs, int threads = kThreadsNarrow);
// Tensor-memory columns of a resident chip kernel's plane.
inline int plane_cols(int threads) { return threads <= 256 ? 128 : 256; }
// Whether the resident kernels of a (dtype, H/S) class keep their plane in
// tensor memory.
bool tmem_plane(int dt, bool hs);
// CTAs of kernel fn (threads per CTA, dynamic shared memory dyn_smem) that
// one SM holds at once, from its registers, shared memory and threads, and
// at most 512 / tmem_cols when it allocates tensor memory (the occupancy
// calculator reports one CTA per SM for any kernel that does).
int resident_ctas_per_sm(const void* fn, int threads, size_t dyn_smem, int tmem_cols);
// Sets a resident chip kernel's dynamic shared-memory limit and asks for the
// largest shared-memory carveout (its CTAs share an SM by shared memory;
// its global accesses bypass L1).
cudaError_t set_resident_attrs(const void* fn, size_t dyn_smem);

// Validates p and derives DevParams; returns SIL_OK or SIL_EINVAL with a
// message stored for sil_last_error().
sil_status derive_params(const sil_params* p, DevParams* dp);
void set_error(const char* fmt, ...);

}  // namespace sil
