// sil_generic.cuh -- labeler for chips larger than 256 x 256 (up to 512).
//
// A 512 x 512 chip's filtered V plane (256 KB) does not fit in shared memory,
// so this variant keeps nothing per pixel: one CTA per chip sweeps the chip
// twice, recomputing V and its 3x3 median from the image in each sweep
// (sweep 1 -> histogram, sweep 2 -> labels and per-pixel counts).  Scalar,
// one pixel per thread step; used only when the statistics chip is set above
// 256.  Same arithmetic as the resident kernel (Sec. III-B filter and
// thresholds), no scratch memory.
#pragma once
#include "sil_chip.cuh"

namespace sil {

// 8-bit V (value) of pixel (y, x) plus nodata; optionally the H/S class mask.
template <int DT, bool HS>
__device__ __forceinline__ int pixel_v(const uint8_t* img, int64_t pitch,
                                       int64_t y, int64_t x, const DevParams& dp,
                                       bool* nodata, uint32_t* hsm) {
  int c[3];
  if (DT == SIL_U8) {
    const uint8_t* p = img + y * pitch + x * 3;
    c[0] = __ldg(p);
    c[1] = __ldg(p + 1);
    c[2] = __ldg(p + 2);
    *nodata = false;
  } else {
    const uint16_t* p = reinterpret_cast<const uint16_t*>(img + y * pitch + x * 6);
    const uint32_t r0 = __ldg(p), r1 = __ldg(p + 1), r2 = __ldg(p + 2);
    *nodata = (r0 | r1 | r2) == 0;
    c[0] = int(u16_to_v8(r0, dp));
    c[1] = int(u16_to_v8(r1, dp));
    c[2] = int(u16_to_v8(r2, dp));
  }
  if (HS) {
    const int ri = dp.bgr ? 2 : 0, bi = dp.bgr ? 0 : 2;
    *hsm = hs_mask(c[ri], c[1], c[bi], dp);
  }
  return max(c[0], max(c[1], c[2]));
}

// Filtered V of chip-local pixel (y, x): 3x3 median clamped to the chip.
template <int DT>
__device__ __forceinline__ int pixel_vf(const uint8_t* img, int64_t pitch,
                                        int64_t y0, int64_t x0, int h, int w,
                                        int y, int x, const DevParams& dp) {
  bool nd;
  uint32_t hm;
  if (!(dp.filter && dp.median)) return pixel_v<DT, false>(img, pitch, y0 + y, x0 + x, dp, &nd, &hm);
  int v[9];
  int n = 0;
#pragma unroll
  for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
    for (int dx = -1; dx <= 1; ++dx) {
      const int yy = min(max(y + dy, 0), h - 1), xx = min(max(x + dx, 0), w - 1);
      v[n++] = pixel_v<DT, false>(img, pitch, y0 + yy, x0 + xx, dp, &nd, &hm);
    }
  // selection of the 5th smallest by partial sorting network
#pragma unroll
  for (int i = 0; i < 5; ++i)
#pragma unroll
    for (int j = i + 1; j < 9; ++j) {
      const int a = v[i], b = v[j];
      v[i] = min(a, b);
      v[j] = max(a, b);
    }
  return v[4];
}

template <int DT, bool HS>
__device__ void label_chip_generic(const Req& r, const DevParams& dp, int chip,
                                   int64_t cy, int64_t cx, ChipStat& sm,
                                   uint8_t* lut) {
  const int tid = threadIdx.x, lane = tid & 31;
  const int64_t y0 = cy * chip, x0 = cx * chip;
  const int h = int(min(int64_t(chip), r.H - y0));
  const int w = int(min(int64_t(chip), r.W - x0));
  const int npx = h * w;
  __syncthreads();
  if (tid < 256) sm.hist[tid] = 0;
  __syncthreads();
  uint32_t nod = 0;
  for (int i = tid; i < npx; i += int(blockDim.x)) {
    const int y = i / w, x = i - y * w;
    bool nd = false;
    uint32_t hm;
    if (DT == SIL_U16) pixel_v<DT, false>(r.img, r.pitch, y0 + y, x0 + x, dp, &nd, &hm);
    const int vf = pixel_vf<DT>(r.img, r.pitch, y0, x0, h, w, y, x, dp);
    if (nd)
      ++nod;
    else
      atomicAdd(&sm.hist[vf], 1u);
  }
  nod = __reduce_add_sync(0xffffffffu, nod);
  if (lane == 0) sm.nod[tid >> 5] = nod;
  __syncthreads();
  if (tid < 32) {
    uint32_t nd = (lane < n_warps()) ? sm.nod[lane] : 0u;
    nd = __reduce_add_sync(0xffffffffu, nd);
    chip_stats_warp(sm, dp, uint32_t(npx) - nd);
  }
  __syncthreads();
  if (tid < 256) lut[tid] = uint8_t(lut_entry<HS>(tid, sm, dp));
  __syncthreads();
  uint32_t cnt[4] = {0, 0, 0, 0};
  for (int i = tid; i < npx; i += int(blockDim.x)) {
    const int y = i / w, x = i - y * w;
    bool nd;
    uint32_t hm = 0;
    pixel_v<DT, HS>(r.img, r.pitch, y0 + y, x0 + x, dp, &nd, &hm);
    const int vf = pixel_vf<DT>(r.img, r.pitch, y0, x0, h, w, y, x, dp);
    const uint32_t e = lut[vf];
    uint32_t lab;
    if (HS) {
      const uint32_t m = e & hm & 7u;
      lab = (m & 1u) ? 0u : (m & 2u) ? 1u : (m & 4u) ? 2u : 3u;
      if (e & 8u) lab = 3u;
    } else {
      lab = e;
    }
    if (nd) lab = 3u;
    cnt[lab] += 1;
    if (r.labels) r.labels[(y0 + y) * r.lpitch + x0 + x] = uint8_t(lab);
    if (r.vprime) r.vprime[(y0 + y) * r.vpitch + x0 + x] = nd ? 0 : uint8_t(vprime_value(vf, sm, dp));
  }
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const uint32_t s = __reduce_add_sync(0xffffffffu, cnt[c]);
    if (lane == 0) sm.red[tid >> 5][c] = s;
  }
  __syncthreads();
  if (tid < 4) {
    const int c = tid;
    uint32_t v = 0;
    for (int k = 0; k < n_warps(); ++k) v += sm.red[k][c];
    if (r.chip_counts) r.chip_counts[(cy * r.gx + cx) * 4 + c] = v;
    atomicAdd(&r.counts[c], (unsigned long long)v);
  }
}

}  // namespace sil
