// sil_api.cu -- C ABI entry points of libsil: parameters, single-request
// labelling (device and host buffers), confusion counts and colour render.
#include <cuda_runtime.h>

#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <mutex>

#include "sil.h"
#include "sil_chip.cuh"
#include "sil_common.h"
#include "sil_label_kernel.cuh"

namespace sil {

static thread_local char g_err[512] = "";

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

sil_status derive_params(const sil_params* p, DevParams* dp) {
  sil_params def;
  if (!p) {
    sil_params_default(&def);
    p = &def;
  }
  for (int k = 0; k < 3; ++k)
    for (int c = 0; c < 3; ++c)
      if (p->lo[k][c] > p->hi[k][c]) {
        set_error("params: lo[%d][%d]=%d > hi[%d][%d]=%d", k, c, p->lo[k][c], k, c, p->hi[k][c]);
        return SIL_EINVAL;
      }
#define SIL_RANGE(f, a, b)                                                \
  if (p->f < (a) || p->f > (b)) {                                         \
    set_error("params: %s=%d outside [%d, %d]", #f, int(p->f), int(a), int(b)); \
    return SIL_EINVAL;                                                    \
  }
  SIL_RANGE(filter, 0, 1)
  SIL_RANGE(chip, 4, 512)
  SIL_RANGE(median, 0, 1)
  SIL_RANGE(mm_min_range, 1, 255)
  SIL_RANGE(mm_min_frac_den, 1, 65536)
  SIL_RANGE(v_trunc, 0, 255)
  SIL_RANGE(max_shift, 0, 255)
  SIL_RANGE(bgr, 0, 1)
  SIL_RANGE(u16_scale, 1, 65535)
#undef SIL_RANGE
  memset(dp, 0, sizeof(*dp));
  memcpy(dp->lo, p->lo, sizeof(dp->lo));
  memcpy(dp->hi, p->hi, sizeof(dp->hi));
  dp->filter = p->filter;
  dp->median = p->median;
  dp->mm_min_range = p->mm_min_range;
  dp->frac_den = p->mm_min_frac_den;
  dp->v_trunc = p->v_trunc;
  dp->max_shift = p->max_shift;
  dp->bgr = p->bgr;
  dp->need_hs = 0;
  for (int k = 0; k < 3; ++k)
    if (p->lo[k][0] > 0 || p->hi[k][0] < 179 || p->lo[k][1] > 0 || p->hi[k][1] < 255)
      dp->need_hs = 1;
  const uint64_t s = uint64_t(p->u16_scale);
  dp->u16_half = uint32_t(s / 2);
  dp->u16_mul = ((uint64_t(1) << 40) + s - 1) / s;
  dp->neg1 = 0xFFFFFFFFu;
  dp->sh8 = 1u << 8;
  dp->sh16 = 1u << 16;
  dp->sh24 = 1u << 24;
  // The quotient by multiplication must be exact on every input it meets.
  static thread_local int checked_scale = -1;
  if (checked_scale != p->u16_scale) {
    for (uint64_t x = 0; x < 65536; ++x) {
      const uint64_t n = x * 255 + dp->u16_half;
      if (((n * dp->u16_mul) >> 40) != n / s) {
        set_error("params: no exact reciprocal for u16_scale=%d", p->u16_scale);
        return SIL_EINVAL;
      }
    }
    checked_scale = p->u16_scale;
  }
  return SIL_OK;
}

static sil_status cuda_fail(cudaError_t e, const char* what) {
  set_error("%s: %s", what, cudaGetErrorString(e));
  return SIL_ECUDA;
}

// ---------------------------------------------------------------------------
// Single-request labelling (kernels: sil_label_kernel.cuh).
// ---------------------------------------------------------------------------
namespace {
struct SmLimits {
  int smem = 0, regs = 0, reserved = 0, blocks = 0, threads = 0;
};
// Per-SM limits of the current device (all devices of a process are taken
// to be alike).
const SmLimits& sm_limits() {
  static std::once_flag once;
  static SmLimits l;
  std::call_once(once, [] {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&l.smem, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    cudaDeviceGetAttribute(&l.regs, cudaDevAttrMaxRegistersPerMultiprocessor, dev);
    cudaDeviceGetAttribute(&l.reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev);
    cudaDeviceGetAttribute(&l.blocks, cudaDevAttrMaxBlocksPerMultiprocessor, dev);
    cudaDeviceGetAttribute(&l.threads, cudaDevAttrMaxThreadsPerMultiProcessor, dev);
    cudaGetLastError();
  });
  return l;
}
}  // namespace

template <int DT, bool HS>
static size_t class_smem_bytes(int threads) {
  using T = ChipSmem<DT, HS>;
  return chip_smem_bytes<Px<DT>::BPP, HS || DT == SIL_U16, T::kSmemPlane>(threads);
}

bool tmem_plane(int dt, bool hs) {
  if (dt == SIL_U8) return hs ? TmemPlane<SIL_U8, true>::value : TmemPlane<SIL_U8, false>::value;
  return hs ? TmemPlane<SIL_U16, true>::value : TmemPlane<SIL_U16, false>::value;
}

size_t resident_smem_bytes(int dt, bool hs, int threads) {
  size_t b;
  if (dt == SIL_U8)
    b = hs ? class_smem_bytes<SIL_U8, true>(threads) : class_smem_bytes<SIL_U8, false>(threads);
  else
    b = hs ? class_smem_bytes<SIL_U16, true>(threads) : class_smem_bytes<SIL_U16, false>(threads);
  if (!tmem_plane(dt, hs)) return b;
  const int max_ctas = 512 / plane_cols(threads);
  const int smem_sm = sm_limits().smem > 0 ? sm_limits().smem : 233472;
  const size_t floor_bytes = size_t(smem_sm / (max_ctas + 1) + 1);
  return b > floor_bytes ? b : floor_bytes;
}

int resident_ctas_per_sm(const void* fn, int threads, size_t dyn_smem, int tmem_cols) {
  const SmLimits& l = sm_limits();
  cudaFuncAttributes fa{};
  if (cudaFuncGetAttributes(&fa, fn) != cudaSuccess || l.regs <= 0 || l.smem <= 0) {
    cudaGetLastError();
    return 1;
  }
  const int warps = (threads + 31) / 32;
  const int warp_regs = ((fa.numRegs * 32 + 255) / 256) * 256;
  int c = warp_regs > 0 ? l.regs / (warp_regs * warps) : l.blocks;
  c = std::min(c, l.smem / int(dyn_smem + fa.sharedSizeBytes + size_t(l.reserved)));
  if (l.threads > 0) c = std::min(c, l.threads / threads);
  if (l.blocks > 0) c = std::min(c, l.blocks);
  if (tmem_cols > 0) c = std::min(c, 512 / tmem_cols);
  return c > 0 ? c : 1;
}

cudaError_t set_resident_attrs(const void* fn, size_t dyn_smem) {
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, int(dyn_smem));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout,
                             int(cudaSharedmemCarveoutMaxShared));
  return e;
}

int device_sm_count();

cudaError_t launch_label(const Req& r, int dt, const DevParams& dp, int chip,
                         int grid, cudaStream_t s) {
  const bool hs = dp.need_hs != 0;
  if (dt == SIL_U8)
    return hs ? LabelKernels<SIL_U8, true>::launch(r, dp, chip, grid, s)
              : LabelKernels<SIL_U8, false>::launch(r, dp, chip, grid, s);
  return hs ? LabelKernels<SIL_U16, true>::launch(r, dp, chip, grid, s)
            : LabelKernels<SIL_U16, false>::launch(r, dp, chip, grid, s);
}

// Shape / pointer checks shared by the request entry points.
sil_status check_request(const void* img, int64_t H, int64_t W, int64_t pitch,
                         sil_dtype dt, const uint8_t* labels, int64_t lpitch,
                         const uint64_t* counts) {
  if (dt != SIL_U8 && dt != SIL_U16) {
    set_error("dtype %d is not SIL_U8 or SIL_U16", int(dt));
    return SIL_EINVAL;
  }
  if (!img || !counts) {
    set_error("img and counts must not be NULL");
    return SIL_EINVAL;
  }
  if (H < 1 || W < 1 || H > (int64_t(1) << 31) || W > (int64_t(1) << 31) ||
      H * W >= (int64_t(1) << 40)) {
    set_error("bad shape %lld x %lld", (long long)H, (long long)W);
    return SIL_EINVAL;
  }
  const int64_t bpp = dt == SIL_U8 ? 3 : 6;
  if (pitch < W * bpp) {
    set_error("pitch_bytes %lld < %lld bytes per row", (long long)pitch, (long long)(W * bpp));
    return SIL_EINVAL;
  }
  if (dt == SIL_U16 && ((reinterpret_cast<uintptr_t>(img) & 1) || (pitch & 1))) {
    set_error("uint16 images need 2-byte aligned img and pitch");
    return SIL_EINVAL;
  }
  if (labels && lpitch < W) {
    set_error("label_pitch %lld < W %lld", (long long)lpitch, (long long)W);
    return SIL_EINVAL;
  }
  return SIL_OK;
}

int device_sm_count() {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms > 0 ? sms : 1;
}

// ---------------------------------------------------------------------------
// Confusion counts and colour render (Sec. IV-A metrics; Sec. III-A colours).
// ---------------------------------------------------------------------------
__global__ void k_confusion(const uint8_t* pred, int64_t pp, const uint8_t* ref,
                            int64_t rp, int64_t H, int64_t W, int chip, int gx,
                            int gy, unsigned long long* conf, uint32_t* chip_conf) {
  __shared__ uint32_t c16[16];
  const int64_t nchips = int64_t(gx) * gy;
  for (int64_t k = blockIdx.x; k < nchips; k += gridDim.x) {
    __syncthreads();
    if (threadIdx.x < 16) c16[threadIdx.x] = 0;
    __syncthreads();
    const int64_t cy = k / gx, cx = k - cy * gx;
    const int64_t y0 = cy * chip, x0 = cx * chip;
    const int h = int(min(int64_t(chip), H - y0)), w = int(min(int64_t(chip), W - x0));
    uint32_t loc[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) loc[i] = 0;
    for (int i = threadIdx.x; i < h * w; i += blockDim.x) {
      const int y = i / w, x = i - y * w;
      const uint32_t a = pred[(y0 + y) * pp + x0 + x], b = ref[(y0 + y) * rp + x0 + x];
      if (a > 3 || b > 3) continue;  // not a label: not counted
      const uint32_t idx = a * 4 + b;
#pragma unroll
      for (int j = 0; j < 16; ++j) loc[j] += (idx == uint32_t(j)) ? 1u : 0u;
    }
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      const uint32_t s = __reduce_add_sync(0xffffffffu, loc[j]);
      if ((threadIdx.x & 31) == 0 && s) atomicAdd(&c16[j], s);
    }
    __syncthreads();
    if (threadIdx.x < 16) {
      if (chip_conf) chip_conf[k * 16 + threadIdx.x] = c16[threadIdx.x];
      atomicAdd(&conf[threadIdx.x], (unsigned long long)c16[threadIdx.x]);
    }
  }
}

__global__ void k_render(const uint8_t* labels, int64_t lp, int64_t H, int64_t W,
                         uint8_t* rgb, int64_t rp) {
  // thick ice red, thin ice blue, open water green, masked black
  const uint32_t pal[4] = {0x0000FFu, 0xFF0000u, 0x00FF00u, 0x000000u};
  const int64_t n = H * W;
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n;
       i += int64_t(gridDim.x) * blockDim.x) {
    const int64_t y = i / W, x = i - y * W;
    const uint32_t l = labels[y * lp + x];
    const uint32_t c = pal[l & 3u];
    uint8_t* o = rgb + y * rp + 3 * x;
    o[0] = uint8_t(c);
    o[1] = uint8_t(c >> 8);
    o[2] = uint8_t(c >> 16);
  }
}

// Chips k0 .. k0 + n - 1 of the chip grid as image chips and colour-mask
// chips (thick ice red, thin ice blue, open water green, masked black; zero
// past the scene's edges).  A thread handles 4 consecutive pixels of one
// chip row: 12 image bytes and 4 labels in, 12 + 12 bytes out as words.
__global__ void k_export(const uint8_t* img, int64_t H, int64_t W, int64_t pitch,
                         const uint8_t* labels, int64_t lp, int chip, int gx, int64_t k0,
                         int64_t n, uint8_t* chips, uint8_t* masks) {
  const uint32_t pal[4] = {0x0000FFu, 0xFF0000u, 0x00FF00u, 0x000000u};
  const int q = chip >> 2;  // groups of 4 pixels per chip row (chip % 4 handled below)
  const int qr = (chip + 3) >> 2;
  const int64_t groups = n * chip * qr;
  for (int64_t g = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; g < groups;
       g += int64_t(gridDim.x) * blockDim.x) {
    const int64_t c = g / (int64_t(chip) * qr);
    const int rem = int(g - c * chip * qr), yy = rem / qr, x4 = 4 * (rem - (rem / qr) * qr);
    const int64_t k = k0 + c;
    const int64_t sy = (k / gx) * chip + yy, sx0 = (k % gx) * chip + x4;
    uint8_t px[12], mk[12];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int64_t sx = sx0 + j;
      const bool in = sy < H && sx < W && x4 + j < chip;
      const uint8_t* s = img + sy * pitch + 3 * sx;
      const uint32_t col = in ? pal[labels[sy * lp + sx] & 3u] : 0u;
      px[3 * j] = in ? s[0] : 0;
      px[3 * j + 1] = in ? s[1] : 0;
      px[3 * j + 2] = in ? s[2] : 0;
      mk[3 * j] = uint8_t(col);
      mk[3 * j + 1] = uint8_t(col >> 8);
      mk[3 * j + 2] = uint8_t(col >> 16);
    }
    const int64_t o = ((c * chip + yy) * chip + x4) * 3;
    const int nb = 3 * min(4, chip - x4);
    if (nb == 12 && ((o & 3) == 0)) {
      uint32_t a[3], b[3];
      memcpy(a, px, 12);
      memcpy(b, mk, 12);
      if (chips) {
        uint32_t* d = reinterpret_cast<uint32_t*>(chips + o);
        d[0] = a[0]; d[1] = a[1]; d[2] = a[2];
      }
      if (masks) {
        uint32_t* d = reinterpret_cast<uint32_t*>(masks + o);
        d[0] = b[0]; d[1] = b[1]; d[2] = b[2];
      }
    } else {
      for (int j = 0; j < nb; ++j) {
        if (chips) chips[o + j] = px[j];
        if (masks) masks[o + j] = mk[j];
      }
    }
  }
  (void)q;
}

}  // namespace sil

using namespace sil;

extern "C" {

sil_status sil_params_default(sil_params* p) {
  if (!p) {
    set_error("sil_params_default: NULL");
    return SIL_EINVAL;
  }
  memset(p, 0, sizeof(*p));
  const uint8_t lo[3][3] = {{0, 0, 205}, {0, 0, 31}, {0, 0, 0}};
  const uint8_t hi[3][3] = {{185, 255, 255}, {185, 255, 204}, {185, 255, 30}};
  memcpy(p->lo, lo, sizeof(lo));
  memcpy(p->hi, hi, sizeof(hi));
  p->filter = 1;
  p->chip = 256;
  p->median = 1;
  p->mm_min_range = 64;
  p->mm_min_frac_den = 16;
  p->v_trunc = 255;
  p->max_shift = 255;
  p->bgr = 0;
  p->u16_scale = 10000;
  return SIL_OK;
}

sil_status sil_params_validate(const sil_params* p) {
  if (!p) {
    set_error("sil_params_validate: NULL");
    return SIL_EINVAL;
  }
  DevParams dp;
  return derive_params(p, &dp);
}

const char* sil_status_string(sil_status s) {
  switch (s) {
    case SIL_OK: return "ok";
    case SIL_EINVAL: return "invalid argument";
    case SIL_ENOMEM: return "out of memory";
    case SIL_ECUDA: return "CUDA error";
    case SIL_ETIMEOUT: return "timed out";
    case SIL_EBUSY: return "busy";
    case SIL_ECANCELED: return "cancelled";
  }
  return "unknown status";
}

const char* sil_last_error(void) { return g_err; }

int sil_version(void) { return SIL_ABI_VERSION; }

sil_status sil_label(const void* img, int64_t H, int64_t W, int64_t pitch_bytes,
                     sil_dtype dt, const sil_params* p, uint8_t* labels,
                     int64_t label_pitch, uint64_t* counts, uint32_t* chip_counts,
                     sil_stream stream) {
  return sil_label_v(img, H, W, pitch_bytes, dt, p, labels, label_pitch, nullptr, 0, counts,
                     chip_counts, stream);
}

sil_status sil_label_v(const void* img, int64_t H, int64_t W, int64_t pitch_bytes,
                       sil_dtype dt, const sil_params* p, uint8_t* labels,
                       int64_t label_pitch, uint8_t* vprime, int64_t vprime_pitch,
                       uint64_t* counts, uint32_t* chip_counts, sil_stream stream) {
  g_err[0] = 0;
  sil_status st = check_request(img, H, W, pitch_bytes, dt, labels, label_pitch, counts);
  if (st != SIL_OK) return st;
  if (vprime && vprime_pitch < W) {
    set_error("sil_label_v: vprime_pitch %lld < W %lld", (long long)vprime_pitch, (long long)W);
    return SIL_EINVAL;
  }
  DevParams dp;
  st = derive_params(p, &dp);
  if (st != SIL_OK) return st;
  const int chip = p ? p->chip : 256;
  Req r;
  r.img = static_cast<const uint8_t*>(img);
  r.H = H;
  r.W = W;
  r.pitch = pitch_bytes;
  r.labels = labels;
  r.lpitch = label_pitch;
  r.counts = reinterpret_cast<unsigned long long*>(counts);
  r.chip_counts = chip_counts;
  r.gx = int32_t((W + chip - 1) / chip);
  r.gy = int32_t((H + chip - 1) / chip);
  r.chip_begin = 0;
  r.vprime = vprime;
  r.vpitch = vprime_pitch;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemsetAsync(counts, 0, 4 * sizeof(uint64_t), s);
  if (e != cudaSuccess) return cuda_fail(e, "sil_label: memset counts");
  const int64_t nchips = int64_t(r.gx) * r.gy;
  const int64_t cap = int64_t(device_sm_count()) * 16;
  const int grid = int(nchips < cap ? nchips : cap);
  e = launch_label(r, dt, dp, chip, grid, s);
  if (e != cudaSuccess) return cuda_fail(e, "sil_label: launch");
  return SIL_OK;
}

// Host-buffer variant: per-thread cached device staging buffers, two copy
// streams and per-stripe events.  The image is cut into stripes of whole
// chip rows; stripe i is copied in on one stream while stripe i-1 is
// labelled on the caller's stream and the labels of stripe i-2 are copied
// out on the other, so the call costs about one pass over the host link.
constexpr int kMaxStripes = 64;
#ifndef SIL_HOST_STRIPES
#define SIL_HOST_STRIPES 12
#endif
struct HostStage {
  int device = -1;
  void* img = nullptr;
  size_t img_bytes = 0;
  uint8_t* lab = nullptr;
  size_t lab_bytes = 0;
  uint64_t* cnt = nullptr;
  uint32_t* cc = nullptr;
  size_t cc_bytes = 0;
  cudaStream_t in = nullptr, out = nullptr;
  cudaEvent_t start = nullptr, ev_in[kMaxStripes] = {}, ev_done[kMaxStripes] = {};
  void release() {
    cudaFree(img);
    cudaFree(lab);
    cudaFree(cnt);
    cudaFree(cc);
    if (in) cudaStreamDestroy(in);
    if (out) cudaStreamDestroy(out);
    if (start) cudaEventDestroy(start);
    for (int i = 0; i < kMaxStripes; ++i) {
      if (ev_in[i]) cudaEventDestroy(ev_in[i]);
      if (ev_done[i]) cudaEventDestroy(ev_done[i]);
      ev_in[i] = ev_done[i] = nullptr;
    }
    device = -1;
    img = nullptr;
    lab = nullptr;
    cnt = nullptr;
    cc = nullptr;
    img_bytes = lab_bytes = cc_bytes = 0;
    in = out = nullptr;
    start = nullptr;
  }
  ~HostStage() { release(); }
};
static thread_local HostStage g_stage;

static sil_status ensure(void** p, size_t* have, size_t need) {
  if (*have >= need && *p) return SIL_OK;
  cudaFree(*p);
  *p = nullptr;
  *have = 0;
  cudaError_t e = cudaMalloc(p, need);
  if (e != cudaSuccess) {
    set_error("cudaMalloc(%zu): %s", need, cudaGetErrorString(e));
    return SIL_ENOMEM;
  }
  *have = need;
  return SIL_OK;
}

// Streams and events of the pipeline, created once per thread and device.
static sil_status ensure_pipe(HostStage& g) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    set_error("sil_label_host: no current device");
    return SIL_ECUDA;
  }
  if (g.device != dev) g.release();  // buffers of another device
  g.device = dev;
  if (g.in) return SIL_OK;
  cudaError_t e = cudaStreamCreateWithFlags(&g.in, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&g.out, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&g.start, cudaEventDisableTiming);
  for (int i = 0; i < kMaxStripes && e == cudaSuccess; ++i) {
    e = cudaEventCreateWithFlags(&g.ev_in[i], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&g.ev_done[i], cudaEventDisableTiming);
  }
  if (e != cudaSuccess) {
    g.release();
    return cuda_fail(e, "sil_label_host: stream/event setup");
  }
  return SIL_OK;
}

sil_status sil_label_host(const void* img, int64_t H, int64_t W, int64_t pitch_bytes,
                          sil_dtype dt, const sil_params* p, uint8_t* labels,
                          int64_t label_pitch, uint64_t* counts,
                          uint32_t* chip_counts, sil_stream stream) {
  g_err[0] = 0;
  sil_status st = check_request(img, H, W, pitch_bytes, dt, labels, label_pitch, counts);
  if (st != SIL_OK) return st;
  DevParams dp;
  st = derive_params(p, &dp);
  if (st != SIL_OK) return st;
  const int chip = p ? p->chip : 256;
  const int64_t bpp = dt == SIL_U8 ? 3 : 6;
  const int64_t row_bytes = W * bpp;
  const int64_t gx = (W + chip - 1) / chip, gy = (H + chip - 1) / chip;
  HostStage& g = g_stage;
  if ((st = ensure_pipe(g)) != SIL_OK) return st;
  // the device copy keeps the host pitch, so each stripe is one contiguous
  // range when the host rows are dense
  if ((st = ensure(&g.img, &g.img_bytes, size_t(pitch_bytes * H))) != SIL_OK) return st;
  if (labels && (st = ensure(reinterpret_cast<void**>(&g.lab), &g.lab_bytes, size_t(W * H))) != SIL_OK)
    return st;
  size_t cnt_bytes = g.cnt ? 32 : 0;
  if ((st = ensure(reinterpret_cast<void**>(&g.cnt), &cnt_bytes, 32)) != SIL_OK) return st;
  if (chip_counts &&
      (st = ensure(reinterpret_cast<void**>(&g.cc), &g.cc_bytes, size_t(gx * gy * 16))) != SIL_OK)
    return st;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  uint8_t* dimg = static_cast<uint8_t*>(g.img);
  const uint8_t* himg = static_cast<const uint8_t*>(img);
  // stripes of whole chip rows: one chip row first and last (the copy in of
  // the first and the labelling and copy out of the last are not overlapped
  // with anything), about SIL_HOST_STRIPES - 2 equal ones between
  int64_t cut[kMaxStripes + 1];
  int nstripes = 0;
  {
    const int64_t mid = gy > 2 ? gy - 2 : 0;
    int64_t ks = mid / (SIL_HOST_STRIPES - 2);
    if (ks < 1) ks = 1;
    if ((mid + ks - 1) / ks > kMaxStripes - 2) ks = (mid + kMaxStripes - 3) / (kMaxStripes - 2);
    int64_t row = 0;
    cut[0] = 0;
    auto add = [&](int64_t rows) {
      row = row + rows < gy ? row + rows : gy;
      cut[++nstripes] = row;
    };
    if (gy > 2) {
      add(1);
      while (row < gy - 1) add(row + ks < gy - 1 ? ks : gy - 1 - row);
      add(1);
    } else {
      while (row < gy) add(1);
    }
  }
  Req r;
  r.W = W;
  r.pitch = pitch_bytes;
  r.lpitch = W;
  r.counts = reinterpret_cast<unsigned long long*>(g.cnt);
  r.gx = int32_t(gx);
  r.chip_begin = 0;
  const int64_t cap = int64_t(device_sm_count()) * 16;
  cudaError_t e = cudaEventRecord(g.start, s);  // the copies follow earlier work on s
  if (e == cudaSuccess) e = cudaStreamWaitEvent(g.in, g.start, 0);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(g.out, g.start, 0);
  if (e == cudaSuccess) e = cudaMemsetAsync(g.cnt, 0, 32, s);
  for (int i = 0; i < nstripes && e == cudaSuccess; ++i) {
    const int64_t r0 = cut[i] * chip;
    const int64_t r1 = cut[i + 1] * chip < H ? cut[i + 1] * chip : H;
    const int64_t rows = r1 - r0;
    // copy in (the last row only up to its last pixel)
    if (pitch_bytes == row_bytes)
      e = cudaMemcpyAsync(dimg + r0 * pitch_bytes, himg + r0 * pitch_bytes, size_t(rows * row_bytes),
                          cudaMemcpyHostToDevice, g.in);
    else
      e = cudaMemcpy2DAsync(dimg + r0 * pitch_bytes, pitch_bytes, himg + r0 * pitch_bytes, pitch_bytes,
                            row_bytes, rows, cudaMemcpyHostToDevice, g.in);
    if (e == cudaSuccess) e = cudaEventRecord(g.ev_in[i], g.in);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, g.ev_in[i], 0);
    if (e != cudaSuccess) break;
    // label the stripe; counts accumulate, chip counts land at its chip rows
    r.img = dimg + r0 * pitch_bytes;
    r.H = rows;
    r.labels = labels ? g.lab + r0 * W : nullptr;
    r.chip_counts = chip_counts ? g.cc + (r0 / chip) * gx * 4 : nullptr;
    r.gy = int32_t((rows + chip - 1) / chip);
    const int64_t nchips = int64_t(r.gx) * r.gy;
    e = launch_label(r, dt, dp, chip, int(nchips < cap ? nchips : cap), s);
    if (e == cudaSuccess) e = cudaEventRecord(g.ev_done[i], s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(g.out, g.ev_done[i], 0);
    if (e == cudaSuccess && labels) {
      if (label_pitch == W)
        e = cudaMemcpyAsync(labels + r0 * W, g.lab + r0 * W, size_t(rows * W), cudaMemcpyDeviceToHost,
                            g.out);
      else
        e = cudaMemcpy2DAsync(labels + r0 * label_pitch, label_pitch, g.lab + r0 * W, W, W, rows,
                              cudaMemcpyDeviceToHost, g.out);
    }
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(counts, g.cnt, 32, cudaMemcpyDeviceToHost, g.out);
  if (e == cudaSuccess && chip_counts)
    e = cudaMemcpyAsync(chip_counts, g.cc, size_t(gx * gy * 16), cudaMemcpyDeviceToHost, g.out);
  // the out stream ends after every stripe's kernel and copy
  const cudaError_t es = cudaStreamSynchronize(g.out);
  const cudaError_t es2 = cudaStreamSynchronize(g.in);
  if (e == cudaSuccess) e = es != cudaSuccess ? es : es2;
  if (e != cudaSuccess) return cuda_fail(e, "sil_label_host");
  return SIL_OK;
}

sil_status sil_confusion(const uint8_t* pred, int64_t pred_pitch, const uint8_t* ref,
                         int64_t ref_pitch, int64_t H, int64_t W, int32_t chip,
                         uint64_t* conf, uint32_t* chip_conf, sil_stream stream) {
  g_err[0] = 0;
  if (!pred || !ref || !conf || H < 1 || W < 1 || pred_pitch < W || ref_pitch < W ||
      chip < 4 || chip > 512) {
    set_error("sil_confusion: invalid arguments");
    return SIL_EINVAL;
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemsetAsync(conf, 0, 16 * sizeof(uint64_t), s);
  if (e != cudaSuccess) return cuda_fail(e, "sil_confusion: memset");
  const int gx = int((W + chip - 1) / chip), gy = int((H + chip - 1) / chip);
  const int64_t nchips = int64_t(gx) * gy;
  const int64_t cap = int64_t(device_sm_count()) * 8;
  k_confusion<<<int(nchips < cap ? nchips : cap), 256, 0, s>>>(
      pred, pred_pitch, ref, ref_pitch, H, W, chip, gx, gy,
      reinterpret_cast<unsigned long long*>(conf), chip_conf);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "sil_confusion: launch");
  return SIL_OK;
}

sil_status sil_render(const uint8_t* labels, int64_t label_pitch, int64_t H, int64_t W,
                      uint8_t* rgb, int64_t rgb_pitch, sil_stream stream) {
  g_err[0] = 0;
  if (!labels || !rgb || H < 1 || W < 1 || label_pitch < W || rgb_pitch < 3 * W) {
    set_error("sil_render: invalid arguments");
    return SIL_EINVAL;
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const int64_t n = H * W;
  const int64_t cap = int64_t(device_sm_count()) * 8;
  const int64_t want = (n + 255) / 256;
  k_render<<<int(want < cap ? want : cap), 256, 0, s>>>(labels, label_pitch, H, W, rgb, rgb_pitch);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "sil_render: launch");
  return SIL_OK;
}

sil_status sil_metrics_from_confusion(const uint64_t* conf, sil_metrics* out) {
  g_err[0] = 0;
  if (!conf || !out) {
    set_error("sil_metrics_from_confusion: NULL argument");
    return SIL_EINVAL;
  }
  memset(out, 0, sizeof(*out));
  auto div = [](double a, double b) { return b != 0.0 ? a / b : 0.0; };
  double col[3] = {0, 0, 0}, row[4] = {0, 0, 0, 0}, total = 0, tp = 0;
  for (int a = 0; a < 4; ++a)
    for (int b = 0; b < 3; ++b) {  // the reference-masked column is left out
      const double v = double(conf[a * 4 + b]);
      col[b] += v;
      row[a] += v;
      total += v;
    }
  for (int k = 0; k < 3; ++k) {
    const double t = double(conf[k * 4 + k]);
    tp += t;
    out->precision[k] = div(t, row[k]);
    out->recall[k] = div(t, col[k]);
    out->f1[k] = div(2.0 * out->precision[k] * out->recall[k], out->precision[k] + out->recall[k]);
    out->support[k] = conf[0 * 4 + k] + conf[1 * 4 + k] + conf[2 * 4 + k] + conf[3 * 4 + k];
    const double w = div(col[k], total);
    out->macro_precision += out->precision[k] / 3.0;
    out->macro_recall += out->recall[k] / 3.0;
    out->macro_f1 += out->f1[k] / 3.0;
    out->weighted_precision += out->precision[k] * w;
    out->weighted_recall += out->recall[k] * w;
    out->weighted_f1 += out->f1[k] * w;
  }
  out->accuracy = div(tp, total);
  for (int a = 0; a < 4; ++a)
    for (int b = 0; b < 3; ++b) out->matrix[a][b] = div(double(conf[a * 4 + b]), col[b]);
  return SIL_OK;
}

sil_status sil_export_chips(const uint8_t* img, int64_t H, int64_t W, int64_t pitch_bytes,
                            const uint8_t* labels, int64_t label_pitch, int32_t chip, int64_t k0,
                            int64_t n, uint8_t* chips, uint8_t* masks, sil_stream stream) {
  g_err[0] = 0;
  if (!img || !labels || H < 1 || W < 1 || pitch_bytes < 3 * W || label_pitch < W || chip < 4 ||
      chip > 512) {
    set_error("sil_export_chips: invalid arguments");
    return SIL_EINVAL;
  }
  const int64_t gx = (W + chip - 1) / chip, gy = (H + chip - 1) / chip;
  if (k0 < 0 || n < 1 || k0 + n > gx * gy) {
    set_error("sil_export_chips: chips %lld..%lld outside the grid of %lld", (long long)k0,
              (long long)(k0 + n - 1), (long long)(gx * gy));
    return SIL_EINVAL;
  }
  if (!chips && !masks) return SIL_OK;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const int64_t groups = n * chip * ((chip + 3) / 4);
  const int64_t cap = int64_t(device_sm_count()) * 8;
  const int64_t want = (groups + 255) / 256;
  k_export<<<int(want < cap ? want : cap), 256, 0, s>>>(img, H, W, pitch_bytes, labels, label_pitch,
                                                        chip, int(gx), k0, n, chips, masks);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "sil_export_chips: launch");
  return SIL_OK;
}

}  // extern "C"
