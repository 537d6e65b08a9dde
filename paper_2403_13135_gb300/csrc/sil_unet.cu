// sil_unet.cu -- U-Net inference on 256 x 256 chips (Sec. III-C "U-Net
// Model Inferencing"), the 3x3 and transposed convolutions as implicit GEMMs
// on the tcgen05 tensor cores.
//
// Convolution kernel (k_conv): a tile is 128 pixels x NT output channels,
// D[p][n] = sum_k A[p][k] B[n][k], with
//   3x3:  k = tap * Ci + c, A[p][k] = x[pixel p shifted by tap][c] (zero
//         outside the image), B[n][k] = w[n][c][tap / 3][tap % 3];
//   2x2 transposed, stride 2:  k = c, A[p][k] = x[p][c], n = (2 i + j) Co + co,
//         B[n][k] = w[c][co][i][j]; column n of input pixel (y, x) is output
//         pixel (2 y + i, 2 x + j), channel co.
// Warps 0-3 gather A for 64-wide K stages with 16-byte cp.async (zero fill
// for padding) straight into the 128-byte-swizzled K-major layout the MMA
// reads; thread 0 also brings the stage's B block (pre-arranged on the host
// in the same layout) with one bulk copy.  Warp 8 issues 4 MMAs
// (128 x NT x 16, bf16 in, f32 accumulate in tensor memory) per stage.
// Stages are handed over with mbarriers (full: 128 cp.async arrivals + the
// bulk copy's bytes; empty: the MMA commit).  CTAs are persistent over the
// tiles and keep two accumulators in tensor memory: while warp 8 fills one,
// the epilogue (warps 4-7, one pixel row per thread) reads the other, adds
// the bias, applies ReLU, rounds to bfloat16 and stores channels-last.
// Every wait is bounded; a wait that runs out counts an error and the CTA
// still frees its tensor memory.
#include <cuda.h>  // CUtensorMap (the encoder is fetched at run time, no -lcuda)
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <vector>

#include "sil.h"
#include "sil_common.h"
#include "sil_unet.h"

namespace sil {
namespace unet {

constexpr int kChip = 256;
constexpr int kBM = 128;           // pixels per tile (MMA M)
constexpr int kBK = 64;            // K per stage: one 128-byte row of bf16
constexpr int kProducers = 128;    // warps 0-3: A and B stages
constexpr int kEpilogue = 128;     // warps 4-7: accumulator -> bf16 output
constexpr int kConvThreads = 288;  // + warp 8: MMA issue
constexpr int kInCh = 8;           // prepared input channels (R, G, B, 5 zeros)
constexpr int kClasses = 3;
constexpr int kMaxCout = 2048;     // widest layer: F = 64 at depth 5

struct ConvArgs {
  const __nv_bfloat16* x;  // input, first channel of pixel 0
  int64_t xs;              // elements between input pixels
  int H, W;                // input height and width
  int cin_log2;            // log2(Ci), Ci a power of two >= 8
  int M;                   // n H W input pixels
  int KT;                  // K stages of 64
  int up;                  // 0: conv, 1: 2x2 stride-2 transposed conv
  int taps;                // 9: 3x3 window (k = tap Ci + c), 1: k = c
  const uint8_t* wblk;     // [N / NT][KT] swizzled NT x 64 bf16 blocks
  const float* bias;       // [cout]
  int cout;                // output channels (per sub-position when up)
  __nv_bfloat16* y;        // output, first channel of pixel 0
  int64_t ys;              // elements between output pixels
  int relu;
  __nv_bfloat16* pool_y;   // optional 2x2 max pool of the output, [n][H/2][W/2][cout]
  const float* head_w;     // optional fused 1x1 head ([3][cout] float32) ...
  const float* head_b;     // ... and its bias; needs NT == cout
  float* logits;           // head scores [n][H][W][3] (nullable)
  uint8_t* labels;         // head argmax [n][H][W] (nullable)
  int tma;                 // A tiles by tensor-map loads: 0 no (per-row gather),
                           // 1 one 64-channel box per stage (Ci multiple of 64),
                           // 2 two 32-channel boxes (two taps) per stage (Ci = 32)
  int fault_it;            // test hook: stage whose A box is never issued (-1: none)
  unsigned int* err;       // count of bounded waits that ran out
  int tw;                  // tile width: 16 (8 rows x 16 pixels of one image) or
                           // 8 (the 8 x 8 pixels of two images; H = W = 8)
};

// A tile is 128 pixels.  Width 16: 8 image rows x 16 pixels of one image,
// tile row r is pixel (y0 + r / 16, x0 + r % 16), and a 2x2 pooling window
// is lanes l, l ^ 1, l ^ 16, l ^ 17 of one epilogue warp.  Width 8 (the
// 8 x 8 maps of the fifth level): the whole 8 x 8 images 2 mt and 2 mt + 1,
// tile row r is pixel (r % 64 / 8, r % 8) of image 2 mt + r / 64.
constexpr int kTileW = 16, kTileH = 8;
__device__ __forceinline__ void tile_origin(int mt, int H, int W, int tw, int& b, int& y0, int& x0) {
  if (tw == 8) {
    b = 2 * mt;
    y0 = x0 = 0;
    return;
  }
  const int tx = W / kTileW, per_img = (H / kTileH) * tx;
  b = mt / per_img;
  const int rem = mt - b * per_img, ty = rem / tx;
  y0 = ty * kTileH;
  x0 = (rem - ty * tx) * kTileW;
}
// Image and pixel of tile row r.
__device__ __forceinline__ void tile_pixel(int r, int tw, int b0, int y0, int x0, int& b, int& y,
                                           int& x) {
  if (tw == 8) {
    b = b0 + (r >> 6);
    y = (r >> 3) & 7;
    x = r & 7;
  } else {
    b = b0;
    y = y0 + (r >> 4);
    x = x0 + (r & 15);
  }
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint32_t a, uint32_t n) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(a), "r"(n) : "memory");
}
// Non-blocking test of the phase of `parity`.
__device__ __forceinline__ bool mbar_test(uint32_t a, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{ .reg .pred p; mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
      : "=r"(ok)
      : "r"(a), "r"(parity)
      : "memory");
  return ok != 0;
}
// One try that may suspend the thread for up to `ns` nanoseconds until the
// phase completes (woken as soon as it does).
__device__ __forceinline__ bool mbar_test_wait(uint32_t a, uint32_t parity, uint32_t ns) {
  uint32_t ok;
  asm volatile(
      "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3; selp.u32 %0, 1, 0, p; }"
      : "=r"(ok)
      : "r"(a), "r"(parity), "r"(ns)
      : "memory");
  return ok != 0;
}
// Waits for the phase of `parity` to complete; gives up (false) after 2^16
// tries of at most 20 us each (about 1.3 s) or soon after another role of
// the CTA has given up.
__device__ __forceinline__ bool mbar_wait(uint32_t a, uint32_t parity, volatile int* failed) {
  if (mbar_test(a, parity)) return true;
  for (int i = 0; i < (1 << 16); ++i) {
    if (mbar_test_wait(a, parity, 20000u)) return true;
    if ((i & 15) == 15 && *failed) return false;
  }
  return false;
}
__device__ __forceinline__ void give_up(volatile int* failed, unsigned int* err) {
  *failed = 1;
  atomicAdd(err, 1u);
}
// 128-byte swizzle, K-major: rows of 128 bytes, 8-row atoms of 1024 bytes,
// stride between atoms (SBO) 1024 bytes, descriptor version 1 (bit 46).
__device__ __forceinline__ uint64_t sw128_desc(uint32_t addr) {
  return uint64_t((addr & 0x3FFFFu) >> 4) | (uint64_t(16 >> 4) << 16) |
         (uint64_t(1024 >> 4) << 32) | (1ull << 46) | (2ull << 61);
}

// 64-byte swizzle, K-major: rows of 64 bytes, 8-row atoms of 512 bytes.
__device__ __forceinline__ uint64_t sw64_desc(uint32_t addr) {
  return uint64_t((addr & 0x3FFFFu) >> 4) | (uint64_t(16 >> 4) << 16) |
         (uint64_t(512 >> 4) << 32) | (1ull << 46) | (4ull << 61);
}

template <int NT>
struct ConvCfg {
  // Narrow tiles (NT <= 32) run three CTAs per SM with three stages each:
  // their per-stage time is set by the single producer and MMA threads'
  // instruction latencies (a stage is only 64 tensor-pipe cycles of work),
  // so more independent CTAs per SM beat a deeper ring; wider tiles run two.
  static constexpr int kMinBlocks = NT <= 32 ? 3 : 2;
  static constexpr int kStages = NT >= 128 ? 3 : (NT <= 32 ? 3 : 4);
  static constexpr int kA = kBM * kBK * 2;
  static constexpr int kB = NT * kBK * 2;
  static constexpr int kStage = kA + kB;
  static constexpr int kSmem = kStages * kStage + 1024;  // + alignment slack
  // two accumulators of NT float32 columns (the epilogue of one tile runs
  // while the next tile accumulates)
  static constexpr int kTmemCols = 2 * NT < 32 ? 32 : 2 * NT;
  // kind::f16 instruction descriptor: D f32, A and B bf16, both K-major,
  // N >> 3 at bit 17, M >> 4 at bit 24.
  static constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) |
                                     (uint32_t(NT >> 3) << 17) | (uint32_t(kBM >> 4) << 24);
};

// Persistent: CTA b handles tiles b, b + gridDim.x, ... (tile t = M tile
// t / ntiles, N tile t % ntiles).  Warps 0-3 produce A/B stages, warps 4-7
// drain the accumulators, warp 8 issues the MMAs.
template <int NT>
__global__ void __launch_bounds__(kConvThreads, ConvCfg<NT>::kMinBlocks)
    k_conv(const ConvArgs a, const __grid_constant__ CUtensorMap tmap, int ntiles, int ntotal) {
  using C = ConvCfg<NT>;
  constexpr int S = C::kStages;
  extern __shared__ uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t full_bar[S], empty_bar[S], acc_full[2], acc_empty[2];
  __shared__ uint32_t tmem_slot;
  __shared__ int failed_s;
  __shared__ float bias_s[kMaxCout];
  __shared__ float head_s[kClasses * 64 + kClasses];
  volatile int* failed = &failed_s;
  uint8_t* smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  for (int i = tid; i < a.cout; i += kConvThreads) bias_s[i] = a.bias[i];
  if (a.head_w)
    for (int i = tid; i < kClasses * (a.cout + 1); i += kConvThreads)
      head_s[i] = i < kClasses * a.cout ? a.head_w[i] : a.head_b[i - kClasses * a.cout];
  if (tid == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(smem_u32(&full_bar[s]), a.tma ? 2 : kProducers + 1);
      mbar_init(smem_u32(&empty_bar[s]), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(smem_u32(&acc_full[b]), 1);
      mbar_init(smem_u32(&acc_empty[b]), kEpilogue);
    }
    failed_s = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_slot)),
                 "r"(C::kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_slot;
  if (warp < 4 && a.tma) {
    // ---- producers, tensor-map path (two threads, each with its own
    // arrival on the stage's full barrier): thread 0 issues per stage one
    // box of 8 x 16 pixels x 64 channels at the tap's offset (zero outside
    // the image, written by the TMA unit in the 128-byte swizzled layout),
    // thread 32 the weight block.  One thread doing both spent about 450
    // of the stage's 800 cycles issuing copies.
    if (tid == 0 || tid == 32) {
      const bool boxes = tid == 0;
      const int cmask = (1 << a.cin_log2) - 1;
      int it = 0;
      bool ok = true;
      for (int t = blockIdx.x; t < ntotal && ok; t += gridDim.x) {
        const int mt = t / ntiles, nt = t - mt * ntiles;
        int b, y0, x0;
        tile_origin(mt, a.H, a.W, a.tw, b, y0, x0);
        for (int kt = 0; kt < a.KT; ++kt, ++it) {
          const int s = it % S;
          if (it >= S && !mbar_wait(smem_u32(&empty_bar[s]), uint32_t((it / S - 1) & 1), failed)) {
            give_up(failed, a.err);
            ok = false;
            break;
          }
          const int k0 = kt * kBK;
          const uint32_t a_s = smem_u32(smem + s * C::kStage), fb = smem_u32(&full_bar[s]);
          asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(fb),
                       "r"(uint32_t(boxes ? C::kA : C::kB))
                       : "memory");
          if (!boxes) {
            asm volatile(
                "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                    a_s + uint32_t(C::kA)),
                "l"(a.wblk + (size_t(nt) * a.KT + kt) * C::kB), "r"(uint32_t(C::kB)), "r"(fb)
                : "memory");
            continue;
          }
          // mode 1: one box, tap k0 / Ci, channels k0 % Ci .. + 63; mode 2:
          // taps 2 kt and 2 kt + 1, all 32 channels each (a tap past the
          // ninth is a box far outside the image: zeros)
          // (the test hook leaves one stage's boxes out: its wait runs out)
          const int nbox = it == a.fault_it ? 0 : (a.tma == 2 ? 2 : 1);
          for (int bx = 0; bx < nbox; ++bx) {
            int tap, c0;
            if (a.tma == 2) {
              tap = 2 * kt + bx;
              c0 = 0;
            } else {
              tap = a.taps == 1 ? 4 : (k0 >> a.cin_log2);
              c0 = a.taps == 1 ? k0 : (k0 & cmask);
            }
            const int yy = tap < 9 ? y0 + tap / 3 - 1 : -4 * kTileH;
            asm volatile(
                "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(
                    a_s + uint32_t(bx * (C::kA / 2))),
                "l"(reinterpret_cast<uint64_t>(&tmap)), "r"(c0), "r"(x0 + tap % 3 - 1), "r"(yy),
                "r"(b), "r"(fb)
                : "memory");
          }
        }
      }
      for (int i = it - S; ok && i < it; ++i)
        if (i >= 0 && !mbar_wait(smem_u32(&empty_bar[i % S]), uint32_t((i / S) & 1), failed)) {
          give_up(failed, a.err);
          ok = false;
        }
    }
  } else if (warp < 4) {
    // ---- producers, gather path: rows 32 warp + 4 i + lane / 8, 16-byte
    // chunk lane % 8
    const int j = lane & 7;
    uint32_t soff[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int r = 32 * warp + 4 * i + (lane >> 3);
      soff[i] = uint32_t((r >> 3) * 1024 + (r & 7) * 128 + ((j ^ (r & 7)) << 4));
    }
    const int cmask = (1 << a.cin_log2) - 1;
    int it = 0;
    bool ok = true;
    for (int t = blockIdx.x; t < ntotal && ok; t += gridDim.x) {
      const int mt = t / ntiles, nt = t - mt * ntiles;
      // per row: element offset of its pixel and which neighbours exist
      // (bit 0 above, 1 below, 2 left, 3 right, 4 the pixel itself)
      int64_t pbase[8];
      uint32_t pfl[8];
      int b0, y0, x0;
      tile_origin(mt, a.H, a.W, a.tw, b0, y0, x0);
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int r = 32 * warp + 4 * i + (lane >> 3);
        int b, y, x;
        tile_pixel(r, a.tw, b0, y0, x0, b, y, x);
        pbase[i] = ((int64_t(b) * a.H + y) * a.W + x) * a.xs;
        pfl[i] = mt * kBM + r < a.M ? (16u | (y > 0 ? 1u : 0u) | (y < a.H - 1 ? 2u : 0u) |
                                       (x > 0 ? 4u : 0u) | (x < a.W - 1 ? 8u : 0u))
                                    : 0u;
      }
      for (int kt = 0; kt < a.KT; ++kt, ++it) {
        const int s = it % S;
        if (it >= S && !mbar_wait(smem_u32(&empty_bar[s]), uint32_t((it / S - 1) & 1), failed)) {
          give_up(failed, a.err);
          ok = false;
          break;
        }
        const uint32_t a_s = smem_u32(smem + s * C::kStage);
        const int k = kt * kBK + 8 * j;
        int tap, c;
        bool tap_ok;
        if (a.taps == 1) {
          tap = 4;
          c = k;
          tap_ok = k <= cmask;
        } else {
          tap = k >> a.cin_log2;
          c = k & cmask;
          tap_ok = tap < 9;
        }
          const int dy = tap / 3 - 1, dx = tap % 3 - 1;
        const uint32_t need = 16u | (dy < 0 ? 1u : 0u) | (dy > 0 ? 2u : 0u) | (dx < 0 ? 4u : 0u) |
                              (dx > 0 ? 8u : 0u);
        const int64_t toff = (int64_t(dy) * a.W + dx) * a.xs + c;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const bool in = tap_ok && (pfl[i] & need) == need;
          const __nv_bfloat16* src = in ? a.x + (pbase[i] + toff) : a.x;
          asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(a_s + soff[i]),
                       "l"(src), "r"(in ? 16 : 0)
                       : "memory");
        }
        asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(
                         smem_u32(&full_bar[s]))
                     : "memory");
        if (tid == 0) {
          const uint32_t fb = smem_u32(&full_bar[s]);
          asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(fb),
                       "r"(uint32_t(C::kB))
                       : "memory");
          asm volatile(
              "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                  a_s + uint32_t(C::kA)),
              "l"(a.wblk + (size_t(nt) * a.KT + kt) * C::kB), "r"(uint32_t(C::kB)), "r"(fb)
              : "memory");
        }
      }
    }
    // tail: the MMA commits of the last stages arrive before the CTA ends
    for (int i = it - S; ok && i < it; ++i)
      if (i >= 0 && !mbar_wait(smem_u32(&empty_bar[i % S]), uint32_t((i / S) & 1), failed)) {
        give_up(failed, a.err);
        ok = false;
      }
    asm volatile("cp.async.wait_all;" ::: "memory");
  } else if (warp < 8) {
    // ---- epilogue: warp w reads accumulator lanes 32 (w % 4) .. + 31
    const int q = warp & 3, r = 32 * q + lane;
    int tl = 0;
    for (int t = blockIdx.x; t < ntotal; t += gridDim.x, ++tl) {
      const int mt = t / ntiles, nt = t - mt * ntiles, buf = tl & 1;
      if (!mbar_wait(smem_u32(&acc_full[buf]), uint32_t((tl >> 1) & 1), failed)) {
        if (lane == 0) give_up(failed, a.err);
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const int p = mt * kBM + r;
      int b0, y0, x0, b, y, x;
      tile_origin(mt, a.H, a.W, a.tw, b0, y0, x0);
      tile_pixel(r, a.tw, b0, y0, x0, b, y, x);
      const bool live = p < a.M;
      float hacc[kClasses];
#pragma unroll
      for (int k = 0; k < kClasses; ++k) hacc[k] = a.head_w ? head_s[kClasses * a.cout + k] : 0.f;
#pragma unroll 1
      for (int c0 = 0; c0 < NT; c0 += 16) {
        uint32_t v[16];
        const uint32_t ta = tmem + (uint32_t(32 * q) << 16) + uint32_t(buf * NT + c0);
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
            : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
              "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]),
              "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
            : "r"(ta));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        const int n = nt * NT + c0;
        int co = n;
        int64_t opix = (int64_t(b) * a.H + y) * a.W + x;
        if (a.up) {
          const int sub = n / a.cout;
          co = n - sub * a.cout;
          opix = (int64_t(b) * 2 * a.H + 2 * y + (sub >> 1)) * (2 * a.W) + 2 * x + (sub & 1);
        }
        uint32_t packed[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          float f0 = __uint_as_float(v[2 * e]) + bias_s[co + 2 * e];
          float f1 = __uint_as_float(v[2 * e + 1]) + bias_s[co + 2 * e + 1];
          if (a.relu) {
            f0 = fmaxf(f0, 0.f);
            f1 = fmaxf(f1, 0.f);
          }
          const __nv_bfloat162 h = __floats2bfloat162_rn(f0, f1);
          packed[e] = *reinterpret_cast<const uint32_t*>(&h);
        }
        if (live && a.y) {
          uint4* dst = reinterpret_cast<uint4*>(a.y + opix * a.ys + co);
          dst[0] = make_uint4(packed[0], packed[1], packed[2], packed[3]);
          dst[1] = make_uint4(packed[4], packed[5], packed[6], packed[7]);
        }
        if (a.head_w) {
          // the head reads the stored (bf16) activation, channels in order
#pragma unroll
          for (int e = 0; e < 8; ++e) {
            const float2 f = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&packed[e]));
#pragma unroll
            for (int k = 0; k < kClasses; ++k) {
              hacc[k] = __fmaf_rn(f.x, head_s[k * a.cout + co + 2 * e], hacc[k]);
              hacc[k] = __fmaf_rn(f.y, head_s[k * a.cout + co + 2 * e + 1], hacc[k]);
            }
          }
        }
        if (a.pool_y) {
          // max over the 2x2 block held by lanes l, l ^ 1, l ^ 16, l ^ 17
          uint32_t m[8];
#pragma unroll
          for (int e = 0; e < 8; ++e) {
            uint32_t t1 = packed[e];
            uint32_t o = __shfl_xor_sync(0xffffffffu, t1, 1);
            __nv_bfloat162 mx = __hmax2(*reinterpret_cast<const __nv_bfloat162*>(&t1),
                                        *reinterpret_cast<const __nv_bfloat162*>(&o));
            t1 = *reinterpret_cast<const uint32_t*>(&mx);
            o = __shfl_xor_sync(0xffffffffu, t1, 16);
            mx = __hmax2(*reinterpret_cast<const __nv_bfloat162*>(&t1),
                         *reinterpret_cast<const __nv_bfloat162*>(&o));
            m[e] = *reinterpret_cast<const uint32_t*>(&mx);
          }
          if (live && (lane & 17) == 0) {
            const int64_t q = (int64_t(b) * (a.H >> 1) + (y >> 1)) * (a.W >> 1) + (x >> 1);
            uint4* dst = reinterpret_cast<uint4*>(a.pool_y + q * a.cout + co);
            dst[0] = make_uint4(m[0], m[1], m[2], m[3]);
            dst[1] = make_uint4(m[4], m[5], m[6], m[7]);
          }
        }
      }
      if (a.head_w && live) {
        const float* sc = hacc;
        int best = 0;
        float top = sc[0];
#pragma unroll
        for (int k = 1; k < kClasses; ++k)
          if (sc[k] > top) {
            top = sc[k];
            best = k;
          }
        const int64_t op = (int64_t(b) * a.H + y) * a.W + x;
        if (a.logits) {
#pragma unroll
          for (int k = 0; k < kClasses; ++k) a.logits[op * kClasses + k] = sc[k];
        }
        if (a.labels) a.labels[op] = uint8_t(best);
      }
      // this accumulator may be overwritten by the tile after next
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&acc_empty[buf])) : "memory");
    }
  } else if (lane == 0) {
    // ---- MMA issue (warp 8, one thread)
    int it = 0, tl = 0;
    bool ok = true;
    for (int t = blockIdx.x; t < ntotal && ok; t += gridDim.x, ++tl) {
      const int buf = tl & 1;
      if (tl >= 2 && !mbar_wait(smem_u32(&acc_empty[buf]), uint32_t(((tl >> 1) - 1) & 1), failed)) {
        give_up(failed, a.err);
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t d = tmem + uint32_t(buf * NT);
      for (int kt = 0; kt < a.KT; ++kt, ++it) {
        const int s = it % S;
        if (!mbar_wait(smem_u32(&full_bar[s]), uint32_t((it / S) & 1), failed)) {
          give_up(failed, a.err);
          ok = false;
          break;
        }
        // the A stage was written through the generic proxy (cp.async)
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t a0 = smem_u32(smem + s * C::kStage), b0 = a0 + uint32_t(C::kA);
#pragma unroll
        for (int kk = 0; kk < kBK / 16; ++kk) {
          // A: 128-byte rows (one box or the per-row gather), or with two
          // 32-channel boxes, box kk / 2 at 32 bytes per K slice
          const uint64_t ad = a.tma == 2 ? sw64_desc(a0 + uint32_t((kk >> 1) * (C::kA / 2) + 32 * (kk & 1)))
                                         : sw128_desc(a0 + 32 * kk);
          const uint64_t bd = sw128_desc(b0 + 32 * kk);
          const uint32_t acc = (kt | kk) ? 1u : 0u;
          asm volatile(
              "{ .reg .pred p; setp.ne.b32 p, %4, 0; tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p; }" ::"r"(
                  d),
              "l"(ad), "l"(bd), "r"(C::kIdesc), "r"(acc)
              : "memory");
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         smem_u32(&empty_bar[s]))
                     : "memory");
      }
      if (ok)
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         smem_u32(&acc_full[buf]))
                     : "memory");
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(C::kTmemCols)
                 : "memory");
}

// R, G, B bytes -> 8 bf16 channels (v / 256, exact; channels 3..7 zero).
__global__ void k_prep(const uint8_t* __restrict__ chips, int64_t P, __nv_bfloat16* __restrict__ x) {
  const int64_t p = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (p >= P) return;
  const uint8_t* s = chips + 3 * p;
  const __nv_bfloat162 rg = __floats2bfloat162_rn(s[0] * (1.f / 256.f), s[1] * (1.f / 256.f));
  const __nv_bfloat162 b0 = __floats2bfloat162_rn(s[2] * (1.f / 256.f), 0.f);
  reinterpret_cast<uint4*>(x)[p] = make_uint4(*reinterpret_cast<const uint32_t*>(&rg),
                                              *reinterpret_cast<const uint32_t*>(&b0), 0u, 0u);
}

// The filtered chip (Sec. III-C): each pixel's R, G, B scaled by V'/V, V the
// largest of them and V' the filter's corrected value, rounded half up
// (c' = floor((2 c V' + V) / (2 V)), 0 when V = 0), then / 256 as k_prep.
__global__ void k_prep_filtered(const uint8_t* __restrict__ chips, const uint8_t* __restrict__ vprime,
                                int64_t P, __nv_bfloat16* __restrict__ x) {
  const int64_t p = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (p >= P) return;
  const uint8_t* s = chips + 3 * p;
  const int v = max(int(s[0]), max(int(s[1]), int(s[2]))), vp = vprime[p];
  float f[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) f[c] = v ? float((2 * int(s[c]) * vp + v) / (2 * v)) * (1.f / 256.f) : 0.f;
  const __nv_bfloat162 rg = __floats2bfloat162_rn(f[0], f[1]);
  const __nv_bfloat162 b0 = __floats2bfloat162_rn(f[2], 0.f);
  reinterpret_cast<uint4*>(x)[p] = make_uint4(*reinterpret_cast<const uint32_t*>(&rg),
                                              *reinterpret_cast<const uint32_t*>(&b0), 0u, 0u);
}

// Chips k0 .. k0 + n - 1 of a scene's 256 x 256 grid (gx chips per row) into
// dense [n][256][256][3] chips and [n][256][256] V' (zero past the scene's
// edges); one thread per chip pixel.
__global__ void k_gather_chips(const uint8_t* __restrict__ img, int64_t H, int64_t W, int64_t pitch,
                               const uint8_t* __restrict__ vp, int64_t vpitch, int64_t k0, int gx,
                               int64_t P, uint8_t* __restrict__ chips, uint8_t* __restrict__ vout) {
  const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t >= P) return;
  const int64_t k = k0 + t / (kChip * kChip);
  const int rem = int(t % (kChip * kChip)), y = rem / kChip, x = rem % kChip;
  const int64_t sy = (k / gx) * kChip + y, sx = (k % gx) * kChip + x;
  const bool in = sy < H && sx < W;
  const uint8_t* s = img + sy * pitch + 3 * sx;
  chips[3 * t] = in ? s[0] : 0;
  chips[3 * t + 1] = in ? s[1] : 0;
  chips[3 * t + 2] = in ? s[2] : 0;
  if (vout) vout[t] = in ? vp[sy * vpitch + sx] : 0;
}

// Chip labels back into the scene's label map (the part inside the scene).
__global__ void k_scatter_labels(const uint8_t* __restrict__ lab, int64_t k0, int gx, int64_t P,
                                 int64_t H, int64_t W, uint8_t* __restrict__ out, int64_t opitch) {
  const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t >= P) return;
  const int64_t k = k0 + t / (kChip * kChip);
  const int rem = int(t % (kChip * kChip)), y = rem / kChip, x = rem % kChip;
  const int64_t sy = (k / gx) * kChip + y, sx = (k % gx) * kChip + x;
  if (sy < H && sx < W) out[sy * opitch + sx] = lab[t];
}

// ---------------------------------------------------------------------------
// Host side.
// ---------------------------------------------------------------------------
struct Tensor {
  __nv_bfloat16* base = nullptr;  // first channel of pixel 0
  int64_t stride = 0;             // elements between pixels
  int H = 0, W = 0, C = 0;
};

struct Layer {
  int kind = 0;  // SIL_UNET_CONV3 / UP / HEAD
  int ci = 0, co = 0, cin_pad = 0, K = 0, KT = 0, N = 0, NT = 0;
  uint8_t* wblk = nullptr;
  float* bias = nullptr;
  Tensor in, out;
  bool relu = false;
  int taps = 9;
  __nv_bfloat16* pool = nullptr;  // fused 2x2 max pool output (encoder second convs)
  bool head = false;              // fused 1x1 head (last decoder conv)
  int tma = 0;                    // A tiles through a tensor map (see ConvArgs::tma)
  int tw = kTileW;                // tile width (see ConvArgs::tw)
  CUtensorMap tmap{};             // 4-D map of the input: {Ci, W, H, max_batch}
};

}  // namespace unet
}  // namespace sil

struct sil_unet {
  int device = 0;
  sil_unet_config cfg{};
  std::vector<sil::unet::Layer> layers;
  std::vector<void*> allocs;
  __nv_bfloat16* x0 = nullptr;
  float* head_w = nullptr;
  float* head_b = nullptr;
  unsigned int* err = nullptr;
  int last_n = 0;
  int fault_layer = -1;  // test hook (sil_unet_set_fault)
  // staging of sil_unet_label_scene: max_batch chips, their V' and labels
  uint8_t* stage_chips = nullptr;
  uint8_t* stage_vp = nullptr;
  uint8_t* stage_lab = nullptr;
};

namespace {

using sil::set_error;
using namespace sil::unet;

bool config_ok(const sil_unet_config* c) {
  return c && (c->base_width == 16 || c->base_width == 32 || c->base_width == 64) &&
         c->depth >= 1 && c->depth <= 5 && c->max_batch >= 1 && c->max_batch <= 4096;
}

int ilog2(int v) {
  int l = 0;
  while ((1 << l) < v) ++l;
  return l;
}

uint16_t f2bf(float f) {
  uint32_t u;
  std::memcpy(&u, &f, 4);
  u += 0x7FFFu + ((u >> 16) & 1u);  // round to nearest, ties to even
  return uint16_t(u >> 16);
}

// byte offset of element (row rr, k) in an NT x 64 block, 128-byte swizzle
size_t sw128_off(int rr, int k) {
  return size_t(rr >> 3) * 1024 + size_t(rr & 7) * 128 + size_t(((k >> 3) ^ (rr & 7)) << 4) +
         size_t(k & 7) * 2;
}

using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                   const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                   const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                   CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// The driver's tensor-map encoder, looked up once through the runtime.
EncodeTiledFn tensor_map_encoder() {
  static EncodeTiledFn fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  }
  return fn;
}

// Tensor map of a layer's input {Ci, W, H, batch} (channels-last, pixel
// stride xs elements), box 64 channels x 16 x 8 pixels with 128-byte swizzle
// (mode 1) or 32 channels with 64-byte swizzle (mode 2); zero fill outside.
bool encode_input_map(Layer& L, int batch) {
  const EncodeTiledFn enc = tensor_map_encoder();
  if (!enc) return false;
  const cuuint64_t dims[4] = {cuuint64_t(L.cin_pad), cuuint64_t(L.in.W), cuuint64_t(L.in.H),
                              cuuint64_t(batch)};
  const cuuint64_t es = 2;
  const cuuint64_t strides[3] = {cuuint64_t(L.in.stride) * es, cuuint64_t(L.in.W) * L.in.stride * es,
                                 cuuint64_t(L.in.H) * L.in.W * L.in.stride * es};
  // a tile of width 16: 16 x 8 pixels of one image; of width 8: two 8 x 8 images
  const cuuint32_t box[4] = {cuuint32_t(L.tma == 2 ? kBK / 2 : kBK), cuuint32_t(L.tw),
                             cuuint32_t(kTileH), cuuint32_t(L.tw == 8 ? 2 : 1)};
  const cuuint32_t estr[4] = {1, 1, 1, 1};
  return enc(&L.tmap, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, L.in.base, dims, strides, box, estr,
             CU_TENSOR_MAP_INTERLEAVE_NONE,
             L.tma == 2 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_128B,
             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int NT>
cudaError_t launch_conv_nt(const ConvArgs& a, const CUtensorMap& tmap, int mtiles, int ntiles,
                           cudaStream_t s) {
  static int ctas_per_sm = 0;  // per process; set before the first launch
  static int sms = 0;
  if (!ctas_per_sm) {
    cudaError_t e = cudaFuncSetAttribute(k_conv<NT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         ConvCfg<NT>::kSmem);
    int dev = 0, smem_sm = 0, regs_sm = 0, reserved = 0;
    cudaFuncAttributes fa{};
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, k_conv<NT>);
    if (e != cudaSuccess) return e;
    // The occupancy calculator reports one CTA per SM for any kernel that
    // allocates tensor memory, so the resident count is derived from the
    // kernel's own shared memory, registers and tensor-memory columns (an
    // SM has 512); extra CTAs of a persistent grid only start later.
    const int by_smem = smem_sm / (ConvCfg<NT>::kSmem + int(fa.sharedSizeBytes) + reserved);
    const int warp_regs = ((fa.numRegs * 32 + 255) / 256) * 256;
    const int by_regs = regs_sm / (warp_regs * (kConvThreads / 32));
    const int by_tmem = 512 / ConvCfg<NT>::kTmemCols;
    int c = by_smem < by_regs ? by_smem : by_regs;
    c = c < by_tmem ? c : by_tmem;
    ctas_per_sm = c > 0 ? c : 1;
  }
  const int ntotal = mtiles * ntiles;
  const int cap = sms * ctas_per_sm;
  const int grid = ntotal < cap ? ntotal : cap;
  k_conv<NT><<<grid, kConvThreads, ConvCfg<NT>::kSmem, s>>>(a, tmap, ntiles, ntotal);
  return cudaGetLastError();
}

cudaError_t run_layer(const Layer& L, int n, unsigned int* err, const float* head_w,
                      const float* head_b, float* logits, uint8_t* labels, bool fault,
                      cudaStream_t s) {
  ConvArgs a;
  a.x = L.in.base;
  a.xs = L.in.stride;
  a.H = L.in.H;
  a.W = L.in.W;
  a.cin_log2 = ilog2(L.cin_pad);
  a.M = n * L.in.H * L.in.W;
  a.KT = L.KT;
  a.up = L.kind == SIL_UNET_UP;
  a.wblk = L.wblk;
  a.bias = L.bias;
  a.cout = L.co;
  a.y = L.out.base;
  a.ys = L.out.stride;
  a.relu = L.relu;
  a.taps = L.taps;
  a.pool_y = L.pool;
  a.head_w = L.head ? head_w : nullptr;
  a.head_b = L.head ? head_b : nullptr;
  a.logits = L.head ? logits : nullptr;
  a.labels = L.head ? labels : nullptr;
  a.tma = L.tma;
  a.fault_it = (fault && L.tma) ? 0 : -1;
  a.err = err;
  a.tw = L.tw;
  const int mtiles = (a.M + kBM - 1) / kBM, ntiles = L.N / L.NT;
  switch (L.NT) {
    case 16: return launch_conv_nt<16>(a, L.tmap, mtiles, ntiles, s);
    case 32: return launch_conv_nt<32>(a, L.tmap, mtiles, ntiles, s);
    case 64: return launch_conv_nt<64>(a, L.tmap, mtiles, ntiles, s);
    default: return launch_conv_nt<128>(a, L.tmap, mtiles, ntiles, s);
  }
}

// Weight shape (PyTorch layout) and kind of layer i; false if out of range.
bool layer_shape(const sil_unet_config& c, int i, int64_t dims[4], int* kind) {
  const int D = c.depth, F = c.base_width;
  auto w = [&](int l) { return int64_t(F) << l; };
  auto set = [&](int64_t a, int64_t b, int64_t k, int kd) {
    dims[0] = a;
    dims[1] = b;
    dims[2] = k;
    dims[3] = k;
    *kind = kd;
    return true;
  };
  if (i < 0) return false;
  if (i < 2 * D) {
    const int l = i / 2;
    if (i % 2 == 0) return set(w(l), l == 0 ? 3 : w(l - 1), 3, SIL_UNET_CONV3);
    return set(w(l), w(l), 3, SIL_UNET_CONV3);
  }
  i -= 2 * D;
  if (i == 0) return set(w(D), w(D - 1), 3, SIL_UNET_CONV3);
  if (i == 1) return set(w(D), w(D), 3, SIL_UNET_CONV3);
  i -= 2;
  if (i < 3 * D) {
    const int l = D - 1 - i / 3;
    if (i % 3 == 0) return set(w(l + 1), w(l), 2, SIL_UNET_UP);
    if (i % 3 == 1) return set(w(l), 2 * w(l), 3, SIL_UNET_CONV3);
    return set(w(l), w(l), 3, SIL_UNET_CONV3);
  }
  i -= 3 * D;
  if (i == 0) return set(kClasses, F, 1, SIL_UNET_HEAD);
  return false;
}

}  // namespace

extern "C" sil_status sil_unet_config_default(sil_unet_config* cfg) {
  if (!cfg) {
    set_error("sil_unet_config_default: NULL");
    return SIL_EINVAL;
  }
  cfg->base_width = 32;
  cfg->depth = 5;
  cfg->max_batch = 32;
  return SIL_OK;
}

extern "C" int32_t sil_unet_num_layers(int32_t depth) {
  return (depth >= 1 && depth <= 5) ? 5 * depth + 3 : -1;
}

extern "C" sil_status sil_unet_layer_shape(const sil_unet_config* cfg, int32_t i, int64_t dims[4],
                                           int32_t* kind) {
  if (!config_ok(cfg) || !dims || !kind) {
    set_error("sil_unet_layer_shape: bad config or NULL output");
    return SIL_EINVAL;
  }
  int k = 0;
  if (!layer_shape(*cfg, i, dims, &k)) {
    set_error("sil_unet_layer_shape: layer %d out of range", int(i));
    return SIL_EINVAL;
  }
  *kind = k;
  return SIL_OK;
}

extern "C" int64_t sil_unet_flops_per_chip(const sil_unet_config* cfg) {
  if (!config_ok(cfg)) return -1;
  int64_t total = 0;
  const int nl = sil_unet_num_layers(cfg->depth);
  for (int i = 0; i < nl; ++i) {
    int64_t d[4];
    int kind = 0;
    layer_shape(*cfg, i, d, &kind);
    // output resolution of the layer
    int level;
    if (i < 2 * cfg->depth) {
      level = i / 2;
    } else if (i < 2 * cfg->depth + 2) {
      level = cfg->depth;
    } else if (i < nl - 1) {
      level = cfg->depth - 1 - (i - 2 * cfg->depth - 2) / 3;
    } else {
      level = 0;
    }
    const int64_t px = int64_t(kChip >> level) * (kChip >> level);
    if (kind == SIL_UNET_CONV3) total += 2 * px * d[0] * d[1] * 9;
    if (kind == SIL_UNET_UP) total += 2 * px * d[0] * d[1];  // every output px: Ci terms
    if (kind == SIL_UNET_HEAD) total += 2 * px * d[0] * d[1];
  }
  return total;
}

extern "C" void sil_unet_destroy(sil_unet* net) {
  if (!net) return;
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(net->device);
  for (void* p : net->allocs) cudaFree(p);
  cudaSetDevice(prev);
  delete net;
}

extern "C" sil_status sil_unet_create(sil_unet** out, const sil_unet_config* cfg,
                                      const float* const* weights, const float* const* biases,
                                      int32_t device) {
  if (!out || !config_ok(cfg) || !weights || !biases) {
    set_error("sil_unet_create: NULL argument or config outside F in {16,32,64}, depth 1..5, "
              "max_batch 1..4096");
    return SIL_EINVAL;
  }
  *out = nullptr;
  const int nl = sil_unet_num_layers(cfg->depth);
  for (int i = 0; i < nl; ++i)
    if (!weights[i] || !biases[i]) {
      set_error("sil_unet_create: NULL weight or bias of layer %d", i);
      return SIL_EINVAL;
    }
  int prev = 0;
  cudaGetDevice(&prev);
  if (cudaSetDevice(device) != cudaSuccess) {
    set_error("sil_unet_create: cudaSetDevice(%d) failed", int(device));
    return SIL_ECUDA;
  }
  sil_unet* net = new (std::nothrow) sil_unet;
  if (!net) {
    cudaSetDevice(prev);
    return SIL_ENOMEM;
  }
  net->device = device;
  net->cfg = *cfg;
  const int D = cfg->depth, F = cfg->base_width, B = cfg->max_batch;
  sil_status st = SIL_OK;
  auto dalloc = [&](size_t bytes) -> void* {
    void* p = nullptr;
    if (st != SIL_OK) return nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
      set_error("sil_unet_create: cudaMalloc(%zu) failed", bytes);
      st = SIL_ENOMEM;
      return nullptr;
    }
    net->allocs.push_back(p);
    return p;
  };
  auto act = [&](int H, int C) {
    Tensor t;
    t.base = static_cast<__nv_bfloat16*>(dalloc(size_t(B) * H * H * C * 2));
    t.stride = C;
    t.H = t.W = H;
    t.C = C;
    return t;
  };
  auto width = [&](int l) { return F << l; };
  // activations
  net->x0 = static_cast<__nv_bfloat16*>(dalloc(size_t(B) * kChip * kChip * kInCh * 2));
  std::vector<Tensor> t(D), cat(D), pool(D), d0(D), d1(D);
  for (int l = 0; l < D; ++l) {
    const int H = kChip >> l;
    t[l] = act(H, width(l));
    cat[l] = act(H, 2 * width(l));
    pool[l] = act(H / 2, width(l));
    d0[l] = act(H, width(l));
    d1[l] = act(H, width(l));
  }
  const Tensor b0 = act(kChip >> D, width(D)), b1 = act(kChip >> D, width(D));
  net->err = static_cast<unsigned int*>(dalloc(sizeof(unsigned int)));
  net->stage_chips = static_cast<uint8_t*>(dalloc(size_t(B) * kChip * kChip * 3));
  net->stage_vp = static_cast<uint8_t*>(dalloc(size_t(B) * kChip * kChip));
  net->stage_lab = static_cast<uint8_t*>(dalloc(size_t(B) * kChip * kChip));
  if (st == SIL_OK && cudaMemset(net->err, 0, sizeof(unsigned int)) != cudaSuccess) st = SIL_ECUDA;
  auto skip_of = [&](int l) {  // encoder output of level l: second half of cat[l]
    Tensor s = cat[l];
    s.base += width(l);
    s.C = width(l);
    return s;
  };
  auto up_of = [&](int l) {  // upsampled half of cat[l]
    Tensor s = cat[l];
    s.C = width(l);
    return s;
  };
  Tensor x0t;
  x0t.base = net->x0;
  x0t.stride = kInCh;
  x0t.H = x0t.W = kChip;
  x0t.C = kInCh;
  // layers
  for (int i = 0; i < nl && st == SIL_OK; ++i) {
    int64_t d[4];
    int kind = 0;
    layer_shape(*cfg, i, d, &kind);
    Layer L;
    L.kind = kind;
    if (kind == SIL_UNET_HEAD) {
      net->head_w = static_cast<float*>(dalloc(sizeof(float) * kClasses * F));
      net->head_b = static_cast<float*>(dalloc(sizeof(float) * kClasses));
      if (st == SIL_OK &&
          (cudaMemcpy(net->head_w, weights[i], sizeof(float) * kClasses * F, cudaMemcpyHostToDevice) !=
               cudaSuccess ||
           cudaMemcpy(net->head_b, biases[i], sizeof(float) * kClasses, cudaMemcpyHostToDevice) !=
               cudaSuccess))
        st = SIL_ECUDA;
      L.in = d1[0];
      net->layers.push_back(L);
      continue;
    }
    const bool up = kind == SIL_UNET_UP;
    L.ci = int(up ? d[0] : d[1]);
    L.co = int(up ? d[1] : d[0]);
    L.cin_pad = L.ci < kInCh ? kInCh : L.ci;
    L.taps = up ? 1 : 9;
    L.K = L.taps == 1 ? L.cin_pad : 9 * L.cin_pad;
    L.KT = (L.K + kBK - 1) / kBK;
    L.N = up ? 4 * L.co : L.co;
    L.tma = (L.cin_pad % kBK == 0) ? 1 : (L.cin_pad == kBK / 2 && !up) ? 2 : 0;
    L.NT = L.N < 128 ? L.N : 128;
    L.relu = !up;
    // inputs and outputs
    if (i < 2 * D) {
      const int l = i / 2;
      if (i % 2 == 0) {
        L.in = l == 0 ? x0t : pool[l - 1];
        L.out = t[l];
      } else {
        L.in = t[l];
        L.out = skip_of(l);
        L.pool = pool[l].base;
      }
    } else if (i == 2 * D) {
      L.in = pool[D - 1];
      L.out = b0;
    } else if (i == 2 * D + 1) {
      L.in = b0;
      L.out = b1;
    } else {
      const int q = i - 2 * D - 2, l = D - 1 - q / 3;
      if (q % 3 == 0) {
        L.in = l == D - 1 ? b1 : d1[l + 1];
        L.out = up_of(l);
      } else if (q % 3 == 1) {
        L.in = cat[l];
        L.out = d0[l];
      } else {
        L.in = d0[l];
        L.out = d1[l];
        L.head = l == 0;
      }
    }
    // the fifth level's 8 x 8 maps are tiled two images at a time
    L.tw = L.in.W >= kTileW ? kTileW : 8;
    if (L.tw == 8 && (L.in.W != 8 || L.in.H != 8 || L.pool || L.head)) st = SIL_EINVAL;
    // inputs whose channel count is a multiple of 64 are read by tensor map
    if (L.tma && !encode_input_map(L, B)) L.tma = 0;
    // weights -> swizzled bf16 blocks [N / NT][KT][NT x 64]
    const size_t blk = size_t(L.NT) * kBK * 2;
    std::vector<uint8_t> h(size_t(L.N / L.NT) * L.KT * blk, 0);
    const float* w = weights[i];
    for (int n = 0; n < L.N; ++n) {
      for (int k = 0; k < L.KT * kBK; ++k) {
        float v = 0.f;
        if (up) {
          const int sub = n / L.co, co = n % L.co, c = k;
          if (c < L.ci) v = w[((size_t(c) * L.co + co) * 2 + (sub >> 1)) * 2 + (sub & 1)];
        } else {
          const int tap = k / L.cin_pad, c = k % L.cin_pad;
          if (tap < 9 && c < L.ci) v = w[((size_t(n) * L.ci + c) * 3 + tap / 3) * 3 + tap % 3];
        }
        const uint16_t bv = f2bf(v);
        const size_t off = (size_t(n / L.NT) * L.KT + k / kBK) * blk + sw128_off(n % L.NT, k % kBK);
        std::memcpy(&h[off], &bv, 2);
      }
    }
    L.wblk = static_cast<uint8_t*>(dalloc(h.size()));
    L.bias = static_cast<float*>(dalloc(sizeof(float) * L.co));
    if (st == SIL_OK &&
        (cudaMemcpy(L.wblk, h.data(), h.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
         cudaMemcpy(L.bias, biases[i], sizeof(float) * L.co, cudaMemcpyHostToDevice) != cudaSuccess))
      st = SIL_ECUDA;
    net->layers.push_back(L);
  }
  cudaSetDevice(prev);
  if (st != SIL_OK) {
    if (st == SIL_ECUDA) set_error("sil_unet_create: weight upload failed");
    sil_unet_destroy(net);
    return st;
  }
  *out = net;
  return SIL_OK;
}

extern "C" sil_status sil_unet_forward(sil_unet* net, const uint8_t* chips, int32_t n,
                                       uint8_t* labels, float* logits, sil_stream stream) {
  return sil_unet_forward_filtered(net, chips, nullptr, n, labels, logits, stream);
}

extern "C" sil_status sil_unet_forward_filtered(sil_unet* net, const uint8_t* chips,
                                                const uint8_t* vprime, int32_t n, uint8_t* labels,
                                                float* logits, sil_stream stream) {
  if (!net || !chips || n < 1 || n > net->cfg.max_batch) {
    set_error("sil_unet_forward: NULL network/chips or n=%d outside 1..max_batch", int(n));
    return SIL_EINVAL;
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const int64_t P = int64_t(n) * kChip * kChip;
  if (vprime)
    k_prep_filtered<<<unsigned((P + 255) / 256), 256, 0, s>>>(chips, vprime, P, net->x0);
  else
    k_prep<<<unsigned((P + 255) / 256), 256, 0, s>>>(chips, P, net->x0);
  cudaError_t e = cudaGetLastError();
  const int nl = int(net->layers.size());
  // the head is fused into the last decoder convolution, the pooling into
  // the encoders' second convolutions
  for (int i = 0; i < nl - 1 && e == cudaSuccess; ++i)
    e = run_layer(net->layers[i], n, net->err, net->head_w, net->head_b, logits, labels,
                  i == net->fault_layer, s);
  if (e != cudaSuccess) {
    set_error("sil_unet_forward: launch failed: %s", cudaGetErrorString(e));
    return SIL_ECUDA;
  }
  net->last_n = n;
  return SIL_OK;
}

extern "C" sil_status sil_unet_set_fault(sil_unet* net, int32_t layer) {
  if (!net || layer < -1 || layer >= int(net->layers.size()) - 1 ||
      (layer >= 0 && !net->layers[layer].tma)) {
    set_error("sil_unet_set_fault: NULL network or layer %d without tensor-map loads", int(layer));
    return SIL_EINVAL;
  }
  net->fault_layer = layer;
  return SIL_OK;
}

extern "C" sil_status sil_unet_label_scene(sil_unet* net, const uint8_t* img, int64_t H,
                                           int64_t W, int64_t pitch, const uint8_t* vprime,
                                           int64_t vprime_pitch, uint8_t* labels,
                                           int64_t label_pitch, sil_stream stream) {
  if (!net || !img || !labels || H < 1 || W < 1 || pitch < 3 * W || label_pitch < W ||
      (vprime && vprime_pitch < W)) {
    set_error("sil_unet_label_scene: NULL pointer or bad geometry");
    return SIL_EINVAL;
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const int gx = int((W + kChip - 1) / kChip), gy = int((H + kChip - 1) / kChip);
  const int64_t nchips = int64_t(gx) * gy;
  for (int64_t k0 = 0; k0 < nchips; k0 += net->cfg.max_batch) {
    const int n = int(nchips - k0 < net->cfg.max_batch ? nchips - k0 : net->cfg.max_batch);
    const int64_t P = int64_t(n) * kChip * kChip;
    const unsigned blocks = unsigned((P + 255) / 256);
    k_gather_chips<<<blocks, 256, 0, s>>>(img, H, W, pitch, vprime, vprime_pitch, k0, gx, P,
                                          net->stage_chips, vprime ? net->stage_vp : nullptr);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
      set_error("sil_unet_label_scene: gather: %s", cudaGetErrorString(e));
      return SIL_ECUDA;
    }
    const sil_status st = sil_unet_forward_filtered(net, net->stage_chips, vprime ? net->stage_vp : nullptr,
                                                    n, net->stage_lab, nullptr, stream);
    if (st != SIL_OK) return st;
    k_scatter_labels<<<blocks, 256, 0, s>>>(net->stage_lab, k0, gx, P, H, W, labels, label_pitch);
    e = cudaGetLastError();
    if (e != cudaSuccess) {
      set_error("sil_unet_label_scene: scatter: %s", cudaGetErrorString(e));
      return SIL_ECUDA;
    }
  }
  return SIL_OK;
}

extern "C" sil_status sil_unet_error_count(sil_unet* net, uint32_t* count) {
  if (!net || !count) {
    set_error("sil_unet_error_count: NULL");
    return SIL_EINVAL;
  }
  unsigned int v = 0;
  const cudaError_t e = cudaMemcpy(&v, net->err, sizeof(v), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) {
    set_error("sil_unet_error_count: %s", cudaGetErrorString(e));
    return SIL_ECUDA;
  }
  *count = v;
  return SIL_OK;
}

namespace {
bool tensor_of(const sil_unet* net, int i, Tensor* t) {
  if (i == -1) {
    t->base = net->x0;
    t->stride = kInCh;
    t->H = t->W = kChip;
    t->C = kInCh;
    return true;
  }
  if (i < 0 || i >= int(net->layers.size()) || net->layers[i].kind == SIL_UNET_HEAD) return false;
  *t = net->layers[i].out;
  return true;
}
}  // namespace

extern "C" sil_status sil_unet_tensor_shape(const sil_unet* net, int32_t i, int64_t dims[4]) {
  Tensor t;
  if (!net || !dims || !tensor_of(net, i, &t)) {
    set_error("sil_unet_tensor_shape: NULL or layer %d has no activation", int(i));
    return SIL_EINVAL;
  }
  dims[0] = net->last_n;
  dims[1] = t.H;
  dims[2] = t.W;
  dims[3] = t.C;
  return SIL_OK;
}

extern "C" sil_status sil_unet_copy_tensor(const sil_unet* net, int32_t i, void* dst,
                                           sil_stream stream) {
  Tensor t;
  if (!net || !dst || !tensor_of(net, i, &t) || net->last_n < 1) {
    set_error("sil_unet_copy_tensor: NULL, no forward yet, or layer %d has no activation", int(i));
    return SIL_EINVAL;
  }
  const size_t rows = size_t(net->last_n) * t.H * t.W;
  const cudaError_t e = cudaMemcpy2DAsync(dst, size_t(t.C) * 2, t.base, size_t(t.stride) * 2,
                                          size_t(t.C) * 2, rows, cudaMemcpyDeviceToDevice,
                                          reinterpret_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) {
    set_error("sil_unet_copy_tensor: %s", cudaGetErrorString(e));
    return SIL_ECUDA;
  }
  return SIL_OK;
}
