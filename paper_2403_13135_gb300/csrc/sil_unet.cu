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
#include <cublas_v2.h>

#include <algorithm>
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
  const __nv_bfloat16* mask;  // optional: output element kept only where this
                              // tensor (same pixel and channel, stride ms) is > 0
                              // (a ReLU's backward pass)
  int64_t ms;
};

// A tile is 128 pixels.  Width 16: 8 image rows x 16 pixels of one image,
// tile row r is pixel (y0 + r / 16, x0 + r % 16), and a 2x2 pooling window
// is lanes l, l ^ 1, l ^ 16, l ^ 17 of one epilogue warp.  Width 8 (the
// 8 x 8 maps of the fifth level): the whole 8 x 8 images 2 mt and 2 mt + 1,
// tile row r is pixel (r % 64 / 8, r % 8) of image 2 mt + r / 64.
constexpr int kTileW = 16, kTileH = 8;
// pixel tiles per work unit of the tensor-map layers (1 or 2, see ConvCfg)
constexpr int kUnitTiles = 2;
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
// Work units of MT tiles that share a stage's weight block: for width 16,
// MT vertically stacked 8 x 16 tiles of one image (tile j at rows y0 + 8 j);
// for width 8, the 2 MT images 2 MT u .. (tile j: images b + 2 j, + 1).
// MT = 1 is tile_origin.
template <int MT>
__device__ __forceinline__ void unit_origin(int u, int H, int W, int tw, int& b, int& y0, int& x0) {
  if (MT == 1) {
    tile_origin(u, H, W, tw, b, y0, x0);
    return;
  }
  if (tw == 8) {
    b = 2 * MT * u;
    y0 = x0 = 0;
    return;
  }
  const int tx = W / kTileW, per_img = (H / (kTileH * MT)) * tx;
  b = u / per_img;
  const int rem = u - b * per_img, ty = rem / tx;
  y0 = ty * kTileH * MT;
  x0 = (rem - ty * tx) * kTileW;
}
// Origin of tile j of a unit.
__device__ __forceinline__ void sub_origin(int j, int tw, int& b, int& y0) {
  if (tw == 8) b += 2 * j;
  else y0 += kTileH * j;
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

template <int NT, int MT = 1>
struct ConvCfg {
  // MT = 1: narrow tiles (NT <= 32) run three CTAs per SM with three stages
  // each: their per-stage time is set by the single producer and MMA
  // threads' instruction latencies (a stage is only 64 tensor-pipe cycles of
  // work), so more independent CTAs per SM beat a deeper ring; wider tiles
  // run two.  MT = 2: a stage holds two pixel tiles (one 16-row box per tap)
  // that share the weight block, halving the box issues and the weight
  // traffic per pixel; two CTAs per SM.
  static constexpr int kMinBlocks = MT == 2 ? 2 : (NT <= 32 ? 3 : 2);
  static constexpr int kStages = MT == 2 ? (NT <= 32 ? 3 : 2) : (NT >= 128 ? 3 : (NT <= 32 ? 3 : 4));
  static constexpr int kA = MT * kBM * kBK * 2;
  static constexpr int kB = NT * kBK * 2;
  static constexpr int kStage = kA + kB;
  static constexpr int kSmem = kStages * kStage + 1024;  // + alignment slack
  static constexpr int kSmemMax = kSmem + kMaxCout * 4;  // + the biases
  // accumulators of MT x NT float32 columns: two (the epilogue of one unit
  // runs while the next accumulates) when they fit in half the tensor
  // memory, else one (the SM's other CTA overlaps instead)
  static constexpr int kAccBufs = 2 * MT * NT <= 256 ? 2 : 1;
  static constexpr int kTmemCols = kAccBufs * MT * NT < 32 ? 32 : kAccBufs * MT * NT;
  // kind::f16 instruction descriptor: D f32, A and B bf16, both K-major,
  // N >> 3 at bit 17, M >> 4 at bit 24.
  static constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) |
                                     (uint32_t(NT >> 3) << 17) | (uint32_t(kBM >> 4) << 24);
};

// Persistent: CTA b handles work items b, b + gridDim.x, ... (item t = M
// unit t / ntiles of MT pixel tiles, N tile t % ntiles).  Warps 0-3 produce
// A/B stages, warps 4-7 drain the accumulators, warp 8 issues the MMAs.
template <int NT, int MT>
__global__ void __launch_bounds__(kConvThreads, (ConvCfg<NT, MT>::kMinBlocks))
    k_conv(const ConvArgs a, const __grid_constant__ CUtensorMap tmap, int ntiles, int ntotal) {
  using C = ConvCfg<NT, MT>;
  constexpr int NB = C::kAccBufs;
  constexpr int S = C::kStages;
  extern __shared__ uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t full_bar[S], empty_bar[S], acc_full[NB], acc_empty[NB];
  __shared__ uint32_t tmem_slot;
  __shared__ int failed_s;
  __shared__ float head_s[kClasses * 64 + kClasses];
  volatile int* failed = &failed_s;
  uint8_t* smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // the layer's biases after the ring (the launch adds cout floats to the
  // dynamic shared memory)
  float* bias_s = reinterpret_cast<float*>(smem + S * C::kStage);
  for (int i = tid; i < a.cout; i += kConvThreads) bias_s[i] = a.bias[i];

  if (a.head_w)
    for (int i = tid; i < kClasses * (a.cout + 1); i += kConvThreads)
      head_s[i] = i < kClasses * a.cout ? a.head_w[i] : a.head_b[i - kClasses * a.cout];
  if (tid == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(smem_u32(&full_bar[s]), a.tma ? 2 : kProducers + 1);
      mbar_init(smem_u32(&empty_bar[s]), 1);
    }
    for (int b = 0; b < NB; ++b) {
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
        unit_origin<MT>(mt, a.H, a.W, a.tw, b, y0, x0);
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
          // ninth is a box far outside the image: zeros); a box covers the
          // unit's MT tiles (8 MT rows, or 2 MT images of 8 x 8)
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
            const int yy = tap < 9 ? y0 + tap / 3 - 1 : -4 * kTileH * MT;
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
    // ---- producers, gather path (one tile per unit; the host gives units
    // of two tiles only to tensor-map layers): rows 32 warp + 4 i + lane /
    // 8, 16-byte chunk lane % 8
    if constexpr (MT == 1) {
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
    }
  } else if (warp < 8) {
    // ---- epilogue: warp w reads accumulator lanes 32 (w % 4) .. + 31
    const int q = warp & 3, r = 32 * q + lane;
    int tl = 0;
    const int nimg = a.M / (a.H * a.W);
    for (int t = blockIdx.x; t < ntotal; t += gridDim.x, ++tl) {
      const int mt = t / ntiles, nt = t - mt * ntiles, buf = tl % NB;
      if (!mbar_wait(smem_u32(&acc_full[buf]), uint32_t((tl / NB) & 1), failed)) {
        if (lane == 0) give_up(failed, a.err);
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      int ub, uy0, ux0;
      unit_origin<MT>(mt, a.H, a.W, a.tw, ub, uy0, ux0);
#pragma unroll 1
      for (int j = 0; j < MT; ++j) {
      int b0 = ub, y0 = uy0, x0 = ux0, b, y, x;
      sub_origin(j, a.tw, b0, y0);
      tile_pixel(r, a.tw, b0, y0, x0, b, y, x);
      const bool live = b < nimg;
      float hacc[kClasses];
#pragma unroll
      for (int k = 0; k < kClasses; ++k) hacc[k] = a.head_w ? head_s[kClasses * a.cout + k] : 0.f;
#pragma unroll 1
      for (int c0 = 0; c0 < NT; c0 += 16) {
        uint32_t v[16];
        const uint32_t ta = tmem + (uint32_t(32 * q) << 16) + uint32_t((buf * MT + j) * NT + c0);
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
        uint32_t mk[8];
        if (a.mask && live) {
          const uint4* mp = reinterpret_cast<const uint4*>(a.mask + opix * a.ms + co);
          const uint4 m0 = mp[0], m1 = mp[1];
          mk[0] = m0.x; mk[1] = m0.y; mk[2] = m0.z; mk[3] = m0.w;
          mk[4] = m1.x; mk[5] = m1.y; mk[6] = m1.z; mk[7] = m1.w;
        }
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          float f0 = __uint_as_float(v[2 * e]) + bias_s[co + 2 * e];
          float f1 = __uint_as_float(v[2 * e + 1]) + bias_s[co + 2 * e + 1];
          if (a.relu) {
            f0 = fmaxf(f0, 0.f);
            f1 = fmaxf(f1, 0.f);
          }
          if (a.mask) {
            // bf16 x > 0 <=> its sign bit is clear and it is not zero
            const uint32_t m = live ? mk[e] : 0u;
            if ((m & 0x8000u) || (m & 0x7FFFu) == 0) f0 = 0.f;
            if ((m & 0x80000000u) || (m & 0x7FFF0000u) == 0) f1 = 0.f;
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
      }  // tile j of the unit
      // this accumulator may be overwritten by the unit after next
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&acc_empty[buf])) : "memory");
    }
  } else if (lane == 0) {
    // ---- MMA issue (warp 8, one thread)
    int it = 0, tl = 0;
    bool ok = true;
    for (int t = blockIdx.x; t < ntotal && ok; t += gridDim.x, ++tl) {
      const int buf = tl % NB;
      if (tl >= NB && !mbar_wait(smem_u32(&acc_empty[buf]), uint32_t(((tl / NB) - 1) & 1), failed)) {
        give_up(failed, a.err);
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t d = tmem + uint32_t(buf * MT * NT);
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
          const uint64_t bd = sw128_desc(b0 + 32 * kk);
          const uint32_t acc = (kt | kk) ? 1u : 0u;
#pragma unroll
          for (int j = 0; j < MT; ++j) {
            // A of tile j: 128-byte rows (one box or the per-row gather),
            // tile j 128 rows further; with two 32-channel boxes, box kk / 2
            // at 32 bytes per K slice, tile j 128 64-byte rows further
            const uint64_t ad =
                a.tma == 2 ? sw64_desc(a0 + uint32_t((kk >> 1) * (C::kA / 2) + j * (kBM * 64) + 32 * (kk & 1)))
                           : sw128_desc(a0 + uint32_t(j * (kBM * 128) + 32 * kk));
            asm volatile(
                "{ .reg .pred p; setp.ne.b32 p, %4, 0; tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p; }" ::"r"(
                    d + uint32_t(j * NT)),
                "l"(ad), "l"(bd), "r"(C::kIdesc), "r"(acc)
                : "memory");
          }
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
  int mt = 1;                     // pixel tiles per work unit (see ConvCfg)
  Tensor mask;                    // ReLU mask of a backward layer (base null: none)
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
  // a tile of width 16: 16 x 8 pixels of one image; of width 8: two 8 x 8
  // images; a box covers the work unit's mt tiles
  const cuuint32_t box[4] = {cuuint32_t(L.tma == 2 ? kBK / 2 : kBK), cuuint32_t(L.tw),
                             cuuint32_t(L.tw == 8 ? kTileH : kTileH * L.mt),
                             cuuint32_t(L.tw == 8 ? 2 * L.mt : 1)};
  const cuuint32_t estr[4] = {1, 1, 1, 1};
  return enc(&L.tmap, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, L.in.base, dims, strides, box, estr,
             CU_TENSOR_MAP_INTERLEAVE_NONE,
             L.tma == 2 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_128B,
             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int NT, int MT>
cudaError_t launch_conv_nt(const ConvArgs& a, const CUtensorMap& tmap, int mtiles, int ntiles,
                           cudaStream_t s) {
  static int ctas_per_sm = 0;  // per process; set before the first launch
  static int sms = 0;
  if (!ctas_per_sm) {
    cudaError_t e = cudaFuncSetAttribute(k_conv<NT, MT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         ConvCfg<NT, MT>::kSmemMax);
    int dev = 0, smem_sm = 0, regs_sm = 0, reserved = 0;
    cudaFuncAttributes fa{};
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, k_conv<NT, MT>);
    if (e != cudaSuccess) return e;
    // The occupancy calculator reports one CTA per SM for any kernel that
    // allocates tensor memory, so the resident count is derived from the
    // kernel's own shared memory, registers and tensor-memory columns (an
    // SM has 512); extra CTAs of a persistent grid only start later.
    const int by_smem =
        smem_sm / (ConvCfg<NT, MT>::kSmem + int(sizeof(float)) * NT + int(fa.sharedSizeBytes) + reserved);
    const int warp_regs = ((fa.numRegs * 32 + 255) / 256) * 256;
    const int by_regs = regs_sm / (warp_regs * (kConvThreads / 32));
    const int by_tmem = 512 / ConvCfg<NT, MT>::kTmemCols;
    int c = by_smem < by_regs ? by_smem : by_regs;
    c = c < by_tmem ? c : by_tmem;
    ctas_per_sm = c > 0 ? c : 1;
  }
  const int ntotal = mtiles * ntiles;
  const int cap = sms * ctas_per_sm;
  const int grid = ntotal < cap ? ntotal : cap;
  k_conv<NT, MT><<<grid, kConvThreads, ConvCfg<NT, MT>::kSmem + int(sizeof(float)) * a.cout, s>>>(
      a, tmap, ntiles, ntotal);
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
  a.mask = L.mask.base;
  a.ms = L.mask.stride;
  const int ntiles = L.N / L.NT;
  if (L.mt == 2) {
    // units of two tiles: 16 x 16 pixels of one image, or four 8 x 8 images
    const int units = L.tw == 8 ? (n + 3) / 4 : n * (L.in.H / (2 * kTileH)) * (L.in.W / kTileW);
    switch (L.NT) {
      case 16: return launch_conv_nt<16, 2>(a, L.tmap, units, ntiles, s);
      case 32: return launch_conv_nt<32, 2>(a, L.tmap, units, ntiles, s);
      case 64: return launch_conv_nt<64, 2>(a, L.tmap, units, ntiles, s);
      default: return launch_conv_nt<128, 2>(a, L.tmap, units, ntiles, s);
    }
  }
  const int mtiles = (a.M + kBM - 1) / kBM;
  switch (L.NT) {
    case 16: return launch_conv_nt<16, 1>(a, L.tmap, mtiles, ntiles, s);
    case 32: return launch_conv_nt<32, 1>(a, L.tmap, mtiles, ntiles, s);
    case 64: return launch_conv_nt<64, 1>(a, L.tmap, mtiles, ntiles, s);
    default: return launch_conv_nt<128, 1>(a, L.tmap, mtiles, ntiles, s);
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
    // inputs whose channel count is a multiple of 64 (or 32) are read by
    // tensor map, two tiles per stage
    L.mt = L.tma && L.NT <= 32 ? kUnitTiles : 1;
    if (L.tma && !encode_input_map(L, B)) {
      L.tma = 0;
      L.mt = 1;
    }
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

// ===========================================================================
// Training step (Sec. III-C "U-Net Model Training": Adam, categorical
// cross-entropy; "Distributed U-Net Model Training using Horovod
// Framework": each worker's gradients are averaged before the update).
//
// Backward pass of a layer y = relu(conv(x) + b):
//   dgrad  dx = conv(ds, w flipped), the same tcgen05 implicit-GEMM kernel
//          as the forward with the weights rearranged (the output channels
//          become the reduction, the spatial taps are mirrored); its
//          epilogue applies the previous layer's ReLU mask, so it writes that
//          layer's ds directly;
//   wgrad  dw[co][tap, ci] = sum_p ds[p][co] x[p + tap][ci]: the taps of x
//          gathered into one matrix (k_im2col), then a plain GEMM (cuBLAS,
//          bf16 in, f32 out) over the batch's pixels; db = ds summed.
// Transposed convolutions: the output gradient is regrouped per input pixel
// (k_space_to_depth), after which dgrad is a 1x1 convolution and wgrad a
// GEMM.  Pooling, the skip connections, the loss and the head have their own
// small kernels.  Activations and activation gradients are bf16, parameter
// gradients, Adam moments and master weights f32; after each update the
// weights are re-packed on the device into the forward and dgrad layouts.
// ===========================================================================
namespace sil {
namespace unet {

constexpr float kAdamB1 = 0.9f, kAdamB2 = 0.999f, kAdamEps = 1e-7f;

__device__ __forceinline__ float bf2f(__nv_bfloat16 v) { return __bfloat162float(v); }

// Pixels whose reference label is a class (0..2): the loss's denominator.
__global__ void k_count_valid(const uint8_t* __restrict__ lab, int64_t P, unsigned int* count) {
  unsigned int c = 0;
  for (int64_t p = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; p < P;
       p += int64_t(gridDim.x) * blockDim.x)
    c += lab[p] < 3 ? 1u : 0u;
  c = __reduce_add_sync(0xffffffffu, c);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(count, c);
}

// Cross-entropy of the scores against the labels: each CTA's loss sum in
// part[CTA] and dz = (softmax - onehot) / count, 0 for left-out pixels.
__global__ void k_ce(const float* __restrict__ z, const uint8_t* __restrict__ lab, int64_t P,
                     const unsigned int* __restrict__ count, float* __restrict__ dz,
                     float* __restrict__ part) {
  const float inv = 1.f / float(max(*count, 1u));
  float acc = 0.f;
  for (int64_t p = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; p < P;
       p += int64_t(gridDim.x) * blockDim.x) {
    const int l = lab[p];
    float d0 = 0.f, d1 = 0.f, d2 = 0.f;
    if (l < 3) {
      const float z0 = z[3 * p], z1 = z[3 * p + 1], z2 = z[3 * p + 2];
      const float m = fmaxf(z0, fmaxf(z1, z2));
      const float e0 = expf(z0 - m), e1 = expf(z1 - m), e2 = expf(z2 - m);
      const float se = e0 + e1 + e2;
      const float zl = l == 0 ? z0 : (l == 1 ? z1 : z2);
      acc += (m + logf(se) - zl);
      d0 = (e0 / se - (l == 0 ? 1.f : 0.f)) * inv;
      d1 = (e1 / se - (l == 1 ? 1.f : 0.f)) * inv;
      d2 = (e2 / se - (l == 2 ? 1.f : 0.f)) * inv;
    }
    dz[3 * p] = d0;
    dz[3 * p + 1] = d1;
    dz[3 * p + 2] = d2;
  }
  // the CTA's loss sum, in a fixed order (k_sum_parts adds the CTAs')
  __shared__ float wsum[32];
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
  if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.f;
    for (int w = 0; w < int(blockDim.x >> 5); ++w) t += wsum[w];
    part[blockIdx.x] = t;
  }
}

// out[o] = sum over CTAs b of part[b width + o], divided by the count of
// left-in pixels when `count` is given: the second half of the loss and
// head-gradient reductions.  One CTA per output: thread t adds parts t,
// t + 256, ..., then a tree in shared memory; the order is fixed, so the
// result is the same bits on every run.
__global__ void k_sum_parts(const float* __restrict__ part, int nparts, int width,
                            const unsigned int* __restrict__ count, float* __restrict__ out) {
  __shared__ float red[256];
  const int o = blockIdx.x, t = threadIdx.x;
  float acc = 0.f;
  for (int b = t; b < nparts; b += 256) acc += part[size_t(b) * width + o];
  red[t] = acc;
  __syncthreads();
  for (int h = 128; h > 0; h >>= 1) {
    if (t < h) red[t] += red[t + h];
    __syncthreads();
  }
  if (t == 0) out[o] = count ? red[0] / float(max(*count, 1u)) : red[0];
}

__device__ __forceinline__ void unpack8(const uint4 v, float* f) {
  const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const float2 t = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&w[e]));
    f[2 * e] = t.x;
    f[2 * e + 1] = t.y;
  }
}
__device__ __forceinline__ uint4 pack8(const float* f) {
  uint32_t w[4];
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(f[2 * e], f[2 * e + 1]);
    w[e] = *reinterpret_cast<const uint32_t*>(&h);
  }
  return make_uint4(w[0], w[1], w[2], w[3]);
}

// Head (1x1, F -> 3): ds of the last decoder convolution = (dz . w) where
// its output is > 0; gw[k][c] = sum_p dz[p][k] y[p][c], gb[k] = sum_p
// dz[p][k].  A CTA stages 256 pixels at a time in shared memory (16-byte
// loads of the activation, 8 channels each); thread o < 3 F + 3 keeps
// output o's partial sum over the CTA's chunks and stores it in
// part[CTA][o] (k_sum_parts adds the CTAs').
__global__ void k_head_bwd(const float* __restrict__ dz, const __nv_bfloat16* __restrict__ y,
                           int64_t ys, int F, int64_t P, const float* __restrict__ hw,
                           __nv_bfloat16* __restrict__ ds, float* __restrict__ part) {
  extern __shared__ float sh[];
  float* sz = sh;              // [256][3]
  float* sy = sh + 256 * 3;    // [256][F]
  const int t = threadIdx.x, chunks = F / 8;
  float acc = 0.f;
  const int o = t, k = o < 3 * F ? o / F : o - 3 * F, c = o < 3 * F ? o - k * F : 0;
  for (int64_t p0 = int64_t(blockIdx.x) * 256; p0 < P; p0 += int64_t(gridDim.x) * 256) {
    __syncthreads();
    for (int q = t; q < 256 * 3; q += 256) sz[q] = p0 + q / 3 < P ? dz[3 * p0 + q] : 0.f;
    for (int q = t; q < 256 * chunks; q += 256) {
      const int pl = q / chunks, ch = q - pl * chunks;
      const int64_t p = p0 + pl;
      const uint4 v = p < P ? *reinterpret_cast<const uint4*>(y + p * ys + 8 * ch) : make_uint4(0, 0, 0, 0);
      unpack8(v, sy + pl * F + 8 * ch);
    }
    __syncthreads();
    for (int q = t; q < 256 * chunks; q += 256) {
      const int pl = q / chunks, ch = q - pl * chunks;
      const int64_t p = p0 + pl;
      if (p >= P) continue;
      float g[8];
      const float z0 = sz[3 * pl], z1 = sz[3 * pl + 1], z2 = sz[3 * pl + 2];
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const int j = 8 * ch + e;
        const float v = z0 * hw[j] + z1 * hw[F + j] + z2 * hw[2 * F + j];
        g[e] = sy[pl * F + j] > 0.f ? v : 0.f;
      }
      *reinterpret_cast<uint4*>(ds + p * F + 8 * ch) = pack8(g);
    }
    if (o < 3 * F)
      for (int i = 0; i < 256; ++i) acc += sz[3 * i + k] * sy[i * F + c];
    else if (o < 3 * F + 3)
      for (int i = 0; i < 256; ++i) acc += sz[3 * i + k];
  }
  if (o < 3 * F + 3) part[size_t(blockIdx.x) * (3 * F + 3) + o] = acc;
}

// Gradient at an encoder level's output (before its 2x2 max pool): the pooled
// gradient routed to the first maximum of each window (order (0,0), (0,1),
// (1,0), (1,1)) plus the skip connection's share, then that output's ReLU
// mask.  y: the output (stride ys), gpool: [n][H/2][W/2][C], gskip: stride
// gss; ds dense.  One thread per window and 8 channels: every input is read
// once, 16 bytes at a time.
__global__ void k_pool_bwd(const __nv_bfloat16* __restrict__ y, int64_t ys,
                           const __nv_bfloat16* __restrict__ gpool,
                           const __nv_bfloat16* __restrict__ gskip, int64_t gss, int H, int W, int C,
                           int64_t windows, __nv_bfloat16* __restrict__ ds) {
  const int chunks = C / 8, Wh = W / 2, Hh = H / 2;
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < windows * chunks;
       i += int64_t(gridDim.x) * blockDim.x) {
    const int ch = int(i % chunks);
    const int64_t win = i / chunks;
    const int wx = int(win % Wh), wy = int((win / Wh) % Hh);
    const int64_t b = win / (int64_t(Wh) * Hh);
    const int64_t p0 = (b * H + 2 * wy) * W + 2 * wx;
    const int64_t pix[4] = {p0, p0 + 1, p0 + W, p0 + W + 1};
    float yv[4][8], sk[4][8], gp[8];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      unpack8(*reinterpret_cast<const uint4*>(y + pix[q] * ys + 8 * ch), yv[q]);
      unpack8(*reinterpret_cast<const uint4*>(gskip + pix[q] * gss + 8 * ch), sk[q]);
    }
    unpack8(*reinterpret_cast<const uint4*>(gpool + win * C + 8 * ch), gp);
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      int arg = 0;
      float m = yv[0][e];
#pragma unroll
      for (int q = 1; q < 4; ++q)
        if (yv[q][e] > m) {
          m = yv[q][e];
          arg = q;
        }
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const float g = sk[q][e] + (q == arg ? gp[e] : 0.f);
        sk[q][e] = yv[q][e] > 0.f ? g : 0.f;
      }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) *reinterpret_cast<uint4*>(ds + pix[q] * C + 8 * ch) = pack8(sk[q]);
  }
}

// Transposed convolution's output gradient regrouped per input pixel:
// r[b][y][x][(2 i + j) C + c] = g[b][2 y + i][2 x + j][c] (g stride gs),
// 8 channels (16 bytes) per thread.
__global__ void k_space_to_depth(const __nv_bfloat16* __restrict__ g, int64_t gs, int H, int W,
                                 int C, int64_t total, __nv_bfloat16* __restrict__ r) {
  const int chunks = C / 8;
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < total;
       i += int64_t(gridDim.x) * blockDim.x) {
    const int ch = int(i % chunks);
    const int64_t rest = i / chunks;
    const int sub = int(rest & 3);
    const int64_t pix = rest >> 2;  // input pixel (H x W)
    const int x = int(pix % W), yy = int((pix / W) % H);
    const int64_t b = pix / (int64_t(W) * H);
    const int64_t op = (b * 2 * H + 2 * yy + (sub >> 1)) * (2 * W) + 2 * x + (sub & 1);
    *reinterpret_cast<uint4*>(r + pix * 4 * C + sub * C + 8 * ch) =
        *reinterpret_cast<const uint4*>(g + op * gs + 8 * ch);
  }
}

// The 3x3 taps of x for pixels p0 .. p0 + np - 1 as one matrix with a
// leading column of ones (its product with ds is the bias gradient):
// row p - p0 = [1, 0 x 7, x[p shifted by tap 0][0 .. Cp), ..., tap 8], zero
// outside the image; ld = 9 Cp + 8.  8 channels (16 bytes) per thread; H, W
// and Cp / 8 are powers of two (shifts and masks, no divisions but by 9).
__global__ void k_im2col(const __nv_bfloat16* __restrict__ x, int64_t xs, int hlog, int wlog,
                         int clog, int64_t p0, int np, __nv_bfloat16* __restrict__ col) {
  const int Cp = 8 << clog, ld = 9 * Cp + 8;
  const uint32_t total = uint32_t(np) * 9u << clog;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
    const uint32_t ch = i & ((1u << clog) - 1u), q = i >> clog;
    const uint32_t pl = q / 9u, tap = q - 9u * pl;
    const int64_t p = p0 + pl;
    const int x0 = int(p & ((1 << wlog) - 1)), y0 = int((p >> wlog) & ((1 << hlog) - 1));
    const int64_t b = p >> (wlog + hlog);
    const int yy = y0 + int(tap) / 3 - 1, xx = x0 + int(tap) % 3 - 1;
    uint4 v = make_uint4(0, 0, 0, 0);
    if (yy >= 0 && yy < (1 << hlog) && xx >= 0 && xx < (1 << wlog))
      v = *reinterpret_cast<const uint4*>(x + ((((b << hlog) + yy) << wlog) + xx) * xs + 8 * ch);
    __nv_bfloat16* row = col + int64_t(pl) * ld;
    *reinterpret_cast<uint4*>(row + 8 + tap * Cp + 8 * ch) = v;
    if (tap == 0 && ch == 0) *reinterpret_cast<uint4*>(row) = make_uint4(0x3F80u, 0, 0, 0);  // bf16 1.0
  }
}

// GEMM results -> the parameter gradient in PyTorch layout.
//   conv:  raw[co + Co (8 + tap Cp + ci)] -> gw[co][ci][tap]; gb[co] = raw[co]
//          (rawb unused)
//   up:    raw[ci + Ci (sub Co + co)] -> gw[ci][co][sub]; gb[co] = sum_sub rawb[sub Co + co]
__global__ void k_wgrad_out(const float* __restrict__ raw, const float* __restrict__ rawb, int up,
                            int Ci, int Co, int Cp, float* __restrict__ gw, float* __restrict__ gb) {
  const int nw = up ? Ci * Co * 4 : Co * Ci * 9;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nw + Co; i += gridDim.x * blockDim.x) {
    if (i >= nw) {
      const int co = i - nw;
      gb[co] = up ? rawb[co] + rawb[Co + co] + rawb[2 * Co + co] + rawb[3 * Co + co] : raw[co];
      continue;
    }
    if (up) {
      const int sub = i % 4, co = (i / 4) % Co, ci = i / (4 * Co);
      gw[i] = raw[ci + size_t(Ci) * (sub * Co + co)];
    } else {
      const int tap = i % 9, ci = (i / 9) % Ci, co = i / (9 * Ci);
      gw[i] = raw[co + size_t(Co) * (8 + tap * Cp + ci)];
    }
  }
}

// One Adam step on the flat parameters: c1 = 1 / (1 - b1^t), c2 = 1 / (1 - b2^t).
__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, int64_t n, float lr, float c1, float c2) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n;
       i += int64_t(gridDim.x) * blockDim.x) {
    const float gi = g[i];
    const float mi = kAdamB1 * m[i] + (1.f - kAdamB1) * gi;
    const float vi = kAdamB2 * v[i] + (1.f - kAdamB2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi * c1) / (sqrtf(vi * c2) + kAdamEps);
  }
}

__device__ __forceinline__ size_t sw128_off_d(int rr, int k) {
  return size_t(rr >> 3) * 1024 + size_t(rr & 7) * 128 + size_t(((k >> 3) ^ (rr & 7)) << 4) +
         size_t(k & 7) * 2;
}

// Weight blocks [N / NT][KT][NT x 64] (bf16, 128-byte swizzle) of a kernel
// from the f32 PyTorch-layout weights w:
//   mode 0 conv forward:  n = co, k = tap Cp + c        <- w[co][c][tap]
//   mode 1 up forward:    n = sub Co + co, k = c        <- w[c][co][sub]
//   mode 2 conv dgrad:    n = ci, k = tap Cop + co      <- w[co][ci][8 - tap]
//   mode 3 up dgrad:      n = ci, k = sub Co + co       <- w[ci][co][sub]
__global__ void k_pack(const float* __restrict__ w, int mode, int Ci, int Co, int Cp, int N, int NT,
                       int KT, uint8_t* __restrict__ blk) {
  // one thread per row n and 8 consecutive k (one 16-byte chunk of a
  // swizzled 128-byte row); Cp and Co are multiples of 8, so the 8 k share
  // their tap / sub-position
  const int64_t total = int64_t(N) * KT * (kBK / 8);
  const size_t bsz = size_t(NT) * kBK * 2;
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < total;
       i += int64_t(gridDim.x) * blockDim.x) {
    const int n = int(i / (int64_t(KT) * (kBK / 8)));
    const int k0 = int(i % (int64_t(KT) * (kBK / 8))) * 8;
    float v[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const int k = k0 + e;
      float u = 0.f;
      if (mode == 0) {
        const int tap = k / Cp, c = k % Cp;
        if (tap < 9 && c < Ci) u = w[(size_t(n) * Ci + c) * 9 + tap];
      } else if (mode == 1) {
        const int sub = n / Co, co = n % Co;
        if (k < Ci) u = w[(size_t(k) * Co + co) * 4 + sub];
      } else if (mode == 2) {
        const int tap = k / Cp, co = k % Cp;  // Cp: the padded output channels of the forward
        if (tap < 9 && co < Co && n < Ci) u = w[(size_t(co) * Ci + n) * 9 + (8 - tap)];
      } else {
        const int sub = k / Co, co = k % Co;
        if (sub < 4 && n < Ci) u = w[(size_t(n) * Co + co) * 4 + sub];
      }
      v[e] = u;
    }
    const int rr = n % NT, kk = k0 % kBK;
    *reinterpret_cast<uint4*>(blk + (size_t(n / NT) * KT + k0 / kBK) * bsz + sw128_off_d(rr, kk)) = pack8(v);
  }
}

}  // namespace unet
}  // namespace sil

struct sil_unet_trainer {
  sil_unet* net = nullptr;
  int device = 0, D = 0, F = 0, B = 0, nl = 0;
  std::vector<void*> allocs;
  std::vector<int64_t> w_off, b_off;
  int64_t nparams = 0;
  float* p = nullptr;  // master weights, PyTorch layout, layer after layer (weight, bias)
  float* m = nullptr;  // Adam moments
  float* v = nullptr;
  std::vector<sil::unet::Layer> bwd;    // dgrad launch of forward layer i (wblk null: none)
  std::vector<sil::unet::Tensor> ds;    // gradient at layer i's pre-activation
  std::vector<sil::unet::Tensor> gcat;  // per level: gradient of the concatenation
  std::vector<sil::unet::Tensor> rr;    // per level: that gradient's first half, per input pixel
  std::vector<sil::unet::Tensor> gpool; // per level: gradient at the pooled output
  __nv_bfloat16* col = nullptr;
  int64_t col_elems = 0;
  float* raw = nullptr;
  float* rawb = nullptr;
  __nv_bfloat16* ones = nullptr;
  float* logits = nullptr;
  float* dz = nullptr;
  unsigned int* count = nullptr;
  float* zero_bias = nullptr;
  float* part = nullptr;  // per-CTA partial sums of the loss and the head gradient
  cublasHandle_t blas = nullptr;
  int last_n = 0;
};

namespace {

int enc_idx(int l, int j) { return 2 * l + j; }
int bott_idx(int D, int j) { return 2 * D + j; }
int up_idx(int D, int l) { return 2 * D + 2 + 3 * (D - 1 - l); }

constexpr int kMaxGrid = 152 * 16;  // CTAs of the grid-stride kernels
int grid_for(int64_t work, int threads) {
  const int64_t g = (work + threads - 1) / threads;
  return int(g < kMaxGrid ? (g > 0 ? g : 1) : kMaxGrid);
}

// out = sum over pixels of a^T b (column-major views, see the callers),
// bf16 inputs, f32 output; beta 0 or 1.
cublasStatus_t gemm_tn(cublasHandle_t h, int m, int n, int k, const void* A, int lda, const void* B,
                       int ldb, float beta, float* C, int ldc, bool b_trans) {
  const float one = 1.f;
  return cublasGemmEx(h, CUBLAS_OP_N, b_trans ? CUBLAS_OP_T : CUBLAS_OP_N, m, n, k, &one, A,
                      CUDA_R_16BF, lda, B, CUDA_R_16BF, ldb, &beta, C, CUDA_R_32F, ldc,
                      CUBLAS_COMPUTE_32F, CUBLAS_GEMM_DEFAULT);
}

// Rewrites the network's forward weight blocks, biases and head and the
// dgrad blocks from the master weights.
cudaError_t repack(sil_unet_trainer* tr, cudaStream_t s) {
  sil_unet* net = tr->net;
  for (int i = 0; i < tr->nl; ++i) {
    const Layer& L = net->layers[i];
    const float* w = tr->p + tr->w_off[i];
    const float* b = tr->p + tr->b_off[i];
    cudaError_t e;
    if (L.kind == SIL_UNET_HEAD) {
      e = cudaMemcpyAsync(net->head_w, w, sizeof(float) * kClasses * tr->F, cudaMemcpyDeviceToDevice, s);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(net->head_b, b, sizeof(float) * kClasses, cudaMemcpyDeviceToDevice, s);
      if (e != cudaSuccess) return e;
      continue;
    }
    const bool up = L.kind == SIL_UNET_UP;
    k_pack<<<grid_for(int64_t(L.N) * L.KT * (kBK / 8), 256), 256, 0, s>>>(w, up ? 1 : 0, L.ci, L.co,
                                                                    L.cin_pad, L.N, L.NT, L.KT, L.wblk);
    e = cudaMemcpyAsync(L.bias, b, sizeof(float) * L.co, cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return e;
    const Layer& G = tr->bwd[i];
    if (G.wblk)
      k_pack<<<grid_for(int64_t(G.N) * G.KT * (kBK / 8), 256), 256, 0, s>>>(w, up ? 3 : 2, L.ci, L.co,
                                                                      G.cin_pad, G.N, G.NT, G.KT, G.wblk);
  }
  return cudaGetLastError();
}

// wgrad of 3x3 layer i: raw = ds^T [1 | col] (Co x (8 + 9 Cp); column 0 is
// the bias gradient), in pixel chunks that fit the im2col buffer; then the
// PyTorch layout.
bool conv_wgrad(sil_unet_trainer* tr, int i, int n, float* grads, cudaStream_t s) {
  const Layer& L = tr->net->layers[i];
  const Tensor& x = L.in;
  const Tensor& g = tr->ds[i];
  const int Cp = L.cin_pad, ld = 9 * Cp + 8, Co = L.co;
  const int64_t P = int64_t(n) * x.H * x.W;
  const int64_t chunk = std::min<int64_t>(P, tr->col_elems / ld);
  bool ok = true;
  for (int64_t p0 = 0; p0 < P && ok; p0 += chunk) {
    const int64_t np = std::min(chunk, P - p0);
    k_im2col<<<grid_for(np * 9 * (Cp / 8), 256), 256, 0, s>>>(x.base, x.stride, ilog2(x.H), ilog2(x.W),
                                                              ilog2(Cp / 8), p0, int(np), tr->col);
    ok = gemm_tn(tr->blas, Co, ld, int(np), g.base + p0 * Co, Co, tr->col, ld, p0 ? 1.f : 0.f,
                 tr->raw, Co, true) == CUBLAS_STATUS_SUCCESS;
  }
  k_wgrad_out<<<grid_for(int64_t(Co) * L.ci * 9 + Co, 256), 256, 0, s>>>(
      tr->raw, nullptr, 0, L.ci, Co, Cp, grads + tr->w_off[i], grads + tr->b_off[i]);
  return ok;
}

// wgrad of the transposed convolution of level l: raw = x^T r (Ci x 4 Co),
// rawb = r^T 1 (4 Co).
bool up_wgrad(sil_unet_trainer* tr, int l, int n, float* grads, cudaStream_t s) {
  const int i = up_idx(tr->D, l);
  const Layer& L = tr->net->layers[i];
  const Tensor& x = L.in;
  const Tensor& r = tr->rr[l];
  const int64_t P = int64_t(n) * x.H * x.W;
  const bool ok =
      gemm_tn(tr->blas, L.ci, 4 * L.co, int(P), x.base, int(x.stride), r.base, 4 * L.co, 0.f, tr->raw,
              L.ci, true) == CUBLAS_STATUS_SUCCESS &&
      gemm_tn(tr->blas, 4 * L.co, 1, int(P), r.base, 4 * L.co, tr->ones, int(P), 0.f, tr->rawb,
              4 * L.co, false) == CUBLAS_STATUS_SUCCESS;
  k_wgrad_out<<<grid_for(int64_t(L.co) * L.ci * 4 + L.co, 256), 256, 0, s>>>(
      tr->raw, tr->rawb, 1, L.ci, L.co, 0, grads + tr->w_off[i], grads + tr->b_off[i]);
  return ok;
}

}  // namespace

extern "C" void sil_unet_trainer_destroy(sil_unet_trainer* tr) {
  if (!tr) return;
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(tr->device);
  if (tr->blas) cublasDestroy(tr->blas);
  for (void* q : tr->allocs) cudaFree(q);
  cudaSetDevice(prev);
  sil_unet_destroy(tr->net);
  delete tr;
}

extern "C" sil_status sil_unet_trainer_create(sil_unet_trainer** out, const sil_unet_config* cfg,
                                              const float* const* weights,
                                              const float* const* biases, int32_t device) {
  if (!out) {
    set_error("sil_unet_trainer_create: NULL");
    return SIL_EINVAL;
  }
  *out = nullptr;
  sil_unet* net = nullptr;
  sil_status st = sil_unet_create(&net, cfg, weights, biases, device);
  if (st != SIL_OK) return st;
  sil_unet_trainer* tr = new (std::nothrow) sil_unet_trainer;
  if (!tr) {
    sil_unet_destroy(net);
    return SIL_ENOMEM;
  }
  tr->net = net;
  tr->device = device;
  tr->D = cfg->depth;
  tr->F = cfg->base_width;
  tr->B = cfg->max_batch;
  tr->nl = int(net->layers.size());
  const int D = tr->D, B = tr->B;
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(device);
  auto dalloc = [&](size_t bytes) -> void* {
    void* q = nullptr;
    if (st != SIL_OK) return nullptr;
    if (cudaMalloc(&q, bytes) != cudaSuccess) {
      set_error("sil_unet_trainer_create: cudaMalloc(%zu) failed", bytes);
      st = SIL_ENOMEM;
      return nullptr;
    }
    tr->allocs.push_back(q);
    return q;
  };
  auto act = [&](int H, int C) {
    Tensor t;
    t.base = static_cast<__nv_bfloat16*>(dalloc(size_t(B) * H * H * C * 2));
    t.stride = C;
    t.H = t.W = H;
    t.C = C;
    return t;
  };
  // parameter offsets (sil_unet_layer_shape order, weight then bias)
  int64_t raw_elems = 0, rawb_elems = 0, col_need = 0;
  for (int i = 0; i < tr->nl; ++i) {
    int64_t d[4];
    int kind = 0;
    layer_shape(*cfg, i, d, &kind);
    tr->w_off.push_back(tr->nparams);
    tr->nparams += d[0] * d[1] * d[2] * d[3];
    tr->b_off.push_back(tr->nparams);
    tr->nparams += kind == SIL_UNET_UP ? d[1] : d[0];
    const Layer& L = net->layers[i];
    if (kind == SIL_UNET_CONV3) {
      raw_elems = std::max<int64_t>(raw_elems, int64_t(L.co) * (9 * L.cin_pad + 8));
      col_need = std::max<int64_t>(col_need, int64_t(B) * L.in.H * L.in.W * (9 * L.cin_pad + 8));
    } else if (kind == SIL_UNET_UP) {
      raw_elems = std::max<int64_t>(raw_elems, int64_t(L.ci) * 4 * L.co);
      rawb_elems = std::max<int64_t>(rawb_elems, 4 * L.co);
    }
  }
  tr->p = static_cast<float*>(dalloc(sizeof(float) * tr->nparams));
  tr->m = static_cast<float*>(dalloc(sizeof(float) * tr->nparams));
  tr->v = static_cast<float*>(dalloc(sizeof(float) * tr->nparams));
  for (int i = 0; i < tr->nl && st == SIL_OK; ++i) {
    const int64_t wl = tr->b_off[i] - tr->w_off[i];
    const int64_t bl = (i + 1 < tr->nl ? tr->w_off[i + 1] : tr->nparams) - tr->b_off[i];
    if (cudaMemcpy(tr->p + tr->w_off[i], weights[i], sizeof(float) * wl, cudaMemcpyHostToDevice) !=
            cudaSuccess ||
        cudaMemcpy(tr->p + tr->b_off[i], biases[i], sizeof(float) * bl, cudaMemcpyHostToDevice) !=
            cudaSuccess)
      st = SIL_ECUDA;
  }
  // the im2col buffer holds at most 1 GiB; larger layers go in pixel chunks
  tr->col_elems = std::min<int64_t>(col_need, int64_t(1) << 29);
  tr->col = static_cast<__nv_bfloat16*>(dalloc(size_t(tr->col_elems) * 2));
  tr->raw = static_cast<float*>(dalloc(sizeof(float) * raw_elems));
  tr->rawb = static_cast<float*>(dalloc(sizeof(float) * rawb_elems));
  const int64_t P0 = int64_t(B) * kChip * kChip;
  tr->ones = static_cast<__nv_bfloat16*>(dalloc(size_t(P0) * 2));
  tr->logits = static_cast<float*>(dalloc(sizeof(float) * P0 * kClasses));
  tr->dz = static_cast<float*>(dalloc(sizeof(float) * P0 * kClasses));
  tr->count = static_cast<unsigned int*>(dalloc(sizeof(unsigned int)));
  tr->zero_bias = static_cast<float*>(dalloc(sizeof(float) * kMaxCout));
  tr->part = static_cast<float*>(dalloc(sizeof(float) * kMaxGrid * (kClasses * (tr->F + 1))));
  if (st == SIL_OK) {
    std::vector<uint16_t> one(size_t(P0), 0x3F80u);  // bfloat16 1.0
    if (cudaMemcpy(tr->ones, one.data(), size_t(P0) * 2, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(tr->zero_bias, 0, sizeof(float) * kMaxCout) != cudaSuccess ||
        cudaMemset(tr->m, 0, sizeof(float) * tr->nparams) != cudaSuccess ||
        cudaMemset(tr->v, 0, sizeof(float) * tr->nparams) != cudaSuccess)
      st = SIL_ECUDA;
  }
  // activation gradients
  tr->ds.resize(tr->nl);
  tr->gcat.resize(D);
  tr->rr.resize(D);
  tr->gpool.resize(D);
  for (int l = 0; l < D; ++l) {
    const int H = kChip >> l, w = tr->F << l;
    tr->gcat[l] = act(H, 2 * w);
    tr->rr[l] = act(H / 2, 4 * w);
    tr->gpool[l] = act(H / 2, w);
  }
  for (int i = 0; i < tr->nl; ++i) {
    const Layer& L = net->layers[i];
    if (L.kind == SIL_UNET_CONV3) {
      tr->ds[i] = act(L.out.H, L.co);
    } else if (L.kind == SIL_UNET_UP) {
      const int l = D - 1 - (i - 2 * D - 2) / 3;
      tr->ds[i] = tr->gcat[l];
      tr->ds[i].C = L.co;
    }
  }
  // dgrad launches: input = ds of the layer, output = the gradient at its
  // input (masked by the producing layer's ReLU where there is one)
  tr->bwd.resize(tr->nl);
  auto dgrad = [&](int i, const Tensor& in, int taps, const Tensor& outt, const Tensor* mask) {
    const Layer& L = net->layers[i];
    Layer G;
    G.kind = SIL_UNET_CONV3;
    G.ci = in.C;
    G.cin_pad = in.C;
    G.co = L.ci;
    G.N = L.ci;
    G.NT = G.N < 128 ? G.N : 128;
    G.taps = taps;
    G.K = taps == 1 ? in.C : 9 * in.C;
    G.KT = (G.K + kBK - 1) / kBK;
    G.relu = false;
    G.in = in;
    G.out = outt;
    if (mask) G.mask = *mask;
    G.tma = (G.cin_pad % kBK == 0) ? 1 : (G.cin_pad == kBK / 2 && taps == 9) ? 2 : 0;
    G.tw = in.W >= kTileW ? kTileW : 8;
    G.mt = G.tma && G.NT <= 32 ? kUnitTiles : 1;
    G.bias = tr->zero_bias;
    G.wblk = static_cast<uint8_t*>(dalloc(size_t(G.N) * G.KT * kBK * 2));
    if (st == SIL_OK && G.tma && !encode_input_map(G, B)) {
      G.tma = 0;
      G.mt = 1;
    }
    tr->bwd[i] = G;
  };
  for (int l = 0; l < D && st == SIL_OK; ++l) {
    const int e0 = enc_idx(l, 0), e1 = enc_idx(l, 1), u = up_idx(D, l);
    dgrad(e1, tr->ds[e1], 9, tr->ds[e0], &net->layers[e0].out);
    if (l > 0) dgrad(e0, tr->ds[e0], 9, tr->gpool[l - 1], nullptr);
    dgrad(u + 2, tr->ds[u + 2], 9, tr->ds[u + 1], &net->layers[u + 1].out);
    dgrad(u + 1, tr->ds[u + 1], 9, tr->gcat[l], nullptr);
    const int below = l == D - 1 ? bott_idx(D, 1) : up_idx(D, l + 1) + 2;
    dgrad(u, tr->rr[l], 1, tr->ds[below], &net->layers[u].in);
  }
  if (st == SIL_OK) {
    const int b0 = bott_idx(D, 0), b1 = bott_idx(D, 1);
    dgrad(b1, tr->ds[b1], 9, tr->ds[b0], &net->layers[b0].out);
    dgrad(b0, tr->ds[b0], 9, tr->gpool[D - 1], nullptr);
  }
  if (st == SIL_OK && cublasCreate(&tr->blas) != CUBLAS_STATUS_SUCCESS) {
    set_error("sil_unet_trainer_create: cublasCreate failed");
    st = SIL_ECUDA;
  }
  if (st == SIL_OK &&
      cudaFuncSetAttribute(k_head_bwd, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           int(sizeof(float)) * 256 * (kClasses + 64)) != cudaSuccess)
    st = SIL_ECUDA;
  if (st == SIL_OK && (repack(tr, nullptr) != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess)) {
    set_error("sil_unet_trainer_create: weight packing failed");
    st = SIL_ECUDA;
  }
  cudaSetDevice(prev);
  if (st != SIL_OK) {
    sil_unet_trainer_destroy(tr);
    return st;
  }
  *out = tr;
  return SIL_OK;
}

extern "C" sil_unet* sil_unet_trainer_net(sil_unet_trainer* tr) { return tr ? tr->net : nullptr; }

extern "C" int64_t sil_unet_trainer_num_params(const sil_unet_trainer* tr) {
  return tr ? tr->nparams : -1;
}

extern "C" sil_status sil_unet_trainer_param_offset(const sil_unet_trainer* tr, int32_t i,
                                                    int64_t* w_off, int64_t* b_off) {
  if (!tr || !w_off || !b_off || i < 0 || i >= tr->nl) {
    set_error("sil_unet_trainer_param_offset: NULL or layer %d out of range", int(i));
    return SIL_EINVAL;
  }
  *w_off = tr->w_off[i];
  *b_off = tr->b_off[i];
  return SIL_OK;
}

extern "C" sil_status sil_unet_trainer_backward(sil_unet_trainer* tr, const uint8_t* chips,
                                                const uint8_t* labels, int32_t n, float* grads,
                                                float* loss, sil_stream stream) {
  if (!tr || !chips || !labels || !grads || !loss || n < 1 || n > tr->B) {
    set_error("sil_unet_trainer_backward: NULL argument or n=%d outside 1..max_batch", int(n));
    return SIL_EINVAL;
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  sil_unet* net = tr->net;
  const int D = tr->D, F = tr->F;
  const int64_t P0 = int64_t(n) * kChip * kChip;
  sil_status st = sil_unet_forward(net, chips, n, nullptr, tr->logits, stream);
  if (st != SIL_OK) return st;
  bool ok = cublasSetStream(tr->blas, s) == CUBLAS_STATUS_SUCCESS;
  const int head = tr->nl - 1;
  cudaError_t e = cudaMemsetAsync(tr->count, 0, sizeof(unsigned int), s);
  if (e != cudaSuccess || !ok) {
    set_error("sil_unet_trainer_backward: %s", ok ? cudaGetErrorString(e) : "cublasSetStream failed");
    return SIL_ECUDA;
  }
  k_count_valid<<<grid_for(P0, 256), 256, 0, s>>>(labels, P0, tr->count);
  const int gce = grid_for(P0, 256);
  k_ce<<<gce, 256, 0, s>>>(tr->logits, labels, P0, tr->count, tr->dz, tr->part);
  k_sum_parts<<<1, 256, 0, s>>>(tr->part, gce, 1, tr->count, loss);
  {
    // head: weight [3][F] then bias [3], contiguous in the flat gradient
    const Layer& L = net->layers[up_idx(D, 0) + 2];
    const int gh = grid_for(P0, 256 * 8), width = kClasses * (F + 1);
    k_head_bwd<<<gh, 256, sizeof(float) * 256 * (kClasses + F), s>>>(
        tr->dz, L.out.base, L.out.stride, F, P0, net->head_w, tr->ds[up_idx(D, 0) + 2].base, tr->part);
    k_sum_parts<<<width, 256, 0, s>>>(tr->part, gh, width, nullptr, grads + tr->w_off[head]);
  }
  auto dgrad = [&](int i) {
    if (e == cudaSuccess)
      e = run_layer(tr->bwd[i], n, net->err, nullptr, nullptr, nullptr, nullptr, false, s);
  };
  for (int l = 0; l < D; ++l) {
    const int u = up_idx(D, l), w = F << l;
    ok = ok && conv_wgrad(tr, u + 2, n, grads, s);
    dgrad(u + 2);
    ok = ok && conv_wgrad(tr, u + 1, n, grads, s);
    dgrad(u + 1);
    const Tensor& g = tr->gcat[l];
    const int h = g.H / 2;
    const int64_t tot = int64_t(n) * h * h * 4 * (w / 8);
    k_space_to_depth<<<grid_for(tot, 256), 256, 0, s>>>(g.base, g.stride, h, h, w, tot, tr->rr[l].base);
    ok = ok && up_wgrad(tr, l, n, grads, s);
    dgrad(u);
  }
  for (int j = 1; j >= 0; --j) {
    ok = ok && conv_wgrad(tr, bott_idx(D, j), n, grads, s);
    dgrad(bott_idx(D, j));
  }
  for (int l = D - 1; l >= 0; --l) {
    const int e0 = enc_idx(l, 0), e1 = enc_idx(l, 1), w = F << l;
    const Layer& L = net->layers[e1];
    const int64_t windows = int64_t(n) * (L.out.H / 2) * (L.out.W / 2);
    k_pool_bwd<<<grid_for(windows * (w / 8), 256), 256, 0, s>>>(
        L.out.base, L.out.stride, tr->gpool[l].base, tr->gcat[l].base + w, tr->gcat[l].stride, L.out.H,
        L.out.W, w, windows, tr->ds[e1].base);
    ok = ok && conv_wgrad(tr, e1, n, grads, s);
    dgrad(e1);
    ok = ok && conv_wgrad(tr, e0, n, grads, s);
    if (l > 0) dgrad(e0);
  }
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess || !ok) {
    set_error("sil_unet_trainer_backward: %s", ok ? cudaGetErrorString(e) : "cuBLAS GEMM failed");
    return SIL_ECUDA;
  }
  tr->last_n = n;
  return SIL_OK;
}

extern "C" sil_status sil_unet_trainer_adam(sil_unet_trainer* tr, const float* grads, float lr,
                                            int32_t t, sil_stream stream) {
  if (!tr || !grads || t < 1 || !(lr >= 0.f)) {
    set_error("sil_unet_trainer_adam: NULL, step t=%d < 1 or negative learning rate", int(t));
    return SIL_EINVAL;
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const float c1 = float(1.0 / (1.0 - std::pow(double(kAdamB1), t)));
  const float c2 = float(1.0 / (1.0 - std::pow(double(kAdamB2), t)));
  k_adam<<<grid_for(tr->nparams, 256), 256, 0, s>>>(tr->p, grads, tr->m, tr->v, tr->nparams, lr, c1, c2);
  const cudaError_t e = repack(tr, s);
  if (e != cudaSuccess) {
    set_error("sil_unet_trainer_adam: %s", cudaGetErrorString(e));
    return SIL_ECUDA;
  }
  return SIL_OK;
}

extern "C" sil_status sil_unet_trainer_get_params(const sil_unet_trainer* tr, float* dst,
                                                  sil_stream stream) {
  if (!tr || !dst) {
    set_error("sil_unet_trainer_get_params: NULL");
    return SIL_EINVAL;
  }
  if (cudaMemcpyAsync(dst, tr->p, sizeof(float) * tr->nparams, cudaMemcpyDeviceToDevice,
                      reinterpret_cast<cudaStream_t>(stream)) != cudaSuccess) {
    set_error("sil_unet_trainer_get_params: copy failed");
    return SIL_ECUDA;
  }
  return SIL_OK;
}

extern "C" sil_status sil_unet_trainer_set_params(sil_unet_trainer* tr, const float* src,
                                                  sil_stream stream) {
  if (!tr || !src) {
    set_error("sil_unet_trainer_set_params: NULL");
    return SIL_EINVAL;
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemcpyAsync(tr->p, src, sizeof(float) * tr->nparams, cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(tr->m, 0, sizeof(float) * tr->nparams, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(tr->v, 0, sizeof(float) * tr->nparams, s);
  if (e == cudaSuccess) e = repack(tr, s);
  if (e != cudaSuccess) {
    set_error("sil_unet_trainer_set_params: %s", cudaGetErrorString(e));
    return SIL_ECUDA;
  }
  return SIL_OK;
}

namespace {
// The stored gradient of kind k (sil_unet_grad_kind) and index i.
bool grad_of(const sil_unet_trainer* tr, int k, int i, Tensor* t) {
  if (!tr) return false;
  if (k == SIL_UNET_GRAD_LAYER && i >= 0 && i < tr->nl - 1) *t = tr->ds[i];
  else if (k == SIL_UNET_GRAD_CAT && i >= 0 && i < tr->D) *t = tr->gcat[i];
  else if (k == SIL_UNET_GRAD_POOL && i >= 0 && i < tr->D) *t = tr->gpool[i];
  else return false;
  return true;
}
}  // namespace

extern "C" sil_status sil_unet_trainer_grad_shape(const sil_unet_trainer* tr, int32_t kind,
                                                  int32_t i, int64_t dims[4]) {
  Tensor t;
  if (!dims || !grad_of(tr, kind, i, &t)) {
    set_error("sil_unet_trainer_grad_shape: NULL or no stored gradient of kind %d, index %d",
              int(kind), int(i));
    return SIL_EINVAL;
  }
  dims[0] = tr->last_n;
  dims[1] = t.H;
  dims[2] = t.W;
  dims[3] = t.C;
  return SIL_OK;
}

extern "C" sil_status sil_unet_trainer_copy_grad(const sil_unet_trainer* tr, int32_t kind,
                                                 int32_t i, void* dst, sil_stream stream) {
  Tensor t;
  if (!dst || !grad_of(tr, kind, i, &t) || tr->last_n < 1) {
    set_error("sil_unet_trainer_copy_grad: NULL, no backward pass yet, or no stored gradient of "
              "kind %d, index %d", int(kind), int(i));
    return SIL_EINVAL;
  }
  const size_t rows = size_t(tr->last_n) * t.H * t.W;
  if (cudaMemcpy2DAsync(dst, size_t(t.C) * 2, t.base, size_t(t.stride) * 2, size_t(t.C) * 2, rows,
                        cudaMemcpyDeviceToDevice, reinterpret_cast<cudaStream_t>(stream)) != cudaSuccess) {
    set_error("sil_unet_trainer_copy_grad: copy failed");
    return SIL_ECUDA;
  }
  return SIL_OK;
}
