// sil_chip.cuh -- the fused per-chip labeler (device code).
//
// One CTA of 256 threads (16 half-warps) labels one chip of at most
// 256 x 256 pixels; a persistent CTA loops over chips.
//
//   pass 1  each half-warp owns a band of rows, each lane 16 columns of them.
//           Rows arrive through a 3-slot shared-memory ring filled by lane-
//           contiguous 16-byte asynchronous copies, so two rows per band are
//           in flight while one is computed.
//           decode -> V = max(R,G,B) -> 3x3 median of V clamped to the chip
//           -> histogram of Vf in shared memory, Vf kept in tensor memory
//           (each thread's own pixels in its own TMEM lane).
//   stats   all threads: lo/hi, exact Otsu threshold (128-bit compares), gate
//   LUT     one thread per value: gated min-max stretch, truncation, class
//           ranges, absdiff override -> label(Vf) table
//   counts  histogram x table (no per-pixel counting)
//   pass 2  Vf from tensor memory -> table -> uint8 label store
//
// Paper passages: Sec. III-B "Filtering Out the Thin Clouds and Shadows"
// (HSV, noise filtering, Otsu, min-max normalisation, truncation, absolute
// difference, binary thresholding, bit-wise ops), Sec. III-B "Auto-labeling
// Method" (inclusive HSV ranges, non-intersecting, one mask per class,
// merged), Sec. III-B "PySpark Map-Reduce" (map = label, reduce = counts).
//
// Pixel values travel through the median as packed u16x2 words whose 16-bit
// lanes carry the 8-bit value in their HIGH byte (the low byte is a copy and
// never decides an order), so one __vimax3_u16x2 / __vimin3_u16x2 handles two
// pixels and three inputs.  A lane's 16 columns are held as 8 words in
// "interleaved" order: word i = [col i, col i+8], so the horizontal
// neighbours of word i are words i-1 and i+1 and only the two segment edges
// need a shuffle.  The median of three is a+b+c-max3-min3, exact in 32-bit
// wrap-around arithmetic because every lane of the result lies in [0,65535].
#pragma once
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

#include "sil_common.h"

namespace sil {

constexpr int kMaxWarps = kMaxThreads / 32;
constexpr int kMaxBands = kMaxThreads / 16;  // one row band per half-warp
// warps and bands of the running CTA (blockDim.x is 256 or 320)
__device__ __forceinline__ int n_warps() { return int(blockDim.x) >> 5; }
__device__ __forceinline__ int n_bands() { return int(blockDim.x) >> 4; }
constexpr int kBinWarps = 256 / 32;  // warps whose threads own a histogram bin
#ifndef SIL_RING
#define SIL_RING 3
#endif
constexpr int kRing = SIL_RING;  // row slots per band
constexpr int kLanePx = 16;

// Per-chip statistics scratch (shared memory).  hist[256 + lane] are bins
// that nothing reads: lanes past a narrow chip's last column count there.
struct ChipStat {
  uint32_t hist[256 + 32];
  uint32_t red[kMaxWarps][4];
  uint32_t nod[kMaxWarps];
  int32_t stat[8];
  uint32_t tmem;  // tensor-memory address of the CTA's Vf plane (resident kernels)
};
// Scratch of the block-wide Otsu search.
struct alignas(16) StatScratch {
  uint32_t wc[kMaxWarps], ws[kMaxWarps];
  uint64_t bnum_lo[kMaxWarps];
  uint32_t bnum_hi[kMaxWarps], bden[kMaxWarps];
  int32_t bt[kMaxWarps], lo[kMaxWarps], hi[kMaxWarps];
  float fmax[kMaxWarps];
  uint32_t n0;
};

// Row slot size: the 16-byte blocks holding one chip row (<= 256 px) of
// bytes-per-pixel BPP plus one block of misalignment.
template <int BPP>
struct Slot {
  static constexpr int kBytes = 16 * ((BPP * 256 + 15) / 16 + 1);
};

// Shared memory of the resident kernel.  The statistics come first so the
// histogram sits at shared offset 0 and a bin's byte offset is its address.
// The row ring comes last: it is declared for the largest CTA, but a launch
// allocates only the blockDim.x / 16 bands it uses (resident_smem_bytes).
// The filtered V plane is here only when SPLANE; otherwise it lives in
// tensor memory (below).
template <int BPP, bool FLAGS, bool SPLANE>
struct ChipSmemT {
  static constexpr bool kSmemPlane = SPLANE;
  ChipStat st;
  StatScratch sc;
  // per row, per lane: 16 nibbles (bits 0-2 class mask of the H/S ranges,
  // bit 3 nodata); uint16 and H/S-narrowed variants only
  uint32_t flags[FLAGS ? 256 : 1][FLAGS ? 16 : 1][FLAGS ? 2 : 1];
  // filtered V in shared memory (plane order, 256 bytes a row)
  alignas(16) uint8_t vf[SPLANE ? 256 * 256 : 16];
  alignas(16) uint8_t ring[kMaxBands][kRing][Slot<BPP>::kBytes];
};
// Bytes of ChipSmemT used by a CTA of nt threads.
template <int BPP, bool FLAGS, bool SPLANE>
constexpr size_t chip_smem_bytes(int nt) {
  using T = ChipSmemT<BPP, FLAGS, SPLANE>;
  return offsetof(T, ring) + size_t(nt / 16) * kRing * Slot<BPP>::kBytes;
}

// ---------------------------------------------------------------------------
// The filtered V plane in tensor memory.  Pass 2 reads back exactly the
// pixels each thread filtered in pass 1, so the plane is per-thread data:
// thread (warp w, lane l) keeps the 4 plane words of each of its band rows
// in TMEM lane 32 (w % 4) + l (the lane quarter warp w may access), columns
// 64 (w / 4) + 4 j .. + 3 for band row j (a band has at most 16 rows).  A
// CTA of up to 8 warps allocates 128 columns (64 KB), of 10 warps 256.
// Keeping the plane out of shared memory leaves a 256-thread u8 CTA about
// 40 KB of shared memory, so three of them (register-bound) share an SM;
// the block scheduler does not count tensor memory, so the host keeps the
// CTAs an SM can hold times these columns within its 512 (see
// resident_smem_bytes).
// ---------------------------------------------------------------------------
// Whether the resident kernels of a (dtype, H/S) class keep the plane in
// tensor memory (else in shared memory).
template <int DT, bool HS>
struct TmemPlane {
  static constexpr bool value = true;
};
template <int NT>
struct PlaneCols {
  static constexpr uint32_t kCols = NT <= 256 ? 128u : 256u;
};
// CTAs per SM the resident kernels of 256 threads are compiled for (the
// register budget): three for 8-bit images without H/S ranges (80
// registers), two for 16-bit images (the ring takes half of an SM's shared
// memory) and for 8-bit images with H/S ranges (which spill at 80), one for
// 16-bit images with H/S ranges (which spill at 128).  CTAs of 320
// threads: two.
template <int DT, bool HS, int NT = kThreadsNarrow>
struct ResidentCtas {
  static constexpr int k = NT != kThreadsNarrow         ? 2
                           : !TmemPlane<DT, HS>::value  ? (DT == SIL_U8 ? 2 : 1)
                           : (DT == SIL_U8 && !HS)      ? 3
                           : (DT == SIL_U16 && HS)      ? 1
                                                        : 2;
};
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
// Allocates the CTA's plane (warp 0) and publishes its address in *slot.
// All threads must call it.
__device__ __forceinline__ void plane_alloc(uint32_t* slot, uint32_t cols) {
  if (threadIdx.x < 32) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_addr(slot)),
                 "r"(cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// Frees it once every thread's plane accesses have completed.  All threads
// must call it.
__device__ __forceinline__ void plane_free(uint32_t base, uint32_t cols) {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (threadIdx.x < 32)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(base), "r"(cols)
                 : "memory");
}
// This thread's plane address (band row 0).
__device__ __forceinline__ uint32_t plane_taddr(uint32_t base) {
  const uint32_t w = threadIdx.x >> 5;
  return base + ((32u * (w & 3u)) << 16) + 64u * (w >> 2);
}
// Warp-wide (every lane, the same column): one band row's 4 plane words.
__device__ __forceinline__ void plane_st(uint32_t taddr, uint4 v) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1, %2, %3, %4};" ::"r"(taddr),
               "r"(v.x), "r"(v.y), "r"(v.z), "r"(v.w)
               : "memory");
}
__device__ __forceinline__ void plane_wait_st() {
  asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}
// Warp-wide: four band rows' plane words (16 columns), waited for.
__device__ __forceinline__ void plane_ld4rows(uint32_t taddr, uint32_t* r) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
      "%12, %13, %14, %15}, [%16];\n\t"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
}

enum { kStatLo = 0, kStatHi, kStatT, kStatN0, kStatGate, kStatN };


__device__ __forceinline__ uint32_t max3(uint32_t a, uint32_t b, uint32_t c) {
  return __vimax3_u16x2(a, b, c);
}
__device__ __forceinline__ uint32_t min3(uint32_t a, uint32_t b, uint32_t c) {
  return __vimin3_u16x2(a, b, c);
}
// a * b + c with b a runtime kernel parameter: stays an integer multiply-add,
// which issues on the multiply-add pipe, beside the min/max/permute pipe.
__device__ __forceinline__ uint32_t imad(uint32_t a, uint32_t b, uint32_t c) { return a * b + c; }
// Four bytes (each < 256) packed into a word, a | b << 8 | c << 16 | d << 24,
// as multiply-adds.
__device__ __forceinline__ uint32_t pack4(uint32_t a, uint32_t b, uint32_t c, uint32_t d,
                                          const DevParams& dp) {
  return imad(d, dp.sh24, imad(c, dp.sh16, imad(b, dp.sh8, a)));
}
// a + b + c - x - y, exact modulo 2^32 (the two subtractions as multiply-adds;
// doing the two additions as multiply-adds too was measured slower: the
// longer dependency chain costs more than the min/max pipe saves)
__device__ __forceinline__ uint32_t sum3m2(uint32_t a, uint32_t b, uint32_t c, uint32_t x,
                                           uint32_t y, const DevParams& dp) {
  return imad(y, dp.neg1, imad(x, dp.neg1, a + b + c));
}
// median of three packed u16x2 words
__device__ __forceinline__ uint32_t med3(uint32_t a, uint32_t b, uint32_t c, const DevParams& dp) {
  return sum3m2(a, b, c, max3(a, b, c), min3(a, b, c), dp);
}

// round(x * 255 / s) clamped to 255, i.e. floor((255 x + s/2) / s) for the
// uint16 scaling; the quotient of n < 2^24 by s < 2^16 is exact as
// (n * ceil(2^40 / s)) >> 40 (checked for every x on the host).
__device__ __forceinline__ uint32_t u16_to_v8(uint32_t x, const DevParams& dp) {
  const uint32_t n = x * 255u + dp.u16_half;
  const uint32_t qv = uint32_t((uint64_t(n) * dp.u16_mul) >> 40);
  return qv > 255u ? 255u : qv;
}

// ---------------------------------------------------------------------------
// Row copies into the ring.  A half-warp copies the 16-byte blocks [A, E)
// that contain a chip row (A = row start rounded down, E = row end rounded
// up) with one 16-byte asynchronous copy per lane and block, lane-contiguous;
// one commit group per row.  A lane waits for its own groups
// (cp.async.wait_group) and the half-warp then synchronises, so no thread
// spins on a flag.
// ---------------------------------------------------------------------------
// One 16-byte asynchronous copy when pred is nonzero (a predicated
// instruction, no branch).
__device__ __forceinline__ void cp16_if(uint32_t dst, uintptr_t src, uint32_t pred) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %2, 0;\n\t"
      "@p cp.async.cg.shared.global [%0], [%1], 16;\n\t}" ::"r"(dst),
      "l"(src), "r"(pred) : "memory");
}
template <int SLOT_BYTES>
__device__ __forceinline__ void copy_row_async(uint8_t* slot, const uint8_t* rowptr,
                                               int row_bytes, int q, bool go) {
  const uintptr_t a = reinterpret_cast<uintptr_t>(rowptr);
  const uintptr_t A = a & ~uintptr_t(15);
  const int nvec = go ? int(((a + uintptr_t(row_bytes) + 15) & ~uintptr_t(15)) - A) >> 4 : 0;
  const uint32_t dst = static_cast<uint32_t>(__cvta_generic_to_shared(slot));
#pragma unroll
  for (int t = 0; t < (SLOT_BYTES / 16 + 15) / 16; ++t) {
    const int v = q + 16 * t;
    cp16_if(dst + 16u * uint32_t(v), A + 16u * uintptr_t(v), v < nvec);
  }
}
// A full-width row (256 px): every lane copies the same number of blocks,
// and the one extra block of a row that does not start on a 16-byte boundary
// (m != 0) is lane 0's.
template <int BPP>
__device__ __forceinline__ void copy_row_full(uint8_t* slot, const uint8_t* rowptr, uint32_t m,
                                              int q, bool go) {
  constexpr int kBlocks = BPP * 256 / 16;  // a multiple of 16
  const uintptr_t A = (reinterpret_cast<uintptr_t>(rowptr) & ~uintptr_t(15)) + 16u * uintptr_t(q);
  const uint32_t dst = static_cast<uint32_t>(__cvta_generic_to_shared(slot)) + 16u * uint32_t(q);
  if constexpr (kBlocks == 48) {
    // one predicate for the lane's three copies
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %2, 0;\n\t"
        "@p cp.async.cg.shared.global [%0], [%1], 16;\n\t"
        "@p cp.async.cg.shared.global [%0+256], [%1+256], 16;\n\t"
        "@p cp.async.cg.shared.global [%0+512], [%1+512], 16;\n\t}" ::"r"(dst),
        "l"(A), "r"(uint32_t(go)) : "memory");
  } else {
#pragma unroll
    for (int t = 0; t < kBlocks / 16; ++t) cp16_if(dst + 256u * uint32_t(t), A + 256u * uintptr_t(t), go);
  }
  cp16_if(dst + 16u * kBlocks, A + 16u * kBlocks, go && q == 0 && m != 0);
}
__device__ __forceinline__ void commit_rows() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void wait_rows() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// ---------------------------------------------------------------------------
// Decode of a lane's 16 pixels from a staged row.  The lane's bytes start at
// slot offset m + 16 BPP q; the words are read from the aligned word below
// and, unless m & 3 == 0, funnel-shifted by 8 (m & 3) bits (the same shift
// for all lanes of the half-warp) so that the gathers below see the row's
// first byte at byte 0 (S = 0).
// ---------------------------------------------------------------------------
// u8: pixel j is bytes 3j..3j+2 after shift S; pair (j, j+8) is 24 bytes = 6
// words apart at the same byte position, so one PRMT lifts both channel bytes
// into the high bytes of a u16x2 word.
template <int S>
__device__ __forceinline__ void gather_u8(const uint32_t* v, uint32_t* V, uint32_t (*G)[3]) {
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    uint32_t g[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const int b = S + 3 * i + c;
      const int wi = b >> 2, p = b & 3;
      const uint32_t sel = p | (p << 4) | ((4 + p) << 8) | ((4 + p) << 12);
      g[c] = __byte_perm(v[wi], v[wi + 6], sel);
      if (G) G[i][c] = g[c];
    }
    V[i] = max3(g[0], g[1], g[2]);
  }
}
// u16: pixel j is bytes 6j..6j+5 after shift S (even); pair (j, j+8) is 48
// bytes = 12 words apart at the same half-word position.
template <int S>
__device__ __forceinline__ void gather_u16(const uint32_t* v, uint32_t* R, uint32_t (*G)[3]) {
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    uint32_t g[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const int b = S + 6 * i + 2 * c;
      const int wi = b >> 2, hh = (b >> 1) & 1;
      g[c] = __byte_perm(v[wi], v[wi + 12], hh ? 0x7632u : 0x5410u);
      if (G) G[i][c] = g[c];
    }
    R[i] = max3(g[0], g[1], g[2]);
  }
}

// Lane value of column j (0..15) of an interleaved segment (16-bit lane).
__device__ __forceinline__ uint32_t seg_get(const uint32_t* V, int j) {
  uint32_t r = 0;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    if (j == i) r = V[i] & 0xFFFFu;
    if (j == i + 8) r = V[i] >> 16;
  }
  return r;
}

// Class mask of the H and S ranges for one pixel (bit k = class k), without
// division: S >= a  <=>  510 d + V >= 2 V a  (V > 0), etc.  H in [0,179] as
// round(hue_degrees / 2) with 180 folded to 0.
__device__ __forceinline__ uint32_t hs_mask(int r, int g, int b, const DevParams& dp) {
  const int v = max(r, max(g, b));
  const int mn = min(r, min(g, b));
  const int d = v - mn;
  // n = hue_degrees * d in [0, 360 d)
  int n = 0;
  if (d > 0) {
    if (v == r)
      n = 60 * (g - b);
    else if (v == g)
      n = 120 * d + 60 * (b - r);
    else
      n = 240 * d + 60 * (r - g);
    if (n < 0) n += 360 * d;
  }
  const bool wraps = d > 0 && (n + d) >= 360 * d;  // rounds to 180 -> 0
  uint32_t mask = 0;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const int sl = dp.lo[k][1], sh = dp.hi[k][1];
    bool s_ok;
    if (v == 0)
      s_ok = (sl == 0);
    else
      s_ok = (510 * d + v >= 2 * v * sl) && (510 * d + v < 2 * v * (sh + 1));
    const int hl = dp.lo[k][0], hh = dp.hi[k][0];
    bool h_ok;
    if (d == 0 || wraps)
      h_ok = (hl == 0);  // H = 0
    else
      h_ok = (n + d >= 2 * d * hl) && (n + d < 2 * d * (hh + 1));
    if (s_ok && h_ok) mask |= 1u << k;
  }
  return mask;
}

template <int DT>
struct Px {
  static constexpr int BPP = DT == SIL_U8 ? 3 : 6;
  static constexpr int NW = DT == SIL_U8 ? 13 : 25;  // words a lane reads
};

// Decode the lane's 16 pixels of the staged row in `slot` (row data starting
// at byte m of the slot) into 8 interleaved V words; F[0], F[1] = per-pixel
// flags of columns 0-7 / 8-15 (nibble: bits 0-2 H/S class mask, bit 3
// nodata) for the variants that need them.  A4: every row of the chip starts
// on a 4-byte boundary (m & 3 == 0), so the realigning shift is left out.
template <int DT, bool HS, bool A4>
__device__ __forceinline__ void decode_row(const uint8_t* slot, int m, int q, int nvalid,
                                           const DevParams& dp, uint32_t* V, uint32_t* F) {
  constexpr int NW = Px<DT>::NW;
  uint32_t G[8][3];
  constexpr bool kNeedG = HS;
  F[0] = F[1] = 0;
  if (DT == SIL_U8) {
    const uint32_t* base = reinterpret_cast<const uint32_t*>(slot) + (m >> 2) + 4 * Px<DT>::BPP * q;
    uint32_t v[NW];
#pragma unroll
    for (int k = 0; k < NW; ++k) v[k] = base[k];
    if (!A4) {
      // realign to the row's first byte: one funnel shift per word, the same
      // for every lane (no per-case code, no divergence between the two
      // half-warps of a warp, whose rows can start at different offsets)
      const uint32_t sh = 8u * uint32_t(m & 3);
#pragma unroll
      for (int k = 0; k < NW - 1; ++k) v[k] = __funnelshift_r(v[k], v[k + 1], sh);
    }
    gather_u8<0>(v, V, kNeedG ? G : nullptr);
  } else {
    const uint32_t* base = reinterpret_cast<const uint32_t*>(slot) + (m >> 2) + 4 * Px<DT>::BPP * q;
    uint32_t v[NW];
#pragma unroll
    for (int k = 0; k < NW; ++k) v[k] = base[k];
    uint32_t R[8];
    if (!A4) {
      const uint32_t sh = 8u * uint32_t(m & 2);
#pragma unroll
      for (int k = 0; k < NW - 1; ++k) v[k] = __funnelshift_r(v[k], v[k + 1], sh);
    }
    gather_u16<0>(v, R, kNeedG ? G : nullptr);
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const uint32_t x0 = R[i] & 0xFFFFu, x1 = R[i] >> 16;
      V[i] = (u16_to_v8(x0, dp) << 8) | (u16_to_v8(x1, dp) << 24);
      F[0] |= (x0 == 0 ? 8u : 0u) << (4 * i);
      F[1] |= (x1 == 0 ? 8u : 0u) << (4 * i);
    }
  }
  if (HS) {
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      int c0[3], c1[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        if (DT == SIL_U8) {
          c0[c] = (G[i][c] >> 8) & 0xFF;
          c1[c] = G[i][c] >> 24;
        } else {
          c0[c] = int(u16_to_v8(G[i][c] & 0xFFFFu, dp));
          c1[c] = int(u16_to_v8(G[i][c] >> 16, dp));
        }
      }
      const int ri = dp.bgr ? 2 : 0, bi = dp.bgr ? 0 : 2;
      F[0] |= hs_mask(c0[ri], c0[1], c0[bi], dp) << (4 * i);
      F[1] |= hs_mask(c1[ri], c1[1], c1[bi], dp) << (4 * i);
    }
  }
  if (nvalid < 16 && nvalid > 0) {
    // replicate the chip's last column into the lane's columns beyond it
    // (the median window is clamped to the chip)
    const uint32_t rep = seg_get(V, nvalid - 1);
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      if (i >= nvalid) V[i] = (V[i] & 0xFFFF0000u) | rep;
      if (i + 8 >= nvalid) V[i] = (V[i] & 0x0000FFFFu) | (rep << 16);
    }
  }
}

// Edge words of a decoded row: EL = [col -1, col 7], ER = [col 8, col 16],
// clamped to the chip (replicated border).  Shuffles stay inside the
// half-warp (hmask).
__device__ __forceinline__ void edge_words(const uint32_t* V, int q, int w, uint32_t hmask,
                                           uint32_t& EL, uint32_t& ER) {
  const uint32_t up = __shfl_up_sync(hmask, V[7], 1, 16);
  const uint32_t dn = __shfl_down_sync(hmask, V[0], 1, 16);
  const uint32_t srcL = (q == 0) ? (V[0] << 16) : up;            // hi lane = col -1
  const uint32_t srcR = (16 * q + 16 >= w) ? (V[7] >> 16) : dn;  // lo lane = col 16
  EL = __byte_perm(srcL, V[7], 0x5432);
  ER = __byte_perm(V[0], srcR, 0x5432);
}

// One decoded row of a lane's 16-pixel segment.
struct RowBuf {
  uint32_t v[8];
  uint32_t eL, eR;
  uint32_t f[2];
};

// Output row y from the window rows (M, Z, P) = (y-1, y, y+1): 3x3 median as
// med3(max3 of column minima, med3 of column medians, min3 of column maxima),
// histogram of Vf, Vf plane row (tensor memory at taddr).  CHECK: the row
// may lie past this half-warp's band (live false: the other half-warp of
// the warp has one row more, and the plane store is warp-wide), so the
// histogram and the flags are skipped then.
template <bool kFlags, int DT, bool FULL, bool CHECK, class SM>
__device__ __forceinline__ void emit_row(const RowBuf& M, const RowBuf& Z, const RowBuf& P,
                                         int y, int q, int nvalid, bool use_median,
                                         const DevParams& dp, SM& sm, uint32_t& n_nodata,
                                         uint32_t taddr, bool live) {
  uint32_t out[8];
  if (use_median) {
    uint32_t L[10], X[10], C[10];
#define SIL_SORT3(k, a, b, c)             \
  {                                       \
    L[k] = min3(a, b, c);                 \
    X[k] = max3(a, b, c);                 \
    C[k] = sum3m2(a, b, c, L[k], X[k], dp);  \
  }
    SIL_SORT3(0, M.eL, Z.eL, P.eL);
#pragma unroll
    for (int i = 0; i < 8; ++i) SIL_SORT3(i + 1, M.v[i], Z.v[i], P.v[i]);
    SIL_SORT3(9, M.eR, Z.eR, P.eR);
#undef SIL_SORT3
#pragma unroll
    for (int i = 0; i < 8; i += 2) {
      // outputs i and i+1 share the middle pair of column medians:
      // med3(x, b, c) = max(min(b, c), min(max(b, c), x))
      const uint32_t pl = __vminu2(C[i + 1], C[i + 2]), ph = __vmaxu2(C[i + 1], C[i + 2]);
      const uint32_t mi0 = __vmaxu2(pl, __vminu2(ph, C[i]));
      const uint32_t mi1 = __vmaxu2(pl, __vminu2(ph, C[i + 3]));
      out[i] = med3(max3(L[i], L[i + 1], L[i + 2]), mi0, min3(X[i], X[i + 1], X[i + 2]), dp);
      out[i + 1] = med3(max3(L[i + 1], L[i + 2], L[i + 3]), mi1, min3(X[i + 1], X[i + 2], X[i + 3]), dp);
    }
  } else {
#pragma unroll
    for (int i = 0; i < 8; ++i) out[i] = Z.v[i];
  }
  // Histogram of Vf over valid, non-nodata pixels; the bin index is byte 1
  // (low lane) or byte 3 (high lane) of each word.
  uint32_t* hist = sm.st.hist;
  if (CHECK && !live) {
    // a row past the band: filtered only for the warp-wide plane store
  } else if (!kFlags && FULL) {
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      // low lane: byte 1 by a permute; high lane: byte 3 = the high word of
      // out * 2^8, a multiply (the two go to different pipes)
      atomicAdd(&hist[__byte_perm(out[i], 0, 0x4441)], 1u);
      atomicAdd(&hist[__umulhi(out[i], dp.sh8)], 1u);
    }
  } else if (!kFlags) {
    // a chip narrower than 256: the same adds in every lane (no branch that
    // would split each half-warp), pixels past the chip's last column
    // counted into the lane's own unread bin
    const uint32_t unread = 256u + (threadIdx.x & 31u);
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      atomicAdd(&hist[i < nvalid ? __byte_perm(out[i], 0, 0x4441) : unread], 1u);
      atomicAdd(&hist[i + 8 < nvalid ? __byte_perm(out[i], 0, 0x4443) : unread], 1u);
    }
  } else {
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const bool nd0 = kFlags && ((Z.f[0] >> (4 * i + 3)) & 1u);
      const bool nd1 = kFlags && ((Z.f[1] >> (4 * i + 3)) & 1u);
      if (i < nvalid && !nd0) atomicAdd(&hist[__byte_perm(out[i], 0, 0x4441)], 1u);
      if (i + 8 < nvalid && !nd1) atomicAdd(&hist[__byte_perm(out[i], 0, 0x4443)], 1u);
      if (DT == SIL_U16) {
        n_nodata += (i < nvalid && nd0) ? 1u : 0u;
        n_nodata += (i + 8 < nvalid && nd1) ? 1u : 0u;
      }
    }
  }
  // Vf plane (plane order: word k = [c2k, c2k+1, c2k+8, c2k+9])
  uint4 pw;
  pw.x = __byte_perm(out[0], out[1], 0x7351);
  pw.y = __byte_perm(out[2], out[3], 0x7351);
  pw.z = __byte_perm(out[4], out[5], 0x7351);
  pw.w = __byte_perm(out[6], out[7], 0x7351);
  if (kFlags && (!CHECK || live)) {
    sm.flags[y][q][0] = Z.f[0];
    sm.flags[y][q][1] = Z.f[1];
  }
  if constexpr (SM::kSmemPlane) {
    if (!CHECK || live) *reinterpret_cast<uint4*>(&sm.vf[y * 256 + 16 * q]) = pw;
  } else {
    if (kFlags || CHECK) __syncwarp();  // the lanes took different branches above
    plane_st(taddr, pw);
  }
}

// The rows one half-warp band streams for one chip: output rows [r0, r1)
// of a chip of h rows and w columns whose pixel (0, 0) is at chip0; streamed
// row k (k = 0 .. r1 - r0 + 1) is chip row clamp(r0 + k - 1, 0, h - 1).
struct Band {
  const uint8_t* chip0;
  int64_t pitch;
  int h, w, r0, r1;
};

__device__ __forceinline__ const uint8_t* band_row(const Band& b, int k) {
  return b.chip0 + int64_t(min(max(b.r0 + k - 1, 0), b.h - 1)) * b.pitch;
}

// Copy streamed row k into slot when go (predicated, no branch); m = the
// row's offset from the 16-byte block below it.  FULL: the chip is 256 wide.
template <int BPP, bool FULL>
__device__ __forceinline__ void band_issue(const Band& b, uint8_t* slot, int k, uint32_t& m,
                                           bool go, int q) {
  const uint8_t* src = band_row(b, k);
  m = uint32_t(reinterpret_cast<uintptr_t>(src)) & 15u;
  if (FULL)
    copy_row_full<BPP>(slot, src, m, q, go);
  else
    copy_row_async<Slot<BPP>::kBytes>(slot, src, BPP * b.w, q, go);
}

// Pass 1 of one half-warp's band: output rows r0..r1-1 of the chip.  The
// band streams its rows through its ring of kRing = 3 row slots: step k
// waits for streamed row k, decodes it from slot k mod 3 and refills that
// slot with row k + 3.  The row loop is unrolled by three so that the window
// rows (y-1, y, y+1) rotate through three register sets and each slot index
// is a constant.  FULL: every lane has 16 columns (chip width 256).  A4:
// every row of the chip starts on a 4-byte boundary.  The two half-warps of
// a warp step through the same number of rows, nmax (their bands differ by
// at most one row, nmin <= r1 - r0 <= nmax), because the plane store is a
// warp-wide instruction: a half-warp's extra row filters a clamped row of
// the chip and stores it to a plane column that pass 2 does not read.
template <int DT, bool HS, bool FULL, bool A4, class SM>
__device__ __forceinline__ void band_pass1(const Band& b, const DevParams& dp, SM& sm,
                                           uint32_t& n_nodata, int nmin, int nmax,
                                           uint32_t taddr) {
  constexpr int BPP = Px<DT>::BPP;
  constexpr bool kFlags = HS || DT == SIL_U16;
  constexpr int SB = Slot<BPP>::kBytes;
  static_assert(kRing == 3, "the row loop is unrolled by the ring size");
  const int lane = threadIdx.x & 31, band = threadIdx.x >> 4;
  const int q = lane & 15;
  const uint32_t hmask = 0xFFFFu << (lane & 16);
  const int w = b.w, r0 = b.r0, own = b.r1 - b.r0;
  const int nvalid = FULL ? 16 : min(max(w - 16 * q, 0), 16);
  const bool use_median = dp.filter && dp.median;
  const int nrows = nmax + 2;  // streamed rows 0 .. nmax + 1
  uint8_t* const s0 = sm.ring[band][0];
  uint8_t* const s1 = s0 + SB;
  uint8_t* const s2 = s1 + SB;
  uint32_t m0, m1, m2;
  band_issue<BPP, FULL>(b, s0, 0, m0, true, q);
  commit_rows();
  band_issue<BPP, FULL>(b, s1, 1, m1, true, q);
  commit_rows();
  band_issue<BPP, FULL>(b, s2, 2, m2, nrows > 2, q);
  commit_rows();
  // step k: decode row k from its slot into B, refill the slot with row k + 3
  auto step = [&](RowBuf& B, uint8_t* slot, uint32_t& m, int k) {
    wait_rows<kRing - 1>();  // this lane's copies of row k have landed
    __syncwarp(hmask);       // ... and every other lane's of the band
    decode_row<DT, HS, A4>(slot, int(m), q, nvalid, dp, B.v, B.f);
    __syncwarp(hmask);  // the slot is free again
    band_issue<BPP, FULL>(b, slot, k + kRing, m, k + kRing < nrows, q);
    commit_rows();
    edge_words(B.v, q, w, hmask, B.eL, B.eR);
  };
#define SIL_EMIT(CHK, M, Z, P, J) \
  emit_row<kFlags, DT, FULL, CHK>(M, Z, P, r0 + (J), q, nvalid, use_median, dp, sm, n_nodata, \
                                  taddr + 4u * uint32_t(J), (J) < own)
  RowBuf B0, B1, B2;
  step(B0, s0, m0, 0);
  step(B1, s1, m1, 1);
  int j = 0;
  for (; j + 3 <= nmin; j += 3) {
    step(B2, s2, m2, j + 2);
    SIL_EMIT(false, B0, B1, B2, j);
    step(B0, s0, m0, j + 3);
    SIL_EMIT(false, B1, B2, B0, j + 1);
    step(B1, s1, m1, j + 4);
    SIL_EMIT(false, B2, B0, B1, j + 2);
  }
  // at most three rows are left (nmin - j <= 2, nmax - nmin <= 1)
  if (j < nmax) {
    step(B2, s2, m2, j + 2);
    SIL_EMIT(true, B0, B1, B2, j);
    if (j + 1 < nmax) {
      step(B0, s0, m0, j + 3);
      SIL_EMIT(true, B1, B2, B0, j + 1);
      if (j + 2 < nmax) {
        step(B1, s1, m1, j + 4);
        SIL_EMIT(true, B2, B0, B1, j + 2);
      }
    }
  }
#undef SIL_EMIT
  // every copy this band issued for the chip has been waited for (the
  // groups committed after the last row's copy are empty)
}

// ---------------------------------------------------------------------------
// Chip statistics (one warp): lo, hi, Otsu t, n0, gate.  Exact: the score
// (S_T w - N s)^2 / (w (N - w)) is compared by 128-bit cross products; ties
// keep the smallest t; no split -> t = lo.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void chip_stats_warp(ChipStat& sm, const DevParams& dp,
                                                uint32_t N) {
  const int lane = threadIdx.x & 31;
  uint32_t c[8];
  uint64_t cnt = 0, sum = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    c[k] = sm.hist[8 * lane + k];
    cnt += c[k];
    sum += uint64_t(8 * lane + k) * c[k];
  }
  // inclusive scans
  uint64_t pc = cnt, ps = sum;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const uint64_t a = __shfl_up_sync(0xffffffffu, pc, off);
    const uint64_t b = __shfl_up_sync(0xffffffffu, ps, off);
    if (lane >= off) { pc += a; ps += b; }
  }
  const uint64_t ST = __shfl_sync(0xffffffffu, ps, 31);
  uint64_t w = pc - cnt, s = ps - sum;  // exclusive prefix
  int best_t = -1;
  unsigned __int128 best_num = 0;
  uint64_t best_den = 1;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const int t = 8 * lane + k;
    w += c[k];
    s += uint64_t(t) * c[k];
    if (t <= 254 && w > 0 && w < N) {
      const int64_t diff = int64_t(ST * w) - int64_t(uint64_t(N) * s);
      const uint64_t ad = diff < 0 ? uint64_t(-diff) : uint64_t(diff);
      const unsigned __int128 num = (unsigned __int128)ad * ad;
      const uint64_t den = w * (uint64_t(N) - w);
      if (best_t < 0 || num * best_den > best_num * den) {
        best_t = t;
        best_num = num;
        best_den = den;
      }
    }
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const uint64_t on_lo = __shfl_xor_sync(0xffffffffu, uint64_t(best_num), off);
    const uint64_t on_hi = __shfl_xor_sync(0xffffffffu, uint64_t(best_num >> 64), off);
    const uint64_t od = __shfl_xor_sync(0xffffffffu, best_den, off);
    const int ot = __shfl_xor_sync(0xffffffffu, best_t, off);
    const unsigned __int128 on = ((unsigned __int128)on_hi << 64) | on_lo;
    bool take = false;
    if (ot >= 0) {
      if (best_t < 0) {
        take = true;
      } else {
        const unsigned __int128 lhs = on * best_den, rhs = best_num * od;
        take = lhs > rhs || (lhs == rhs && ot < best_t);
      }
    }
    if (take) {
      best_t = ot;
      best_num = on;
      best_den = od;
    }
  }
  // lo / hi
  bool any = false;
  int my_lo = 255, my_hi = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    if (c[k]) {
      any = true;
      my_lo = min(my_lo, 8 * lane + k);
      my_hi = max(my_hi, 8 * lane + k);
    }
  }
  const uint32_t bal = __ballot_sync(0xffffffffu, any);
  int lo = 0, hi = 0;
  if (bal) {
    lo = __shfl_sync(0xffffffffu, my_lo, __ffs(bal) - 1);
    hi = __shfl_sync(0xffffffffu, my_hi, 31 - __clz(bal));
  }
  const int t = best_t < 0 ? lo : best_t;
  // n0 = #(Vf <= t)
  uint32_t mine = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k)
    if (8 * lane + k <= t) mine += c[k];
  const uint32_t n0 = __reduce_add_sync(0xffffffffu, mine);
  const uint32_t n1 = N - n0;
  const int gate = (hi - lo >= dp.mm_min_range) &&
                   (uint64_t(dp.frac_den) * n0 >= N) &&
                   (uint64_t(dp.frac_den) * n1 >= N) && N > 0;
  if (lane == 0) {
    sm.stat[kStatLo] = lo;
    sm.stat[kStatHi] = hi;
    sm.stat[kStatT] = t;
    sm.stat[kStatN0] = int(n0);
    sm.stat[kStatGate] = gate;
    sm.stat[kStatN] = int(N);
  }
}

// The same statistics computed by all threads of the CTA (thread t < 256
// owns histogram bin t), for chips of at most 65536 pixels: block-wide
// prefix sums, one score per thread, block-wide argmax.  Scores:
// D = S_T w - N s < 2^40, num = D^2 < 2^80, den = w (N - w) <= 2^32, cross
// products < 2^112.  Contains __syncthreads(); every thread must call it.
__device__ __forceinline__ bool better(uint64_t nlo_a, uint32_t nhi_a, uint32_t den_a, int t_a,
                                       uint64_t nlo_b, uint32_t nhi_b, uint32_t den_b, int t_b) {
  // is candidate a strictly better than b (ties: smaller t)?
  if (t_a < 0) return false;
  if (t_b < 0) return true;
  const unsigned __int128 na = ((unsigned __int128)nhi_a << 64) | nlo_a;
  const unsigned __int128 nb = ((unsigned __int128)nhi_b << 64) | nlo_b;
  const unsigned __int128 l = na * den_b, r = nb * den_a;
  return l > r || (l == r && t_a < t_b);
}

__device__ __forceinline__ void chip_stats_block(ChipStat& st, StatScratch& sc,
                                                 const DevParams& dp, uint32_t N) {
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const uint32_t hv = tid < 256 ? st.hist[tid] : 0u;
  uint32_t c = hv, s = uint32_t(tid) * hv;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const uint32_t a = __shfl_up_sync(0xffffffffu, c, off);
    const uint32_t b = __shfl_up_sync(0xffffffffu, s, off);
    if (lane >= off) {
      c += a;
      s += b;
    }
  }
  const uint32_t nz = __ballot_sync(0xffffffffu, hv != 0);
  if (lane == 31) {
    sc.wc[wid] = c;
    sc.ws[wid] = s;
  }
  if (lane == 0) {
    sc.lo[wid] = nz ? wid * 32 + __ffs(nz) - 1 : 256;
    sc.hi[wid] = nz ? wid * 32 + 31 - __clz(nz) : -1;
  }
  __syncthreads();
  // only the first 8 warps own histogram bins (threads 256.. contribute
  // nothing to the sums, the extremes or the scores)
  uint32_t ST = 0, pc = 0, ps = 0;
  int lo = 256, hi = -1;
#pragma unroll
  for (int k = 0; k < kBinWarps; ++k) {
    if (k < wid) {
      pc += sc.wc[k];
      ps += sc.ws[k];
    }
    ST += sc.ws[k];
    lo = min(lo, sc.lo[k]);
    hi = max(hi, sc.hi[k]);
  }
  c += pc;  // pixels with Vf <= tid
  s += ps;
  if (hi < 0) {  // no pixel: the statistics of an empty chip
    lo = 0;
    hi = 0;
  }
  int t = -1;
  uint64_t nlo = 0;
  uint32_t nhi = 0, den = 0;
  float f = -1.f;
  if (tid <= 254 && c > 0 && c < N) {
    const uint64_t D = uint64_t(ST) * c - uint64_t(N) * s;  // >= 0
    const unsigned __int128 num = (unsigned __int128)D * D;
    nlo = uint64_t(num);
    nhi = uint32_t(num >> 64);
    den = c * (N - c);
    t = tid;
    const float fd = float(D);
    f = fd * fd / float(den);
  }
  // Float pre-filter: each float score is within 3e-7 (relative) of the
  // exact one (three roundings and two conversions of 2^-24 each), so every
  // threshold whose exact score is the largest has a float score within
  // 4e-6 of the largest float score.  Only those candidates are compared
  // exactly; when there is one, it is the answer.
  float m = f;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, off));
  if (lane == 0) sc.fmax[wid] = m;
  __syncthreads();
  float M = -1.f;
#pragma unroll
  for (int k = 0; k < kBinWarps; ++k) M = fmaxf(M, sc.fmax[k]);
  const bool cand = t >= 0 && f >= M * (1.0f - 4e-6f);
  const int ncand = __syncthreads_count(cand);
  if (ncand <= 1) {
    // one candidate, or none (no split: t = lo); that thread's inclusive
    // prefix count is n0
    if (ncand == 1 ? cand : tid == lo) {
      const uint32_t n0 = c, n1 = N - n0;
      st.stat[kStatLo] = lo;
      st.stat[kStatHi] = hi;
      st.stat[kStatT] = tid;
      st.stat[kStatN] = int(N);
      st.stat[kStatN0] = int(n0);
      st.stat[kStatGate] = (hi - lo >= dp.mm_min_range) && (uint64_t(dp.frac_den) * n0 >= N) &&
                           (uint64_t(dp.frac_den) * n1 >= N) && N > 0;
    }
    __syncthreads();
    return;
  }
  // several candidates (ties or near-ties): exact argmax among them
  if (!cand) t = -1;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const uint64_t o_lo = __shfl_xor_sync(0xffffffffu, nlo, off);
    const uint32_t o_hi = __shfl_xor_sync(0xffffffffu, nhi, off);
    const uint32_t o_d = __shfl_xor_sync(0xffffffffu, den, off);
    const int o_t = __shfl_xor_sync(0xffffffffu, t, off);
    if (better(o_lo, o_hi, o_d, o_t, nlo, nhi, den, t)) {
      nlo = o_lo;
      nhi = o_hi;
      den = o_d;
      t = o_t;
    }
  }
  if (lane == 0) {
    sc.bnum_lo[wid] = nlo;
    sc.bnum_hi[wid] = nhi;
    sc.bden[wid] = den;
    sc.bt[wid] = t;
  }
  __syncthreads();
  if (wid == 0) {
    const bool own = lane < kBinWarps;
    nlo = own ? sc.bnum_lo[lane] : 0;
    nhi = own ? sc.bnum_hi[lane] : 0;
    den = own ? sc.bden[lane] : 0;
    t = own ? sc.bt[lane] : -1;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      const uint64_t o_lo = __shfl_xor_sync(0xffffffffu, nlo, off);
      const uint32_t o_hi = __shfl_xor_sync(0xffffffffu, nhi, off);
      const uint32_t o_d = __shfl_xor_sync(0xffffffffu, den, off);
      const int o_t = __shfl_xor_sync(0xffffffffu, t, off);
      if (better(o_lo, o_hi, o_d, o_t, nlo, nhi, den, t)) {
        nlo = o_lo;
        nhi = o_hi;
        den = o_d;
        t = o_t;
      }
    }
    if (lane == 0) {
      if (hi < 0) {
        lo = 0;
        hi = 0;
      }
      st.stat[kStatLo] = lo;
      st.stat[kStatHi] = hi;
      st.stat[kStatT] = t < 0 ? lo : t;
      st.stat[kStatN] = int(N);
    }
  }
  __syncthreads();
  const int tt = st.stat[kStatT];
  if (tid == tt) sc.n0 = c;
  __syncthreads();
  if (tid == 0) {
    const uint32_t n0 = sc.n0, n1 = N - n0;
    const int lo2 = st.stat[kStatLo], hi2 = st.stat[kStatHi];
    st.stat[kStatN0] = int(n0);
    st.stat[kStatGate] = (hi2 - lo2 >= dp.mm_min_range) && (uint64_t(dp.frac_den) * n0 >= N) &&
                         (uint64_t(dp.frac_den) * n1 >= N) && N > 0;
  }
  __syncthreads();
}

// V' of filtered value vf: the gated min-max stretch (round half up) and the
// truncation (Sec. III-B); vf itself when the filter is off.
__device__ __forceinline__ int vprime_value(int vf, const ChipStat& sm, const DevParams& dp) {
  int vp = vf;
  if (dp.filter) {
    const int lo = sm.stat[kStatLo], hi = sm.stat[kStatHi];
    if (sm.stat[kStatGate]) {
      const int x = min(max(vf, lo), hi);
      const int rg = hi - lo;
      vp = ((x - lo) * 510 + rg) / (2 * rg);
    }
    vp = min(vp, dp.v_trunc);
  }
  return vp;
}

// Label table entry for filtered value vf (thread per value).
// Non-H/S variant: the label code.  H/S variant: bits 0-2 = classes whose V
// range holds V', bit 3 = absdiff override.
template <bool HS>
__device__ __forceinline__ uint32_t lut_entry(int vf, const ChipStat& sm,
                                              const DevParams& dp) {
  const int vp = vprime_value(vf, sm, dp);
  uint32_t vm = 0;
#pragma unroll
  for (int k = 0; k < 3; ++k)
    if (vp >= dp.lo[k][2] && vp <= dp.hi[k][2]) vm |= 1u << k;
  const bool ovr = dp.filter && abs(vp - vf) > dp.max_shift;
  if (HS) return vm | (ovr ? 8u : 0u);
  if (ovr) return 3u;
  return (vm & 1u) ? 0u : (vm & 2u) ? 1u : (vm & 4u) ? 2u : 3u;
}

// ---------------------------------------------------------------------------
// Pass 2: Vf plane -> labels (+ per-pixel counts for the H/S variant).
// ---------------------------------------------------------------------------
__device__ __forceinline__ void store_row16(uint8_t* dst, int nvalid, uint4 lab) {
  const uintptr_t a = reinterpret_cast<uintptr_t>(dst);
  if (nvalid == 16) {
    if ((a & 15) == 0) {
      *reinterpret_cast<uint4*>(dst) = lab;
      return;
    }
    if ((a & 3) == 0) {
      uint32_t* d = reinterpret_cast<uint32_t*>(dst);
      d[0] = lab.x;
      d[1] = lab.y;
      d[2] = lab.z;
      d[3] = lab.w;
      return;
    }
  }
  const uint32_t wv[4] = {lab.x, lab.y, lab.z, lab.w};
#pragma unroll
  for (int j = 0; j < 16; ++j)
    if (j < nvalid) dst[j] = uint8_t(wv[j >> 2] >> (8 * (j & 3)));
}

// Store of a lane's 16 labels.  store: every label row of the chip starts
// on a 16-byte (16) or 4-byte (4) boundary, or neither (1); known per chip
// (a branch every lane of the chip takes alike).  Lanes with fewer than 16
// columns left (the right edge of a narrow chip) store bytes.
__device__ __forceinline__ void store_labels(uint8_t* dst, int nvalid, uint4 lab, int store) {
  if (store == 16 && nvalid == 16) {
    *reinterpret_cast<uint4*>(dst) = lab;
  } else if (store == 4 && nvalid == 16) {
    uint32_t* d = reinterpret_cast<uint32_t*>(dst);
    d[0] = lab.x;
    d[1] = lab.y;
    d[2] = lab.z;
    d[3] = lab.w;
  } else {
    const uint32_t wv[4] = {lab.x, lab.y, lab.z, lab.w};
#pragma unroll
    for (int j = 0; j < 16; ++j)
      if (j < nvalid) dst[j] = uint8_t(wv[j >> 2] >> (8 * (j & 3)));
  }
}

// Rows are read from the plane four at a time (one warp-wide load of 16
// columns; the warp steps through nmax rows, see band_pass1); rows past the
// half-warp's band and lanes past the chip's last column store nothing.
template <int DT, bool HS, class SM>
__device__ __forceinline__ void band_pass2(uint8_t* labels, int64_t lpitch, int64_t y0, int64_t x0,
                                           int w, int r0, int r1, int nmax, uint32_t taddr,
                                           const uint8_t* lut, const SM& sm, uint32_t* cnt,
                                           const DevParams& dp, int store) {
  constexpr bool kFlags = HS || DT == SIL_U16;
  const int q = threadIdx.x & 15;
  const int nvalid = min(max(w - 16 * q, 0), 16);
  const int own = nvalid > 0 ? r1 - r0 : 0;
  uint8_t* dst = labels ? labels + (y0 + r0) * lpitch + x0 + 16 * q : nullptr;
  for (int j0 = 0; j0 < nmax; j0 += 4) {
    uint32_t pr[16];
    if constexpr (SM::kSmemPlane) {
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        if (j0 + i < own) {
          const uint4 pw = *reinterpret_cast<const uint4*>(&sm.vf[(r0 + j0 + i) * 256 + 16 * q]);
          pr[4 * i] = pw.x;
          pr[4 * i + 1] = pw.y;
          pr[4 * i + 2] = pw.z;
          pr[4 * i + 3] = pw.w;
        }
      }
    } else {
      __syncwarp();
      plane_ld4rows(taddr + 4u * uint32_t(j0), pr);
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
    if (j0 + i >= own) break;
    // one row's table lookups at a time (kept from being hoisted above the
    // previous row's stores, which would hold 64 lookups in registers)
    asm volatile("" ::: "memory");
    const int y = r0 + j0 + i;
    // plane word k holds columns (2k, 2k+1, 2k+8, 2k+9)
    const uint32_t p[4] = {pr[4 * i], pr[4 * i + 1], pr[4 * i + 2], pr[4 * i + 3]};
    uint32_t l[16];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      l[2 * k] = lut[__byte_perm(p[k], 0, 0x4440)];
      l[2 * k + 1] = lut[__byte_perm(p[k], 0, 0x4441)];
      l[2 * k + 8] = lut[__byte_perm(p[k], 0, 0x4442)];
      l[2 * k + 9] = lut[__umulhi(p[k], dp.sh8)];  // byte 3
    }
    if (kFlags) {
      const uint32_t f0 = sm.flags[y][q][0], f1 = sm.flags[y][q][1];
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const uint32_t fj = ((j < 8 ? f0 : f1) >> (4 * (j & 7))) & 0xFu;
        uint32_t lab;
        if (HS) {
          const uint32_t e = l[j];
          const uint32_t mm = e & fj & 7u;
          lab = (mm & 1u) ? 0u : (mm & 2u) ? 1u : (mm & 4u) ? 2u : 3u;
          if (e & 8u) lab = 3u;
        } else {
          lab = l[j];
        }
        if (fj & 8u) lab = 3u;
        l[j] = lab;
        if (HS && j < nvalid) cnt[lab] += 1;
      }
    }
    if (dst) {
      uint4 lab;
      lab.x = pack4(l[0], l[1], l[2], l[3], dp);
      lab.y = pack4(l[4], l[5], l[6], l[7], dp);
      lab.z = pack4(l[8], l[9], l[10], l[11], dp);
      lab.w = pack4(l[12], l[13], l[14], l[15], dp);
      store_labels(dst, nvalid, lab, store);
      dst += lpitch;
    }
    }
  }
}

// Optional output of the filter's corrected value: V' = vlut[Vf] per pixel
// (0 for nodata), rows r0..r1-1 of the band.
template <bool kFlags, class SM>
__device__ __forceinline__ void band_vprime(uint8_t* out, int64_t pitch, int64_t y0, int64_t x0,
                                            int w, int r0, int r1, int nmax, uint32_t taddr,
                                            const uint8_t* vlut, const SM& sm) {
  const int q = threadIdx.x & 15;
  const int nvalid = min(max(w - 16 * q, 0), 16);
  const int own = nvalid > 0 ? r1 - r0 : 0;
  uint8_t* dst = out + (y0 + r0) * pitch + x0 + 16 * q;
  for (int j0 = 0; j0 < nmax; j0 += 4) {
    uint32_t pr[16];
    if constexpr (SM::kSmemPlane) {
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        if (j0 + i < own) {
          const uint4 pw = *reinterpret_cast<const uint4*>(&sm.vf[(r0 + j0 + i) * 256 + 16 * q]);
          pr[4 * i] = pw.x;
          pr[4 * i + 1] = pw.y;
          pr[4 * i + 2] = pw.z;
          pr[4 * i + 3] = pw.w;
        }
      }
    } else {
      __syncwarp();
      plane_ld4rows(taddr + 4u * uint32_t(j0), pr);
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
    if (j0 + i >= own) break;
    const int y = r0 + j0 + i;
    const uint32_t p[4] = {pr[4 * i], pr[4 * i + 1], pr[4 * i + 2], pr[4 * i + 3]};
    uint32_t l[16];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      l[2 * k] = vlut[__byte_perm(p[k], 0, 0x4440)];
      l[2 * k + 1] = vlut[__byte_perm(p[k], 0, 0x4441)];
      l[2 * k + 8] = vlut[__byte_perm(p[k], 0, 0x4442)];
      l[2 * k + 9] = vlut[__byte_perm(p[k], 0, 0x4443)];
    }
    if (kFlags) {
      const uint32_t f0 = sm.flags[y][q][0], f1 = sm.flags[y][q][1];
#pragma unroll
      for (int j = 0; j < 16; ++j)
        if ((((j < 8 ? f0 : f1) >> (4 * (j & 7))) & 8u) != 0) l[j] = 0;
    }
    uint4 v;
    v.x = __byte_perm(__byte_perm(l[0], l[1], 0x0040), __byte_perm(l[2], l[3], 0x0040), 0x5410);
    v.y = __byte_perm(__byte_perm(l[4], l[5], 0x0040), __byte_perm(l[6], l[7], 0x0040), 0x5410);
    v.z = __byte_perm(__byte_perm(l[8], l[9], 0x0040), __byte_perm(l[10], l[11], 0x0040), 0x5410);
    v.w = __byte_perm(__byte_perm(l[12], l[13], 0x0040), __byte_perm(l[14], l[15], 0x0040), 0x5410);
    store_row16(dst, nvalid, v);
    dst += pitch;
    }
  }
}

// ---------------------------------------------------------------------------
// The whole chip.  All threads of the CTA must call it.
// kSplit > 1: the CTA is rank q of a cluster of kSplit CTAs that label the
// chip together; it filters rows [q h / kSplit, (q + 1) h / kSplit) (the
// median's neighbours outside that slice are read from the image like any
// other row, clamped to the chip), the slices' histograms are summed through
// distributed shared memory, every CTA derives the same statistics and
// table from the sum, labels its own rows, and rank 0 alone writes the
// chip's counts.  (8-bit images without H/S ranges only: those keep no
// per-pixel flags.)
// ---------------------------------------------------------------------------
// This half-warp's band of chip (cy, cx) of request r (rank's row slice of
// it when kSplit CTAs share the chip): balanced row bands, one per half-warp.
template <int DT>
__device__ __forceinline__ Band chip_band(const Req& r, int chip, int64_t cy, int64_t cx,
                                          int kSplit, unsigned rank) {
  const int band = threadIdx.x >> 4;
  const int64_t y0 = cy * chip, x0 = cx * chip;
  Band b;
  b.h = int(min(int64_t(chip), r.H - y0));
  b.w = int(min(int64_t(chip), r.W - x0));
  b.pitch = r.pitch;
  b.chip0 = r.img + x0 * Px<DT>::BPP + y0 * r.pitch;
  const int s0 = int(rank) * b.h / kSplit, s1 = (int(rank) + 1) * b.h / kSplit;
  b.r0 = s0 + (band * (s1 - s0)) / n_bands();
  b.r1 = s0 + ((band + 1) * (s1 - s0)) / n_bands();
  return b;
}

template <int DT, bool HS, int kSplit = 1, class SM>
__device__ __forceinline__ void label_chip(const Req& r, const DevParams& dp, int chip,
                                           int64_t cy, int64_t cx, SM& sm, uint8_t* lut,
                                           uint8_t* vlut) {
  static_assert(kSplit == 1 || (DT == SIL_U8 && !HS), "split chips: 8-bit, no H/S ranges");
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int64_t y0 = cy * chip, x0 = cx * chip;
  const int h = int(min(int64_t(chip), r.H - y0));
  const int w = int(min(int64_t(chip), r.W - x0));
  unsigned rank = 0;
  if (kSplit > 1) rank = cooperative_groups::this_cluster().block_rank();
  const Band bd = chip_band<DT>(r, chip, cy, cx, kSplit, rank);
  const int r0 = bd.r0, r1 = bd.r1;
  // rows of this half-warp's band and of the other half-warp's (the warp
  // steps through nmax rows in both passes)
  const int own = r1 - r0, other = __shfl_xor_sync(0xffffffffu, own, 16);
  const int nmin = min(own, other), nmax = max(own, other);
  const uint32_t taddr = plane_taddr(sm.st.tmem);

  __syncthreads();  // the previous chip of a persistent CTA is done with sm
  if (tid < 256) sm.st.hist[tid] = 0;
  __syncthreads();
  uint32_t n_nodata = 0;
  if (nmax > 0) {
    // rows start on 4-byte boundaries when the base, the pitch and the chip's
    // first column (x0 * 3 or x0 * 6 bytes) do
    const bool a4 = ((reinterpret_cast<uintptr_t>(r.img) | uint64_t(r.pitch) | uint64_t(x0)) & 3) == 0;
#define SIL_PASS1(F, A) band_pass1<DT, HS, F, A>(bd, dp, sm, n_nodata, nmin, nmax, taddr)
    if (w == 256) {
      if (a4)
        SIL_PASS1(true, true);
      else
        SIL_PASS1(true, false);
    } else {
      if (a4)
        SIL_PASS1(false, true);
      else
        SIL_PASS1(false, false);
    }
#undef SIL_PASS1
  }
  if constexpr (!SM::kSmemPlane) plane_wait_st();  // this thread's plane rows are in tensor memory
  if (DT == SIL_U16) {
    n_nodata = __reduce_add_sync(0xffffffffu, n_nodata);
    if (lane == 0) sm.st.nod[wid] = n_nodata;
  }
  __syncthreads();
  if (kSplit > 1) {
    // the chip's histogram = the sum of the slices' histograms
    cooperative_groups::cluster_group cl = cooperative_groups::this_cluster();
    cl.sync();  // every slice's histogram is complete
    uint32_t v = 0;
    if (tid < 256) {
#pragma unroll
      for (int q = 0; q < kSplit; ++q) v += cl.map_shared_rank(sm.st.hist, q)[tid];
    }
    cl.sync();  // every CTA has read every histogram
    if (tid < 256) sm.st.hist[tid] = v;
    __syncthreads();
  }
  {
    uint32_t nd = 0;
    if (DT == SIL_U16) {
#pragma unroll
      for (int k = 0; k < kMaxWarps; ++k) nd += k < n_warps() ? sm.st.nod[k] : 0u;
    }
    chip_stats_block(sm.st, sm.sc, dp, uint32_t(h * w) - nd);
  }
  uint32_t e = 0;
  if (tid < 256) {
    e = lut_entry<HS>(tid, sm.st, dp);
    lut[tid] = uint8_t(e);
    if (r.vprime) vlut[tid] = uint8_t(vprime_value(tid, sm.st, dp));
  }
  if (!HS && tid < 256) {
    // counts = histogram x label table (nodata pixels are added below)
    const uint32_t hv = sm.st.hist[tid];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const uint32_t s = __reduce_add_sync(0xffffffffu, e == uint32_t(c) ? hv : 0u);
      if (lane == 0) sm.st.red[wid][c] = s;
    }
  }
  __syncthreads();
  // A chip whose every present value maps to one label (common inside a
  // floe) is filled with that label instead of being looked up pixel by pixel.
  bool uniform = false;
  if (!HS) {
    const int lo = sm.st.stat[kStatLo], hi = sm.st.stat[kStatHi];
    const bool nodata = uint32_t(sm.st.stat[kStatN]) != uint32_t(h * w);
    const bool same = (tid >= lo && tid <= hi && tid < 256) ? (lut[tid] == lut[lo]) : true;
    uniform = __syncthreads_and(same && !nodata) != 0;
  }
  uint32_t cnt[4] = {0, 0, 0, 0};
  if (uniform) {
    if (r0 < r1 && r.labels) {
      const int q = tid & 15;
      const int nvalid = min(max(w - 16 * q, 0), 16);
      const uint32_t cw = uint32_t(lut[sm.st.stat[kStatLo]]) * 0x01010101u;
      if (nvalid > 0) {
        uint8_t* dst = r.labels + (y0 + r0) * r.lpitch + x0 + 16 * q;
        for (int y = r0; y < r1; ++y, dst += r.lpitch) store_row16(dst, nvalid, make_uint4(cw, cw, cw, cw));
      }
    }
  } else if (nmax > 0 && (HS || r.labels)) {
    const uint64_t la = reinterpret_cast<uintptr_t>(r.labels) + uint64_t(x0);
    const int store = ((la | uint64_t(r.lpitch)) & 15) == 0 ? 16 : ((la | uint64_t(r.lpitch)) & 3) == 0 ? 4 : 1;
    band_pass2<DT, HS>(r.labels, r.lpitch, y0, x0, w, r0, r1, nmax, taddr, lut, sm, cnt, dp, store);
  }
  if (r.vprime && nmax > 0)
    band_vprime<HS || DT == SIL_U16>(r.vprime, r.vpitch, y0, x0, w, r0, r1, nmax, taddr, vlut, sm);
  if (HS) {
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const uint32_t s = __reduce_add_sync(0xffffffffu, cnt[c]);
      if (lane == 0) sm.st.red[wid][c] = s;
    }
    __syncthreads();
  }
  if (tid < 4) {
    const int c = tid;
    const int nw = HS ? n_warps() : kBinWarps;
    uint32_t v = 0;
    for (int k = 0; k < nw; ++k) v += sm.st.red[k][c];
    // nodata pixels are left out of the histogram and always masked
    if (!HS && c == 3) v += uint32_t(h * w) - uint32_t(sm.st.stat[kStatN]);
    if (rank == 0) {
      if (r.chip_counts) r.chip_counts[(cy * r.gx + cx) * 4 + c] = v;
      atomicAdd(&r.counts[c], (unsigned long long)v);
    }
  }
}

template <int DT, bool HS>
using ChipSmem = ChipSmemT<Px<DT>::BPP, HS || DT == SIL_U16, !TmemPlane<DT, HS>::value>;

}  // namespace sil
