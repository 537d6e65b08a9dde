// sil_chip.cuh -- the fused per-chip labeler (device code).
//
// One CTA of 256 threads labels one chip of at most 256 x 256 pixels:
//
//   pass 1  (per half-warp row band, 16 px per lane, rows streamed top to
//           bottom with a rolling 3-row window in registers)
//           decode -> V = max(R,G,B) -> 3x3 median of V clamped to the chip
//           -> histogram of Vf in shared memory, Vf kept in a shared plane
//   stats   one warp: lo/hi, exact Otsu threshold (128-bit compares), gate
//   LUT     256 threads: V' = gated min-max stretch, truncation, class ranges,
//           absdiff override  ->  label(Vf) table
//   counts  from histogram x LUT (no per-pixel counting)
//   pass 2  Vf plane -> LUT -> uint8 label store
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
// pixels and three inputs.  A lane-local segment of 16 pixels is held as 8
// words in "interleaved" order: word i = [col i, col i+8], so the horizontal
// neighbours of word i are words i-1 and i+1 and only the two segment edges
// need a shuffle.  The median of three is a+b+c-max3-min3, exact in 32-bit
// wrap-around arithmetic because every lane of the result lies in [0,65535].
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "sil_common.h"

namespace sil {

constexpr int kPlaneStride = 256;

// Per-chip statistics scratch (shared memory).
struct ChipStat {
  uint32_t hist[256];
  uint32_t red[kThreads / 32][4];
  uint32_t nod[kThreads / 32];
  int32_t stat[8];
};
// Scratch of the block-wide Otsu search.
struct alignas(16) StatScratch {
  uint32_t wc[kThreads / 32], ws[kThreads / 32];
  uint64_t bnum_lo[kThreads / 32];
  uint32_t bnum_hi[kThreads / 32], bden[kThreads / 32];
  int32_t bt[kThreads / 32], lo[kThreads / 32], hi[kThreads / 32];
  uint32_t n0;
};

// The statistics come first so the histogram sits at shared offset 0 and a
// bin's byte offset is its address.
struct ChipSmem {
  ChipStat st;
  StatScratch sc;
  uint8_t vf[kResidentChip * kPlaneStride];  // filtered V, plane order
};
static_assert(sizeof(ChipStat) % 16 == 0 && (sizeof(ChipStat) + sizeof(StatScratch)) % 16 == 0,
              "plane must stay 16-byte aligned");
// Per row, per lane: 16 nibbles (bits 0-2 class mask of H/S ranges, bit 3
// nodata); only used by the uint16 and H/S-narrowed variants.
struct ChipFlags {
  uint32_t f[kResidentChip][16][2];
};

enum { kStatLo = 0, kStatHi, kStatT, kStatN0, kStatGate, kStatN };

__device__ __forceinline__ uint32_t max3(uint32_t a, uint32_t b, uint32_t c) {
  return __vimax3_u16x2(a, b, c);
}
__device__ __forceinline__ uint32_t min3(uint32_t a, uint32_t b, uint32_t c) {
  return __vimin3_u16x2(a, b, c);
}
__device__ __forceinline__ uint32_t med3(uint32_t a, uint32_t b, uint32_t c) {
  return a + b + c - max3(a, b, c) - min3(a, b, c);
}
// a * b + c with b a runtime kernel parameter: stays an integer multiply-add.
__device__ __forceinline__ uint32_t imad(uint32_t a, uint32_t b, uint32_t c) {
  return a * b + c;
}
#ifndef SIL_MED_IMAD
#define SIL_MED_IMAD 0
#endif
#ifndef SIL_HIST_IMAD
#define SIL_HIST_IMAD 0
#endif
#ifndef SIL_P2_IMAD
#define SIL_P2_IMAD 0
#endif
// a + b + c - x - y (exact modulo 2^32), on the multiply-add pipe.
__device__ __forceinline__ uint32_t sum3m2(uint32_t a, uint32_t b, uint32_t c,
                                           uint32_t x, uint32_t y, const DevParams& dp) {
#if SIL_MED_IMAD == 1
  uint32_t s = imad(a, dp.one, b);
  s = imad(c, dp.one, s);
  s = imad(x, dp.neg1, s);
  return imad(y, dp.neg1, s);
#elif SIL_MED_IMAD == 2
  return imad(y, dp.neg1, imad(x, dp.neg1, a + b + c));
#else
  return a + b + c - x - y;
#endif
}
// median of three packed u16x2 words: 2 min/max + 4 multiply-adds.
__device__ __forceinline__ uint32_t med3m(uint32_t a, uint32_t b, uint32_t c,
                                          const DevParams& dp) {
  return sum3m2(a, b, c, max3(a, b, c), min3(a, b, c), dp);
}

// ---------------------------------------------------------------------------
// Row fetch.  The lane's bytes start at window offset m (0..15) of a
// 16-byte aligned window; only vectors that overlap the row's data are read,
// so no read leaves the 16-byte blocks that hold image bytes.
// ---------------------------------------------------------------------------
template <int NV>
struct Raw {
  uint4 v[NV];
};

template <int BPP, int NV>
__device__ __forceinline__ void fetch_row(const uint8_t* rowptr, int q, int w,
                                          Raw<NV>& raw) {
  const uintptr_t a = reinterpret_cast<uintptr_t>(rowptr);
  const uintptr_t A = a & ~uintptr_t(15);
  const int m = int(a & 15);
  const int lim = m + BPP * w;  // data bytes end, relative to A
  const int lane_off = 16 * BPP * q;
  const uint4* base = reinterpret_cast<const uint4*>(A + lane_off);
#pragma unroll
  for (int j = 0; j < NV; ++j) {
    if (lane_off + 16 * j < lim)
      raw.v[j] = __ldg(base + j);
    else
      raw.v[j] = make_uint4(0, 0, 0, 0);
  }
}

// Ask L2 to start fetching a chip row that will be decoded a few steps later,
// so that more of the image is in flight than the registers can hold.  Only
// 16-byte blocks that contain bytes of the row are named.
#ifndef SIL_L2PF
#define SIL_L2PF 0
#endif
#ifndef SIL_PFD
#define SIL_PFD 4
#endif
template <int BPP>
__device__ __forceinline__ void prefetch_row_l2(const uint8_t* rowptr, int q, int w) {
  const uintptr_t a = reinterpret_cast<uintptr_t>(rowptr);
  const uintptr_t A = a & ~uintptr_t(15);
  const uint32_t bytes = uint32_t(((a + uintptr_t(BPP) * w + 15) & ~uintptr_t(15)) - A);
#if SIL_L2PF == 1
  // one 128-byte line per lane
  if (uint32_t(q) * 128u < bytes)
    asm volatile("prefetch.global.L2 [%0];" ::"l"(A + uintptr_t(q) * 128u));
#elif SIL_L2PF == 2
  // one bulk prefetch per row, issued by the first lane of the band
  if (q == 0)
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(A), "r"(bytes) : "memory");
#endif
}

// u8: pixel j of the segment is bytes 3j..3j+2 after offset M.  For pair
// (i, i+8) and channel c the two bytes are 24 bytes = 6 words apart at the
// same byte position, so one PRMT lifts both into the high bytes of a u16x2.
template <int M>
__device__ __forceinline__ void gather_u8(const uint32_t* v, uint32_t* V,
                                          uint32_t (*G)[3]) {
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    uint32_t g[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const int b = M + 3 * i + c;
      const int wi = b >> 2, p = b & 3;
      const uint32_t sel = p | (p << 4) | ((4 + p) << 8) | ((4 + p) << 12);
      g[c] = __byte_perm(v[wi], v[wi + 6], sel);
      if (G) G[i][c] = g[c];
    }
    V[i] = max3(g[0], g[1], g[2]);
  }
}

// u16: pixel j is bytes 6j..6j+5 after offset M (even); pair (i, i+8) is 48
// bytes = 12 words apart at the same half-word position.
template <int M>
__device__ __forceinline__ void gather_u16(const uint32_t* v, uint32_t* R,
                                           uint32_t (*G)[3]) {
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    uint32_t g[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const int b = M + 6 * i + 2 * c;
      const int wi = b >> 2, hh = (b >> 1) & 1;
      g[c] = __byte_perm(v[wi], v[wi + 12], hh ? 0x7632u : 0x5410u);
      if (G) G[i][c] = g[c];
    }
    R[i] = max3(g[0], g[1], g[2]);
  }
}

#define SIL_CASE16(F, ...)                                               \
  case 0: F<0>(__VA_ARGS__); break; case 1: F<1>(__VA_ARGS__); break;    \
  case 2: F<2>(__VA_ARGS__); break; case 3: F<3>(__VA_ARGS__); break;    \
  case 4: F<4>(__VA_ARGS__); break; case 5: F<5>(__VA_ARGS__); break;    \
  case 6: F<6>(__VA_ARGS__); break; case 7: F<7>(__VA_ARGS__); break;    \
  case 8: F<8>(__VA_ARGS__); break; case 9: F<9>(__VA_ARGS__); break;    \
  case 10: F<10>(__VA_ARGS__); break; case 11: F<11>(__VA_ARGS__); break; \
  case 12: F<12>(__VA_ARGS__); break; case 13: F<13>(__VA_ARGS__); break; \
  case 14: F<14>(__VA_ARGS__); break; default: F<15>(__VA_ARGS__); break;

#define SIL_CASE16_EVEN(F, ...)                                          \
  case 0: F<0>(__VA_ARGS__); break; case 2: F<2>(__VA_ARGS__); break;    \
  case 4: F<4>(__VA_ARGS__); break; case 6: F<6>(__VA_ARGS__); break;    \
  case 8: F<8>(__VA_ARGS__); break; case 10: F<10>(__VA_ARGS__); break;  \
  case 12: F<12>(__VA_ARGS__); break; default: F<14>(__VA_ARGS__); break;

// round(x * 255 / s) clamped to 255, i.e. floor((255 x + s/2) / s) for the
// uint16 scaling; the quotient of n < 2^24 by s < 2^16 is exact as
// (n * ceil(2^40 / s)) >> 40 (checked for every x on the host).
__device__ __forceinline__ uint32_t u16_to_v8(uint32_t x, const DevParams& dp) {
  const uint32_t n = x * 255u + dp.u16_half;
  const uint32_t qv = uint32_t((uint64_t(n) * dp.u16_mul) >> 40);
  return qv > 255u ? 255u : qv;
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

// ---------------------------------------------------------------------------
// Row decode: raw bytes -> 8 interleaved V words (+ flags for u16 / H-S).
// ---------------------------------------------------------------------------
template <int DT, bool HS>
struct RowDec {
  static constexpr int BPP = DT == SIL_U8 ? 3 : 6;
  static constexpr int NV = DT == SIL_U8 ? 4 : 7;
};

template <int DT, bool HS>
__device__ __forceinline__ void decode_row(const Raw<RowDec<DT, HS>::NV>& raw,
                                           int m, int nvalid,
                                           const DevParams& dp, uint32_t* V,
                                           uint32_t* F) {
  const uint32_t* v = reinterpret_cast<const uint32_t*>(raw.v);
  uint32_t G[8][3];
  constexpr bool kNeedG = HS;
  if (DT == SIL_U8) {
    switch (m) { SIL_CASE16(gather_u8, v, V, kNeedG ? G : nullptr) }
  } else {
    uint32_t R[8];
    switch (m) { SIL_CASE16_EVEN(gather_u16, v, R, kNeedG ? G : nullptr) }
    uint32_t nd0 = 0, nd1 = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const uint32_t x0 = R[i] & 0xFFFFu, x1 = R[i] >> 16;
      V[i] = (u16_to_v8(x0, dp) << 8) | (u16_to_v8(x1, dp) << 24);
      nd0 |= (x0 == 0 ? 8u : 0u) << (4 * i);
      nd1 |= (x1 == 0 ? 8u : 0u) << (4 * i);
    }
    F[0] = nd0;
    F[1] = nd1;
  }
  if (HS) {
    uint32_t f0 = 0, f1 = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      int c0[3], c1[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        if (DT == SIL_U8) {
          c0[c] = (G[i][c] >> 8) & 0xFF;
          c1[c] = G[i][c] >> 24;
        } else {
          c0[c] = u16_to_v8(G[i][c] & 0xFFFFu, dp);
          c1[c] = u16_to_v8(G[i][c] >> 16, dp);
        }
      }
      const int ri = dp.bgr ? 2 : 0, bi = dp.bgr ? 0 : 2;
      f0 |= hs_mask(c0[ri], c0[1], c0[bi], dp) << (4 * i);
      f1 |= hs_mask(c1[ri], c1[1], c1[bi], dp) << (4 * i);
    }
    if (DT == SIL_U8) {
      F[0] = f0;
      F[1] = f1;
    } else {
      F[0] |= f0;
      F[1] |= f1;
    }
  }
  if (nvalid < 16 && nvalid > 0) {
    // Replicate the chip's last column into the lane's columns beyond it
    // (the median window is clamped to the chip).
    const uint32_t rep = seg_get(V, nvalid - 1);
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      if (i >= nvalid) V[i] = (V[i] & 0xFFFF0000u) | rep;
      if (i + 8 >= nvalid) V[i] = (V[i] & 0x0000FFFFu) | (rep << 16);
    }
  }
}

// Edge words of a decoded row: EL = [col -1, col 7], ER = [col 8, col 16],
// clamped to the chip (replicated border).
__device__ __forceinline__ void edge_words(const uint32_t* V, int q, int w,
                                          uint32_t hmask, uint32_t& EL,
                                          uint32_t& ER) {
  const uint32_t up = __shfl_up_sync(hmask, V[7], 1, 16);
  const uint32_t dn = __shfl_down_sync(hmask, V[0], 1, 16);
  const uint32_t srcL = (q == 0) ? (V[0] << 16) : up;           // hi lane = col -1
  const uint32_t srcR = (16 * q + 16 >= w) ? (V[7] >> 16) : dn; // lo lane = col 16
  EL = __byte_perm(srcL, V[7], 0x5432);
  ER = __byte_perm(V[0], srcR, 0x5432);
}

// ---------------------------------------------------------------------------
// Pass 1 for one half-warp band.
// ---------------------------------------------------------------------------
// One decoded row of a lane's 16-pixel segment: 8 interleaved words, the two
// edge words and (uint16 / H-S variants) the per-pixel flags.
struct RowBuf {
  uint32_t v[8];
  uint32_t eL, eR;
  uint32_t f[2];
};

// Sorted column (min, median, max) of three packed rows.
struct Col {
  uint32_t l, c, x;
};
__device__ __forceinline__ Col sort_col(uint32_t a, uint32_t b, uint32_t c,
                                        const DevParams& dp) {
  Col r;
  r.l = min3(a, b, c);
  r.x = max3(a, b, c);
  r.c = sum3m2(a, b, c, r.l, r.x, dp);
  return r;
}

// Output row y from the window rows (M, Z, P) = (y-1, y, y+1): 3x3 median
// as med3(max3 of column minima, med3 of column medians, min3 of column
// maxima), histogram of Vf, Vf plane row.  Column sorts are produced one
// word ahead of the output that needs them (three live at a time).
template <bool kFlags, int DT>
__device__ __forceinline__ void emit_row(const RowBuf& M, const RowBuf& Z,
                                         const RowBuf& P, int y, int q,
                                         int nvalid, bool use_median,
                                         const DevParams& dp, ChipSmem& sm,
                                         ChipFlags* fl, uint32_t& n_nodata) {
  uint32_t out[8];
  if (use_median) {
    Col a = sort_col(M.eL, Z.eL, P.eL, dp);
    Col b = sort_col(M.v[0], Z.v[0], P.v[0], dp);
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const Col c = (i < 7) ? sort_col(M.v[i + 1], Z.v[i + 1], P.v[i + 1], dp)
                            : sort_col(M.eR, Z.eR, P.eR, dp);
      const uint32_t lo = max3(a.l, b.l, c.l);
      const uint32_t hi = min3(a.x, b.x, c.x);
      const uint32_t mi = med3m(a.c, b.c, c.c, dp);
      out[i] = med3m(lo, mi, hi, dp);
      a = b;
      b = c;
    }
  } else {
#pragma unroll
    for (int i = 0; i < 8; ++i) out[i] = Z.v[i];
  }
  // Histogram of Vf over valid, non-nodata pixels.
  char* hist = reinterpret_cast<char*>(sm.st.hist);
  if (!kFlags && nvalid == 16) {
#pragma unroll
    for (int i = 0; i < 8; ++i) {
#if SIL_HIST_IMAD
      const uint32_t c = out[i] & 0xFF00FF00u;
      const uint32_t a1 = __umulhi(c, dp.k10);
      const uint32_t a0 = __umulhi(imad(c, dp.k16, 0u), dp.k10);
#else
      const uint32_t a0 = (out[i] >> 6) & 0x3FCu;
      const uint32_t a1 = (out[i] >> 22) & 0x3FCu;
#endif
      atomicAdd(reinterpret_cast<uint32_t*>(hist + a0), 1u);
      atomicAdd(reinterpret_cast<uint32_t*>(hist + a1), 1u);
    }
  } else {
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const uint32_t a0 = (out[i] >> 6) & 0x3FCu;
      const uint32_t a1 = (out[i] >> 22) & 0x3FCu;
      const bool nd0 = kFlags && ((Z.f[0] >> (4 * i + 3)) & 1u);
      const bool nd1 = kFlags && ((Z.f[1] >> (4 * i + 3)) & 1u);
      if (i < nvalid && !nd0) atomicAdd(reinterpret_cast<uint32_t*>(hist + a0), 1u);
      if (i + 8 < nvalid && !nd1) atomicAdd(reinterpret_cast<uint32_t*>(hist + a1), 1u);
      if (DT == SIL_U16) {
        n_nodata += (i < nvalid && nd0) ? 1u : 0u;
        n_nodata += (i + 8 < nvalid && nd1) ? 1u : 0u;
      }
    }
  }
  // Vf plane (plane order: word k = [c2k, c2k+1, c2k+8, c2k+9]).
  uint4 pw;
  pw.x = __byte_perm(out[0], out[1], 0x7351);
  pw.y = __byte_perm(out[2], out[3], 0x7351);
  pw.z = __byte_perm(out[4], out[5], 0x7351);
  pw.w = __byte_perm(out[6], out[7], 0x7351);
  *reinterpret_cast<uint4*>(&sm.vf[y * kPlaneStride + 16 * q]) = pw;
  if (kFlags) {
    fl->f[y][q][0] = Z.f[0];
    fl->f[y][q][1] = Z.f[1];
  }
}

// Pass 1 of one half-warp band: rows r0..r1-1 of the chip.  The band streams
// rows r0-1 .. r1 (clamped to the chip) through a single decode site; the
// row after the one being decoded is already in flight.
template <int DT, bool HS>
__device__ __forceinline__ void band_pass1(const uint8_t* img, int64_t pitch,
                                           int64_t y0, int64_t x0, int h, int w,
                                           int r0, int r1, int q, uint32_t hmask,
                                           const DevParams& dp, ChipSmem& sm,
                                           ChipFlags* fl, uint32_t& n_nodata) {
  constexpr int BPP = RowDec<DT, HS>::BPP;
  constexpr int NV = RowDec<DT, HS>::NV;
  constexpr bool kFlags = HS || DT == SIL_U16;
  const int nvalid = min(max(w - 16 * q, 0), 16);
  const bool use_median = dp.filter && dp.median;
  // row sequence: max(r0-1,0), r0, r0+1, ..., min(r1, h-1)
  const int nrows = r1 - r0 + 2;
  int fy = max(r0 - 1, 0);
  const uint8_t* fp = img + x0 * BPP + (y0 + fy) * pitch;
#ifndef SIL_PREFETCH
#define SIL_PREFETCH 1
#endif
  Raw<NV> raw;
#if SIL_PREFETCH
  if (nvalid > 0) fetch_row<BPP, NV>(fp, q, w, raw);
#endif
  RowBuf M, Z, P;
  for (int k = 0; k < nrows; ++k) {
#if !SIL_PREFETCH
    if (nvalid > 0) fetch_row<BPP, NV>(fp, q, w, raw);
#endif
    decode_row<DT, HS>(raw, int(reinterpret_cast<uintptr_t>(fp) & 15), nvalid, dp, P.v, P.f);
    edge_words(P.v, q, w, hmask, P.eL, P.eR);
#if SIL_L2PF
    if (k + SIL_PFD < nrows && nvalid > 0) {
      const int py = min(r0 + k + SIL_PFD - 1, h - 1);  // row of element k+PFD
      prefetch_row_l2<BPP>(img + x0 * BPP + (y0 + py) * pitch, q, w);
    }
#endif
    if (k + 1 < nrows) {
      const int ny = min(r0 + k, h - 1);  // row index of element k+1
      if (ny != fy) {
        fp += pitch;
        fy = ny;
      }
#if SIL_PREFETCH
      if (nvalid > 0) fetch_row<BPP, NV>(fp, q, w, raw);
#endif
    }
    if (k >= 2)
      emit_row<kFlags, DT>(M, Z, P, r0 + k - 2, q, nvalid, use_median, dp, sm, fl, n_nodata);
    M = Z;
    Z = P;
  }
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

// The same statistics computed by all 256 threads of the CTA (thread t owns
// histogram bin t), for chips of at most 65536 pixels: block-wide prefix
// sums, one score per thread, block-wide argmax.  Scores: D = S_T w - N s
// < 2^40, num = D^2 < 2^80, den = w (N - w) <= 2^32, cross products
// < 2^112.  Contains __syncthreads(); every thread of the CTA must call it.

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
  const uint32_t hv = st.hist[tid];
  uint32_t c = hv, s = uint32_t(tid) * hv;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const uint32_t a = __shfl_up_sync(0xffffffffu, c, off);
    const uint32_t b = __shfl_up_sync(0xffffffffu, s, off);
    if (lane >= off) { c += a; s += b; }
  }
  const uint32_t nz = __ballot_sync(0xffffffffu, hv != 0);
  if (lane == 31) { sc.wc[wid] = c; sc.ws[wid] = s; }
  if (lane == 0) {
    sc.lo[wid] = nz ? wid * 32 + __ffs(nz) - 1 : 256;
    sc.hi[wid] = nz ? wid * 32 + 31 - __clz(nz) : -1;
  }
  __syncthreads();
  uint32_t ST = 0, pc = 0, ps = 0;
  int lo = 256, hi = -1;
#pragma unroll
  for (int k = 0; k < kThreads / 32; ++k) {
    if (k < wid) { pc += sc.wc[k]; ps += sc.ws[k]; }
    ST += sc.ws[k];
    lo = min(lo, sc.lo[k]);
    hi = max(hi, sc.hi[k]);
  }
  c += pc;  // pixels with Vf <= tid
  s += ps;
  // score of threshold t = tid
  int t = -1;
  uint64_t nlo = 0;
  uint32_t nhi = 0, den = 0;
  if (tid <= 254 && c > 0 && c < N) {
    const uint64_t D = uint64_t(ST) * c - uint64_t(N) * s;  // >= 0
    const unsigned __int128 num = (unsigned __int128)D * D;
    nlo = uint64_t(num);
    nhi = uint32_t(num >> 64);
    den = c * (N - c);
    t = tid;
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const uint64_t o_lo = __shfl_xor_sync(0xffffffffu, nlo, off);
    const uint32_t o_hi = __shfl_xor_sync(0xffffffffu, nhi, off);
    const uint32_t o_d = __shfl_xor_sync(0xffffffffu, den, off);
    const int o_t = __shfl_xor_sync(0xffffffffu, t, off);
    if (better(o_lo, o_hi, o_d, o_t, nlo, nhi, den, t)) {
      nlo = o_lo; nhi = o_hi; den = o_d; t = o_t;
    }
  }
  if (lane == 0) {
    sc.bnum_lo[wid] = nlo; sc.bnum_hi[wid] = nhi; sc.bden[wid] = den; sc.bt[wid] = t;
  }
  __syncthreads();
  if (wid == 0) {
    const int k = lane & 7;
    nlo = sc.bnum_lo[k]; nhi = sc.bnum_hi[k]; den = sc.bden[k]; t = sc.bt[k];
#pragma unroll
    for (int off = 4; off > 0; off >>= 1) {
      const uint64_t o_lo = __shfl_xor_sync(0xffffffffu, nlo, off);
      const uint32_t o_hi = __shfl_xor_sync(0xffffffffu, nhi, off);
      const uint32_t o_d = __shfl_xor_sync(0xffffffffu, den, off);
      const int o_t = __shfl_xor_sync(0xffffffffu, t, off);
      if (better(o_lo, o_hi, o_d, o_t, nlo, nhi, den, t)) {
        nlo = o_lo; nhi = o_hi; den = o_d; t = o_t;
      }
    }
    if (lane == 0) {
      if (hi < 0) { lo = 0; hi = 0; }
      const int tt = t < 0 ? lo : t;
      st.stat[kStatLo] = lo;
      st.stat[kStatHi] = hi;
      st.stat[kStatT] = tt;
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
    st.stat[kStatGate] = (hi2 - lo2 >= dp.mm_min_range) &&
                         (uint64_t(dp.frac_den) * n0 >= N) &&
                         (uint64_t(dp.frac_den) * n1 >= N) && N > 0;
  }
  __syncthreads();
}

// Label table entry for filtered value vf (thread per value).
// Non-H/S variant: the label code.  H/S variant: bits 0-2 = classes whose V
// range holds V', bit 3 = absdiff override.
template <bool HS>
__device__ __forceinline__ uint32_t lut_entry(int vf, const ChipStat& sm,
                                              const DevParams& dp) {
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
      d[0] = lab.x; d[1] = lab.y; d[2] = lab.z; d[3] = lab.w;
      return;
    }
  }
  const uint32_t wv[4] = {lab.x, lab.y, lab.z, lab.w};
#pragma unroll
  for (int j = 0; j < 16; ++j)
    if (j < nvalid) dst[j] = uint8_t(wv[j >> 2] >> (8 * (j & 3)));
}

// Byte k of w, zero-extended, on the multiply-add pipe: (w << 8(3-k)) >> 24.
__device__ __forceinline__ uint32_t byte_of(uint32_t w, int k, const DevParams& dp) {
#if SIL_P2_IMAD == 0
  return __byte_perm(w, 0, 0x4440 + k);
#endif
  if (k == 3) return __umulhi(w, dp.k8);
  if (k == 2) return __umulhi(imad(w, dp.k8, 0u), dp.k8);
  if (k == 1) return __umulhi(imad(w, dp.k16, 0u), dp.k8);
  return w & 0xFFu;
}

template <int DT, bool HS>
__device__ __forceinline__ void band_pass2(uint8_t* labels, int64_t lpitch,
                                           int64_t y0, int64_t x0, int w, int r0,
                                           int r1, int q, const uint8_t* lut,
                                           const ChipSmem& sm, const ChipFlags* fl,
                                           uint32_t* cnt, const DevParams& dp) {
  constexpr bool kFlags = HS || DT == SIL_U16;
  const int nvalid = min(max(w - 16 * q, 0), 16);
  if (nvalid == 0) return;
  uint8_t* dst = labels ? labels + (y0 + r0) * lpitch + x0 + 16 * q : nullptr;
  for (int y = r0; y < r1; ++y) {
    const uint4 pw = *reinterpret_cast<const uint4*>(&sm.vf[y * kPlaneStride + 16 * q]);
    // plane word k holds columns (2k, 2k+1, 2k+8, 2k+9)
    const uint32_t p[4] = {pw.x, pw.y, pw.z, pw.w};
    uint32_t l[16];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      l[2 * k] = lut[byte_of(p[k], 0, dp)];
      l[2 * k + 1] = lut[byte_of(p[k], 1, dp)];
      l[2 * k + 8] = lut[byte_of(p[k], 2, dp)];
      l[2 * k + 9] = lut[byte_of(p[k], 3, dp)];
    }
    if (kFlags) {
      const uint32_t f0 = fl->f[y][q][0], f1 = fl->f[y][q][1];
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const uint32_t f = ((j < 8 ? f0 : f1) >> (4 * (j & 7))) & 0xFu;
        uint32_t lab;
        if (HS) {
          const uint32_t e = l[j];
          const uint32_t m = e & f & 7u;
          lab = (m & 1u) ? 0u : (m & 2u) ? 1u : (m & 4u) ? 2u : 3u;
          if (e & 8u) lab = 3u;
        } else {
          lab = l[j];
        }
        if (f & 8u) lab = 3u;
        l[j] = lab;
        if (HS && j < nvalid) cnt[lab] += 1;
      }
    }
    if (dst) {
      // label bytes in natural column order, assembled by multiply-adds
      uint4 lab;
#if SIL_P2_IMAD == 0
      lab.x = __byte_perm(__byte_perm(l[0], l[1], 0x0040), __byte_perm(l[2], l[3], 0x0040), 0x5410);
      lab.y = __byte_perm(__byte_perm(l[4], l[5], 0x0040), __byte_perm(l[6], l[7], 0x0040), 0x5410);
      lab.z = __byte_perm(__byte_perm(l[8], l[9], 0x0040), __byte_perm(l[10], l[11], 0x0040), 0x5410);
      lab.w = __byte_perm(__byte_perm(l[12], l[13], 0x0040), __byte_perm(l[14], l[15], 0x0040), 0x5410);
#else
      lab.x = imad(l[3], dp.k24, imad(l[2], dp.k16, imad(l[1], dp.k8, l[0])));
      lab.y = imad(l[7], dp.k24, imad(l[6], dp.k16, imad(l[5], dp.k8, l[4])));
      lab.z = imad(l[11], dp.k24, imad(l[10], dp.k16, imad(l[9], dp.k8, l[8])));
      lab.w = imad(l[15], dp.k24, imad(l[14], dp.k16, imad(l[13], dp.k8, l[12])));
#endif
      store_row16(dst, nvalid, lab);
      dst += lpitch;
    }
  }
}

// ---------------------------------------------------------------------------
// The whole chip.  All 256 threads of the CTA must call it.
// ---------------------------------------------------------------------------
template <int DT, bool HS>
__device__ __forceinline__ void label_chip(const Req& r, const DevParams& dp,
                                           int chip, int64_t cy, int64_t cx,
                                           ChipSmem& sm, ChipFlags* fl,
                                           uint8_t* lut) {
  const int tid = threadIdx.x;
  const int lane = tid & 31, q = lane & 15, band = tid >> 4;
  const uint32_t hmask = 0xFFFFu << (lane & 16);
  const int64_t y0 = cy * chip, x0 = cx * chip;
  const int h = int(min(int64_t(chip), r.H - y0));
  const int w = int(min(int64_t(chip), r.W - x0));
  const int bh = (h + 15) >> 4;
  const int r0 = min(band * bh, h), r1 = min(h, r0 + bh);

  __syncthreads();  // the previous chip of a persistent CTA is done with sm
  sm.st.hist[tid] = 0;
  __syncthreads();
  uint32_t n_nodata = 0;
  if (r0 < r1)
    band_pass1<DT, HS>(r.img, r.pitch, y0, x0, h, w, r0, r1, q, hmask, dp, sm, fl,
                       n_nodata);
  if (DT == SIL_U16) {
    n_nodata = __reduce_add_sync(0xffffffffu, n_nodata);
    if (lane == 0) sm.st.nod[tid >> 5] = n_nodata;
  }
  __syncthreads();
  {
    uint32_t nd = 0;
    if (DT == SIL_U16) {
#pragma unroll
      for (int k = 0; k < kThreads / 32; ++k) nd += sm.st.nod[k];
    }
    chip_stats_block(sm.st, sm.sc, dp, uint32_t(h * w) - nd);
  }
  const uint32_t e = lut_entry<HS>(tid, sm.st, dp);
  lut[tid] = uint8_t(e);
  uint32_t cnt[4] = {0, 0, 0, 0};
  if (!HS) {
    // counts = histogram x label table (+ nodata pixels, always masked)
    const uint32_t hv = sm.st.hist[tid];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const uint32_t s = __reduce_add_sync(0xffffffffu, e == uint32_t(c) ? hv : 0u);
      if (lane == 0) sm.st.red[tid >> 5][c] = s;
    }
  }
  __syncthreads();
  if (r0 < r1 && (HS || r.labels))
    band_pass2<DT, HS>(r.labels, r.lpitch, y0, x0, w, r0, r1, q, lut, sm, fl, cnt, dp);
  if (HS) {
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const uint32_t s = __reduce_add_sync(0xffffffffu, cnt[c]);
      if (lane == 0) sm.st.red[tid >> 5][c] = s;
    }
    __syncthreads();
  }
  if (tid < 32) {
    const int c = lane & 3, wv = lane >> 2;  // 8 warps x 4 classes
    uint32_t v = sm.st.red[wv][c];
#pragma unroll
    for (int off = 4; off < 32; off <<= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    // nodata pixels are left out of the histogram and always masked
    if (!HS && c == 3) v += uint32_t(h * w) - uint32_t(sm.st.stat[kStatN]);
    if (lane < 4) {
      if (r.chip_counts) r.chip_counts[(cy * r.gx + cx) * 4 + c] = v;
      atomicAdd(&r.counts[c], (unsigned long long)v);
    }
  }
}

}  // namespace sil
