/*
 * sil_oracle.c -- plain, slow, single-threaded CPU oracle of the sea-ice
 * auto-labeling path (thin-cloud/shadow filter, HSV colour-threshold
 * segmentation, per-chip and per-request class counts).
 *
 * THIS IS TEST INFRASTRUCTURE.  Only the tests, the smoke check and the
 * CPU-baseline leg of the benchmark may load it.  It shares no code, header,
 * table or helper with the CUDA library; it is written step by step in the
 * order of the method so that a reader can check it against the paper:
 *
 *   Sec. III-B "Filtering Out the Thin Clouds and Shadows": the filter is a
 *     composition of RGB->HSV conversion, noise filtering, Otsu thresholding,
 *     min-max normalisation, truncated / binary thresholding, absolute
 *     difference and bit-wise operations.  The paper gives no order, channel
 *     or parameters; this file implements the project's reading "F1":
 *       V = max(R,G,B) -> 3x3 median of V inside the chip -> per-chip Otsu
 *       and min/max -> gated min-max stretch -> truncation -> absdiff mask.
 *   Sec. III-B "Auto-labeling Method": inclusive HSV ranges per class,
 *     thick ice (0,0,205)-(185,255,255), thin ice (0,0,31)-(185,255,204),
 *     open water (0,0,0)-(185,255,30); one mask per class, masks merged.
 *   Sec. III-B "PySpark Map-Reduce": map = label one image, reduce = collect
 *     results; here the reduce is the class count per chip and per request.
 *   Sec. III-A / Sec. III-C inference: images are 256x256 chips cut from
 *     scenes; statistics (Otsu, min/max) are taken per chip.
 *
 * Label codes: 0 thick/snow-covered ice, 1 young/thin ice, 2 open water,
 * 3 masked (no class matched, S2 nodata, or the absdiff override).
 *
 * Every arithmetic step is integer; no floating point appears anywhere.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct sil_oracle_params {
  uint8_t lo[3][3]; /* [thick, thin, water][H, S, V], inclusive */
  uint8_t hi[3][3];
  int32_t filter;          /* 0: thresholds on raw HSV; 1: filter F1 */
  int32_t chip;            /* statistics / count chip side */
  int32_t median;          /* 1: 3x3 median of V inside the chip */
  int32_t mm_min_range;    /* stretch only if hi - lo >= this */
  int32_t mm_min_frac_den; /* ... and each Otsu class holds >= N / den */
  int32_t v_trunc;         /* truncation level applied after the stretch */
  int32_t max_shift;       /* mask pixels whose V moved by more than this */
  int32_t bgr;             /* 1: byte order B,G,R */
  int32_t u16_scale;       /* uint16 reflectance that maps to 255 */
} sil_oracle_params;

enum { ORC_OK = 0, ORC_EINVAL = 1 };

/* Defaults: the class ranges of Sec. III-B "Auto-labeling Method"; the filter
 * constants are the project's reading of the filter paragraph, which names
 * operations but no parameters. */
int sil_oracle_params_default(sil_oracle_params* p) {
  if (!p) return ORC_EINVAL;
  memset(p, 0, sizeof(*p));
  /* thick ice (0,0,205)-(185,255,255) */
  p->lo[0][0] = 0; p->lo[0][1] = 0; p->lo[0][2] = 205;
  p->hi[0][0] = 185; p->hi[0][1] = 255; p->hi[0][2] = 255;
  /* thin ice (0,0,31)-(185,255,204) */
  p->lo[1][0] = 0; p->lo[1][1] = 0; p->lo[1][2] = 31;
  p->hi[1][0] = 185; p->hi[1][1] = 255; p->hi[1][2] = 204;
  /* open water (0,0,0)-(185,255,30) */
  p->lo[2][0] = 0; p->lo[2][1] = 0; p->lo[2][2] = 0;
  p->hi[2][0] = 185; p->hi[2][1] = 255; p->hi[2][2] = 30;
  p->filter = 1;
  p->chip = 256;
  p->median = 1;
  p->mm_min_range = 64;
  p->mm_min_frac_den = 16;
  p->v_trunc = 255;
  p->max_shift = 255;
  p->bgr = 0;
  p->u16_scale = 10000;
  return ORC_OK;
}

int sil_oracle_params_check(const sil_oracle_params* p) {
  if (!p) return ORC_EINVAL;
  for (int k = 0; k < 3; ++k)
    for (int c = 0; c < 3; ++c)
      if (p->lo[k][c] > p->hi[k][c]) return ORC_EINVAL;
  if (p->filter != 0 && p->filter != 1) return ORC_EINVAL;
  if (p->chip < 4 || p->chip > 512) return ORC_EINVAL;
  if (p->median != 0 && p->median != 1) return ORC_EINVAL;
  if (p->mm_min_range < 1 || p->mm_min_range > 255) return ORC_EINVAL;
  if (p->mm_min_frac_den < 1 || p->mm_min_frac_den > 65536) return ORC_EINVAL;
  if (p->v_trunc < 0 || p->v_trunc > 255) return ORC_EINVAL;
  if (p->max_shift < 0 || p->max_shift > 255) return ORC_EINVAL;
  if (p->bgr != 0 && p->bgr != 1) return ORC_EINVAL;
  if (p->u16_scale < 1 || p->u16_scale > 65535) return ORC_EINVAL;
  return ORC_OK;
}

/* Sec. III-A: 8-bit true colour.  uint16 reflectance is brought to 8 bit by
 * round-half-up of v * 255 / scale, clamped to 255 (the paper is silent on
 * this scaling; this is the project's reading). */
int sil_oracle_u16_to_u8(int v, int scale) {
  long long q = ((long long)v * 255 + scale / 2) / scale;
  return q > 255 ? 255 : (int)q;
}

/* Sec. III-B: RGB -> HSV in the 8-bit convention implied by the class bounds
 * (H in [0,179] as degrees / 2, S and V in [0,255]); integer, round half up.
 *   V = max, d = V - min, S = round(255 d / V),
 *   H = round(hue_degrees / 2) with 180 folded to 0. */
void sil_oracle_hsv(int r, int g, int b, int* h_out, int* s_out, int* v_out) {
  int v = r;
  if (g > v) v = g;
  if (b > v) v = b;
  int mn = r;
  if (g < mn) mn = g;
  if (b < mn) mn = b;
  int d = v - mn;

  int s = 0;
  if (v > 0) s = (510 * d + v) / (2 * v);

  int h = 0;
  if (d > 0) {
    int n; /* hue in degrees, times d */
    if (v == r)
      n = 60 * (g - b);
    else if (v == g)
      n = 120 * d + 60 * (b - r);
    else
      n = 240 * d + 60 * (r - g);
    if (n < 0) n += 360 * d;
    h = (n + d) / (2 * d);
    if (h == 180) h = 0;
  }
  *h_out = h;
  *s_out = s;
  *v_out = v;
}

/* Noise filtering (Sec. III-B filter paragraph): 3x3 median of the V plane
 * of one chip, window coordinates clamped to the chip (replicated border).
 * V and out are h x w, row-major, contiguous. */
static int cmp_int(const void* a, const void* b) {
  int x = *(const int*)a, y = *(const int*)b;
  return (x > y) - (x < y);
}

void sil_oracle_median3x3(const uint8_t* V, int h, int w, uint8_t* out) {
  for (int y = 0; y < h; ++y) {
    for (int x = 0; x < w; ++x) {
      int win[9];
      int n = 0;
      for (int dy = -1; dy <= 1; ++dy) {
        for (int dx = -1; dx <= 1; ++dx) {
          int yy = y + dy, xx = x + dx;
          if (yy < 0) yy = 0;
          if (yy > h - 1) yy = h - 1;
          if (xx < 0) xx = 0;
          if (xx > w - 1) xx = w - 1;
          win[n++] = V[(size_t)yy * w + xx];
        }
      }
      qsort(win, 9, sizeof(int), cmp_int);
      out[(size_t)y * w + x] = (uint8_t)win[4];
    }
  }
}

/* Otsu thresholding (Sec. III-B filter paragraph): the global threshold t of
 * a 256-bin histogram that maximises the between-class variance.  With
 * N = sum h, S_T = sum k h[k], w(t) = sum_{k<=t} h[k], s(t) = sum_{k<=t} k h[k],
 * the between-class variance is proportional to
 *     (S_T w - N s)^2 / (w (N - w)),
 * compared exactly by cross multiplication in 128-bit integers.  Thresholds
 * with an empty class are skipped; ties keep the smallest t; if no t splits
 * the pixels (a constant chip) the result is `fallback`.  Returns t. */
int sil_oracle_otsu(const uint64_t hist[256], int fallback) {
  uint64_t N = 0, ST = 0;
  for (int k = 0; k < 256; ++k) {
    N += hist[k];
    ST += (uint64_t)k * hist[k];
  }
  int best_t = -1;
  unsigned __int128 best_num = 0, best_den = 1;
  uint64_t w = 0, s = 0;
  for (int t = 0; t <= 254; ++t) {
    w += hist[t];
    s += (uint64_t)t * hist[t];
    if (w == 0 || w == N) continue;
    int64_t diff = (int64_t)(ST * w) - (int64_t)(N * s);
    uint64_t ad = diff < 0 ? (uint64_t)(-diff) : (uint64_t)diff;
    unsigned __int128 num = (unsigned __int128)ad * ad;
    unsigned __int128 den = (unsigned __int128)w * (N - w);
    if (best_t < 0 || num * best_den > best_num * den) {
      best_t = t;
      best_num = num;
      best_den = den;
    }
  }
  return best_t < 0 ? fallback : best_t;
}

/* Min-max normalisation (Sec. III-B filter paragraph): map [lo, hi] onto
 * [0, 255], round half up: floor(((v - lo) * 510 + (hi - lo)) / (2 (hi - lo))). */
int sil_oracle_stretch(int v, int lo, int hi) {
  int r = hi - lo;
  return ((v - lo) * 510 + r) / (2 * r);
}

/* Per-chip statistics, exported for tests. */
typedef struct sil_oracle_chip_stats {
  int32_t n;      /* pixels that are not nodata */
  int32_t lo, hi; /* min / max of the filtered V */
  int32_t t;      /* Otsu threshold */
  int32_t n0, n1; /* pixels at or below / above t */
  int32_t gate;   /* 1 if the min-max stretch is applied */
} sil_oracle_chip_stats;

/* Read pixel (y, x) as 8-bit R, G, B plus a nodata flag.  dtype 0 = uint8,
 * 1 = uint16 (little-endian); layout H x W x 3 interleaved, row pitch in
 * bytes. */
static void read_pixel(const uint8_t* img, int64_t pitch, int dtype, int64_t y,
                       int64_t x, const sil_oracle_params* p, int* r, int* g,
                       int* b, int* nodata) {
  int c[3];
  *nodata = 0;
  if (dtype == 0) {
    const uint8_t* px = img + y * pitch + x * 3;
    c[0] = px[0];
    c[1] = px[1];
    c[2] = px[2];
  } else {
    const uint8_t* px = img + y * pitch + x * 6;
    int raw[3];
    for (int i = 0; i < 3; ++i) raw[i] = px[2 * i] | (px[2 * i + 1] << 8);
    if (raw[0] == 0 && raw[1] == 0 && raw[2] == 0) *nodata = 1;
    for (int i = 0; i < 3; ++i) c[i] = sil_oracle_u16_to_u8(raw[i], p->u16_scale);
  }
  if (p->bgr) {
    *r = c[2];
    *g = c[1];
    *b = c[0];
  } else {
    *r = c[0];
    *g = c[1];
    *b = c[2];
  }
}

/* The whole path on one request (Sec. III-B filter + auto-labeling, and the
 * map-reduce count).  img: H x W x 3 (uint8 or uint16), pitch bytes per row.
 * labels: H x W uint8 with label_pitch bytes per row (may be NULL).
 * vprime: H x W uint8 with vprime_pitch bytes per row (may be NULL): the
 * filter's corrected value V' of every pixel (V when the filter is off, 0 for
 * nodata), the value the class ranges are applied to.
 * counts: uint64[4] (overwritten).  chip_counts: uint32[ceil(H/C)][ceil(W/C)][4]
 * (may be NULL).  stats: one entry per chip, same order (may be NULL).
 * Returns 0, or 1 for invalid arguments. */
int sil_oracle_label_v(const void* img_v, int64_t H, int64_t W, int64_t pitch,
                       int dtype, const sil_oracle_params* p, uint8_t* labels,
                       int64_t label_pitch, uint8_t* vprime_out, int64_t vprime_pitch,
                       uint64_t* counts, uint32_t* chip_counts,
                       sil_oracle_chip_stats* stats) {
  const uint8_t* img = (const uint8_t*)img_v;
  if (!img || !p || !counts || H < 1 || W < 1) return ORC_EINVAL;
  if (dtype != 0 && dtype != 1) return ORC_EINVAL;
  if (sil_oracle_params_check(p) != ORC_OK) return ORC_EINVAL;
  int bpp = dtype == 0 ? 3 : 6;
  if (pitch < W * bpp) return ORC_EINVAL;
  if (labels && label_pitch < W) return ORC_EINVAL;
  if (vprime_out && vprime_pitch < W) return ORC_EINVAL;

  const int C = p->chip;
  const int64_t gy = (H + C - 1) / C, gx = (W + C - 1) / C;
  for (int k = 0; k < 4; ++k) counts[k] = 0;

  uint8_t* Hc = (uint8_t*)malloc((size_t)C * C);
  uint8_t* Sc = (uint8_t*)malloc((size_t)C * C);
  uint8_t* Vc = (uint8_t*)malloc((size_t)C * C);
  uint8_t* Vf = (uint8_t*)malloc((size_t)C * C);
  uint8_t* ND = (uint8_t*)malloc((size_t)C * C);
  if (!Hc || !Sc || !Vc || !Vf || !ND) {
    free(Hc); free(Sc); free(Vc); free(Vf); free(ND);
    return ORC_EINVAL;
  }

  for (int64_t cy = 0; cy < gy; ++cy) {
    for (int64_t cx = 0; cx < gx; ++cx) {
      const int64_t y0 = cy * C, x0 = cx * C;
      const int h = (int)((y0 + C <= H) ? C : H - y0);
      const int w = (int)((x0 + C <= W) ? C : W - x0);

      /* Step 1-2: decode and convert every pixel of the chip to HSV. */
      for (int y = 0; y < h; ++y) {
        for (int x = 0; x < w; ++x) {
          int r, g, b, nd, hh, ss, vv;
          read_pixel(img, pitch, dtype, y0 + y, x0 + x, p, &r, &g, &b, &nd);
          sil_oracle_hsv(r, g, b, &hh, &ss, &vv);
          Hc[y * w + x] = (uint8_t)hh;
          Sc[y * w + x] = (uint8_t)ss;
          Vc[y * w + x] = (uint8_t)vv;
          ND[y * w + x] = (uint8_t)nd;
        }
      }

      /* Step 3: noise filter. */
      if (p->filter && p->median)
        sil_oracle_median3x3(Vc, h, w, Vf);
      else
        memcpy(Vf, Vc, (size_t)h * w);

      /* Step 4: chip statistics over pixels that are not nodata. */
      sil_oracle_chip_stats st;
      memset(&st, 0, sizeof(st));
      uint64_t hist[256];
      memset(hist, 0, sizeof(hist));
      st.lo = 255;
      st.hi = 0;
      for (int i = 0; i < h * w; ++i) {
        if (ND[i]) continue;
        hist[Vf[i]] += 1;
        st.n += 1;
        if (Vf[i] < st.lo) st.lo = Vf[i];
        if (Vf[i] > st.hi) st.hi = Vf[i];
      }
      if (st.n == 0) { st.lo = 0; st.hi = 0; }
      st.t = sil_oracle_otsu(hist, st.lo);
      for (int i = 0; i < h * w; ++i)
        if (!ND[i] && Vf[i] <= st.t) st.n0 += 1;
      st.n1 = st.n - st.n0;

      /* Step 5: the gate for the min-max stretch. */
      st.gate = (st.hi - st.lo >= p->mm_min_range) &&
                ((int64_t)p->mm_min_frac_den * st.n0 >= st.n) &&
                ((int64_t)p->mm_min_frac_den * st.n1 >= st.n) && st.n > 0;
      if (stats) stats[cy * gx + cx] = st;

      uint32_t cc[4] = {0, 0, 0, 0};
      for (int y = 0; y < h; ++y) {
        for (int x = 0; x < w; ++x) {
          const int i = y * w + x;
          int vprime;
          if (p->filter) {
            vprime = st.gate ? sil_oracle_stretch(Vf[i], st.lo, st.hi) : Vf[i];
            if (vprime > p->v_trunc) vprime = p->v_trunc;
          } else {
            vprime = Vc[i];
          }
          /* Step 6: one inclusive mask per class, merged with precedence
           * thick > thin > water; no match -> masked. */
          int label = 3;
          for (int k = 0; k < 3; ++k) {
            int in = Hc[i] >= p->lo[k][0] && Hc[i] <= p->hi[k][0] &&
                     Sc[i] >= p->lo[k][1] && Sc[i] <= p->hi[k][1] &&
                     vprime >= p->lo[k][2] && vprime <= p->hi[k][2];
            if (in) { label = k; break; }
          }
          /* Step 7: overrides. */
          if (ND[i]) label = 3;
          if (p->filter && abs(vprime - (int)Vf[i]) > p->max_shift) label = 3;
          /* Step 8: map-reduce counts. */
          cc[label] += 1;
          if (labels) labels[(y0 + y) * label_pitch + (x0 + x)] = (uint8_t)label;
          if (vprime_out)
            vprime_out[(y0 + y) * vprime_pitch + (x0 + x)] = (uint8_t)(ND[i] ? 0 : vprime);
        }
      }
      for (int k = 0; k < 4; ++k) counts[k] += cc[k];
      if (chip_counts)
        for (int k = 0; k < 4; ++k) chip_counts[(cy * gx + cx) * 4 + k] = cc[k];
    }
  }
  free(Hc); free(Sc); free(Vc); free(Vf); free(ND);
  return ORC_OK;
}

int sil_oracle_label(const void* img_v, int64_t H, int64_t W, int64_t pitch,
                     int dtype, const sil_oracle_params* p, uint8_t* labels,
                     int64_t label_pitch, uint64_t* counts,
                     uint32_t* chip_counts, sil_oracle_chip_stats* stats) {
  return sil_oracle_label_v(img_v, H, W, pitch, dtype, p, labels, label_pitch, NULL, 0, counts,
                            chip_counts, stats);
}

/* Confusion counts of one label map against a reference map (Sec. IV-A,
 * evaluation metrics): conf[pred * 4 + ref] += 1 over all pixels, with
 * per-chip copies when chip_conf is not NULL.  Labels outside 0..3 are
 * invalid. */
int sil_oracle_confusion(const uint8_t* pred, int64_t pred_pitch,
                         const uint8_t* ref, int64_t ref_pitch, int64_t H,
                         int64_t W, int chip, uint64_t* conf,
                         uint32_t* chip_conf) {
  if (!pred || !ref || !conf || H < 1 || W < 1 || chip < 4 || chip > 512)
    return ORC_EINVAL;
  const int64_t gx = (W + chip - 1) / chip;
  const int64_t gy = (H + chip - 1) / chip;
  for (int k = 0; k < 16; ++k) conf[k] = 0;
  if (chip_conf)
    for (int64_t i = 0; i < gx * gy * 16; ++i) chip_conf[i] = 0;
  for (int64_t y = 0; y < H; ++y) {
    for (int64_t x = 0; x < W; ++x) {
      int a = pred[y * pred_pitch + x], b = ref[y * ref_pitch + x];
      if (a > 3 || b > 3) return ORC_EINVAL;
      conf[a * 4 + b] += 1;
      if (chip_conf) chip_conf[((y / chip) * gx + x / chip) * 16 + a * 4 + b] += 1;
    }
  }
  return ORC_OK;
}
