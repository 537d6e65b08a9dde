/*
 * sil.h -- C ABI of the GB300 sea-ice auto-labeler (libsil.so).
 *
 * The library labels Sentinel-2 true-colour imagery per pixel as thick /
 * snow-covered ice, young / thin ice, open water or masked, after a thin
 * cloud and shadow filter, and reduces the labels to per-chip and per-request
 * class counts, in one fused pass on the GPU.  It follows
 *   "A Parallel Workflow for Polar Sea-Ice Classification using Auto-labeling
 *    of Sentinel-2 Imagery" (arXiv 2403.13135):
 *   - Sec. III-A: inputs are bands 2/3/4 (blue, green, red) at 10 m, cut into
 *     256 x 256 chips;
 *   - Sec. III-B "Filtering Out the Thin Clouds and Shadows": the filter is
 *     built from HSV conversion, noise filtering, Otsu thresholding, min-max
 *     normalisation, truncated / binary thresholding, absolute difference and
 *     bit-wise operations (composition "F1", described at sil_params);
 *   - Sec. III-B "Auto-labeling Method": inclusive HSV ranges per class,
 *     thick (0,0,205)-(185,255,255), thin (0,0,31)-(185,255,204),
 *     water (0,0,0)-(185,255,30), one mask per class, masks merged;
 *   - Sec. III-B "PySpark Map-Reduce": map = label an image, reduce =
 *     collect; here the reduce is a class count per chip and per request.
 *
 * Label codes: 0 thick ice, 1 thin ice, 2 open water, 3 masked.
 *
 * Conventions for every call:
 *   - Image, label and count buffers are owned by the caller.  Unless a
 *     function says otherwise they are DEVICE pointers of the current device.
 *   - Calls are asynchronous on the given stream (NULL = legacy default
 *     stream); a returned SIL_OK means the work was enqueued.
 *   - Arguments are validated on the host before anything is launched; a bad
 *     argument returns SIL_EINVAL and launches nothing.  CUDA errors return
 *     SIL_ECUDA.  sil_last_error() gives a message for the calling thread.
 *   - All arithmetic is integer; results are bit-exact and do not depend on
 *     launch configuration, stream or batching.
 */
#ifndef SIL_H_
#define SIL_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SIL_ABI_VERSION 2

/* cudaStream_t is `struct CUstream_st*`; declared here so this header does
 * not need the CUDA headers. */
typedef struct CUstream_st* sil_stream;

typedef enum sil_status {
  SIL_OK = 0,
  SIL_EINVAL = 1,    /* invalid argument (nothing launched) */
  SIL_ENOMEM = 2,    /* device or host allocation failed */
  SIL_ECUDA = 3,     /* a CUDA call failed */
  SIL_ETIMEOUT = 4,  /* a bounded wait ran out */
  SIL_EBUSY = 5,     /* no free slot / memory right now; retry later */
  SIL_ECANCELED = 6  /* request cancelled or server shut down */
} sil_status;

typedef enum sil_dtype {
  SIL_U8 = 0,  /* 3 x uint8 per pixel (8-bit true colour) */
  SIL_U16 = 1  /* 3 x uint16 per pixel (S2 reflectance, little-endian) */
} sil_dtype;

/* Parameters.  Defaults (sil_params_default) are the paper's class ranges
 * (Sec. III-B) and the filter reading F1:
 *   V = max(R,G,B); Vf = 3x3 median of V inside the chip (replicated
 *   border) [noise filtering]; per chip over non-nodata pixels: lo/hi =
 *   min/max of Vf, Otsu threshold t [Otsu]; stretch Vf to [0,255] when
 *   hi - lo >= mm_min_range and both Otsu classes hold >= N/mm_min_frac_den
 *   pixels [min-max normalisation]; V' = min(stretched, v_trunc)
 *   [truncated threshold]; class masks by inclusive ranges on (H, S, V')
 *   merged with precedence thick > thin > water, no match -> masked
 *   [binary thresholds, bit-wise ops]; a pixel whose |V' - Vf| > max_shift
 *   is masked [absolute difference].
 * H is hue in degrees / 2 (0..179), S and V are 0..255, all rounded half up.
 * filter = 0 skips every filter step (classes on raw H, S, V).
 * uint16 input is brought to 8 bit by round(v * 255 / u16_scale) clamped to
 * 255; a pixel with all three raw channels 0 is S2 nodata and is masked. */
typedef struct sil_params {
  uint8_t lo[3][3];        /* [thick, thin, water][H, S, V], inclusive */
  uint8_t hi[3][3];        /* lo <= hi required */
  int32_t filter;          /* 0 or 1 (default 1) */
  int32_t chip;            /* statistics / count chip side, 4..512 (256) */
  int32_t median;          /* 0 or 1 (1) */
  int32_t mm_min_range;    /* 1..255 (64) */
  int32_t mm_min_frac_den; /* 1..65536 (16) */
  int32_t v_trunc;         /* 0..255 (255 = no truncation) */
  int32_t max_shift;       /* 0..255 (255 = never masks) */
  int32_t bgr;             /* 0: bytes are R,G,B; 1: B,G,R (OpenCV order) */
  int32_t u16_scale;       /* 1..65535 (10000) */
} sil_params;

/* Fill *p with the defaults.  Returns SIL_EINVAL if p is NULL. */
sil_status sil_params_default(sil_params* p);

/* SIL_OK if every field is in range, else SIL_EINVAL (message in
 * sil_last_error). */
sil_status sil_params_validate(const sil_params* p);

/* Static text for a status code; never NULL. */
const char* sil_status_string(sil_status s);

/* Message of the last failed call on this host thread ("" if none). */
const char* sil_last_error(void);

/* Library ABI version (SIL_ABI_VERSION). */
int sil_version(void);

/* Label one request (a tile or a scene), fused single pass on the GPU.
 *   img          device, H x W pixels, 3 interleaved channels of dt, rows
 *                pitch_bytes apart (pitch_bytes >= 3 W sizeof(dt)); uint16
 *                images need 2-byte aligned img and pitch.  No alignment is
 *                required otherwise.
 *   H, W         >= 1, H * W < 2^40.
 *   p            host pointer; NULL = defaults.
 *   labels       device, H x W uint8 codes with label_pitch >= W bytes per
 *                row; NULL = do not write labels (counts only).
 *   counts       device uint64[4], OVERWRITTEN with the request's totals
 *                (thick, thin, water, masked); required.
 *   chip_counts  device uint32[ceil(H/chip)][ceil(W/chip)][4] row-major, one
 *                entry per chip of the grid anchored at (0,0); may be NULL.
 * Statistics (Otsu, min/max) are taken per chip (Sec. III-A / III-C: the
 * paper filters 256 x 256 chips).  Nothing is allocated; the call only
 * enqueues a memset of counts and one kernel.  (uint8 requests without H/S
 * ranges whose chips number at most a quarter of the device's resident
 * CTAs run on clusters of four CTAs per chip, one row slice each; the
 * results are the same bit for bit.) */
sil_status sil_label(const void* img, int64_t H, int64_t W, int64_t pitch_bytes,
                     sil_dtype dt, const sil_params* p, uint8_t* labels,
                     int64_t label_pitch, uint64_t* counts,
                     uint32_t* chip_counts, sil_stream stream);

/* sil_label plus the filter's corrected value: vprime = DEVICE uint8 H x W
 * with vprime_pitch bytes per row (NULL: none) receives V' of every pixel,
 * the value the class ranges are applied to (Sec. III-B): V after the 3x3
 * median, the gated min-max stretch and the truncation; V when the filter is
 * off; 0 for nodata.  Scaling a pixel's R, G, B by V'/V gives the filtered
 * image the paper feeds to its U-Net (Sec. III-C; see
 * sil_unet_forward_filtered).  SIL_EINVAL also when vprime_pitch < W. */
sil_status sil_label_v(const void* img, int64_t H, int64_t W, int64_t pitch_bytes,
                       sil_dtype dt, const sil_params* p, uint8_t* labels,
                       int64_t label_pitch, uint8_t* vprime, int64_t vprime_pitch,
                       uint64_t* counts, uint32_t* chip_counts, sil_stream stream);

/* Same as sil_label but the image, labels and counts are HOST buffers; the
 * library stages them through its own device buffers and returns when the
 * results are in host memory.  The image is cut into stripes of whole chip
 * rows: the copy in of a stripe, the labelling of the previous one (on
 * `stream`) and the copy back of the one before run concurrently (two
 * internal streams ordered after earlier work on `stream`).  Pinned host
 * memory gives the fastest copies.  labels and chip_counts may be NULL.
 * Device buffers, streams and events are cached per host thread and device
 * and reused across calls. */
sil_status sil_label_host(const void* img, int64_t H, int64_t W,
                          int64_t pitch_bytes, sil_dtype dt, const sil_params* p,
                          uint8_t* labels, int64_t label_pitch,
                          uint64_t* counts, uint32_t* chip_counts,
                          sil_stream stream);

/* ---------------------------------------------------------------------
 * Batched labeling (one persistent launch over a work queue of uneven
 * tiles, captured in a CUDA graph).  Mirrors the paper's PySpark map over
 * a collection of images (Sec. III-B "PySpark Map-Reduce"): each tile is
 * labelled independently and reduced to its own counts.
 * ------------------------------------------------------------------- */
typedef struct sil_tile {
  const void* img;       /* device */
  int64_t H, W, pitch_bytes;
  uint8_t* labels;       /* device, may be NULL */
  int64_t label_pitch;
  uint64_t* counts;      /* device uint64[4], overwritten */
  uint32_t* chip_counts; /* device, may be NULL */
} sil_tile;

typedef struct sil_ctx sil_ctx;

/* Create a context on `device` (the current device is restored on return).
 * The context owns the batch work queue, tile descriptors, graph cache and
 * autotune results; it is not thread-safe (one host thread at a time). */
sil_status sil_ctx_create(sil_ctx** ctx, int device);
void sil_ctx_destroy(sil_ctx* ctx);

/* Label n tiles (host array of descriptors) with one persistent kernel.
 * All tiles share dt and p.  The launch is recorded once into a CUDA graph
 * per (n, dt, params, tile list) and replayed when the same batch comes
 * again.  Returns after enqueueing on `stream`. */
sil_status sil_label_batch(const sil_tile* tiles, int32_t n, sil_dtype dt,
                           const sil_params* p, sil_ctx* ctx, sil_stream stream);

/* Batched labelling that allocates nothing (the paper has no counterpart;
 * this exists for callers of this library that may not allocate device
 * memory: code running inside a framework whose caching allocator owns all
 * device memory, plug-ins and callbacks that must not call cudaMalloc
 * because it can block or synchronise the device, and hosts with a fixed
 * device-memory budget set up front).  Same work and results as
 * sil_label_batch, without a context: the request descriptors, chip prefix
 * sums and work-queue head live in one fixed device array inside the
 * library (about 22.5 KB, kept by every GPU that loads the library until
 * the process exits).
 *   tiles  host array of n descriptors, 1 <= n <= 256; more is rejected
 *          with SIL_EINVAL and a message naming the limit.
 * The first call on a device looks up the array's device address (once per
 * device and CUDA context, with that device current; again after the
 * context has been replaced, e.g. by cudaDeviceReset).  Every call shares
 * the array and leaves the last call's descriptors in it (the queue head
 * and each tile's counts are zeroed by the call itself): calls whose work
 * overlaps on the GPU -- for example on two streams without ordering
 * between them -- race and must not be made; calls on one stream are
 * ordered.  The descriptors are copied to the array from the call's own
 * stack (pageable memory), so the call may block the host until earlier
 * work on `stream` has drained, and it returns SIL_EINVAL without doing
 * anything while `stream` is being captured (a recorded copy would read
 * that stack after the call returned).  Calls no cudaMalloc, cudaFree or
 * other allocating routine.  Asynchronous on `stream` otherwise. */
sil_status sil_label_batch_noalloc(const sil_tile* tiles, int32_t n, sil_dtype dt,
                                   const sil_params* p, sil_stream stream);

/* A schedule of the batched kernel (sil_label_batch). */
typedef struct sil_tuning {
  int32_t schedule;    /* 0: persistent CTAs, fixed chip stride;
                          1: persistent CTAs taking chips from a work queue;
                          2: one CTA per chip (the hardware hands chips to
                             free slots) */
  int32_t ctas_per_sm; /* CTAs per SM of schedules 0 and 1; 0 for schedule 2 */
  int32_t threads;     /* threads per CTA: 256 (16 row bands) or 320 (20) */
  float us;            /* time of one batch when tuned (0: not tuned) */
} sil_tuning;

/* Pick the batched kernel's schedule for the given batch by timing every
 * candidate on `stream`: threads per CTA (256, 320) x {one CTA per chip;
 * persistent CTAs with a work queue or a fixed stride at each number of
 * CTAs per SM that fits}.  The winner is kept in ctx for the batch's class
 * -- device name, dtype, H/S ranges narrowed or not, chip size, and the
 * batch's tile count, chip count and chips per tile rounded down to powers
 * of two -- so that later sil_label_batch calls of that class use it, and
 * is saved to a cache file that sil_ctx_create loads: SIL_AUTOTUNE_CACHE if
 * set (empty: no file), else $XDG_CACHE_HOME/sil-autotune.txt or
 * $HOME/.cache/sil-autotune.txt (one text line per class).  Blocks until
 * the timing is done.  best (may be NULL) receives the winner.  Untuned
 * classes run one 256-thread CTA per chip.  (Pixels per thread, 16, and
 * the row-staging depth, 3 slots, are fixed by the kernel's design.) */
sil_status sil_autotune_ex(const sil_tile* tiles, int32_t n, sil_dtype dt,
                           const sil_params* p, sil_ctx* ctx, sil_stream stream,
                           sil_tuning* best);

/* sil_autotune_ex reporting only the winner's CTAs per SM (0 when one CTA
 * per chip won); best_ctas_per_sm may be NULL. */
sil_status sil_autotune(const sil_tile* tiles, int32_t n, sil_dtype dt,
                        const sil_params* p, sil_ctx* ctx, sil_stream stream,
                        int32_t* best_ctas_per_sm);

/* The schedule sil_label_batch would use for this batch (no launch);
 * *tuned (may be NULL) = 1 if it comes from a tuning, 0 if the default. */
sil_status sil_batch_tuning(const sil_tile* tiles, int32_t n, sil_dtype dt,
                            const sil_params* p, sil_ctx* ctx, sil_tuning* out,
                            int32_t* tuned);

/* ---------------------------------------------------------------------
 * Served labeling: a continuous-batching request loop.  Requests arrive at
 * any time with HOST images (pinned memory recommended); they are admitted
 * in arrival order when device memory and a request slot are free, and
 * copied in on an ingest stream.  After its image copy, each request is
 * published to a device-resident request ring: its descriptor, its "ready"
 * word and the ring's count of published chips are written by copies that
 * follow the image copy on the same stream.  A persistent kernel (one CTA
 * per resident slot) claims published chips one at a time, in publication
 * order, with an atomic compare-and-swap on the ring's claim counter, so
 * requests that arrive while others run are taken up by the running kernel
 * without a new launch; the CTA that finishes a request's last chip marks
 * the request complete in host-mapped memory, and its results are copied
 * back on an egress stream.  Every device wait is bounded: a CTA with no
 * published chip for idle_timeout_us exits (the host relaunches the kernel
 * when work arrives), and a chip whose request's ready word has not arrived
 * within ready_timeout_ms is skipped and its request ends with
 * SIL_ETIMEOUT.
 * ------------------------------------------------------------------- */
typedef struct sil_server sil_server;

typedef struct sil_server_config {
  int32_t device;             /* CUDA device */
  int32_t max_inflight;       /* request slots (default 64) */
  int64_t device_mem_budget;  /* bytes of device memory for request buffers;
                                 0 = 50% of free memory at create */
  int32_t max_batch;          /* unused (the ring kernel takes requests one
                                 chip at a time); kept for compatibility */
  int32_t want_labels;        /* 1: copy labels back (default 1) */
  int32_t ready_timeout_ms;   /* device wait for a published request's
                                 image (default 2000) */
  int32_t idle_timeout_us;    /* a kernel CTA with no work exits after this
                                 (default 5000) */
} sil_server_config;

typedef struct sil_request_result {
  int64_t id;
  sil_status status;
  uint64_t counts[4];
  double t_submit_ms, t_admit_ms, t_done_ms; /* host monotonic clock */
} sil_request_result;

sil_status sil_server_config_default(sil_server_config* cfg);
sil_status sil_server_create(sil_server** srv, const sil_server_config* cfg,
                             sil_dtype dt, const sil_params* p);
/* Submit one request.  img and labels are HOST buffers that must stay valid
 * until the request completes (labels may be NULL).  chip_counts (host, may
 * be NULL) receives the per-chip counts.  *id receives the request id.
 * Returns SIL_EBUSY if the request can never fit the memory budget. */
sil_status sil_server_submit(sil_server* srv, const void* img, int64_t H,
                             int64_t W, int64_t pitch_bytes, uint8_t* labels,
                             int64_t label_pitch, uint32_t* chip_counts,
                             int64_t* id);
/* Wait up to timeout_ms (-1 = no limit) for request `id` to complete.
 * SIL_OK once it has completed, whatever its outcome: out->status is the
 * request's own status (SIL_OK; SIL_ETIMEOUT when the device's wait for its
 * image ran out; SIL_ECANCELED; SIL_ECUDA), and the request is released.
 * SIL_ETIMEOUT if it did not complete within timeout_ms (it stays
 * queryable); SIL_EINVAL for an unknown id. */
sil_status sil_server_wait(sil_server* srv, int64_t id, int64_t timeout_ms,
                           sil_request_result* out);
/* Non-blocking: SIL_OK and *out filled (out->status = the request's
 * status) if done, SIL_EBUSY if not yet, SIL_EINVAL for an unknown id. */
sil_status sil_server_poll(sil_server* srv, int64_t id, sil_request_result* out);
/* Cancel a request that has not been admitted yet (SIL_EBUSY if it is
 * already running). */
sil_status sil_server_cancel(sil_server* srv, int64_t id);
/* Persistent-kernel launches since the server was created and chips
 * published to its ring (either pointer may be NULL).  Requests that arrive
 * while the kernel runs are taken up without a launch. */
sil_status sil_server_stats(sil_server* srv, int64_t* kernel_launches,
                            int64_t* chips_published);

/* Test hook for the bounded device waits (no GPU fault): while set, the
 * next request to be published gets its descriptor and chips published but
 * never its ready word, so every chip of it waits ready_timeout_ms and the
 * request completes with SIL_ETIMEOUT; later requests are unaffected.
 * skip_ready = 0 clears the hook. */
sil_status sil_server_set_fault(sil_server* srv, int32_t skip_ready);

/* Stop accepting work, cancel pending requests, wait for running ones and
 * free everything. */
void sil_server_destroy(sil_server* srv);

/* ---------------------------------------------------------------------
 * Confusion counts of a label map against a reference map (Sec. IV-A:
 * accuracy, precision, recall, F1 and the confusion matrix are computed from
 * these counts).  conf: device uint64[4][4] indexed [pred][ref], overwritten;
 * chip_conf: device uint32[gy][gx][4][4] or NULL.  Labels must be 0..3.
 * ------------------------------------------------------------------- */
sil_status sil_confusion(const uint8_t* pred, int64_t pred_pitch,
                         const uint8_t* ref, int64_t ref_pitch, int64_t H,
                         int64_t W, int32_t chip, uint64_t* conf,
                         uint32_t* chip_conf, sil_stream stream);

/* Render labels as the paper's colour masks (Sec. III-B: each class mask
 * gets its own colour; Fig. 3 legend: thick ice red, thin ice blue, open
 * water green; masked pixels black).  rgb: device, H x W x 3 uint8 with
 * rgb_pitch bytes per row. */
sil_status sil_render(const uint8_t* labels, int64_t label_pitch, int64_t H,
                      int64_t W, uint8_t* rgb, int64_t rgb_pitch,
                      sil_stream stream);

/* ---------------------------------------------------------------------
 * Evaluation metrics (Sec. IV-A "Evaluation Metrics"): accuracy,
 * precision, recall, F1 score, and the confusion matrix whose element in
 * row A, column B is the number of pixels predicted as A over the number of
 * pixels of reference class B (each column adds up to 1).  Computed on the
 * host from the counts of sil_confusion.  Over the paper's three classes:
 * pixels whose reference is masked (code 3) are left out; a prediction of
 * masked counts as a miss of the pixel's reference class (row 3 of the
 * matrix).  A ratio whose denominator is zero is 0.  The paper reports one
 * precision / recall / F1 figure per model; macro_* are the unweighted
 * means over the three classes, weighted_* the means weighted by each
 * class's reference pixel count.
 * ------------------------------------------------------------------- */
typedef struct sil_metrics {
  double accuracy;
  double precision[3], recall[3], f1[3];  /* thick, thin, water */
  double macro_precision, macro_recall, macro_f1;
  double weighted_precision, weighted_recall, weighted_f1;
  double matrix[4][4];  /* [pred][ref]; columns 0..2 sum to 1, column 3 is 0 */
  uint64_t support[3];  /* reference pixels of each class */
} sil_metrics;

/* conf: HOST uint64[4][4] indexed [pred][ref] (as sil_confusion writes it,
 * copied to the host).  SIL_EINVAL on NULL. */
sil_status sil_metrics_from_confusion(const uint64_t* conf, sil_metrics* out);

/* The paper's training pairs (Sec. III-A colour masks; Sec. III-C cuts
 * scenes into 256 x 256 images): chips k0 .. k0 + n - 1 of the chip grid
 * of side `chip` anchored at (0, 0), row-major over the grid, each as the
 * image chip and its colour-mask chip (red thick ice, blue thin ice, green
 * open water, black masked), zero past the scene's right and bottom edges.
 *   img      DEVICE uint8 H x W x 3, pitch_bytes per row (>= 3 W)
 *   labels   DEVICE uint8 H x W codes 0..3, label_pitch per row (>= W)
 *   chips    DEVICE uint8 [n][chip][chip][3] or NULL
 *   masks    DEVICE uint8 [n][chip][chip][3] or NULL
 * chip 4..512; 0 <= k0, k0 + n <= the grid's chip count, n >= 1.
 * Asynchronous on `stream`. */
sil_status sil_export_chips(const uint8_t* img, int64_t H, int64_t W,
                            int64_t pitch_bytes, const uint8_t* labels,
                            int64_t label_pitch, int32_t chip, int64_t k0,
                            int64_t n, uint8_t* chips, uint8_t* masks,
                            sil_stream stream);

#ifdef __cplusplus
}
#endif
#endif /* SIL_H_ */
