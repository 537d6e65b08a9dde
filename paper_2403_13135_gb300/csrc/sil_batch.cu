// sil_batch.cu -- batched labelling of uneven tiles with one persistent
// kernel over a device work queue of (tile, chip) items, launched through a
// captured CUDA graph; the schedule is picked by an autotuner.
//
// The paper maps an auto-labelling UDF over a distributed collection of
// images and reduces the results (Sec. III-B "PySpark Map-Reduce"); here the
// collection is a batch of device tiles, the map is one chip of one tile per
// work item and the reduce is each tile's class counts.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cstring>
#include <vector>

#include "sil.h"
#include "sil_batch.h"
#include "sil_chip.cuh"
#include "sil_common.h"
#include "sil_generic.cuh"

namespace sil {

size_t resident_smem_bytes(int dt, bool hs);
int device_sm_count();
sil_status check_request(const void* img, int64_t H, int64_t W, int64_t pitch,
                         sil_dtype dt, const uint8_t* labels, int64_t lpitch,
                         const uint64_t* counts);

// Zero every tile's counts and the work-queue head.
__global__ void k_batch_prologue(const Req* reqs, int n, unsigned long long* head) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0) *head = 0ull;
  if (i < n) {
#pragma unroll
    for (int c = 0; c < 4; ++c) reqs[i].counts[c] = 0ull;
  }
}

// Tile holding global chip k: largest t with prefix[t] <= k.
__device__ __forceinline__ int find_tile(const int64_t* prefix, int n, int64_t k) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (prefix[mid] <= k)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

template <int DT, bool HS, bool RESIDENT>
__global__ void __launch_bounds__(kThreads, (DT == SIL_U8) ? 2 : 1)
    k_label_batch(const Req* __restrict__ reqs, const int64_t* __restrict__ prefix,
                  int n, DevParams dp, int chip, unsigned long long* head,
                  int dynamic) {
  extern __shared__ __align__(128) uint8_t smem_raw[];
  __shared__ uint8_t lut[256];
  __shared__ long long s_next;
  __shared__ __align__(16) ChipStat st_generic;
  const int64_t total = prefix[n];
  int64_t k = blockIdx.x;
  if (dynamic) {
    if (threadIdx.x == 0) s_next = (long long)atomicAdd(head, 1ull);
    __syncthreads();
    k = s_next;
  }
  while (k < total) {
    const int t = find_tile(prefix, n, k);
    const Req& r = reqs[t];
    const int64_t local = k - prefix[t];
    const int64_t cy = local / r.gx, cx = local - cy * r.gx;
    if (RESIDENT) {
      ChipSmem<DT, HS>& sm = *reinterpret_cast<ChipSmem<DT, HS>*>(smem_raw);
      label_chip<DT, HS>(r, dp, chip, cy, cx, sm, lut, lut);  // (batches have no V' output)
    } else {
      label_chip_generic<DT, HS>(r, dp, chip, cy, cx, st_generic, lut);
    }
    if (dynamic) {
      __syncthreads();  // everyone has read s_next
      if (threadIdx.x == 0) s_next = (long long)atomicAdd(head, 1ull);
      __syncthreads();
      k = s_next;
    } else {
      k += gridDim.x;
    }
  }
}

template <int DT, bool HS, bool RESIDENT>
static cudaError_t launch_batch_t(const BatchLaunch& b, cudaStream_t s) {
  const size_t smem = RESIDENT ? resident_smem_bytes(DT, HS) : 0;
  k_batch_prologue<<<(b.n + 255) / 256, 256, 0, s>>>(b.reqs, b.n, b.head);
  k_label_batch<DT, HS, RESIDENT><<<b.grid, kThreads, smem, s>>>(
      b.reqs, b.prefix, b.n, b.dp, b.chip, b.head, b.dynamic);
  return cudaGetLastError();
}

cudaError_t launch_batch(const BatchLaunch& b, cudaStream_t s) {
  const bool hs = b.dp.need_hs != 0;
  const bool res = b.chip <= kResidentChip;
#define SIL_DISPATCH(DT)                                                  \
  if (hs)                                                                 \
    return res ? launch_batch_t<DT, true, true>(b, s)                     \
               : launch_batch_t<DT, true, false>(b, s);                   \
  return res ? launch_batch_t<DT, false, true>(b, s)                      \
             : launch_batch_t<DT, false, false>(b, s);
  if (b.dt == SIL_U8) {
    SIL_DISPATCH(SIL_U8)
  }
  SIL_DISPATCH(SIL_U16)
#undef SIL_DISPATCH
}

// Resident CTAs per SM the hardware allows for the batch kernel.
int batch_max_ctas_per_sm(int dt, bool hs, int chip) {
  int n = 0;
  const bool res = chip <= kResidentChip;
  const size_t smem = res ? resident_smem_bytes(dt, hs) : 0;
  const void* f = nullptr;
#define SIL_F(DT, HS, R) reinterpret_cast<const void*>(k_label_batch<DT, HS, R>)
  if (dt == SIL_U8)
    f = hs ? (res ? SIL_F(SIL_U8, true, true) : SIL_F(SIL_U8, true, false))
           : (res ? SIL_F(SIL_U8, false, true) : SIL_F(SIL_U8, false, false));
  else
    f = hs ? (res ? SIL_F(SIL_U16, true, true) : SIL_F(SIL_U16, true, false))
           : (res ? SIL_F(SIL_U16, false, true) : SIL_F(SIL_U16, false, false));
#undef SIL_F
  if (res) cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, f, kThreads, smem) != cudaSuccess || n < 1)
    n = 1;
  return n;
}

}  // namespace sil

// ---------------------------------------------------------------------------
// Context: work queue head, descriptor buffers, graph cache, tuning.
// ---------------------------------------------------------------------------
using namespace sil;

struct CachedGraph {
  std::vector<uint8_t> key;
  Req* d_reqs = nullptr;
  int64_t* d_prefix = nullptr;
  unsigned long long* d_head = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  uint64_t last_use = 0;
};

struct sil_ctx {
  int device = 0;
  int sms = 1;
  std::vector<CachedGraph> graphs;
  uint64_t tick = 0;
  // tuning: CTAs per SM and queue policy, per dtype (-1 = not tuned)
  int tuned_ctas[2] = {-1, -1};
  int tuned_dynamic[2] = {1, 1};
};

namespace {

struct DeviceGuard {
  int prev = 0;
  explicit DeviceGuard(int dev) {
    cudaGetDevice(&prev);
    cudaSetDevice(dev);
  }
  ~DeviceGuard() { cudaSetDevice(prev); }
};

void free_graph(CachedGraph& g) {
  if (g.exec) cudaGraphExecDestroy(g.exec);
  if (g.graph) cudaGraphDestroy(g.graph);
  cudaFree(g.d_reqs);
  cudaFree(g.d_prefix);
  cudaFree(g.d_head);
  g = CachedGraph();
}

// Builds the request descriptors and chip prefix sums of a batch.
sil_status build_batch(const sil_tile* tiles, int n, sil_dtype dt, const sil_params* p,
                       std::vector<Req>& reqs, std::vector<int64_t>& prefix) {
  const int chip = p ? p->chip : 256;
  reqs.resize(n);
  prefix.assign(n + 1, 0);
  for (int i = 0; i < n; ++i) {
    const sil_tile& t = tiles[i];
    sil_status st = check_request(t.img, t.H, t.W, t.pitch_bytes, dt, t.labels, t.label_pitch,
                                  t.counts);
    if (st != SIL_OK) return st;
    Req& r = reqs[i];
    r.img = static_cast<const uint8_t*>(t.img);
    r.H = t.H;
    r.W = t.W;
    r.pitch = t.pitch_bytes;
    r.labels = t.labels;
    r.lpitch = t.label_pitch;
    r.counts = reinterpret_cast<unsigned long long*>(t.counts);
    r.chip_counts = t.chip_counts;
    r.gx = int32_t((t.W + chip - 1) / chip);
    r.gy = int32_t((t.H + chip - 1) / chip);
    r.chip_begin = prefix[i];
    prefix[i + 1] = prefix[i] + int64_t(r.gx) * r.gy;
  }
  return SIL_OK;
}

std::vector<uint8_t> batch_key(const sil_tile* tiles, int n, sil_dtype dt, const sil_params* p,
                               int grid, int dynamic) {
  sil_params def;
  if (!p) {
    sil_params_default(&def);
    p = &def;
  }
  std::vector<uint8_t> k(sizeof(int) * 4 + sizeof(sil_params) + sizeof(sil_tile) * size_t(n));
  int hdr[4] = {n, int(dt), grid, dynamic};
  memcpy(k.data(), hdr, sizeof(hdr));
  memcpy(k.data() + sizeof(hdr), p, sizeof(sil_params));
  memcpy(k.data() + sizeof(hdr) + sizeof(sil_params), tiles, sizeof(sil_tile) * size_t(n));
  return k;
}

sil_status cuda_err(cudaError_t e, const char* what) {
  set_error("%s: %s", what, cudaGetErrorString(e));
  return SIL_ECUDA;
}

// Uploads descriptors (synchronously) and records prologue + persistent
// kernel into a graph.
sil_status make_graph(sil_ctx* ctx, const std::vector<Req>& reqs,
                      const std::vector<int64_t>& prefix, int dt, const DevParams& dp,
                      int chip, int grid, int dynamic, CachedGraph& g) {
  const int n = int(reqs.size());
  cudaError_t e;
  if ((e = cudaMalloc(&g.d_reqs, sizeof(Req) * n)) != cudaSuccess ||
      (e = cudaMalloc(&g.d_prefix, sizeof(int64_t) * (n + 1))) != cudaSuccess ||
      (e = cudaMalloc(&g.d_head, sizeof(unsigned long long))) != cudaSuccess) {
    free_graph(g);
    set_error("batch descriptors: %s", cudaGetErrorString(e));
    return SIL_ENOMEM;
  }
  if ((e = cudaMemcpy(g.d_reqs, reqs.data(), sizeof(Req) * n, cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMemcpy(g.d_prefix, prefix.data(), sizeof(int64_t) * (n + 1),
                      cudaMemcpyHostToDevice)) != cudaSuccess) {
    free_graph(g);
    return cuda_err(e, "batch descriptors upload");
  }
  cudaStream_t cs;
  if ((e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking)) != cudaSuccess) {
    free_graph(g);
    return cuda_err(e, "capture stream");
  }
  BatchLaunch b{g.d_reqs, g.d_prefix, n, dt, dp, chip, g.d_head, grid, dynamic};
  e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    cudaError_t le = launch_batch(b, cs);
    e = cudaStreamEndCapture(cs, &g.graph);
    if (le != cudaSuccess) e = le;
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&g.exec, g.graph, 0);
  cudaStreamDestroy(cs);
  if (e != cudaSuccess) {
    free_graph(g);
    return cuda_err(e, "batch graph capture");
  }
  (void)ctx;
  return SIL_OK;
}

}  // namespace

extern "C" {

sil_status sil_ctx_create(sil_ctx** ctx, int device) {
  if (!ctx) {
    set_error("sil_ctx_create: NULL");
    return SIL_EINVAL;
  }
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    set_error("sil_ctx_create: no CUDA device %d", device);
    return SIL_EINVAL;
  }
  sil_ctx* c = new sil_ctx();
  c->device = device;
  cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, device);
  if (c->sms < 1) c->sms = 1;
  *ctx = c;
  return SIL_OK;
}

void sil_ctx_destroy(sil_ctx* ctx) {
  if (!ctx) return;
  {
    DeviceGuard g(ctx->device);
    for (auto& cg : ctx->graphs) free_graph(cg);
  }
  delete ctx;
}

sil_status sil_label_batch(const sil_tile* tiles, int32_t n, sil_dtype dt,
                           const sil_params* p, sil_ctx* ctx, sil_stream stream) {
  if (!ctx || !tiles || n < 1) {
    set_error("sil_label_batch: NULL context/tiles or n < 1");
    return SIL_EINVAL;
  }
  DeviceGuard guard(ctx->device);
  DevParams dp;
  sil_status st = derive_params(p, &dp);
  if (st != SIL_OK) return st;
  if (dt != SIL_U8 && dt != SIL_U16) {
    set_error("dtype %d", int(dt));
    return SIL_EINVAL;
  }
  const int chip = p ? p->chip : 256;
  const int maxc = batch_max_ctas_per_sm(dt, dp.need_hs != 0, chip);
  const int ti = dt == SIL_U8 ? 0 : 1;
  const int cps = ctx->tuned_ctas[ti] > 0 ? std::min(ctx->tuned_ctas[ti], maxc) : maxc;
  const int dynamic = ctx->tuned_dynamic[ti];
  std::vector<Req> reqs;
  std::vector<int64_t> prefix;
  if ((st = build_batch(tiles, n, dt, p, reqs, prefix)) != SIL_OK) return st;
  const int64_t total = prefix[n];
  const int grid = int(std::min<int64_t>(total, int64_t(ctx->sms) * cps));
  std::vector<uint8_t> key = batch_key(tiles, n, dt, p, grid, dynamic);
  CachedGraph* hit = nullptr;
  for (auto& g : ctx->graphs)
    if (g.key == key) hit = &g;
  if (!hit) {
    CachedGraph g;
    if ((st = make_graph(ctx, reqs, prefix, dt, dp, chip, grid, dynamic, g)) != SIL_OK) return st;
    g.key = std::move(key);
    if (ctx->graphs.size() >= 16) {
      auto old = std::min_element(ctx->graphs.begin(), ctx->graphs.end(),
                                  [](const CachedGraph& a, const CachedGraph& b) {
                                    return a.last_use < b.last_use;
                                  });
      free_graph(*old);
      *old = std::move(g);
      hit = &*old;
    } else {
      ctx->graphs.push_back(std::move(g));
      hit = &ctx->graphs.back();
    }
  }
  hit->last_use = ++ctx->tick;
  cudaError_t e = cudaGraphLaunch(hit->exec, reinterpret_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_err(e, "sil_label_batch: graph launch");
  return SIL_OK;
}

sil_status sil_autotune(const sil_tile* tiles, int32_t n, sil_dtype dt, const sil_params* p,
                        sil_ctx* ctx, sil_stream stream, int32_t* best_ctas_per_sm) {
  if (!ctx || !tiles || n < 1) {
    set_error("sil_autotune: NULL context/tiles or n < 1");
    return SIL_EINVAL;
  }
  DeviceGuard guard(ctx->device);
  DevParams dp;
  sil_status st = derive_params(p, &dp);
  if (st != SIL_OK) return st;
  if (dt != SIL_U8 && dt != SIL_U16) {
    set_error("dtype %d", int(dt));
    return SIL_EINVAL;
  }
  const int chip = p ? p->chip : 256;
  const int maxc = batch_max_ctas_per_sm(dt, dp.need_hs != 0, chip);
  const int ti = dt == SIL_U8 ? 0 : 1;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best = 1e30f;
  int best_c = maxc, best_d = 1;
  for (int c = 1; c <= maxc; ++c) {
    for (int d = 0; d <= 1; ++d) {
      ctx->tuned_ctas[ti] = c;
      ctx->tuned_dynamic[ti] = d;
      // warm-up (also builds the graph), then the median of 3 timed runs
      if ((st = sil_label_batch(tiles, n, dt, p, ctx, stream)) != SIL_OK) goto done;
      float t[3];
      for (int rep = 0; rep < 3; ++rep) {
        cudaEventRecord(e0, s);
        if ((st = sil_label_batch(tiles, n, dt, p, ctx, stream)) != SIL_OK) goto done;
        cudaEventRecord(e1, s);
        if (cudaEventSynchronize(e1) != cudaSuccess) {
          st = cuda_err(cudaGetLastError(), "sil_autotune: timing");
          goto done;
        }
        cudaEventElapsedTime(&t[rep], e0, e1);
      }
      std::sort(t, t + 3);
      if (t[1] < best) {
        best = t[1];
        best_c = c;
        best_d = d;
      }
    }
  }
  ctx->tuned_ctas[ti] = best_c;
  ctx->tuned_dynamic[ti] = best_d;
  if (best_ctas_per_sm) *best_ctas_per_sm = best_c;
done:
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return st;
}

}  // extern "C"
