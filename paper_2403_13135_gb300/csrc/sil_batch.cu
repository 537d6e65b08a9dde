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
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <string>
#include <sys/stat.h>
#include <unistd.h>
#include <vector>

#include "sil.h"
#include "sil_batch.h"
#include "sil_batch_kernel.cuh"
#include "sil_common.h"

namespace sil {

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

cudaError_t launch_batch(const BatchLaunch& b, cudaStream_t s) {
  k_batch_prologue<<<(b.n + 255) / 256, 256, 0, s>>>(b.reqs, b.n, b.head);
  const bool hs = b.dp.need_hs != 0;
  if (b.dt == SIL_U8)
    return hs ? BatchKernels<SIL_U8, true>::launch(b, s) : BatchKernels<SIL_U8, false>::launch(b, s);
  return hs ? BatchKernels<SIL_U16, true>::launch(b, s) : BatchKernels<SIL_U16, false>::launch(b, s);
}

// The batch kernel instance of a (dtype, H/S, resident, threads) class.
static const void* batch_fn(int dt, bool hs, bool res, int threads) {
  if (dt == SIL_U8)
    return hs ? BatchKernels<SIL_U8, true>::fn(res, threads) : BatchKernels<SIL_U8, false>::fn(res, threads);
  return hs ? BatchKernels<SIL_U16, true>::fn(res, threads) : BatchKernels<SIL_U16, false>::fn(res, threads);
}

// Resident CTAs per SM the hardware allows for the batch kernel with
// `threads` threads per CTA; also sets both CTA sizes' shared-memory limits.
int batch_max_ctas_per_sm(int dt, bool hs, int chip, int threads) {
  const bool res = chip <= kResidentChip;
  int n = 0;
  for (int nt : {kThreadsNarrow, kThreadsWide}) {
    const size_t smem = res ? resident_smem_bytes(dt, hs, nt) : 0;
    const void* f = batch_fn(dt, hs, res, nt);
    if (res) set_resident_attrs(f, smem);
    if (nt != threads) continue;
    if (res) {
      n = resident_ctas_per_sm(f, nt, smem, tmem_plane(dt, hs) ? plane_cols(nt) : 0);
    } else if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, f, nt, 0) != cudaSuccess) {
      n = 1;
    }
  }
  cudaGetLastError();
  return n > 0 ? n : 1;
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

// A schedule of the batch kernel and its measured time.
struct Tuning {
  int schedule = kSchedPerChip;  // kSched*
  int ctas = -1;                 // CTAs per SM of the persistent schedules (-1: all that fit)
  int threads = kThreadsNarrow;  // threads per CTA
  float us = 0.f;                // time of one batch when it was tuned
};

struct sil_ctx {
  int device = 0;
  int sms = 1;
  std::string gpu;  // device name, part of every tuning key
  std::vector<CachedGraph> graphs;
  uint64_t tick = 0;
  // tuned schedules by batch class (tune_key); loaded from and saved to the
  // cache file (empty path: not persisted)
  std::map<std::string, Tuning> tuned;
  std::string cache_path;
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
                               int grid, int schedule, int threads) {
  sil_params def;
  if (!p) {
    sil_params_default(&def);
    p = &def;
  }
  std::vector<uint8_t> k(sizeof(int) * 5 + sizeof(sil_params) + sizeof(sil_tile) * size_t(n));
  int hdr[5] = {n, int(dt), grid, schedule, threads};
  memcpy(k.data(), hdr, sizeof(hdr));
  memcpy(k.data() + sizeof(hdr), p, sizeof(sil_params));
  memcpy(k.data() + sizeof(hdr) + sizeof(sil_params), tiles, sizeof(sil_tile) * size_t(n));
  return k;
}

sil_status cuda_err(cudaError_t e, const char* what) {
  set_error("%s: %s", what, cudaGetErrorString(e));
  return SIL_ECUDA;
}

int log2_bucket(int64_t v) {
  int b = 0;
  while (v > 1) {
    v >>= 1;
    ++b;
  }
  return b;
}

// Class of a batch for the tuning cache: the device, the kernel instance
// (dtype, H/S ranges, chip) and the batch's shape in powers of two (tiles,
// chips, chips per tile); the best schedule depends on these, not on the
// image contents.
std::string tune_key(const sil_ctx* ctx, int dt, bool hs, int chip, int n, int64_t chips) {
  char buf[256];
  snprintf(buf, sizeof(buf), "%s|dt%d|hs%d|chip%d|n%d|c%d|p%d", ctx->gpu.c_str(), dt, int(hs), chip,
           log2_bucket(n), log2_bucket(chips), log2_bucket(chips / (n > 0 ? n : 1)));
  std::string k(buf);
  for (char& c : k)
    if (c == ' ' || c == '\t' || c == '\n') c = '_';
  return k;
}

// Cache file: SIL_AUTOTUNE_CACHE if set (empty: none), else
// $XDG_CACHE_HOME/sil-autotune.txt or $HOME/.cache/sil-autotune.txt.
std::string cache_file() {
  const char* e = getenv("SIL_AUTOTUNE_CACHE");
  if (e) return std::string(e);
  const char* x = getenv("XDG_CACHE_HOME");
  if (x && *x) return std::string(x) + "/sil-autotune.txt";
  const char* h = getenv("HOME");
  if (h && *h) return std::string(h) + "/.cache/sil-autotune.txt";
  return std::string();
}

// One line per batch class: "<key> <schedule> <ctas> <threads> <us>".
std::map<std::string, Tuning> load_tuning(const std::string& path) {
  std::map<std::string, Tuning> m;
  if (path.empty()) return m;
  FILE* f = fopen(path.c_str(), "r");
  if (!f) return m;
  char key[256];
  Tuning t;
  while (fscanf(f, "%255s %d %d %d %f", key, &t.schedule, &t.ctas, &t.threads, &t.us) == 5) {
    if (t.schedule < kSchedStride || t.schedule > kSchedPerChip) continue;
    if (t.threads != kThreadsNarrow && t.threads != kThreadsWide) continue;
    m[key] = t;
  }
  fclose(f);
  return m;
}

// Merges the context's entries into the file (written whole to a temporary
// file, then renamed over it).  Failing to write is not an error of the
// tuning itself.
void save_tuning(const sil_ctx* ctx) {
  const std::string& path = ctx->cache_path;
  if (path.empty()) return;
  std::map<std::string, Tuning> m = load_tuning(path);
  for (const auto& kv : ctx->tuned) m[kv.first] = kv.second;
  const size_t slash = path.rfind('/');
  if (slash != std::string::npos && slash > 0) mkdir(path.substr(0, slash).c_str(), 0755);
  const std::string tmp = path + ".tmp" + std::to_string(long(getpid()));
  FILE* f = fopen(tmp.c_str(), "w");
  if (!f) return;
  for (const auto& kv : m)
    fprintf(f, "%s %d %d %d %.3f\n", kv.first.c_str(), kv.second.schedule, kv.second.ctas,
            kv.second.threads, kv.second.us);
  const bool ok = fclose(f) == 0;
  if (ok)
    rename(tmp.c_str(), path.c_str());
  else
    remove(tmp.c_str());
}

// Uploads descriptors (synchronously) and records prologue + persistent
// kernel into a graph.
sil_status make_graph(sil_ctx* ctx, const std::vector<Req>& reqs,
                      const std::vector<int64_t>& prefix, int dt, const DevParams& dp,
                      int chip, int grid, int schedule, int threads, CachedGraph& g) {
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
  BatchLaunch b{g.d_reqs, g.d_prefix, n, dt, dp, chip, g.d_head, grid, schedule, threads};
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

// The schedule a batch of this class runs with: the tuned one if there is
// one, else one CTA per chip of 256 threads.
Tuning batch_tuning(const sil_ctx* ctx, const std::string& key, int maxc) {
  auto it = ctx->tuned.find(key);
  Tuning t = it != ctx->tuned.end() ? it->second : Tuning();
  t.ctas = t.ctas > 0 ? std::min(t.ctas, maxc) : maxc;
  return t;
}

// Records (if needed) and replays the batch's graph for tuning t.
sil_status run_batch(const sil_tile* tiles, int32_t n, sil_dtype dt, const sil_params* p,
                     sil_ctx* ctx, cudaStream_t stream, const DevParams& dp,
                     const std::vector<Req>& reqs, const std::vector<int64_t>& prefix,
                     const Tuning& t) {
  const int chip = p ? p->chip : 256;
  const int64_t total = prefix[n];
  int schedule = t.schedule;
  if (schedule == kSchedPerChip && total > int64_t(0x7fffffff)) schedule = kSchedQueue;
  // CTAs per SM of a persistent schedule: at most what fits with this CTA size
  const int ctas = std::min(t.ctas, batch_max_ctas_per_sm(int(dt), dp.need_hs != 0, chip, t.threads));
  const int grid = schedule == kSchedPerChip ? int(total)
                                             : int(std::min<int64_t>(total, int64_t(ctx->sms) * ctas));
  std::vector<uint8_t> key = batch_key(tiles, n, dt, p, grid, schedule, t.threads);
  CachedGraph* hit = nullptr;
  for (auto& g : ctx->graphs)
    if (g.key == key) hit = &g;
  if (!hit) {
    CachedGraph g;
    sil_status st = make_graph(ctx, reqs, prefix, dt, dp, chip, grid, schedule, t.threads, g);
    if (st != SIL_OK) return st;
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
  cudaError_t e = cudaGraphLaunch(hit->exec, stream);
  if (e != cudaSuccess) return cuda_err(e, "sil_label_batch: graph launch");
  return SIL_OK;
}

// Shared argument checks and descriptor building of the batch entry points.
sil_status prepare_batch(const char* who, const sil_tile* tiles, int32_t n, sil_dtype dt,
                         const sil_params* p, sil_ctx* ctx, DevParams* dp, std::vector<Req>& reqs,
                         std::vector<int64_t>& prefix, std::string* key, int* maxc) {
  if (!ctx || !tiles || n < 1) {
    set_error("%s: NULL context/tiles or n < 1", who);
    return SIL_EINVAL;
  }
  sil_status st = derive_params(p, dp);
  if (st != SIL_OK) return st;
  if (dt != SIL_U8 && dt != SIL_U16) {
    set_error("%s: dtype %d", who, int(dt));
    return SIL_EINVAL;
  }
  if ((st = build_batch(tiles, n, dt, p, reqs, prefix)) != SIL_OK) return st;
  const int chip = p ? p->chip : 256;
  *maxc = batch_max_ctas_per_sm(dt, dp->need_hs != 0, chip, kThreadsNarrow);
  *key = tune_key(ctx, int(dt), dp->need_hs != 0, chip, n, prefix[n]);
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
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, device) == cudaSuccess) c->gpu = prop.name;
  if (c->gpu.empty()) c->gpu = "gpu";
  c->cache_path = cache_file();
  c->tuned = load_tuning(c->cache_path);
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
  if (!ctx) {
    set_error("sil_label_batch: NULL context");
    return SIL_EINVAL;
  }
  DeviceGuard guard(ctx->device);
  DevParams dp;
  std::vector<Req> reqs;
  std::vector<int64_t> prefix;
  std::string key;
  int maxc = 1;
  sil_status st = prepare_batch("sil_label_batch", tiles, n, dt, p, ctx, &dp, reqs, prefix, &key, &maxc);
  if (st != SIL_OK) return st;
  return run_batch(tiles, n, dt, p, ctx, reinterpret_cast<cudaStream_t>(stream), dp, reqs, prefix,
                   batch_tuning(ctx, key, maxc));
}

sil_status sil_batch_tuning(const sil_tile* tiles, int32_t n, sil_dtype dt, const sil_params* p,
                            sil_ctx* ctx, sil_tuning* out, int32_t* tuned) {
  if (!ctx || !out) {
    set_error("sil_batch_tuning: NULL context or output");
    return SIL_EINVAL;
  }
  DeviceGuard guard(ctx->device);
  DevParams dp;
  std::vector<Req> reqs;
  std::vector<int64_t> prefix;
  std::string key;
  int maxc = 1;
  sil_status st = prepare_batch("sil_batch_tuning", tiles, n, dt, p, ctx, &dp, reqs, prefix, &key, &maxc);
  if (st != SIL_OK) return st;
  const Tuning t = batch_tuning(ctx, key, maxc);
  out->schedule = t.schedule;
  out->ctas_per_sm = t.schedule == kSchedPerChip ? 0 : t.ctas;
  out->threads = t.threads;
  out->us = t.us;
  if (tuned) *tuned = ctx->tuned.count(key) ? 1 : 0;
  return SIL_OK;
}

sil_status sil_autotune_ex(const sil_tile* tiles, int32_t n, sil_dtype dt, const sil_params* p,
                           sil_ctx* ctx, sil_stream stream, sil_tuning* best_out) {
  if (!ctx) {
    set_error("sil_autotune: NULL context");
    return SIL_EINVAL;
  }
  DeviceGuard guard(ctx->device);
  DevParams dp;
  std::vector<Req> reqs;
  std::vector<int64_t> prefix;
  std::string key;
  int maxc = 1;
  sil_status st = prepare_batch("sil_autotune", tiles, n, dt, p, ctx, &dp, reqs, prefix, &key, &maxc);
  if (st != SIL_OK) return st;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  // candidates: for each CTA size, one CTA per chip and the persistent
  // schedules (queue, stride) at every CTAs-per-SM count that fits
  std::vector<Tuning> cand;
  for (int threads : {kThreadsNarrow, kThreadsWide}) {
    Tuning t;
    t.threads = threads;
    t.schedule = kSchedPerChip;
    const int maxt = batch_max_ctas_per_sm(int(dt), dp.need_hs != 0, p ? p->chip : 256, threads);
    t.ctas = maxt;
    cand.push_back(t);
    for (int c = 1; c <= maxt; ++c) {
      t.ctas = c;
      t.schedule = kSchedQueue;
      cand.push_back(t);
      t.schedule = kSchedStride;
      cand.push_back(t);
    }
  }
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  Tuning best;
  best.us = 1e30f;
  for (Tuning& t : cand) {
    // warm-up (also records the graph), then the median of 3 timed runs
    if ((st = run_batch(tiles, n, dt, p, ctx, s, dp, reqs, prefix, t)) != SIL_OK) break;
    float ms[3];
    for (int rep = 0; rep < 3 && st == SIL_OK; ++rep) {
      cudaEventRecord(e0, s);
      st = run_batch(tiles, n, dt, p, ctx, s, dp, reqs, prefix, t);
      cudaEventRecord(e1, s);
      if (st == SIL_OK && cudaEventSynchronize(e1) != cudaSuccess)
        st = cuda_err(cudaGetLastError(), "sil_autotune: timing");
      if (st == SIL_OK) cudaEventElapsedTime(&ms[rep], e0, e1);
    }
    if (st != SIL_OK) break;
    std::sort(ms, ms + 3);
    t.us = ms[1] * 1000.f;
    if (t.us < best.us) best = t;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != SIL_OK) return st;
  ctx->tuned[key] = best;
  save_tuning(ctx);
  if (best_out) {
    best_out->schedule = best.schedule;
    best_out->ctas_per_sm = best.schedule == kSchedPerChip ? 0 : best.ctas;
    best_out->threads = best.threads;
    best_out->us = best.us;
  }
  return SIL_OK;
}

sil_status sil_autotune(const sil_tile* tiles, int32_t n, sil_dtype dt, const sil_params* p,
                        sil_ctx* ctx, sil_stream stream, int32_t* best_ctas_per_sm) {
  sil_tuning t;
  const sil_status st = sil_autotune_ex(tiles, n, dt, p, ctx, stream, &t);
  if (st == SIL_OK && best_ctas_per_sm) *best_ctas_per_sm = t.ctas_per_sm;
  return st;
}

}  // extern "C"
