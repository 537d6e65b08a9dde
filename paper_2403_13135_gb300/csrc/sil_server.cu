// sil_server.cu -- continuous-batching labelling server (host runtime).
//
// Requests carry HOST images.  A worker thread admits them in arrival order
// while a request slot and room in a device arena are free, copies each
// image into the arena on an ingest stream, and launches the persistent
// batch kernel over every admitted request whose copy has been issued
// (waiting on their copy events, not on the host).  Results go back on an
// egress stream; completion is observed through events.  Requests that
// arrive while others are on the GPU are admitted as memory frees up, and
// their copies overlap the running kernels.  The paper's equivalent is the
// Spark driver distributing images to executors and collecting the labelled
// results (Sec. III-B "PySpark Map-Reduce").
//
// No kernel waits on the host or on another kernel: the only waits are host
// waits on CUDA events and condition variables, all of them bounded by the
// caller's timeout.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "sil.h"
#include "sil_batch.h"
#include "sil_common.h"

namespace sil {
sil_status check_request(const void* img, int64_t H, int64_t W, int64_t pitch,
                         sil_dtype dt, const uint8_t* labels, int64_t lpitch,
                         const uint64_t* counts);
}

using namespace sil;

namespace {

double now_ms() {
  using namespace std::chrono;
  return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

// First-fit allocator over one device arena (offsets, 256-byte granules).
class Arena {
 public:
  explicit Arena(size_t bytes) : size_(bytes) { free_[0] = bytes; }
  bool alloc(size_t bytes, size_t* off) {
    bytes = (bytes + 255) & ~size_t(255);
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= bytes) {
        *off = it->first;
        const size_t rest = it->second - bytes;
        const size_t at = it->first + bytes;
        free_.erase(it);
        if (rest) free_[at] = rest;
        used_ += bytes;
        return true;
      }
    }
    return false;
  }
  void release(size_t off, size_t bytes) {
    bytes = (bytes + 255) & ~size_t(255);
    used_ -= bytes;
    auto it = free_.emplace(off, bytes).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }
  size_t size() const { return size_; }

 private:
  size_t size_;
  size_t used_ = 0;
  std::map<size_t, size_t> free_;
};

enum class St { kPending, kAdmitted, kRunning, kDone, kCanceled };

struct Request {
  int64_t id = 0;
  const void* img = nullptr;
  int64_t H = 0, W = 0, pitch = 0;
  uint8_t* labels = nullptr;
  int64_t lpitch = 0;
  uint32_t* chip_counts = nullptr;
  int gx = 0, gy = 0;
  // device layout inside the arena
  size_t off = 0, bytes = 0, dpitch = 0, o_lab = 0, o_cnt = 0, o_cc = 0;
  int slot = -1;  // index into the pinned result area
  St st = St::kPending;
  sil_status status = SIL_OK;
  uint64_t counts[4] = {0, 0, 0, 0};
  double t_submit = 0, t_admit = 0, t_done = 0;
  cudaEvent_t ev_in = nullptr, ev_done = nullptr;
};

constexpr int kDescSlots = 8;

}  // namespace

struct sil_server {
  sil_server_config cfg{};
  sil_dtype dt = SIL_U8;
  sil_params params{};
  DevParams dp{};
  int bpp = 3;
  int grid = 1;
  uint8_t* arena_mem = nullptr;
  std::unique_ptr<Arena> arena;
  cudaStream_t s_in = nullptr, s_comp = nullptr, s_out = nullptr;
  // pinned per-slot results: counts (4 x u64)
  uint64_t* h_counts = nullptr;
  std::vector<int> free_slots;
  // descriptor ring for batch launches
  Req* d_reqs[kDescSlots] = {};
  int64_t* d_prefix[kDescSlots] = {};
  unsigned long long* d_head[kDescSlots] = {};
  Req* h_reqs[kDescSlots] = {};
  int64_t* h_prefix[kDescSlots] = {};
  cudaEvent_t desc_done[kDescSlots] = {};
  int desc_next = 0;

  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Request*> pending;
  std::vector<Request*> admitted;  // copy issued, not yet launched
  std::vector<Request*> running;
  std::unordered_map<int64_t, std::unique_ptr<Request>> all;
  int64_t next_id = 1;
  bool stop = false;
  std::thread worker;
  std::atomic<int> worker_error{0};

  void run();
  void finish(Request* r, sil_status st);
};

namespace {

size_t request_bytes(const sil_server* s, Request* r) {
  const int64_t row = r->W * s->bpp;
  r->dpitch = size_t((row + 127) / 128 * 128);
  size_t off = r->dpitch * size_t(r->H);
  off = (off + 255) & ~size_t(255);
  r->o_lab = off;
  if (r->labels && s->cfg.want_labels) off += size_t(r->W * r->H);
  off = (off + 255) & ~size_t(255);
  r->o_cnt = off;
  off += 32;
  off = (off + 255) & ~size_t(255);
  r->o_cc = off;
  off += size_t(r->gx) * r->gy * 16;
  return off;
}

}  // namespace

void sil_server::finish(Request* r, sil_status st) {
  r->status = st;
  r->t_done = now_ms();
  r->st = (st == SIL_ECANCELED) ? St::kCanceled : St::kDone;
}

void sil_server::run() {
  cudaSetDevice(cfg.device);
  std::unique_lock<std::mutex> lk(mu);
  while (true) {
    if (stop && pending.empty() && admitted.empty() && running.empty()) break;
    bool progressed = false;
    // 1. admission: arrival order, while a slot and arena room are free
    while (!pending.empty() && !free_slots.empty()) {
      Request* r = pending.front();
      size_t off;
      if (!arena->alloc(r->bytes, &off)) break;
      pending.pop_front();
      r->off = off;
      r->slot = free_slots.back();
      free_slots.pop_back();
      r->st = St::kAdmitted;
      r->t_admit = now_ms();
      cudaError_t e = cudaMemcpy2DAsync(arena_mem + r->off, r->dpitch, r->img, r->pitch,
                                        r->W * bpp, r->H, cudaMemcpyHostToDevice, s_in);
      if (e == cudaSuccess) e = cudaEventRecord(r->ev_in, s_in);
      if (e != cudaSuccess) {
        arena->release(r->off, r->bytes);
        free_slots.push_back(r->slot);
        finish(r, SIL_ECUDA);
        cv_done.notify_all();
        continue;
      }
      admitted.push_back(r);
      progressed = true;
    }
    // 2. launch one persistent kernel over the admitted requests
    if (!admitted.empty()) {
      const int nb = std::min<int>(int(admitted.size()), std::max(1, cfg.max_batch));
      std::vector<Request*> batch(admitted.begin(), admitted.begin() + nb);
      admitted.erase(admitted.begin(), admitted.begin() + nb);
      const int ds = desc_next;
      desc_next = (desc_next + 1) % kDescSlots;
      lk.unlock();
      cudaEventSynchronize(desc_done[ds]);  // previous use of this slot done
      Req* hr = h_reqs[ds];
      int64_t* hp = h_prefix[ds];
      hp[0] = 0;
      for (int i = 0; i < nb; ++i) {
        Request* r = batch[i];
        Req& q = hr[i];
        q.img = arena_mem + r->off;
        q.H = r->H;
        q.W = r->W;
        q.pitch = int64_t(r->dpitch);
        q.labels = (r->labels && cfg.want_labels) ? arena_mem + r->off + r->o_lab : nullptr;
        q.lpitch = r->W;
        q.counts = reinterpret_cast<unsigned long long*>(arena_mem + r->off + r->o_cnt);
        q.chip_counts = reinterpret_cast<uint32_t*>(arena_mem + r->off + r->o_cc);
        q.gx = r->gx;
        q.gy = r->gy;
        q.chip_begin = hp[i];
        hp[i + 1] = hp[i] + int64_t(r->gx) * r->gy;
        cudaStreamWaitEvent(s_comp, r->ev_in, 0);
      }
      cudaError_t e = cudaMemcpyAsync(d_reqs[ds], hr, sizeof(Req) * nb, cudaMemcpyHostToDevice, s_comp);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_prefix[ds], hp, sizeof(int64_t) * (nb + 1), cudaMemcpyHostToDevice, s_comp);
      if (e == cudaSuccess) {
        BatchLaunch b{d_reqs[ds], d_prefix[ds], nb, int(dt), dp, params.chip, d_head[ds],
                      int(std::min<int64_t>(hp[nb], grid)), 1};
        e = launch_batch(b, s_comp);
      }
      if (e == cudaSuccess) e = cudaEventRecord(desc_done[ds], s_comp);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(s_out, desc_done[ds], 0);
      for (int i = 0; i < nb && e == cudaSuccess; ++i) {
        Request* r = batch[i];
        if (r->labels && cfg.want_labels)
          e = cudaMemcpy2DAsync(r->labels, r->lpitch, arena_mem + r->off + r->o_lab, r->W, r->W,
                                r->H, cudaMemcpyDeviceToHost, s_out);
        if (e == cudaSuccess)
          e = cudaMemcpyAsync(h_counts + 4 * r->slot, arena_mem + r->off + r->o_cnt, 32,
                              cudaMemcpyDeviceToHost, s_out);
        if (e == cudaSuccess && r->chip_counts)
          e = cudaMemcpyAsync(r->chip_counts, arena_mem + r->off + r->o_cc,
                              size_t(r->gx) * r->gy * 16, cudaMemcpyDeviceToHost, s_out);
        if (e == cudaSuccess) e = cudaEventRecord(r->ev_done, s_out);
      }
      lk.lock();
      for (Request* r : batch) {
        if (e != cudaSuccess) {
          worker_error = 1;
          finish(r, SIL_ECUDA);
          continue;
        }
        r->st = St::kRunning;
        running.push_back(r);
      }
      if (e != cudaSuccess) cv_done.notify_all();
      progressed = true;
    }
    // 3. completions
    bool done_any = false;
    for (size_t i = 0; i < running.size();) {
      Request* r = running[i];
      const cudaError_t q = cudaEventQuery(r->ev_done);
      if (q == cudaErrorNotReady) {
        ++i;
        continue;
      }
      if (q == cudaSuccess) memcpy(r->counts, h_counts + 4 * r->slot, 32);
      arena->release(r->off, r->bytes);
      free_slots.push_back(r->slot);
      finish(r, q == cudaSuccess ? SIL_OK : SIL_ECUDA);
      running[i] = running.back();
      running.pop_back();
      done_any = true;
    }
    if (done_any) {
      cv_done.notify_all();
      progressed = true;
    }
    if (!progressed) {
      // nothing to admit or launch: sleep until new work or a short poll tick
      cv_work.wait_for(lk, std::chrono::microseconds(running.empty() ? 2000 : 50));
    }
  }
}

extern "C" {

sil_status sil_server_config_default(sil_server_config* cfg) {
  if (!cfg) {
    set_error("sil_server_config_default: NULL");
    return SIL_EINVAL;
  }
  cfg->device = 0;
  cfg->max_inflight = 64;
  cfg->device_mem_budget = 0;
  cfg->max_batch = 32;
  cfg->want_labels = 1;
  return SIL_OK;
}

sil_status sil_server_create(sil_server** out, const sil_server_config* cfg_in, sil_dtype dt,
                             const sil_params* p) {
  if (!out) {
    set_error("sil_server_create: NULL");
    return SIL_EINVAL;
  }
  *out = nullptr;
  sil_server_config cfg;
  if (cfg_in)
    cfg = *cfg_in;
  else
    sil_server_config_default(&cfg);
  if (dt != SIL_U8 && dt != SIL_U16) {
    set_error("sil_server_create: dtype %d", int(dt));
    return SIL_EINVAL;
  }
  if (cfg.max_inflight < 1 || cfg.max_inflight > 4096 || cfg.max_batch < 1 ||
      cfg.device_mem_budget < 0) {
    set_error("sil_server_create: bad config");
    return SIL_EINVAL;
  }
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || cfg.device < 0 || cfg.device >= ndev) {
    set_error("sil_server_create: no CUDA device %d", cfg.device);
    return SIL_EINVAL;
  }
  auto s = std::make_unique<sil_server>();
  if (p)
    s->params = *p;
  else
    sil_params_default(&s->params);
  sil_status st = derive_params(&s->params, &s->dp);
  if (st != SIL_OK) return st;
  s->cfg = cfg;
  s->dt = dt;
  s->bpp = dt == SIL_U8 ? 3 : 6;
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(cfg.device);
  size_t fr = 0, tot = 0;
  cudaMemGetInfo(&fr, &tot);
  size_t budget = cfg.device_mem_budget > 0 ? size_t(cfg.device_mem_budget) : fr / 2;
  budget &= ~size_t(255);
  cudaError_t e = cudaMalloc(&s->arena_mem, budget);
  if (e != cudaSuccess) {
    cudaSetDevice(prev);
    set_error("sil_server_create: arena of %zu bytes: %s", budget, cudaGetErrorString(e));
    return SIL_ENOMEM;
  }
  s->arena.reset(new Arena(budget));
  e = cudaMallocHost(&s->h_counts, sizeof(uint64_t) * 4 * cfg.max_inflight);
  for (int i = 0; i < cfg.max_inflight; ++i) s->free_slots.push_back(cfg.max_inflight - 1 - i);
  for (int i = 0; i < kDescSlots && e == cudaSuccess; ++i) {
    e = cudaMalloc(&s->d_reqs[i], sizeof(Req) * cfg.max_batch);
    if (e == cudaSuccess) e = cudaMalloc(&s->d_prefix[i], sizeof(int64_t) * (cfg.max_batch + 1));
    if (e == cudaSuccess) e = cudaMalloc(&s->d_head[i], sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMallocHost(&s->h_reqs[i], sizeof(Req) * cfg.max_batch);
    if (e == cudaSuccess) e = cudaMallocHost(&s->h_prefix[i], sizeof(int64_t) * (cfg.max_batch + 1));
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->desc_done[i], cudaEventDisableTiming);
  }
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->s_in, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->s_comp, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->s_out, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    sil_server* raw = s.release();
    raw->stop = true;
    sil_server_destroy(raw);
    cudaSetDevice(prev);
    set_error("sil_server_create: %s", cudaGetErrorString(e));
    return SIL_ENOMEM;
  }
  int sms = 1;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, cfg.device);
  s->grid = sms * batch_max_ctas_per_sm(dt, s->dp.need_hs != 0, s->params.chip);
  cudaSetDevice(prev);
  sil_server* raw = s.release();
  raw->worker = std::thread([raw] { raw->run(); });
  *out = raw;
  return SIL_OK;
}

sil_status sil_server_submit(sil_server* srv, const void* img, int64_t H, int64_t W,
                             int64_t pitch_bytes, uint8_t* labels, int64_t label_pitch,
                             uint32_t* chip_counts, int64_t* id) {
  if (!srv || !id) {
    set_error("sil_server_submit: NULL");
    return SIL_EINVAL;
  }
  uint64_t dummy;
  sil_status st = check_request(img, H, W, pitch_bytes, srv->dt, labels, label_pitch, &dummy);
  if (st != SIL_OK) return st;
  auto r = std::make_unique<Request>();
  r->img = img;
  r->H = H;
  r->W = W;
  r->pitch = pitch_bytes;
  r->labels = labels;
  r->lpitch = label_pitch;
  r->chip_counts = chip_counts;
  r->gx = int((W + srv->params.chip - 1) / srv->params.chip);
  r->gy = int((H + srv->params.chip - 1) / srv->params.chip);
  r->bytes = request_bytes(srv, r.get());
  if (r->bytes > srv->arena->size()) {
    set_error("sil_server_submit: request needs %zu bytes, budget is %zu", r->bytes,
              srv->arena->size());
    return SIL_EBUSY;
  }
  if (cudaEventCreateWithFlags(&r->ev_in, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&r->ev_done, cudaEventDisableTiming) != cudaSuccess) {
    if (r->ev_in) cudaEventDestroy(r->ev_in);
    set_error("sil_server_submit: event creation failed");
    return SIL_ECUDA;
  }
  r->t_submit = now_ms();
  {
    std::lock_guard<std::mutex> g(srv->mu);
    if (srv->stop) {
      cudaEventDestroy(r->ev_in);
      cudaEventDestroy(r->ev_done);
      set_error("sil_server_submit: server is shutting down");
      return SIL_ECANCELED;
    }
    r->id = srv->next_id++;
    *id = r->id;
    srv->pending.push_back(r.get());
    srv->all.emplace(r->id, std::move(r));
  }
  srv->cv_work.notify_one();
  return SIL_OK;
}

static void fill_result(const Request* r, sil_request_result* out) {
  if (!out) return;
  out->id = r->id;
  out->status = r->status;
  memcpy(out->counts, r->counts, sizeof(out->counts));
  out->t_submit_ms = r->t_submit;
  out->t_admit_ms = r->t_admit;
  out->t_done_ms = r->t_done;
}

static void release_request(sil_server* srv, int64_t id) {
  auto it = srv->all.find(id);
  if (it == srv->all.end()) return;
  cudaEventDestroy(it->second->ev_in);
  cudaEventDestroy(it->second->ev_done);
  srv->all.erase(it);
}

sil_status sil_server_wait(sil_server* srv, int64_t id, int64_t timeout_ms,
                           sil_request_result* out) {
  if (!srv) {
    set_error("sil_server_wait: NULL");
    return SIL_EINVAL;
  }
  std::unique_lock<std::mutex> lk(srv->mu);
  auto it = srv->all.find(id);
  if (it == srv->all.end()) {
    set_error("sil_server_wait: unknown request %lld", (long long)id);
    return SIL_EINVAL;
  }
  Request* r = it->second.get();
  auto done = [r] { return r->st == St::kDone || r->st == St::kCanceled; };
  if (timeout_ms < 0)
    srv->cv_done.wait(lk, done);
  else if (!srv->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), done)) {
    set_error("sil_server_wait: request %lld not done after %lld ms", (long long)id,
              (long long)timeout_ms);
    return SIL_ETIMEOUT;
  }
  fill_result(r, out);
  const sil_status st = r->status;
  release_request(srv, id);
  return st == SIL_OK ? SIL_OK : st;
}

sil_status sil_server_poll(sil_server* srv, int64_t id, sil_request_result* out) {
  if (!srv) {
    set_error("sil_server_poll: NULL");
    return SIL_EINVAL;
  }
  std::lock_guard<std::mutex> g(srv->mu);
  auto it = srv->all.find(id);
  if (it == srv->all.end()) {
    set_error("sil_server_poll: unknown request %lld", (long long)id);
    return SIL_EINVAL;
  }
  Request* r = it->second.get();
  if (r->st != St::kDone && r->st != St::kCanceled) return SIL_EBUSY;
  fill_result(r, out);
  const sil_status st = r->status;
  release_request(srv, id);
  return st;
}

sil_status sil_server_cancel(sil_server* srv, int64_t id) {
  if (!srv) {
    set_error("sil_server_cancel: NULL");
    return SIL_EINVAL;
  }
  {
    std::lock_guard<std::mutex> g(srv->mu);
    auto it = srv->all.find(id);
    if (it == srv->all.end()) {
      set_error("sil_server_cancel: unknown request %lld", (long long)id);
      return SIL_EINVAL;
    }
    Request* r = it->second.get();
    if (r->st != St::kPending) {
      set_error("sil_server_cancel: request %lld already admitted", (long long)id);
      return SIL_EBUSY;
    }
    srv->pending.erase(std::find(srv->pending.begin(), srv->pending.end(), r));
    srv->finish(r, SIL_ECANCELED);
  }
  srv->cv_done.notify_all();
  return SIL_OK;
}

void sil_server_destroy(sil_server* srv) {
  if (!srv) return;
  {
    std::lock_guard<std::mutex> g(srv->mu);
    srv->stop = true;
    for (Request* r : srv->pending) srv->finish(r, SIL_ECANCELED);
    srv->pending.clear();
  }
  srv->cv_done.notify_all();
  srv->cv_work.notify_all();
  if (srv->worker.joinable()) srv->worker.join();
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(srv->cfg.device);
  if (srv->s_in) cudaStreamSynchronize(srv->s_in);
  if (srv->s_comp) cudaStreamSynchronize(srv->s_comp);
  if (srv->s_out) cudaStreamSynchronize(srv->s_out);
  for (auto& kv : srv->all) {
    cudaEventDestroy(kv.second->ev_in);
    cudaEventDestroy(kv.second->ev_done);
  }
  srv->all.clear();
  for (int i = 0; i < kDescSlots; ++i) {
    cudaFree(srv->d_reqs[i]);
    cudaFree(srv->d_prefix[i]);
    cudaFree(srv->d_head[i]);
    cudaFreeHost(srv->h_reqs[i]);
    cudaFreeHost(srv->h_prefix[i]);
    if (srv->desc_done[i]) cudaEventDestroy(srv->desc_done[i]);
  }
  cudaFreeHost(srv->h_counts);
  cudaFree(srv->arena_mem);
  if (srv->s_in) cudaStreamDestroy(srv->s_in);
  if (srv->s_comp) cudaStreamDestroy(srv->s_comp);
  if (srv->s_out) cudaStreamDestroy(srv->s_out);
  cudaSetDevice(prev);
  delete srv;
}

}  // extern "C"
