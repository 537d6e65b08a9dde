// sil_server.cu -- continuous-batching labelling server: a device-resident
// request ring read by a persistent kernel, and the host runtime around it.
//
// Host (one worker thread): admits requests in arrival order while a slot
// and room in a device arena are free, copies each image into the arena on
// the ingest stream and then publishes the request to the ring with more
// copies on the same stream (so they land after the image): the slot's
// descriptor with its ready word, its counts zeroed, a log entry (sequence
// number, chip count, slot) and the ring's count of published requests.  It keeps one
// persistent kernel running while there is published work, polls the
// completion words the kernel writes into host-mapped memory, and copies
// each finished request's labels, counts and status back on the egress
// stream.
//
// Device (k_served): every CTA claims its next chip from the oldest
// published request that has chips left (an atomic counter per request; an
// exhausted request moves the ring's cursor on by a compare-and-swap),
// checks the request's ready word, labels the chip with the same per-chip
// code as every other entry point, and counts it done; the CTA that
// finishes a request's last chip writes its completion word.  Every wait is
// bounded: no published chip for idle_ns -> the CTA exits; a ready word
// that does not arrive within ready_ns -> the request is marked timed out
// and its chips are skipped.
//
// The paper's equivalent is the Spark driver distributing images to
// executors and collecting the labelled results (Sec. III-B "PySpark
// Map-Reduce").
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
#include "sil_common.h"
#include "sil_served_kernel.cuh"

namespace sil {
sil_status check_request(const void* img, int64_t H, int64_t W, int64_t pitch,
                         sil_dtype dt, const uint8_t* labels, int64_t lpitch,
                         const uint64_t* counts);
int device_sm_count();

}  // namespace sil

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
        return true;
      }
    }
    return false;
  }
  void release(size_t off, size_t bytes) {
    bytes = (bytes + 255) & ~size_t(255);
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
  std::map<size_t, size_t> free_;
};

enum class St { kPending, kPublished, kCopyBack, kDone, kCanceled };

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
  int slot = -1;
  uint64_t seq = 0;
  St st = St::kPending;
  sil_status status = SIL_OK;
  uint64_t counts[4] = {0, 0, 0, 0};
  double t_submit = 0, t_admit = 0, t_done = 0;
  cudaEvent_t ev_done = nullptr;
};

// Pinned host staging of one slot's copies (stable until the slot is reused).
struct SlotHost {
  SlotDev desc;
  uint64_t counts[4];     // results copied back
  unsigned int status;    // the slot's status word copied back
};

}  // namespace

struct sil_server {
  sil_server_config cfg{};
  sil_dtype dt = SIL_U8;
  sil_params params{};
  DevParams dp{};
  int bpp = 3;
  int grid = 1;
  size_t smem = 0;
  uint8_t* arena_mem = nullptr;
  std::unique_ptr<Arena> arena;
  cudaStream_t s_in = nullptr, s_comp = nullptr, s_out = nullptr;
  // ring
  RingCtl* d_ctl = nullptr;
  LogEntry* d_log = nullptr;
  SlotDev* d_slots = nullptr;
  unsigned int* h_complete = nullptr;  // host-mapped, written by the kernel
  unsigned int* d_complete = nullptr;  // its device alias
  SlotHost* h_slot = nullptr;          // pinned staging per slot
  LogEntry* h_log = nullptr;           // pinned staging per log entry
  unsigned long long* h_tail = nullptr;  // pinned staging of the published request count, per log entry
  unsigned int* h_zero = nullptr;        // pinned zeros (the ring's idle and quit words at each launch)
  int L = 0;
  uint64_t next_seq = 0;    // next publication
  uint64_t published = 0;   // chips published
  cudaEvent_t ev_kernel = nullptr;
  bool kernel_live = false;
  int64_t launches = 0;  // kernel launches so far
  std::atomic<int> skip_ready{0};  // test hook
  std::vector<int> free_slots;
  Request* by_slot[4096] = {};

  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Request*> pending;
  std::vector<Request*> running;  // published or copying back
  std::unordered_map<int64_t, std::unique_ptr<Request>> all;
  int64_t next_id = 1;
  bool stop = false;
  std::thread worker;

  void run();
  void finish(Request* r, sil_status st);
  cudaError_t launch();
};

namespace {

// Device layout of a request: the image keeps the host's row pitch, so it
// arrives by one plain copy of its bytes (a pitched copy may run as a
// kernel, which would wait for the persistent kernel's CTAs to leave the
// SMs); labels at W bytes per row (one plain copy back when the caller's
// label rows are dense too), counts, chip counts.
size_t request_bytes(const sil_server* s, Request* r) {
  r->dpitch = size_t(r->pitch);
  size_t off = size_t(r->H - 1) * r->dpitch + size_t(r->W) * s->bpp;
  off = (off + 255) & ~size_t(255);
  r->o_lab = off;
  off += size_t(r->W * r->H);  // labels are always written (the kernel labels whole chips)
  off = (off + 255) & ~size_t(255);
  r->o_cnt = off;
  off += 32;
  off = (off + 255) & ~size_t(255);
  r->o_cc = off;
  off += size_t(r->gx) * r->gy * 16;
  return off;
}

}  // namespace

namespace {

// (dt, H/S) -> the kernel class
template <template <int, bool> class F, class... A>
cudaError_t dispatch_served(int dt, bool hs, A... a) {
  if (dt == SIL_U8) return hs ? F<SIL_U8, true>::run(a...) : F<SIL_U8, false>::run(a...);
  return hs ? F<SIL_U16, true>::run(a...) : F<SIL_U16, false>::run(a...);
}
template <int DT, bool HS>
struct LaunchServed {
  static cudaError_t run(const sil_server* s, cudaStream_t st) {
    return ServedKernels<DT, HS>::launch(
        s->params.chip <= kResidentChip, s->grid, s->smem, st, s->d_ctl, s->d_log, s->L, s->d_slots,
        s->d_complete, s->dp, s->params.chip, (long long)s->cfg.ready_timeout_ms * 1000000ll,
        (long long)s->cfg.idle_timeout_us * 1000ll);
  }
};
template <int DT, bool HS>
struct PrepareServed {
  static cudaError_t run(bool res, size_t smem, int* per_sm) {
    return ServedKernels<DT, HS>::prepare(res, smem, per_sm);
  }
};

}  // namespace

cudaError_t sil_server::launch() {
  // a new grid starts with no idle CTA and no quit word (the previous grid
  // has ended: its event completed); a copy from pinned zeros, in stream
  // order before the kernel
  cudaError_t e = cudaMemcpyAsync(&d_ctl->idle, h_zero, 3 * sizeof(unsigned int), cudaMemcpyHostToDevice,
                                  s_comp);
  if (e == cudaSuccess)
    e = dispatch_served<LaunchServed>(int(dt), dp.need_hs != 0, static_cast<const sil_server*>(this),
                                      s_comp);
  if (e == cudaSuccess) e = cudaEventRecord(ev_kernel, s_comp);
  if (e == cudaSuccess) {
    kernel_live = true;
    ++launches;
  }
  return e;
}

void sil_server::finish(Request* r, sil_status st) {
  r->status = st;
  r->t_done = now_ms();
  r->st = (st == SIL_ECANCELED) ? St::kCanceled : St::kDone;
}

void sil_server::run() {
  cudaSetDevice(cfg.device);
  std::unique_lock<std::mutex> lk(mu);
  while (true) {
    if (stop && pending.empty() && running.empty()) break;
    bool progressed = false;
    cudaError_t e = cudaSuccess;
    // 1. admission in arrival order, then publication on the ingest stream:
    //    image, slot descriptor (+ ready word), counts = 0, log entry,
    //    published chip count -- in that order, all by the copy engines
    while (!pending.empty() && !free_slots.empty()) {
      Request* r = pending.front();
      size_t off;
      if (!arena->alloc(r->bytes, &off)) break;
      pending.pop_front();
      r->off = off;
      r->slot = free_slots.back();
      free_slots.pop_back();
      r->t_admit = now_ms();
      r->seq = next_seq++;
      by_slot[r->slot] = r;
      const int64_t chips = int64_t(r->gx) * r->gy;
      SlotHost& hs = h_slot[r->slot];
      memset(&hs.desc, 0, sizeof(hs.desc));
      Req& q = hs.desc.req;
      q.img = arena_mem + r->off;
      q.H = r->H;
      q.W = r->W;
      q.pitch = int64_t(r->dpitch);
      q.labels = arena_mem + r->off + r->o_lab;
      q.lpitch = r->W;
      q.counts = reinterpret_cast<unsigned long long*>(arena_mem + r->off + r->o_cnt);
      q.chip_counts = reinterpret_cast<uint32_t*>(arena_mem + r->off + r->o_cc);
      q.gx = r->gx;
      q.gy = r->gy;
      q.chip_begin = int64_t(published);
      hs.desc.ready = skip_ready.exchange(0) ? 0u : unsigned(r->seq + 1);
      hs.desc.claimw = uint64_t(unsigned(r->seq + 1)) << 32;
      hs.desc.done = 0;
      hs.desc.status = 0;
      const int li = int(r->seq % uint64_t(L));
      h_log[li].seq1 = r->seq + 1;
      h_log[li].c = unsigned(chips);
      h_log[li].slot = unsigned(r->slot);
      published += uint64_t(chips);
      h_tail[li] = r->seq + 1;  // requests published
      h_complete[r->slot] = 0;
      e = cudaMemcpyAsync(arena_mem + r->off, r->img, size_t(r->H - 1) * r->dpitch + size_t(r->W) * bpp,
                          cudaMemcpyHostToDevice, s_in);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(&d_slots[r->slot], &hs.desc, sizeof(SlotDev), cudaMemcpyHostToDevice, s_in);
      // (a copy, not a memset: a memset is a kernel, which would wait for
      // the persistent kernel's CTAs to leave the SMs)
      memset(hs.counts, 0, sizeof(hs.counts));
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(arena_mem + r->off + r->o_cnt, hs.counts, 32, cudaMemcpyHostToDevice, s_in);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(&d_log[li], &h_log[li], sizeof(LogEntry), cudaMemcpyHostToDevice, s_in);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(&d_ctl->pub, &h_tail[li], sizeof(unsigned long long), cudaMemcpyHostToDevice,
                            s_in);
      r->st = St::kPublished;
      running.push_back(r);
      progressed = true;
      if (e != cudaSuccess) break;
    }
    // 2. keep a kernel running while published chips may be unclaimed
    if (e == cudaSuccess && kernel_live && cudaEventQuery(ev_kernel) == cudaSuccess) kernel_live = false;
    if (e == cudaSuccess && !kernel_live) {
      bool work = false;
      for (const Request* r : running)
        if (r->st == St::kPublished) work = true;
      if (work) {
        // the kernel has ended (its CTAs found no chip for idle_timeout_us)
        // while published requests are unfinished: start it again (the
        // ring's cursor and claim words carry over)
        e = launch();
        progressed = true;
      }
    }
    // 3. completions: the kernel's completion word -> copy the results back
    for (size_t i = 0; i < running.size() && e == cudaSuccess; ++i) {
      Request* r = running[i];
      if (r->st != St::kPublished) continue;
      if (*reinterpret_cast<volatile unsigned int*>(&h_complete[r->slot]) != unsigned(r->seq + 1))
        continue;
      SlotHost& hs = h_slot[r->slot];
      if (r->labels && cfg.want_labels) {
        if (r->lpitch == r->W)
          e = cudaMemcpyAsync(r->labels, arena_mem + r->off + r->o_lab, size_t(r->W) * r->H,
                              cudaMemcpyDeviceToHost, s_out);
        else
          e = cudaMemcpy2DAsync(r->labels, r->lpitch, arena_mem + r->off + r->o_lab, r->W, r->W, r->H,
                                cudaMemcpyDeviceToHost, s_out);
      }
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(hs.counts, arena_mem + r->off + r->o_cnt, 32, cudaMemcpyDeviceToHost, s_out);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(&hs.status, &d_slots[r->slot].status, 4, cudaMemcpyDeviceToHost, s_out);
      if (e == cudaSuccess && r->chip_counts)
        e = cudaMemcpyAsync(r->chip_counts, arena_mem + r->off + r->o_cc, size_t(r->gx) * r->gy * 16,
                            cudaMemcpyDeviceToHost, s_out);
      if (e == cudaSuccess) e = cudaEventRecord(r->ev_done, s_out);
      r->st = St::kCopyBack;
      progressed = true;
    }
    bool done_any = false;
    for (size_t i = 0; i < running.size() && e == cudaSuccess;) {
      Request* r = running[i];
      if (r->st != St::kCopyBack) {
        ++i;
        continue;
      }
      const cudaError_t q = cudaEventQuery(r->ev_done);
      if (q == cudaErrorNotReady) {
        ++i;
        continue;
      }
      const SlotHost& hs = h_slot[r->slot];
      memcpy(r->counts, hs.counts, 32);
      sil_status st = q == cudaSuccess ? SIL_OK : SIL_ECUDA;
      if (st == SIL_OK && hs.status != 0) st = SIL_ETIMEOUT;
      arena->release(r->off, r->bytes);
      free_slots.push_back(r->slot);
      by_slot[r->slot] = nullptr;
      finish(r, st);
      running[i] = running.back();
      running.pop_back();
      done_any = true;
    }
    if (e != cudaSuccess) {
      // a CUDA failure ends every request in flight
      for (Request* r : running) {
        arena->release(r->off, r->bytes);
        free_slots.push_back(r->slot);
        finish(r, SIL_ECUDA);
      }
      running.clear();
      cudaGetLastError();
      done_any = true;
    }
    if (done_any) {
      cv_done.notify_all();
      progressed = true;
    }
    if (!progressed) {
      // nothing to admit, launch or complete: sleep until new work or a
      // short poll tick (completion words are polled)
      cv_work.wait_for(lk, std::chrono::microseconds(running.empty() ? 2000 : 20));
    } else {
      // let submit / wait / poll in between busy iterations
      lk.unlock();
      std::this_thread::yield();
      lk.lock();
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
  cfg->ready_timeout_ms = 2000;
  cfg->idle_timeout_us = 5000;
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
  if (cfg.max_inflight < 1 || cfg.max_inflight > 4096 || cfg.device_mem_budget < 0 ||
      cfg.ready_timeout_ms < 1 || cfg.ready_timeout_ms > 600000 || cfg.idle_timeout_us < 1 ||
      cfg.idle_timeout_us > 10000000) {
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
  s->L = kLogFactor * cfg.max_inflight;
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
  const int R = cfg.max_inflight;
  for (int i = 0; i < R; ++i) s->free_slots.push_back(R - 1 - i);
  e = cudaMalloc(&s->d_ctl, sizeof(RingCtl));
  if (e == cudaSuccess) e = cudaMemset(s->d_ctl, 0, sizeof(RingCtl));
  if (e == cudaSuccess) e = cudaMalloc(&s->d_log, sizeof(LogEntry) * s->L);
  if (e == cudaSuccess) e = cudaMemset(s->d_log, 0, sizeof(LogEntry) * s->L);
  if (e == cudaSuccess) e = cudaMalloc(&s->d_slots, sizeof(SlotDev) * R);
  if (e == cudaSuccess) e = cudaMemset(s->d_slots, 0, sizeof(SlotDev) * R);
  if (e == cudaSuccess) e = cudaHostAlloc(&s->h_complete, sizeof(unsigned int) * R, cudaHostAllocMapped);
  if (e == cudaSuccess) memset(s->h_complete, 0, sizeof(unsigned int) * R);
  if (e == cudaSuccess) e = cudaHostGetDevicePointer(reinterpret_cast<void**>(&s->d_complete), s->h_complete, 0);
  if (e == cudaSuccess) e = cudaMallocHost(&s->h_slot, sizeof(SlotHost) * R);
  if (e == cudaSuccess) e = cudaMallocHost(&s->h_log, sizeof(LogEntry) * s->L);
  if (e == cudaSuccess) e = cudaMallocHost(&s->h_tail, sizeof(unsigned long long) * s->L);
  if (e == cudaSuccess) e = cudaMallocHost(&s->h_zero, 4 * sizeof(unsigned int));
  if (e == cudaSuccess) memset(s->h_zero, 0, 4 * sizeof(unsigned int));
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->ev_kernel, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->s_in, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->s_comp, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->s_out, cudaStreamNonBlocking);
  int per_sm = 0;
  if (e == cudaSuccess) {
    const bool hs = s->dp.need_hs != 0;
    s->smem = resident_smem_bytes(dt, hs);
    e = dispatch_served<PrepareServed>(int(dt), hs, s->params.chip <= kResidentChip, s->smem, &per_sm);
  }
  if (e != cudaSuccess) {
    sil_server* raw = s.release();
    raw->stop = true;
    sil_server_destroy(raw);
    cudaSetDevice(prev);
    set_error("sil_server_create: %s", cudaGetErrorString(e));
    return SIL_ENOMEM;
  }
  s->grid = (per_sm > 0 ? per_sm : 1) * device_sm_count();
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
  if (cudaEventCreateWithFlags(&r->ev_done, cudaEventDisableTiming) != cudaSuccess) {
    set_error("sil_server_submit: event creation failed");
    return SIL_ECUDA;
  }
  r->t_submit = now_ms();
  {
    std::lock_guard<std::mutex> g(srv->mu);
    if (srv->stop) {
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
  release_request(srv, id);
  return SIL_OK;
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
  release_request(srv, id);
  return SIL_OK;
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

sil_status sil_server_stats(sil_server* srv, int64_t* kernel_launches, int64_t* chips_published) {
  if (!srv) {
    set_error("sil_server_stats: NULL");
    return SIL_EINVAL;
  }
  std::lock_guard<std::mutex> g(srv->mu);
  if (kernel_launches) *kernel_launches = srv->launches;
  if (chips_published) *chips_published = int64_t(srv->published);
  return SIL_OK;
}

sil_status sil_server_set_fault(sil_server* srv, int32_t skip_ready) {
  if (!srv) {
    set_error("sil_server_set_fault: NULL");
    return SIL_EINVAL;
  }
  srv->skip_ready = skip_ready ? 1 : 0;
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
  // the worker leaves when nothing is in flight; the kernel ends on its own
  // (no work for idle_timeout_us)
  if (srv->s_in) cudaStreamSynchronize(srv->s_in);
  if (srv->s_comp) cudaStreamSynchronize(srv->s_comp);
  if (srv->s_out) cudaStreamSynchronize(srv->s_out);
  for (auto& kv : srv->all) cudaEventDestroy(kv.second->ev_done);
  srv->all.clear();
  cudaFree(srv->d_ctl);
  cudaFree(srv->d_log);
  cudaFree(srv->d_slots);
  cudaFreeHost(srv->h_complete);
  cudaFreeHost(srv->h_slot);
  cudaFreeHost(srv->h_log);
  cudaFreeHost(srv->h_tail);
  cudaFreeHost(srv->h_zero);
  if (srv->ev_kernel) cudaEventDestroy(srv->ev_kernel);
  cudaFree(srv->arena_mem);
  if (srv->s_in) cudaStreamDestroy(srv->s_in);
  if (srv->s_comp) cudaStreamDestroy(srv->s_comp);
  if (srv->s_out) cudaStreamDestroy(srv->s_out);
  cudaSetDevice(prev);
  delete srv;
}

}  // extern "C"
