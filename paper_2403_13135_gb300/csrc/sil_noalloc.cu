// sil_noalloc.cu -- batched labelling that allocates nothing.
//
// Same persistent kernel as sil_label_batch, but its scratch (request
// descriptors, chip prefix sums, work-queue head) lives in one file-scope
// device array instead of context-owned allocations, for callers that are
// not allowed to call cudaMalloc (see the declaration in sil.h).
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>

#include "sil.h"
#include "sil_batch.h"
#include "sil_common.h"

namespace sil {
int device_sm_count();
sil_status check_request(const void* img, int64_t H, int64_t W, int64_t pitch,
                         sil_dtype dt, const uint8_t* labels, int64_t lpitch,
                         const uint64_t* counts);
}  // namespace sil

using namespace sil;

namespace {

constexpr int kNoAllocMaxTiles = 256;
constexpr size_t kReqBytes = sizeof(Req) * kNoAllocMaxTiles;
constexpr size_t kPrefixOff = (kReqBytes + 255) & ~size_t(255);
constexpr size_t kHeadOff = (kPrefixOff + sizeof(int64_t) * (kNoAllocMaxTiles + 1) + 255) & ~size_t(255);
constexpr size_t kScratchBytes = kHeadOff + 256;

// Shared by every call on a device and kept until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
void* g_scratch_addr[kMaxDevices] = {};
unsigned long long g_scratch_ctx[kMaxDevices] = {};

// Identity of the device's current context (cuCtxGetCurrent + cuCtxGetId,
// fetched through the runtime so the library does not link libcuda): a
// cudaDeviceReset in this process ends the context and reloads the module,
// after which the array has a new address.  0 if unavailable.
unsigned long long current_context_id() {
  using GetCurrentFn = int (*)(void**);
  using GetIdFn = int (*)(void*, unsigned long long*);
  static GetCurrentFn get_current = nullptr;
  static GetIdFn get_id = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess && q == cudaDriverEntryPointSuccess)
      get_current = reinterpret_cast<GetCurrentFn>(p);
    p = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess && q == cudaDriverEntryPointSuccess)
      get_id = reinterpret_cast<GetIdFn>(p);
  });
  void* ctx = nullptr;
  unsigned long long id = 0;
  if (!get_current || !get_id || get_current(&ctx) != 0 || !ctx || get_id(ctx, &id) != 0) return 0;
  return id;
}

// Device address of the scratch array on the current device (the host-side
// name is not a device address).  Looked up once per device and context:
// again after the device's context has been replaced.
sil_status scratch_address(int dev, unsigned char** out) {
  if (dev < 0 || dev >= kMaxDevices) {
    set_error("sil_label_batch_noalloc: device %d out of range", dev);
    return SIL_EINVAL;
  }
  const unsigned long long ctx = current_context_id();
  std::lock_guard<std::mutex> g(g_setup_mu);
  if (!g_scratch_addr[dev] || ctx == 0 || g_scratch_ctx[dev] != ctx) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      set_error("sil_label_batch_noalloc: cudaGetSymbolAddress: %s", cudaGetErrorString(e));
      return SIL_ECUDA;
    }
    g_scratch_addr[dev] = p;
    // the lookup creates the device's context if there was none yet
    g_scratch_ctx[dev] = current_context_id();
  }
  *out = static_cast<unsigned char*>(g_scratch_addr[dev]);
  return SIL_OK;
}

}  // namespace

extern "C" sil_status sil_label_batch_noalloc(const sil_tile* tiles, int32_t n, sil_dtype dt,
                                              const sil_params* p, sil_stream stream) {
  if (!tiles || n < 1) {
    set_error("sil_label_batch_noalloc: NULL tiles or n < 1");
    return SIL_EINVAL;
  }
  if (n > kNoAllocMaxTiles) {
    set_error("sil_label_batch_noalloc: %d tiles, at most %d fit its fixed scratch", int(n),
              kNoAllocMaxTiles);
    return SIL_EINVAL;
  }
  if (dt != SIL_U8 && dt != SIL_U16) {
    set_error("sil_label_batch_noalloc: dtype %d", int(dt));
    return SIL_EINVAL;
  }
  DevParams dp;
  sil_status st = derive_params(p, &dp);
  if (st != SIL_OK) return st;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  // The descriptors are copied from this call's stack: a copy recorded into
  // a graph would read that memory after the call has returned.
  cudaStreamCaptureStatus cap_st = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cap_st) != cudaSuccess || cap_st != cudaStreamCaptureStatusNone) {
    cudaGetLastError();
    set_error("sil_label_batch_noalloc: the stream is being captured; this call cannot be captured");
    return SIL_EINVAL;
  }
  const int chip = p ? p->chip : 256;
  // descriptors built on the stack, copied into the device array
  Req reqs[kNoAllocMaxTiles];
  int64_t prefix[kNoAllocMaxTiles + 1];
  prefix[0] = 0;
  for (int i = 0; i < n; ++i) {
    const sil_tile& t = tiles[i];
    st = check_request(t.img, t.H, t.W, t.pitch_bytes, dt, t.labels, t.label_pitch, t.counts);
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
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    set_error("sil_label_batch_noalloc: no current device");
    return SIL_ECUDA;
  }
  unsigned char* base = nullptr;
  if ((st = scratch_address(dev, &base)) != SIL_OK) return st;
  Req* d_reqs = reinterpret_cast<Req*>(base);
  int64_t* d_prefix = reinterpret_cast<int64_t*>(base + kPrefixOff);
  unsigned long long* d_head = reinterpret_cast<unsigned long long*>(base + kHeadOff);
  // Copies from pageable memory return once the source bytes are staged
  // (which can block the host until earlier work on the stream is done), so
  // the stack arrays may go out of scope afterwards.
  cudaError_t e = cudaMemcpyAsync(d_reqs, reqs, sizeof(Req) * n, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(d_prefix, prefix, sizeof(int64_t) * (n + 1), cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) {
    set_error("sil_label_batch_noalloc: descriptor copy: %s", cudaGetErrorString(e));
    return SIL_ECUDA;
  }
  const int cps = batch_max_ctas_per_sm(dt, dp.need_hs != 0, chip, kThreadsNarrow);
  const int64_t total = prefix[n];
  const int64_t cap = int64_t(device_sm_count()) * cps;
  const int grid = int(total < cap ? total : cap);
  BatchLaunch b{d_reqs, d_prefix, int(n), int(dt), dp, chip, d_head, grid, 1};
  e = launch_batch(b, s);  // the prologue zeroes the head and every counts[4]
  if (e != cudaSuccess) {
    set_error("sil_label_batch_noalloc: launch: %s", cudaGetErrorString(e));
    return SIL_ECUDA;
  }
  return SIL_OK;
}
