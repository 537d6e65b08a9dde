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

// Device address of the scratch array on the current device, looked up once
// per device (the host-side name is not a device address).
sil_status scratch_address(int dev, unsigned char** out) {
  if (dev < 0 || dev >= kMaxDevices) {
    set_error("sil_label_batch_noalloc: device %d out of range", dev);
    return SIL_EINVAL;
  }
  std::lock_guard<std::mutex> g(g_setup_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      set_error("sil_label_batch_noalloc: cudaGetSymbolAddress: %s", cudaGetErrorString(e));
      return SIL_ECUDA;
    }
    g_scratch_addr[dev] = p;
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
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  // Pageable-source copies return once the source bytes are staged, so the
  // stack arrays may go out of scope afterwards.
  cudaError_t e = cudaMemcpyAsync(d_reqs, reqs, sizeof(Req) * n, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(d_prefix, prefix, sizeof(int64_t) * (n + 1), cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) {
    set_error("sil_label_batch_noalloc: descriptor copy: %s", cudaGetErrorString(e));
    return SIL_ECUDA;
  }
  const int cps = batch_max_ctas_per_sm(dt, dp.need_hs != 0, chip);
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
