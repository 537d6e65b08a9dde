// sil_served_kernel.cuh -- the served kernel and the device-resident ring
// it reads (internal).  Each (dtype, H/S) class of the kernel is compiled in
// a translation unit of its own (sil_served_k_*.cu), so the library builds
// in parallel.
#pragma once
#include <cuda_runtime.h>

#include "sil.h"
#include "sil_chip.cuh"
#include "sil_common.h"
#include "sil_generic.cuh"

namespace sil {

// ---------------------------------------------------------------------------
// Ring layout (device memory unless stated).
// ---------------------------------------------------------------------------
struct RingCtl {
  unsigned long long pub;   // requests published (written by the ingest stream)
  unsigned long long cur;   // oldest request that may still have unclaimed chips
  unsigned int err;         // log entries found missing (0 in normal operation)
  unsigned int idle;        // CTAs that found no chip for idle_ns (reset per launch)
  unsigned int quit;        // set once every CTA was idle at the same time: all leave
  unsigned int pad;
};
// One publication: request sequence number + 1 (0 = never written), its chip
// count and slot.
struct LogEntry {
  unsigned long long seq1;
  unsigned int c;
  unsigned int slot;
};
// One request slot: descriptor, the claim word (high half: the low 32 bits
// of seq + 1 of the request it belongs to, low half: chips claimed), the
// ready word (seq + 1 once the image is in place), chips done, status (1:
// the ready wait ran out).  Tagging the claim word with the request makes a
// claim that raced with the slot's reuse by a newer request fail instead of
// taking that request's chip.
struct SlotDev {
  Req req;
  unsigned long long claimw;
  unsigned int ready;
  unsigned int done;
  unsigned int status;
  unsigned int pad;
};
constexpr int kLogFactor = 4;  // log entries per request slot

__device__ __forceinline__ unsigned long long gtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ unsigned long long ld_acquire(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ unsigned int ld_acquire32(const unsigned int* p) {
  unsigned int v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

template <int DT, bool HS, bool RESIDENT>
__global__ void __launch_bounds__(kThreadsNarrow, RESIDENT ? ResidentCtas<DT, HS>::k : ((DT == SIL_U8) ? 2 : 1))
    k_served(RingCtl* ctl, const LogEntry* log, int L, SlotDev* slots, unsigned int* complete,
             DevParams dp, int chip, long long ready_ns, long long idle_ns) {
  extern __shared__ __align__(128) uint8_t smem_raw[];
  __shared__ uint8_t lut[256];
  __shared__ Req s_req;
  __shared__ long long s_local;
  __shared__ int s_slot, s_ok, s_got;
  __shared__ unsigned int s_c, s_seq32;
  __shared__ __align__(16) ChipStat st_generic;
  constexpr uint32_t kCols = PlaneCols<kThreadsNarrow>::kCols;
  ChipSmem<DT, HS>& sm = *reinterpret_cast<ChipSmem<DT, HS>*>(smem_raw);
  if (RESIDENT && !ChipSmem<DT, HS>::kSmemPlane) plane_alloc(&sm.st.tmem, kCols);
  while (true) {
    if (threadIdx.x == 0) {
      // claim a chip: the oldest published request with chips left hands
      // out its next chip (a per-request counter); an exhausted request
      // moves the ring's cursor on.  No published chip for idle_ns -> leave.
      int got = 0;
      const unsigned long long t0 = gtimer();
      // idle polls back off from 1 to 32 us: a few hundred CTAs polling the
      // ring's two control words every microsecond load one L2 line hard
      // enough to slow the chips being labelled and the copies.  The grid
      // leaves only as a whole: a CTA idle for idle_ns counts itself idle
      // and keeps polling; when every CTA is idle at once, the first to see
      // it sets the quit word and all leave.  (CTAs leaving one by one left
      // a kernel of a few CTAs that stayed live under a steady trickle of
      // requests, so the host never relaunched the full grid.)
      unsigned int backoff = 1000;
      bool counted = false;
      while (true) {
        if (ld_acquire32(&ctl->quit)) break;
        const unsigned long long pub = ld_acquire(&ctl->pub);
        const unsigned long long cur = ld_acquire(&ctl->cur);
        if (cur < pub && counted) {
          atomicSub(&ctl->idle, 1u);
          counted = false;
        }
        if (cur < pub) {
          const LogEntry* le = &log[cur % (unsigned long long)L];
          if (ld_acquire(&le->seq1) != cur + 1) {
            atomicAdd(&ctl->err, 1u);  // overwritten: cannot happen with <= L requests in flight
            break;
          }
          const unsigned int c = *reinterpret_cast<const volatile unsigned int*>(&le->c);
          const unsigned int slot = *reinterpret_cast<const volatile unsigned int*>(&le->slot);
          const unsigned long long tag = (cur + 1ull) << 32;
          unsigned long long w = ld_acquire(&slots[slot].claimw);
          bool exhausted = false;
          while ((w & ~0xffffffffull) == (tag & 0xffffffff00000000ull)) {
            const unsigned int k = unsigned(w);
            if (k >= c) {
              exhausted = true;
              break;
            }
            const unsigned long long seen = atomicCAS(&slots[slot].claimw, w, w + 1ull);
            if (seen == w) {
              got = 1;
              s_slot = int(slot);
              s_local = (long long)k;
              s_c = c;
              s_seq32 = unsigned(cur + 1);
              break;
            }
            w = seen;
            if ((long long)(gtimer() - t0) > idle_ns + ready_ns) break;
          }
          if (got) break;
          // every chip of it is claimed, or the slot already holds a newer
          // request (this cursor value is stale): move the cursor on
          if (exhausted || (w >> 32) != ((cur + 1ull) & 0xffffffffull)) atomicCAS(&ctl->cur, cur, cur + 1ull);
        } else {
          if (!counted && (long long)(gtimer() - t0) > idle_ns) {
            atomicAdd(&ctl->idle, 1u);
            counted = true;
          }
          if (counted && ld_acquire32(&ctl->idle) >= gridDim.x) {
            atomicExch(&ctl->quit, 1u);
            break;
          }
          __nanosleep(backoff);
          backoff = backoff < 32000u ? 2u * backoff : 32000u;
        }
        if ((long long)(gtimer() - t0) > idle_ns + ready_ns) break;  // bounded in every case
      }
      s_got = got;
      s_ok = 0;
      if (got) {
        SlotDev* sd = &slots[s_slot];
        // the request's image is in place once its ready word is set
        bool ok = ld_acquire32(&sd->status) == 0;
        const unsigned long long t1 = gtimer();
        while (ok && ld_acquire32(&sd->ready) != s_seq32) {
          if (ld_acquire32(&sd->status) != 0) {
            ok = false;  // another CTA's wait for this request ran out
          } else if ((long long)(gtimer() - t1) > ready_ns) {
            atomicExch(&sd->status, 1u);
            ok = false;
          } else {
            __nanosleep(2000);
          }
        }
        s_ok = ok && ld_acquire32(&sd->status) == 0;
        if (s_ok) {
          // the descriptor through L2 (an earlier request's copy of this
          // slot may still sit in this SM's L1)
          const unsigned long long* src = reinterpret_cast<const unsigned long long*>(&sd->req);
          unsigned long long* dst = reinterpret_cast<unsigned long long*>(&s_req);
          for (int w = 0; w < int(sizeof(Req) / 8); ++w) dst[w] = __ldcg(src + w);
        }
      }
    }
    __syncthreads();
    if (!s_got) break;
    if (s_ok) {
      const Req r = s_req;
      const int64_t cy = s_local / r.gx, cx = s_local - cy * r.gx;
      if (RESIDENT) {
        label_chip<DT, HS>(r, dp, chip, cy, cx, sm, lut, lut);
      } else {
        label_chip_generic<DT, HS>(r, dp, chip, cy, cx, st_generic, lut);
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      SlotDev* sd = &slots[s_slot];
      __threadfence();  // this chip's labels and counts before its done count
      const unsigned int old = atomicAdd(&sd->done, 1u);
      if (old + 1u == s_c) {
        __threadfence();  // every chip's results before the completion word
        *reinterpret_cast<volatile unsigned int*>(&complete[s_slot]) = s_seq32;
        __threadfence_system();
      }
    }
  }
  if (RESIDENT && !ChipSmem<DT, HS>::kSmemPlane) plane_free(sm.st.tmem, kCols);
}

// The served kernel's instances of one (dtype, H/S) class.
template <int DT, bool HS>
struct ServedKernels {
  // Enqueues the persistent kernel (resident when the chip fits in shared
  // memory; smem = its dynamic shared memory then).
  static cudaError_t launch(bool resident, int grid, size_t smem, cudaStream_t st, RingCtl* ctl,
                            const LogEntry* log, int L, SlotDev* slots, unsigned int* complete,
                            const DevParams& dp, int chip, long long ready_ns, long long idle_ns);
  // Sets the shared-memory limit and returns the resident CTAs per SM.
  static cudaError_t prepare(bool resident, size_t smem, int* per_sm);
};

template <int DT, bool HS>
cudaError_t ServedKernels<DT, HS>::launch(bool resident, int grid, size_t smem, cudaStream_t st,
                                          RingCtl* ctl, const LogEntry* log, int L, SlotDev* slots,
                                          unsigned int* complete, const DevParams& dp, int chip,
                                          long long ready_ns, long long idle_ns) {
  if (resident)
    k_served<DT, HS, true><<<grid, kThreadsNarrow, smem, st>>>(ctl, log, L, slots, complete, dp,
                                                               chip, ready_ns, idle_ns);
  else
    k_served<DT, HS, false><<<grid, kThreadsNarrow, 0, st>>>(ctl, log, L, slots, complete, dp,
                                                             chip, ready_ns, idle_ns);
  return cudaGetLastError();
}

template <int DT, bool HS>
cudaError_t ServedKernels<DT, HS>::prepare(bool resident, size_t smem, int* per_sm) {
  cudaError_t e = cudaSuccess;
  if (resident) {
    e = set_resident_attrs(reinterpret_cast<const void*>(k_served<DT, HS, true>), smem);
    if (e == cudaSuccess)
      *per_sm = resident_ctas_per_sm(reinterpret_cast<const void*>(k_served<DT, HS, true>),
                                     kThreadsNarrow, smem, tmem_plane(DT, HS) ? plane_cols(kThreadsNarrow) : 0);
  } else {
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, k_served<DT, HS, false>,
                                                      kThreadsNarrow, 0);
  }
  return e;
}

extern template struct ServedKernels<SIL_U8, false>;
extern template struct ServedKernels<SIL_U8, true>;
extern template struct ServedKernels<SIL_U16, false>;
extern template struct ServedKernels<SIL_U16, true>;

}  // namespace sil
