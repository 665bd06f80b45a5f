// ihist_device.cuh -- device-side building blocks shared by the scan and
// query kernels: control words, memory-model helpers, bounded waits and the
// packed warp scans.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace ihist {

constexpr int kChunk = 128;               // columns per warp chunk: 32 lanes x 4
constexpr uint32_t kFull = 0xffffffffu;

// Carry-flag states.  A flag word is (epoch << 2) | state, so flags left
// from an earlier launch never match the current one and the flags need no
// clearing between launches.
enum : uint32_t { kStateAgg = 1u, kStateIncl = 2u, kStatePoison = 3u };

// Device status codes (mirror the IHIST_* values of ihist.h).
enum : int { kStatusOk = 0, kStatusTimeout = 5, kStatusBadRect = 6, kStatusCheck = 7 };

// Per-plan control block in device memory (zeroed once at plan creation).
struct Ctrl {
  unsigned int ticket;    // next work item of the running launch
  unsigned int done;      // CTAs of the running launch that have finished
  unsigned int epoch;     // launch counter carried in every flag
  int status;             // first device error latched since the last read
  unsigned int timeouts;  // number of waits that gave up
  unsigned int pad[3];
};

// Checked builds (compiled with -DIHIST_CHECKED, the stand-in for a memory
// sanitizer): each guarded access is tested first; a failed test latches
// kStatusCheck in the status word and the access is skipped.  Other builds
// compile the guards away.
#ifdef IHIST_CHECKED
#define IHIST_GUARD(ctrl, cond) ::ihist::guard_access((ctrl), (cond))
#else
#define IHIST_GUARD(ctrl, cond) true
#endif

__device__ __forceinline__ uint32_t ld_acquire_gpu(const uint32_t *p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_release_gpu(uint32_t *p, uint32_t v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// L2-coherent 128-bit load of data another CTA published (never a stale L1 line).
__device__ __forceinline__ uint4 ld_relaxed_v4(const uint32_t *p) {
  uint4 v;
  asm volatile("ld.relaxed.gpu.global.v4.u32 {%0, %1, %2, %3}, [%4];"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "l"(p)
               : "memory");
  return v;
}

// Coherent 32-bit / 64-bit loads (L2, never a possibly stale L1 or
// read-only-cache line) for descriptors that other agents wrote.
__device__ __forceinline__ uint32_t ld_relaxed_u32(const void *p) {
  uint32_t v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ unsigned long long ld_relaxed_u64(const void *p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

// Streaming (evict-first) 128-bit store for the write-once output.
__device__ __forceinline__ void st_stream_v4(uint32_t *p, uint32_t a, uint32_t b, uint32_t c,
                                             uint32_t d) {
  asm volatile("st.global.cs.v4.u32 [%0], {%1, %2, %3, %4};" ::"l"(p), "r"(a), "r"(b), "r"(c),
               "r"(d)
               : "memory");
}

// Streaming 256-bit store (32-byte aligned p): one full DRAM sector.
__device__ __forceinline__ void st_stream_v8(uint32_t *p, uint4 a, uint4 b) {
  asm volatile("st.global.cs.v8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"l"(p), "r"(a.x), "r"(a.y),
               "r"(a.z), "r"(a.w), "r"(b.x), "r"(b.y), "r"(b.z), "r"(b.w)
               : "memory");
}

__device__ __forceinline__ void st_stream(uint32_t *p, uint32_t a) {
  asm volatile("st.global.cs.u32 [%0], %1;" ::"l"(p), "r"(a) : "memory");
}

// Programmatic dependent launch: wait until the grids this one depends on
// have completed (a no-op without such a dependency), then let the next
// grid's CTAs start.
__device__ __forceinline__ void griddep_wait_and_release() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// Named barrier over `count` threads (whole, converged warps) of the CTA;
// ids 1..15 (0 is __syncthreads).
__device__ __forceinline__ void named_bar_sync(int id, int count) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}

// The same barrier, returning whether `pred` held in every thread that took part.
__device__ __forceinline__ bool named_bar_and(int id, int count, bool pred) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\t"
      "setp.ne.u32 p, %1, 0;\n\t"
      "bar.red.and.pred q, %2, %3, p;\n\t"
      "selp.u32 %0, 1, 0, q;\n\t}"
      : "=r"(r)
      : "r"((uint32_t)pred), "r"(id), "r"(count)
      : "memory");
  return r != 0u;
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// a << s with PTX semantics: shift amounts >= 32 (including "negative"
// amounts seen as large unsigned values) give 0.  This makes one-hot byte
// lanes without a compare: byte j of shl_clamp(1, 8*j - 32*q) is set only
// when bin 4q + j is the pixel's bin.
__device__ __forceinline__ uint32_t shl_clamp(uint32_t a, uint32_t s) {
  uint32_t r;
  asm("shl.b32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(s));
  return r;
}

// Inclusive warp scan of 32-bit words (each byte or half-word lane scans
// independently as long as no lane overflows).
__device__ __forceinline__ uint32_t warp_scan_incl(uint32_t v, int lane) {
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    uint32_t n = __shfl_up_sync(kFull, v, d);
    if (lane >= d) v += n;
  }
  return v;
}

// Latch the first device error into the status word.
__device__ __forceinline__ void latch_status(Ctrl *ctrl, int code) {
  atomicCAS(&ctrl->status, kStatusOk, code);
}

__device__ __forceinline__ bool guard_access(Ctrl *ctrl, bool ok) {
  if (!ok) latch_status(ctrl, kStatusCheck);
  return ok;
}

// Wait (all lanes of a warp, same address) until the flag carries this
// epoch and a non-zero state.  Every lane performs its own acquire load and
// the wait ends only when all lanes saw the same published word, so each
// lane is ordered after the publisher's release.  Bounded: after timeout_ns
// it records a timeout and returns kStatePoison, so no wait is endless.
__device__ __forceinline__ uint32_t wait_flag(const uint32_t *flag, uint32_t epoch, Ctrl *ctrl,
                                              unsigned long long timeout_ns) {
  unsigned long long t0 = 0;
  unsigned int backoff = 32;
  for (;;) {
    const uint32_t f = ld_acquire_gpu(flag);
    const uint32_t f0 = __shfl_sync(kFull, f, 0);
    const bool ok = (f == f0) && ((f >> 2) == epoch) && ((f & 3u) != 0u);
    if (__all_sync(kFull, ok)) return f0 & 3u;
    const unsigned long long now = __shfl_sync(kFull, global_ns(), 0);
    if (t0 == 0) {
      t0 = now;
    } else if (now - t0 > timeout_ns) {
      if ((threadIdx.x & 31) == 0) {
        latch_status(ctrl, kStatusTimeout);
        atomicAdd(&ctrl->timeouts, 1u);
      }
      return kStatePoison;
    }
    __nanosleep(backoff);
    if (backoff < 1024) backoff <<= 1;
  }
}

// ---- TMA + mbarrier (per-warp tile staging) ------------------------------

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// Make mbarrier initialisation visible to the async (TMA) proxy.
__device__ __forceinline__ void mbar_init_fence() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Order this thread's earlier generic-proxy shared-memory accesses before
// later async-proxy (TMA) writes to the same buffer.
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// One lane: arm the barrier for `bytes` and start a 2-D tiled TMA load of
// the box at (x, y) (x in elements, x * 1 byte a multiple of 16) into dst.
__device__ __forceinline__ void tma_load_2d(const void *tmap, void *dst, uint64_t *bar, int x, int y,
                                            uint32_t bytes) {
  asm volatile(
      "{\n\t.reg .b64 st;\n\t"
      "mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(smem_u32(bar)),
      "r"(bytes)
      : "memory");
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, "
      "%3}], [%4];" ::"r"(smem_u32(dst)),
      "l"(tmap), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

// Wait for the barrier phase with the given parity.  Bounded: gives up
// after timeout_ns (returns false), so a lost completion cannot hang the GPU.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity,
                                          unsigned long long timeout_ns) {
  const uint32_t a = smem_u32(bar);
  unsigned long long t0 = 0;
  for (;;) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
    const unsigned long long now = global_ns();
    if (t0 == 0) {
      t0 = now;
    } else if (now - t0 > timeout_ns) {
      return false;
    }
  }
}

}  // namespace ihist
