// Device helpers shared by the kernels: deterministic warp/block sums, the
// "last CTA finishes the reduction" pattern, and the sticky error word.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace kg {

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
  // Butterfly: every lane ends with the same bits (each step adds the same two
  // operands in commuted order).
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sum over the CTA, returned to every thread.  scratch: >= 32 entries of shared
// memory.  Fixed association order, so bitwise reproducible.
template <typename T>
__device__ __forceinline__ T block_sum(T v, T* scratch) {
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  __syncthreads();
  if (lane == 0) scratch[w] = v;
  __syncthreads();
  T r = lane < nw ? scratch[lane] : T(0);
  return warp_sum(r);
}

// Each CTA contributes `partial`; the CTA that arrives last sums all partials
// in CTA-index order (deterministic), writes *out (as T) and resets the
// arrival counter for the next launch.  The arrival is a single atomicAdd per
// CTA and nobody waits: the last CTA to arrive does the work.
template <typename T>
__device__ __forceinline__ void finish_sum(double partial, double* fpart, unsigned* counter,
                                           T* out, int accumulate, double* scratch) {
  __shared__ bool s_last;
  if (threadIdx.x == 0) {
    fpart[blockIdx.x] = partial;
    __threadfence();
    unsigned t = atomicAdd(counter, 1u);
    s_last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  double s = 0.0;
  for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) s += __ldcg(&fpart[i]);
  s = block_sum(s, scratch);
  if (threadIdx.x == 0) {
    if (out) *out = accumulate ? (T)((double)*out + s) : (T)s;
    *counter = 0u;
  }
}

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void set_error(unsigned* err, unsigned bit) {
  if (err) atomicOr(err, bit);
}

template <typename T>
__device__ __forceinline__ T load_seed(const T* seed) {
  return seed ? *seed : T(1);
}

// Streaming load that does not allocate in L1 (data is read once).
template <typename T>
__device__ __forceinline__ T ld_stream(const T* p) {
  return __ldcs(p);
}

}  // namespace kg

// ---------------------------------------------------------------------------
// TMA bulk copies and mbarriers (inline PTX, sm_90+ / sm_103a).
// ---------------------------------------------------------------------------
namespace kg {

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// Makes the initialised barriers visible to the async (TMA) proxy.
__device__ __forceinline__ void fence_barrier_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Orders this thread's generic-proxy shared-memory writes before later
// async-proxy (TMA) accesses of the same memory.
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Waits for the phase of `bar` with the given parity to complete; gives up
// (returns false) after about one second of wall time.
constexpr uint64_t kWaitLimitNs = 1000000000ull;
// The clock is read on every 64th failed try only: spinning warps then issue
// little besides the try-wait itself.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity,
                                                  uint64_t limit_ns = kWaitLimitNs) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  for (uint32_t i = 1;; ++i) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((i & 63u) == 0u && global_ns() - t0 > limit_ns) return false;
  }
}

// Grid barrier of a cooperative launch (every CTA resident), for thread 0 of
// each CTA after a __syncthreads: the CTA's writes are made visible, it counts
// itself in at arrive[0] and waits, bounded, until every CTA has.  Returns
// false (ERRBIT_TIMEOUT set in err) when the wait gives up.
__device__ __forceinline__ bool grid_arrive_and_wait(unsigned* arrive, unsigned* err, unsigned bit) {
  __threadfence();
  atomicAdd(arrive, 1u);
  const uint64_t t0 = global_ns();
  while (ld_acquire_u32(arrive) < gridDim.x) {
    if (global_ns() - t0 > kWaitLimitNs) {
      set_error(err, bit);
      return false;
    }
  }
  __threadfence();
  return true;
}

// Thread 0 counts the CTA out of the barrier's work at depart[0]; the last CTA
// resets both counters for the next launch.
__device__ __forceinline__ void grid_depart(unsigned* arrive, unsigned* depart) {
  __threadfence();
  if (atomicAdd(depart, 1u) == gridDim.x - 1) {
    *arrive = 0u;
    *depart = 0u;
  }
}

// In a kernel launched with programmatic stream serialization: blocks until
// the preceding grid on the stream has completed and its memory operations
// are visible (returns at once otherwise).
__device__ __forceinline__ void grid_dependency_wait() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
}

// Global floating-point add whose old value is not wanted: PTX red (a
// reduction at L2 that returns nothing to the SM), where atomicAdd's atom form
// also brings the old value back.  p points to global memory.
__device__ __forceinline__ void red_add(float* p, float v) {
  asm volatile("red.global.add.f32 [%0], %1;" ::"l"(__cvta_generic_to_global(p)), "f"(v) : "memory");
}
__device__ __forceinline__ void red_add(double* p, double v) {
  asm volatile("red.global.add.f64 [%0], %1;" ::"l"(__cvta_generic_to_global(p)), "d"(v) : "memory");
}

// 1-D bulk copy global -> shared (TMA), completing `bytes` on `bar`.
// dst and src 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void tma_load_1d(void* dst, const void* src, uint32_t bytes,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// Bulk prefetch of [src, src + bytes) into L2 (16-byte aligned, multiple of 16).
__device__ __forceinline__ void prefetch_l2_bulk(const void* src, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}

// Barrier over `nthreads` threads on hardware barrier `id` (1..15) that also
// ORs a predicate across them.  Non-aligned form: the threads of a warp may
// arrive at different times (e.g. while one lane issues TMA copies).
__device__ __forceinline__ bool named_barrier_or(int id, int nthreads, bool pred) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\t"
      "setp.ne.u32 p, %1, 0;\n\t"
      "barrier.red.or.pred q, %2, %3, p;\n\t"
      "selp.u32 %0, 1, 0, q;\n\t}"
      : "=r"(r)
      : "r"((uint32_t)pred), "r"(id), "r"(nthreads)
      : "memory");
  return r != 0;
}

__device__ __forceinline__ void named_barrier(int id, int nthreads) {
  asm volatile("barrier.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

}  // namespace kg
