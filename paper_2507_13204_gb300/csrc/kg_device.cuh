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
