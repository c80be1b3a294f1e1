// Device characterisation: the arithmetic and reduction rates that set the
// ALU roofline of the native-FP64 kernels and explain the float-pair design.
//
//   - FP64 and FP32 FMA rates: every thread runs eight independent FMA chains
//     in registers (enough independent work per warp scheduler to keep either
//     pipe busy), over a few waves of CTAs on every SM;
//   - FP64 log1p and division rates, in the same chained pattern;
//   - FP64 and FP32 reduction rates: every thread issues red.global.add to
//     pseudo-random slots (xorshift) of an 8 MiB array, the scatter-add pattern
//     of the tet and sparse gradients at an L2-resident footprint;
//   - FP64 and FP32 gather rates: the same slots read by independent loads
//     (eight in flight a thread), the sparse forward's x gathers.
// Each kernel is timed with CUDA events after one warm-up launch (best of
// three).  The results are kept live by a store that the data never triggers
// (the compiler cannot prove it), so the loops are not removed.
#include <cuda_runtime.h>

#include <algorithm>

#include "kg_device.cuh"
#include "kg_internal.h"

namespace kg {
namespace {

constexpr int kChains = 8;
constexpr int kBoxBlock = 256;

template <typename T>
__global__ void __launch_bounds__(kBoxBlock) fma_rate_kernel(T* sink, int iters, T a, T b) {
  T v[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) v[c] = (T)(threadIdx.x + c) * (T)1e-3;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) v[c] = fma(v[c], a, b);
  }
  T s = 0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += v[c];
  if (s == (T)-1234.5) sink[0] = s;  // never true for these inputs
}

// FP64 log1p and division: eight independent chains per thread, each step
// feeding the previous result back (log1p of a value in [0, 2); a / b with b
// in [1, 2)), so that neither is hoisted out of the loop.
__global__ void __launch_bounds__(kBoxBlock) log1p_rate_kernel(double* sink, int iters) {
  double v[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) v[c] = 0.5 + 1e-3 * (threadIdx.x + c);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) v[c] = log1p(v[c] + 1.0);
  }
  double s = 0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += v[c];
  if (s == -1234.5) sink[0] = s;
}

__global__ void __launch_bounds__(kBoxBlock) div_rate_kernel(double* sink, int iters, double b) {
  double v[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) v[c] = 1.0 + 1e-3 * (threadIdx.x + c);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) v[c] = (v[c] + 1.0) / b;
  }
  double s = 0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += v[c];
  if (s == -1234.5) sink[0] = s;
}

template <typename T>
__global__ void __launch_bounds__(kBoxBlock) red_rate_kernel(T* slots, uint32_t mask, int per_thread) {
  uint32_t x = 0x9E3779B9u ^ (blockIdx.x * kBoxBlock + threadIdx.x) * 2654435761u;
  for (int k = 0; k < per_thread; ++k) {
    x ^= x << 13;
    x ^= x >> 17;
    x ^= x << 5;
    red_add(slots + (x & mask), (T)1);
  }
}

template <typename T>
__global__ void __launch_bounds__(kBoxBlock) gather_rate_kernel(const T* __restrict__ slots, uint32_t mask,
                                                                int per_thread, T* sink) {
  uint32_t x = 0x7F4A7C15u ^ (blockIdx.x * kBoxBlock + threadIdx.x) * 2654435761u;
  T acc = 0;
  for (int k = 0; k < per_thread; k += kChains) {
    T v[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) {
      x ^= x << 13;
      x ^= x >> 17;
      x ^= x << 5;
      v[c] = __ldg(slots + (x & mask));
    }
#pragma unroll
    for (int c = 0; c < kChains; ++c) acc += v[c];
  }
  if (acc == (T)-1234.5) sink[0] = acc;  // the slots hold zeros: never true
}

template <typename K>
kg_status time_best(K launch, cudaStream_t s, float* best_ms) {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    return fail(KG_ERR_CUDA, "kg_measure_box: event creation");
  }
  launch();  // warm-up
  float best = 1e30f;
  cudaError_t e = cudaSuccess;
  for (int r = 0; r < 3 && e == cudaSuccess; ++r) {
    cudaEventRecord(e0, s);
    launch();
    cudaEventRecord(e1, s);
    e = cudaEventSynchronize(e1);
    float t = 0.f;
    if (e == cudaSuccess && cudaEventElapsedTime(&t, e0, e1) == cudaSuccess) best = std::min(best, t);
  }
  if (e == cudaSuccess) e = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess) return cuda_fail(e, "kg_measure_box");
  *best_ms = best;
  return KG_OK;
}

}  // namespace
}  // namespace kg

using namespace kg;

extern "C" kg_status kg_measure_box(kg_box_rates* out, kg_stream stream) {
  if (!out) return fail(KG_ERR_INVALID_ARG, "kg_measure_box: out is NULL");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  int dev = 0, sms = 0, l2 = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev);
  if (e != cudaSuccess) return cuda_fail(e, "kg_measure_box: device attributes");
  constexpr uint32_t kSlots = 1u << 20;  // 8 MiB of doubles
  void* buf = nullptr;
  if ((e = cudaMalloc(&buf, kSlots * sizeof(double))) != cudaSuccess)
    return cuda_fail(e, "kg_measure_box: scratch");
  cudaMemsetAsync(buf, 0, kSlots * sizeof(double), s);
  kg_status rc = KG_OK;
  float ms = 0.f;
  const int grid = sms * 4;
  const double threads = (double)grid * kBoxBlock;
  const int it64 = 1024, it32 = 65536;
  rc = time_best([&] { fma_rate_kernel<double><<<grid, kBoxBlock, 0, s>>>(
                           static_cast<double*>(buf), it64, 0.999999, 1e-6); }, s, &ms);
  if (rc == KG_OK) out->fp64_fma_tflops = 2.0 * threads * it64 * kChains / (ms * 1e-3) / 1e12;
  if (rc == KG_OK)
    rc = time_best([&] { fma_rate_kernel<float><<<grid, kBoxBlock, 0, s>>>(
                             static_cast<float*>(buf), it32, 0.999999f, 1e-6f); }, s, &ms);
  if (rc == KG_OK) out->fp32_fma_tflops = 2.0 * threads * it32 * kChains / (ms * 1e-3) / 1e12;
  const int rgrid = sms * 8, per = 256;
  const double reds = (double)rgrid * kBoxBlock * per;
  if (rc == KG_OK)
    rc = time_best([&] { red_rate_kernel<double><<<rgrid, kBoxBlock, 0, s>>>(
                             static_cast<double*>(buf), kSlots - 1, per); }, s, &ms);
  if (rc == KG_OK) out->fp64_red_gops = reds / (ms * 1e-3) / 1e9;
  if (rc == KG_OK)
    rc = time_best([&] { red_rate_kernel<float><<<rgrid, kBoxBlock, 0, s>>>(
                             static_cast<float*>(buf), kSlots - 1, per); }, s, &ms);
  if (rc == KG_OK) out->fp32_red_gops = reds / (ms * 1e-3) / 1e9;
  // the red kernels left the slots at small integers; the gathers want zeros
  if (rc == KG_OK && cudaMemsetAsync(buf, 0, kSlots * sizeof(double), s) != cudaSuccess)
    rc = fail(KG_ERR_CUDA, "kg_measure_box: scratch reset");
  if (rc == KG_OK)
    rc = time_best([&] { gather_rate_kernel<double><<<rgrid, kBoxBlock, 0, s>>>(
                             static_cast<const double*>(buf), kSlots - 1, per, static_cast<double*>(buf)); }, s, &ms);
  if (rc == KG_OK) out->fp64_gather_gops = reds / (ms * 1e-3) / 1e9;
  if (rc == KG_OK)
    rc = time_best([&] { gather_rate_kernel<float><<<rgrid, kBoxBlock, 0, s>>>(
                             static_cast<const float*>(buf), kSlots - 1, per, static_cast<float*>(buf)); }, s, &ms);
  if (rc == KG_OK) out->fp32_gather_gops = reds / (ms * 1e-3) / 1e9;
  const int itl = 64;
  if (rc == KG_OK)
    rc = time_best([&] { log1p_rate_kernel<<<grid, kBoxBlock, 0, s>>>(static_cast<double*>(buf), itl); }, s,
                   &ms);
  if (rc == KG_OK) out->fp64_log1p_gops = threads * itl * kChains / (ms * 1e-3) / 1e9;
  if (rc == KG_OK)
    rc = time_best([&] { div_rate_kernel<<<grid, kBoxBlock, 0, s>>>(static_cast<double*>(buf), itl, 1.25); }, s,
                   &ms);
  if (rc == KG_OK) out->fp64_div_gops = threads * itl * kChains / (ms * 1e-3) / 1e9;
  out->sms = sms;
  out->l2_bytes = l2;
  cudaStreamSynchronize(s);
  cudaFree(buf);
  return rc;
}
