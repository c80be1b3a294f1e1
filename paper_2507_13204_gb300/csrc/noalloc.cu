// Allocation-free value-and-gradient of f(x) = ||A x||^2 (FP64).
//
// Some callers cannot allocate device memory when they need a gradient: code
// under a memory manager that owns the whole device heap, a plug-in that must
// not grow the process's device footprint once it is running, or a real-time
// loop that must never enter the allocator.  They cannot use kg_create, which
// allocates the problem's workspaces.  This
// entry point instead takes all of its scratch from one array compiled into
// the library, so the call itself allocates nothing: the caller passes only
// its inputs and outputs.
//
// The array (kNoAllocScratchBytes, 16 MiB) lives in device memory on every GPU
// that loads the library, until the process exits.  Its contents persist from
// call to call; the kernels write every location they later read within the
// same call, so nothing needs clearing.  All calls share it: calls that run at
// the same time on the GPU (different streams, or different host threads)
// race on it and must be serialised by the caller.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "kg_internal.h"

namespace {

constexpr size_t kNoAllocScratchBytes = size_t(16) << 20;
constexpr size_t kNoAllocScratchDoubles = kNoAllocScratchBytes / sizeof(double);

// Device-side scratch.  In host code this name is only a stand-in for the
// symbol; its device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocScratchDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double* g_scratch_ptr[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device, looked up once
// per device (with that device current) and cached.  The first call on a
// device does this look-up; it should come before any stream capture.
kg_status scratch_for_current_device(double** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return kg::cuda_fail(e, "kg_quadform_grad_noalloc: cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices)
    return kg::fail(KG_ERR_UNSUPPORTED, "kg_quadform_grad_noalloc: device index >= 64");
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p)
      return kg::cuda_fail(e != cudaSuccess ? e : cudaErrorInvalidSymbol,
                           "kg_quadform_grad_noalloc: cudaGetSymbolAddress");
    g_scratch_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_ptr[dev];
  return KG_OK;
}

}  // namespace

extern "C" kg_status kg_quadform_grad_noalloc(const double* A, int64_t m, int64_t n,
                                              const double* x, double* f, double* gx,
                                              kg_stream s) {
  kg::reset_launch_count();
  if (!A || !x || !gx) return kg::fail(KG_ERR_INVALID_ARG, "kg_quadform_grad_noalloc: NULL argument");
  if (m < 1 || n < 1 || m >= (int64_t(1) << 31) || n > 12288)
    return kg::fail(KG_ERR_INVALID_ARG,
                    "kg_quadform_grad_noalloc: need 1 <= m < 2^31 and 1 <= n <= 12288");
  double* scratch = nullptr;
  kg_status rc = scratch_for_current_device(&scratch);
  if (rc != KG_OK) return rc;
  return kg::qf_native_fused_on_scratch(A, m, n, x, f, gx, scratch, kNoAllocScratchDoubles,
                                        reinterpret_cast<cudaStream_t>(s));
}
