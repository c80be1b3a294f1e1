// The paper's example (Sec. 4, Fig. "function_f"): f(x, b) = ||A (3 x) - b||^2
// with A = tridiag(-1, 2, -1), rows 0 and n-1 truncated.
//
// KG_STRATEGY_ATOMIC follows the structure of the paper's generated gradient
// (Fig. "grad_f"): three forward kernels (scale, stencil + square, sum) and
// three reverse kernels in reverse order (broadcast of the sum's adjoint; the
// stencil's reverse with atomic scatter to the neighbours, because the
// stencil reads x at three different loop-index expressions, the paper's
// second race rule; the reverse of the scale).
// KG_STRATEGY_FUSED (default) is the single-kernel value-and-grad: the
// stencil's transpose is again a 3-point stencil, so each thread gathers
// xbar_j = 3 (2 ybar_j - ybar_{j-1} - ybar_{j+1}) with no atomics (the
// rescheduling and kernel fusion of Sec. 5).
// KG_MODE_TAPE adds the taped chain: kg_eval_tape records y in the forward
// kernel, kg_grad_from_tape runs the reverse chain from the tape alone.
#include <cuda_runtime.h>

#include <algorithm>

#include "kg_device.cuh"
#include "kg_internal.h"

namespace kg {

template <typename T>
__device__ __forceinline__ T lap_y(const T* __restrict__ x, const T* __restrict__ b, int j, int n) {
  T v = T(2) * (T(3) * x[j]) - b[j];
  if (j != 0) v -= T(3) * x[j - 1];
  if (j != n - 1) v -= T(3) * x[j + 1];
  return v;
}

template <typename T>
__global__ void __launch_bounds__(256) lap_eval_kernel(const T* __restrict__ x, const T* __restrict__ b,
                                                       int n, double* fpart, unsigned* counter, T* f) {
  __shared__ double scratch[32];
  double acc = 0.0;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
    const T y = lap_y(x, b, j, n);
    acc += (double)(y * y);
  }
  acc = block_sum(acc, scratch);
  finish_sum<T>(acc, fpart, counter, f, 0, scratch);
}

template <typename T>
__global__ void __launch_bounds__(256) lap_fused_kernel(const T* __restrict__ x, const T* __restrict__ b,
                                                        int n, const T* seed, double* fpart,
                                                        unsigned* counter, T* f, T* gx, T* gb,
                                                        int accumulate) {
  __shared__ double scratch[32];
  const T fb = load_seed(seed);
  double acc = 0.0;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
    const T y = lap_y(x, b, j, n);
    acc += (double)(y * y);
    const T yb = T(2) * fb * y;
    T x3b = T(2) * yb;
    if (j != 0) x3b -= T(2) * fb * lap_y(x, b, j - 1, n);
    if (j != n - 1) x3b -= T(2) * fb * lap_y(x, b, j + 1, n);
    const T g = T(3) * x3b;
    gx[j] = accumulate ? gx[j] + g : g;
    if (gb) gb[j] = accumulate ? gb[j] - yb : -yb;
  }
  acc = block_sum(acc, scratch);
  finish_sum<T>(acc, fpart, counter, f, 0, scratch);
}

// ---- TAPE mode: the chain x -> y -> y^2 -> sum with y taped ----------------
// The forward writes y (the only value the reverse of the chain needs: the
// reverse of y^2 is 2 y ybar) to a tape of n values allocated once at
// kg_create (Sec. 5, third restriction); the reverse reads the tape instead of
// re-running the stencil: xbar_j = 3 (2 ybar_j - ybar_{j-1} - ybar_{j+1}) with
// ybar = 2 fbar y, b unread.
template <typename T>
__global__ void __launch_bounds__(256) lap_tape_kernel(const T* __restrict__ x, const T* __restrict__ b,
                                                       int n, T* tape, double* fpart,
                                                       unsigned* counter, T* f) {
  __shared__ double scratch[32];
  double acc = 0.0;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
    const T y = lap_y(x, b, j, n);
    tape[j] = y;
    acc += (double)(y * y);
  }
  acc = block_sum(acc, scratch);
  finish_sum<T>(acc, fpart, counter, f, 0, scratch);
}

template <typename T>
__global__ void __launch_bounds__(256) lap_from_tape_kernel(const T* __restrict__ tape, int n,
                                                            const T* seed, T* gx, int accumulate) {
  const T fb2 = T(2) * load_seed(seed);
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
    T x3b = T(2) * (fb2 * tape[j]);
    if (j != 0) x3b -= fb2 * tape[j - 1];
    if (j != n - 1) x3b -= fb2 * tape[j + 1];
    const T g = T(3) * x3b;
    gx[j] = accumulate ? gx[j] + g : g;
  }
}

// Hessian-vector product: the tangent (direction v) of the fused value-and-
// gradient; f is quadratic in x, so x and b drop out: ydot_j = (A (3v))_j and
// hv_j = 3 (2 ybd_j - ybd_{j-1} - ybd_{j+1}) with ybd = 2 fbar ydot.
template <typename T>
__device__ __forceinline__ T lap_ydot(const T* __restrict__ v, int j, int n) {
  T t = T(2) * (T(3) * v[j]);
  if (j != 0) t -= T(3) * v[j - 1];
  if (j != n - 1) t -= T(3) * v[j + 1];
  return t;
}

template <typename T>
__global__ void __launch_bounds__(256) lap_hvp_kernel(const T* __restrict__ v, int n, const T* seed,
                                                      T* hv, int accumulate) {
  const T fb2 = T(2) * load_seed(seed);
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
    T x3b = T(2) * (fb2 * lap_ydot(v, j, n));
    if (j != 0) x3b -= fb2 * lap_ydot(v, j - 1, n);
    if (j != n - 1) x3b -= fb2 * lap_ydot(v, j + 1, n);
    const T g = T(3) * x3b;
    hv[j] = accumulate ? hv[j] + g : g;
  }
}

// ---- the six kernels of the paper's generated gradient ------------------
template <typename T>
__global__ void lap_k1_scale(const T* x, T* x3, int n) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x)
    x3[j] = T(3) * x[j];
}
template <typename T>
__global__ void lap_k2_stencil(const T* x3, const T* b, T* y, T* y2, int n) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
    T v = T(2) * x3[j] - b[j];
    if (j != 0) v -= x3[j - 1];
    if (j != n - 1) v -= x3[j + 1];
    y[j] = v;
    y2[j] = v * v;
  }
}
template <typename T>
__global__ void __launch_bounds__(256) lap_k3_sum(const T* y2, int n, double* fpart, unsigned* counter,
                                                  T* f) {
  __shared__ double scratch[32];
  double acc = 0.0;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x)
    acc += (double)y2[j];
  acc = block_sum(acc, scratch);
  finish_sum<T>(acc, fpart, counter, f, 0, scratch);
}
// reverse of the sum: broadcast fbar into y2bar (y2bar += fbar)
template <typename T>
__global__ void lap_k3t_broadcast(const T* seed, T* y2b, int n) {
  const T fb = load_seed(seed);
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x)
    y2b[j] += fb;
}
// reverse of stencil + square; the neighbour updates race, so they are atomic
template <typename T>
__global__ void lap_k2t_stencil(const T* y, T* y2b, T* yb, T* x3b, T* gb, int n, int accumulate) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
    const T r = y2b[j];
    y2b[j] -= r;
    yb[j] += T(2) * y[j] * r;
    const T ry = yb[j];
    if (j != n - 1) red_add(x3b + j + 1, -ry);
    if (j != 0) red_add(x3b + j - 1, -ry);
    yb[j] -= ry;
    red_add(x3b + j, T(2) * ry);
    if (gb) gb[j] = accumulate ? gb[j] - ry : -ry;
  }
}
// reverse of the scale
template <typename T>
__global__ void lap_k1t_scale(const T* x3b, T* gx, int n, int accumulate) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
    const T g = T(3) * x3b[j];
    gx[j] = accumulate ? gx[j] + g : g;
  }
}

// ---------------------------------------------------------------- host ----
static int lap_grid(int64_t n) {
  return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, (int64_t)num_sms() * 8));
}

kg_status lap_setup(kg_problem* p, cudaStream_t s) {
  if (p->strategy == KG_STRATEGY_AUTO) p->strategy = KG_STRATEGY_FUSED;
  if (p->strategy != KG_STRATEGY_FUSED && p->strategy != KG_STRATEGY_ATOMIC)
    return fail(KG_ERR_UNSUPPORTED, "LAPLACE1D: strategy must be FUSED or ATOMIC");
  // TAPE on request only: the fused recompute is one pass over x and b either way
  p->mode = p->mode == KG_MODE_TAPE ? KG_MODE_TAPE : KG_MODE_RECOMPUTE;
  if (p->arith == KG_ARITH_AUTO) p->arith = KG_ARITH_NATIVE;
  kg_status rc = ws_common(p, lap_grid(p->n), s);
  if (rc != KG_OK) return rc;
  if (p->mode == KG_MODE_TAPE &&
      (rc = ws_alloc(p, &p->tape, p->esize * (size_t)p->n, "1-D tape y")) != KG_OK)
    return rc;
  if (p->strategy == KG_STRATEGY_ATOMIC) {
    // x3, y, y2 (forward "views") and their shadows y2bar, ybar, x3bar
    rc = ws_alloc(p, &p->y, p->esize * 6 * (size_t)p->n, "1-D views and shadows");
    if (rc != KG_OK) return rc;
  }
  return KG_OK;
}

template <typename T>
static kg_status lap_eval_t(kg_problem* p, const void* x, void* f, cudaStream_t s) {
  const int n = (int)p->n;
  prof_begin(s, "lap_eval_kernel");
  struct End { cudaStream_t s; ~End() { prof_end(s); } } end{s};
  lap_eval_kernel<T><<<lap_grid(n), 256, 0, s>>>(static_cast<const T*>(x),
                                                 static_cast<const T*>(p->data0), n, p->fpart,
                                                 p->counter, static_cast<T*>(f));
  count_launch();
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? KG_OK : cuda_fail(e, "1-D forward kernel");
}

kg_status lap_eval(kg_problem* p, const void* x, void* f, cudaStream_t s) {
  return p->dtype == KG_F64 ? lap_eval_t<double>(p, x, f, s) : lap_eval_t<float>(p, x, f, s);
}

template <typename T>
static kg_status lap_grad_t(kg_problem* p, const void* xv, void* f, void* gx, void* gb,
                            const void* seed, int accumulate, cudaStream_t s) {
  const int n = (int)p->n, g = lap_grid(n);
  const T* x = static_cast<const T*>(xv);
  const T* b = static_cast<const T*>(p->data0);
  cudaError_t e;
  if (p->strategy == KG_STRATEGY_FUSED) {
    prof_begin(s, "lap_fused_kernel");
    struct End { cudaStream_t s; ~End() { prof_end(s); } } end{s};
    lap_fused_kernel<T><<<g, 256, 0, s>>>(x, b, n, static_cast<const T*>(seed), p->fpart, p->counter,
                                          static_cast<T*>(f), static_cast<T*>(gx),
                                          static_cast<T*>(gb), accumulate);
    count_launch();
    e = cudaGetLastError();
    return e == cudaSuccess ? KG_OK : cuda_fail(e, "1-D fused kernel");
  }
  T* w = static_cast<T*>(p->y);
  T *x3 = w, *y = w + n, *y2 = w + 2 * n, *y2b = w + 3 * n, *yb = w + 4 * n, *x3b = w + 5 * n;
  // shadows start at zero (Sec. 3.1: the shadow of a constructed view)
  // timed as one unit: the generated gradient's six kernels and the shadow zeroing
  prof_begin(s, "lap generated gradient (memset + 6 kernels)");
  struct End { cudaStream_t s; ~End() { prof_end(s); } } end{s};
  if ((e = cudaMemsetAsync(y2b, 0, sizeof(T) * 3 * (size_t)n, s)) != cudaSuccess)
    return cuda_fail(e, "zero shadows");
  lap_k1_scale<T><<<g, 256, 0, s>>>(x, x3, n);
  lap_k2_stencil<T><<<g, 256, 0, s>>>(x3, b, y, y2, n);
  lap_k3_sum<T><<<g, 256, 0, s>>>(y2, n, p->fpart, p->counter, static_cast<T*>(f));
  lap_k3t_broadcast<T><<<g, 256, 0, s>>>(static_cast<const T*>(seed), y2b, n);
  lap_k2t_stencil<T><<<g, 256, 0, s>>>(y, y2b, yb, x3b, static_cast<T*>(gb), n, accumulate);
  lap_k1t_scale<T><<<g, 256, 0, s>>>(x3b, static_cast<T*>(gx), n, accumulate);
  count_launch(7);
  e = cudaGetLastError();
  return e == cudaSuccess ? KG_OK : cuda_fail(e, "1-D generated-gradient kernels");
}

kg_status lap_grad(kg_problem* p, const void* x, void* f, void* gx, void* gb, const void* seed,
                   int accumulate, cudaStream_t s) {
  return p->dtype == KG_F64 ? lap_grad_t<double>(p, x, f, gx, gb, seed, accumulate, s)
                            : lap_grad_t<float>(p, x, f, gx, gb, seed, accumulate, s);
}

template <typename T>
static kg_status lap_eval_tape_t(kg_problem* p, const void* x, void* f, cudaStream_t s) {
  const int n = (int)p->n;
  prof_begin(s, "lap_tape_kernel");
  lap_tape_kernel<T><<<lap_grid(n), 256, 0, s>>>(static_cast<const T*>(x),
                                                 static_cast<const T*>(p->data0), n,
                                                 static_cast<T*>(p->tape), p->fpart, p->counter,
                                                 static_cast<T*>(f));
  prof_end(s);
  count_launch();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "1-D taping forward kernel");
  p->tape_valid = true;
  p->tape_gen += 1;
  return KG_OK;
}

template <typename T>
static kg_status lap_grad_from_tape_t(kg_problem* p, void* gx, const void* seed, int accumulate,
                                      cudaStream_t s) {
  const int n = (int)p->n;
  prof_begin(s, "lap_from_tape_kernel");
  lap_from_tape_kernel<T><<<lap_grid(n), 256, 0, s>>>(static_cast<const T*>(p->tape), n,
                                                      static_cast<const T*>(seed),
                                                      static_cast<T*>(gx), accumulate);
  prof_end(s);
  count_launch();
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? KG_OK : cuda_fail(e, "1-D reverse from tape");
}

kg_status lap_eval_tape(kg_problem* p, const void* x, void* f, cudaStream_t s) {
  return p->dtype == KG_F64 ? lap_eval_tape_t<double>(p, x, f, s) : lap_eval_tape_t<float>(p, x, f, s);
}

kg_status lap_grad_from_tape(kg_problem* p, void* gx, const void* seed, int accumulate,
                             cudaStream_t s) {
  return p->dtype == KG_F64 ? lap_grad_from_tape_t<double>(p, gx, seed, accumulate, s)
                            : lap_grad_from_tape_t<float>(p, gx, seed, accumulate, s);
}

template <typename T>
static kg_status lap_hvp_t(kg_problem* p, const void* v, void* hv, const void* seed, int accumulate,
                           cudaStream_t s) {
  const int n = (int)p->n;
  prof_begin(s, "lap_hvp_kernel");
  lap_hvp_kernel<T><<<lap_grid(n), 256, 0, s>>>(static_cast<const T*>(v), n,
                                                static_cast<const T*>(seed), static_cast<T*>(hv),
                                                accumulate);
  prof_end(s);
  count_launch();
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? KG_OK : cuda_fail(e, "1-D Hessian-vector kernel");
}

kg_status lap_hvp(kg_problem* p, const void* v, void* hv, const void* seed, int accumulate,
                  cudaStream_t s) {
  return p->dtype == KG_F64 ? lap_hvp_t<double>(p, v, hv, seed, accumulate, s)
                            : lap_hvp_t<float>(p, v, hv, seed, accumulate, s);
}

}  // namespace kg
