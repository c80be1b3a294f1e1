// Unstructured tet-mesh energy f(u) = sum_e log1p(|G_e u_e|^2) and its
// reverse-mode gradient.
//
// Forward: u_e = u[conn[e][0..3]] is a read through an index map (Sec. 3.3,
// first race rule), g_e = G_e u_e, f = sum_e log1p(|g_e|^2) (a parallel_sum).
// Reverse: fbar is broadcast to every element (Sec. 3.2), the element adjoint
// is c_e = G_e^T (2 fbar g_e / (1 + |g_e|^2)), and each gathered read becomes
// the scatter-add gu[conn[e][k]] += c_e[k] -- atomic when the reverse reuses
// the forward schedule (KG_STRATEGY_ATOMIC, the paper's choice), or an
// atomic-free gather over the transposed connectivity (KG_STRATEGY_CSR: the
// rescheduling proposed in Sec. 5).  In TAPE mode the forward stores c_e (for
// fbar = 1) so that the reverse pass reads neither G nor u (Sec. 5, taping
// allocated once outside the kernel).
#include <cuda_runtime.h>

#include <algorithm>
#include <string>

#include "kg_device.cuh"
#include "kg_internal.h"

namespace kg {

template <typename T>
__device__ __forceinline__ T log1p_t(T v) {
  if constexpr (sizeof(T) == 8) return log1p(v);
  else return log1pf(v);
}

template <typename T>
struct TetArgs {
  const int4* conn;
  const T* G;
  const T* u;
  int64_t ne;
  int nv;
  const T* seed;
  T* gu;
  T* tape;  // [ne][4]
  double* fpart;
  unsigned* counter;
  T* f;
  unsigned* err;
  int check;
};

enum { TET_EVAL = 0, TET_GRAD = 1, TET_TAPE = 2 };

// Loads the 12 entries of G_e (row-major 3x4) with 16-byte loads.
template <typename T>
__device__ __forceinline__ void load_G(const T* __restrict__ Ge, T g[12]) {
  if constexpr (sizeof(T) == 8) {
    const double2* p = reinterpret_cast<const double2*>(Ge);
#pragma unroll
    for (int i = 0; i < 6; ++i) {
      double2 v = __ldcs(p + i);
      g[2 * i] = v.x;
      g[2 * i + 1] = v.y;
    }
  } else {
    const float4* p = reinterpret_cast<const float4*>(Ge);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      float4 v = __ldcs(p + i);
      g[4 * i] = v.x;
      g[4 * i + 1] = v.y;
      g[4 * i + 2] = v.z;
      g[4 * i + 3] = v.w;
    }
  }
}

// One thread per element (grid-stride).  EVAL: f.  GRAD: f and the atomic
// scatter of fbar * c_e.  TAPE: f and c_e (fbar = 1) stored to the tape.
template <typename T, int MODE>
__global__ void __launch_bounds__(256) tet_kernel(TetArgs<T> a) {
  __shared__ double scratch[32];
  const T fb = MODE == TET_GRAD ? load_seed(a.seed) : T(1);
  T facc = T(0);
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < a.ne; e += stride) {
    const int4 c = __ldcs(a.conn + e);
    if (a.check) {
      if ((unsigned)c.x >= (unsigned)a.nv || (unsigned)c.y >= (unsigned)a.nv ||
          (unsigned)c.z >= (unsigned)a.nv || (unsigned)c.w >= (unsigned)a.nv) {
        set_error(a.err, ERRBIT_BOUNDS);
        continue;
      }
    }
    T G[12];
    load_G<T>(a.G + e * 12, G);
    const T u0 = __ldg(a.u + c.x), u1 = __ldg(a.u + c.y), u2 = __ldg(a.u + c.z),
            u3 = __ldg(a.u + c.w);
    const T g0 = G[0] * u0 + G[1] * u1 + G[2] * u2 + G[3] * u3;
    const T g1 = G[4] * u0 + G[5] * u1 + G[6] * u2 + G[7] * u3;
    const T g2 = G[8] * u0 + G[9] * u1 + G[10] * u2 + G[11] * u3;
    const T s = g0 * g0 + g1 * g1 + g2 * g2;
    facc += log1p_t(s);
    if constexpr (MODE != TET_EVAL) {
      const T w = T(2) * fb / (T(1) + s);
      const T w0 = w * g0, w1 = w * g1, w2 = w * g2;
      const T c0 = G[0] * w0 + G[4] * w1 + G[8] * w2;
      const T c1 = G[1] * w0 + G[5] * w1 + G[9] * w2;
      const T c2 = G[2] * w0 + G[6] * w1 + G[10] * w2;
      const T c3 = G[3] * w0 + G[7] * w1 + G[11] * w2;
      if constexpr (MODE == TET_GRAD) {
        atomicAdd(a.gu + c.x, c0);
        atomicAdd(a.gu + c.y, c1);
        atomicAdd(a.gu + c.z, c2);
        atomicAdd(a.gu + c.w, c3);
      } else {
        T* t = a.tape + e * 4;
        if constexpr (sizeof(T) == 8) {
          __stcs(reinterpret_cast<double2*>(t), make_double2(c0, c1));
          __stcs(reinterpret_cast<double2*>(t) + 1, make_double2(c2, c3));
        } else {
          __stcs(reinterpret_cast<float4*>(t), make_float4(c0, c1, c2, c3));
        }
      }
    }
  }
  const double fcta = block_sum((double)facc, scratch);
  finish_sum<T>(fcta, a.fpart, a.counter, a.f, 0, scratch);
}

// Reverse from the tape with the forward schedule: atomic scatter of fbar*c_e.
template <typename T>
__global__ void __launch_bounds__(256) tet_tape_scatter_kernel(const int4* __restrict__ conn,
                                                               const T* __restrict__ tape,
                                                               int64_t ne, const T* seed, T* gu) {
  const T fb = load_seed(seed);
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < ne; e += stride) {
    const int4 c = __ldcs(conn + e);
    const T* t = tape + e * 4;
    atomicAdd(gu + c.x, fb * t[0]);
    atomicAdd(gu + c.y, fb * t[1]);
    atomicAdd(gu + c.z, fb * t[2]);
    atomicAdd(gu + c.w, fb * t[3]);
  }
}

// Atomic-free reverse: thread per vertex gathers its incidences, in ascending
// (e, k) order, from the tape: gu[v] (+)= fbar * sum_p tape[inc[p]].
template <typename T>
__global__ void __launch_bounds__(256) tet_csr_gather_kernel(const int* __restrict__ rowptr,
                                                             const int* __restrict__ inc,
                                                             const T* __restrict__ tape, int nv,
                                                             const T* seed, T* gu, int accumulate) {
  const T fb = load_seed(seed);
  const int stride = gridDim.x * blockDim.x;
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < nv; v += stride) {
    const int p0 = rowptr[v], p1 = rowptr[v + 1];
    T s = T(0);
    for (int p = p0; p < p1; ++p) s += tape[inc[p]];
    const T r = fb * s;
    gu[v] = accumulate ? gu[v] + r : r;
  }
}

// ------------------------------------------------- set-up kernels ---------
__global__ void tet_validate_kernel(const int* __restrict__ conn, int64_t n4, int nv,
                                    unsigned* err) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += stride)
    if ((unsigned)conn[i] >= (unsigned)nv) set_error(err, ERRBIT_BOUNDS);
}

__global__ void csr_degree_kernel(const int* __restrict__ conn, int64_t n4, int* deg) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += stride)
    atomicAdd(deg + conn[i], 1);
}

// In-place exclusive scan of deg[0..n) into rowptr[0..n] (rowptr[n] = total),
// one CTA of 1024 threads walking the array in chunks (set-up only).
__global__ void __launch_bounds__(1024) csr_scan_kernel(int* data, int n) {
  __shared__ int wsum[32];
  __shared__ int carry_s;
  if (threadIdx.x == 0) carry_s = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int base = 0; base < n; base += 1024) {
    const int i = base + threadIdx.x;
    const int v = i < n ? data[i] : 0;
    int incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int t = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += t;
    }
    if (lane == 31) wsum[w] = incl;
    __syncthreads();
    if (w == 0) {
      int ws = wsum[lane];
      int wi = ws;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        int t = __shfl_up_sync(0xffffffffu, wi, o);
        if (lane >= o) wi += t;
      }
      wsum[lane] = wi - ws;  // exclusive warp offsets
    }
    __syncthreads();
    const int carry = carry_s;
    if (i < n) data[i] = carry + wsum[w] + incl - v;
    __syncthreads();
    if (threadIdx.x == 1023) carry_s = carry + wsum[31] + incl;
    __syncthreads();
  }
  if (threadIdx.x == 0) data[n] = carry_s;
}

__global__ void csr_fill_kernel(const int* __restrict__ conn, int64_t n4, int* cursor, int* inc) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += stride) {
    const int pos = atomicAdd(cursor + conn[i], 1);
    inc[pos] = (int)i;  // i = 4 e + k = (e << 2) | k
  }
}

// Sort each vertex's incidence list ascending so that the gather order (and
// thus the rounding) does not depend on the order atomics filled it.
__global__ void csr_sort_kernel(const int* __restrict__ rowptr, int nv, int* inc) {
  const int stride = gridDim.x * blockDim.x;
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < nv; v += stride) {
    const int p0 = rowptr[v], p1 = rowptr[v + 1];
    for (int p = p0 + 1; p < p1; ++p) {
      const int key = inc[p];
      int q = p - 1;
      while (q >= p0 && inc[q] > key) {
        inc[q + 1] = inc[q];
        --q;
      }
      inc[q + 1] = key;
    }
  }
}

// ---------------------------------------------------------------- host ----
static int grid_for(int64_t work, int block, int per_sm) {
  int64_t g = (work + block - 1) / block;
  return (int)std::max<int64_t>(1, std::min<int64_t>(g, (int64_t)num_sms() * per_sm));
}

kg_status tet_setup(kg_problem* p, cudaStream_t s) {
  if (p->m * 4 >= (int64_t(1) << 31))
    return fail(KG_ERR_INVALID_ARG, "TETENERGY: 4 * N_e must be < 2^31");
  if (p->strategy == KG_STRATEGY_AUTO) p->strategy = KG_STRATEGY_ATOMIC;
  if (p->strategy != KG_STRATEGY_ATOMIC && p->strategy != KG_STRATEGY_CSR)
    return fail(KG_ERR_UNSUPPORTED, "TETENERGY: strategy must be ATOMIC or CSR");
  const size_t tape_bytes = p->esize * 4 * (size_t)p->m;
  const size_t budget = p->opt.tape_budget_bytes ? p->opt.tape_budget_bytes : (size_t(1) << 30);
  if (p->mode == KG_MODE_AUTO) p->mode = tape_bytes <= budget ? KG_MODE_TAPE : KG_MODE_RECOMPUTE;
  if (p->arith == KG_ARITH_AUTO) p->arith = KG_ARITH_NATIVE;
  p->tet_block = p->opt.block ? p->opt.block : 256;
  if (p->tet_block != 256) return fail(KG_ERR_UNSUPPORTED, "TETENERGY: block must be 256");
  p->tet_grid = grid_for(p->m, p->tet_block, 8);
  kg_status rc = ws_common(p, p->tet_grid, s);
  if (rc != KG_OK) return rc;
  if (p->mode == KG_MODE_TAPE || p->strategy == KG_STRATEGY_CSR) {
    if ((rc = ws_alloc(p, &p->tape, tape_bytes, "tape c_e")) != KG_OK) return rc;
  }
  const int64_t n4 = 4 * p->m;
  const int* conn = static_cast<const int*>(p->data0);
  tet_validate_kernel<<<grid_for(n4, 256, 8), 256, 0, s>>>(conn, n4, (int)p->n, p->err);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "validate connectivity");
  if (p->strategy == KG_STRATEGY_CSR) {
    // the connectivity must be in range before it is used as an index
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_fail(e, "validate connectivity");
    unsigned h = 0;
    if ((e = cudaMemcpy(&h, p->err, sizeof(h), cudaMemcpyDeviceToHost)) != cudaSuccess)
      return cuda_fail(e, "read error word");
    if (h & ERRBIT_BOUNDS) return fail(KG_ERR_BOUNDS, "kg_create: connectivity entry outside [0, N_v)");
    if ((rc = ws_alloc(p, (void**)&p->rowptr, sizeof(int) * (size_t)(p->n + 1), "CSR rowptr")) != KG_OK)
      return rc;
    if ((rc = ws_alloc(p, (void**)&p->inc, sizeof(int) * (size_t)n4, "CSR incidences")) != KG_OK)
      return rc;
    int* cursor = nullptr;
    if ((e = dev_alloc((void**)&cursor, sizeof(int) * (size_t)p->n)) != cudaSuccess)
      return fail(KG_ERR_OOM, "CSR build cursor allocation failed");
    bool ok = cudaMemsetAsync(p->rowptr, 0, sizeof(int) * (size_t)(p->n + 1), s) == cudaSuccess;
    if (ok) {
      csr_degree_kernel<<<grid_for(n4, 256, 8), 256, 0, s>>>(conn, n4, p->rowptr);
      csr_scan_kernel<<<1, 1024, 0, s>>>(p->rowptr, (int)p->n);
      ok = cudaMemcpyAsync(cursor, p->rowptr, sizeof(int) * (size_t)p->n, cudaMemcpyDeviceToDevice,
                           s) == cudaSuccess;
    }
    if (ok) {
      csr_fill_kernel<<<grid_for(n4, 256, 8), 256, 0, s>>>(conn, n4, cursor, p->inc);
      csr_sort_kernel<<<grid_for(p->n, 256, 8), 256, 0, s>>>(p->rowptr, (int)p->n, p->inc);
    }
    e = cudaGetLastError();
    cudaError_t e2 = cudaStreamSynchronize(s);
    cudaFree(cursor);
    if (!ok || e != cudaSuccess || e2 != cudaSuccess)
      return cuda_fail(e != cudaSuccess ? e : e2, "CSR build");
  }
  return KG_OK;
}

template <typename T>
static TetArgs<T> tet_args(kg_problem* p, const void* x, const void* seed, void* f) {
  TetArgs<T> a{};
  a.conn = static_cast<const int4*>(p->data0);
  a.G = static_cast<const T*>(p->data1);
  a.u = static_cast<const T*>(x);
  a.ne = p->m;
  a.nv = (int)p->n;
  a.seed = static_cast<const T*>(seed);
  a.tape = static_cast<T*>(p->tape);
  a.fpart = p->fpart;
  a.counter = p->counter;
  a.f = static_cast<T*>(f);
  a.err = p->err;
  a.check = p->opt.check;
  return a;
}

template <typename T>
static kg_status tet_eval_t(kg_problem* p, const void* x, void* f, bool tape, cudaStream_t s) {
  TetArgs<T> a = tet_args<T>(p, x, nullptr, f);
  prof_begin(s, tape ? "tet_kernel<tape>" : "tet_kernel<eval>");
  if (tape) tet_kernel<T, TET_TAPE><<<p->tet_grid, p->tet_block, 0, s>>>(a);
  else tet_kernel<T, TET_EVAL><<<p->tet_grid, p->tet_block, 0, s>>>(a);
  prof_end(s);
  count_launch();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "tet forward kernel");
  if (tape) p->tape_valid = true;
  return KG_OK;
}

kg_status tet_eval(kg_problem* p, const void* x, void* f, bool tape, cudaStream_t s) {
  return p->dtype == KG_F64 ? tet_eval_t<double>(p, x, f, tape, s)
                            : tet_eval_t<float>(p, x, f, tape, s);
}

template <typename T>
static kg_status tet_scatter_t(kg_problem* p, void* gx, const void* seed, int accumulate,
                               cudaStream_t s) {
  cudaError_t e;
  if (p->strategy == KG_STRATEGY_CSR) {
    prof_begin(s, "tet_csr_gather_kernel");
    tet_csr_gather_kernel<T><<<grid_for(p->n, 256, 8), 256, 0, s>>>(
        p->rowptr, p->inc, static_cast<const T*>(p->tape), (int)p->n, static_cast<const T*>(seed),
        static_cast<T*>(gx), accumulate);
    prof_end(s);
    count_launch();
  } else {
    if (!accumulate) {
      if ((e = cudaMemsetAsync(gx, 0, sizeof(T) * (size_t)p->n, s)) != cudaSuccess)
        return cuda_fail(e, "zero gu");
      count_launch();
    }
    prof_begin(s, "tet_tape_scatter_kernel");
    tet_tape_scatter_kernel<T><<<p->tet_grid, 256, 0, s>>>(
        static_cast<const int4*>(p->data0), static_cast<const T*>(p->tape), p->m,
        static_cast<const T*>(seed), static_cast<T*>(gx));
    prof_end(s);
    count_launch();
  }
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "tet reverse kernel");
  return KG_OK;
}

template <typename T>
static kg_status tet_grad_t(kg_problem* p, const void* x, void* f, void* gx, const void* seed,
                            int accumulate, cudaStream_t s) {
  if (p->strategy == KG_STRATEGY_CSR) {
    kg_status rc = tet_eval_t<T>(p, x, f, true, s);
    if (rc != KG_OK) return rc;
    return tet_scatter_t<T>(p, gx, seed, accumulate, s);
  }
  cudaError_t e;
  if (!accumulate) {
    if ((e = cudaMemsetAsync(gx, 0, sizeof(T) * (size_t)p->n, s)) != cudaSuccess)
      return cuda_fail(e, "zero gu");
    count_launch();
  }
  TetArgs<T> a = tet_args<T>(p, x, seed, f);
  a.gu = static_cast<T*>(gx);
  prof_begin(s, "tet_kernel<grad>");
  tet_kernel<T, TET_GRAD><<<p->tet_grid, p->tet_block, 0, s>>>(a);
  prof_end(s);
  count_launch();
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "tet fused value-and-grad kernel");
  return KG_OK;
}

kg_status tet_grad(kg_problem* p, const void* x, void* f, void* gx, const void* seed,
                   int accumulate, cudaStream_t s) {
  return p->dtype == KG_F64 ? tet_grad_t<double>(p, x, f, gx, seed, accumulate, s)
                            : tet_grad_t<float>(p, x, f, gx, seed, accumulate, s);
}

kg_status tet_grad_from_tape(kg_problem* p, void* gx, const void* seed, int accumulate,
                             cudaStream_t s) {
  return p->dtype == KG_F64 ? tet_scatter_t<double>(p, gx, seed, accumulate, s)
                            : tet_scatter_t<float>(p, gx, seed, accumulate, s);
}

}  // namespace kg
