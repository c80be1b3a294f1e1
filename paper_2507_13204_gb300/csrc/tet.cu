// Unstructured tet-mesh energy f(u) = sum_e log1p(|G_e u_e|^2) and its
// reverse-mode gradient.
//
// Forward: u_e = u[conn[e][0..3]] is a read through an index map (Sec. 3.3,
// first race rule), g_e = G_e u_e, f = sum_e log1p(|g_e|^2) (a parallel_sum).
// Reverse: fbar is broadcast to every element (Sec. 3.2), the element adjoint
// is c_e = G_e^T (2 fbar g_e / (1 + |g_e|^2)), and each gathered read becomes
// the scatter-add gu[conn[e][k]] += c_e[k] -- atomic when the reverse reuses
// the forward schedule (KG_STRATEGY_ATOMIC, the paper's choice), or an
// atomic-free, reproducible reverse over per-tile transposed connectivity
// (KG_STRATEGY_CSR, tet_tile.cu: the rescheduling proposed in Sec. 5).  In TAPE mode the forward stores c_e (for
// fbar = 1) so that the reverse pass reads neither G nor u (Sec. 5, taping
// allocated once outside the kernel).
//
// This file holds the set-up (validation, CSR build, prepared copies), the
// tape scatter and CSR gather kernels, the direct FP32 kernels and the
// dispatch; the FP64 and staged kernels are in tet_pair.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <string>

#include "kg_device.cuh"
#include "kg_internal.h"
#include "kg_pair.cuh"
#include "kg_tet_elem.cuh"

namespace kg {

// Reverse from the tape with the forward schedule: scatter of fbar*c_e, each
// contribution an atomic (ATOMIC, SHARED, FP64 WARP) or combined within the
// warp first (FP32 WARP, see warp_combine).  The loop is uniform per block so that every lane
// of a warp reaches the warp-level combine.
template <typename T, bool WARPC>
__global__ void __launch_bounds__(256) tet_tape_scatter_kernel(const int4* __restrict__ conn,
                                                               const T* __restrict__ tape,
                                                               int64_t ne, const T* seed, T* gu) {
  const T fb = load_seed(seed);
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e0 = (int64_t)blockIdx.x * blockDim.x; e0 < ne; e0 += stride) {
    const int64_t e = e0 + threadIdx.x;
    const bool act = e < ne;
    int4 c = make_int4(-1, -1, -1, -1);
    T t[4] = {T(0), T(0), T(0), T(0)};
    if (act) {
      c = __ldcs(conn + e);
      if constexpr (sizeof(T) == 8) {
        const double2 a = __ldcs(reinterpret_cast<const double2*>(tape) + 2 * e);
        const double2 b = __ldcs(reinterpret_cast<const double2*>(tape) + 2 * e + 1);
        t[0] = a.x, t[1] = a.y, t[2] = b.x, t[3] = b.y;
      } else {
        const float4 a = __ldcs(reinterpret_cast<const float4*>(tape) + e);
        t[0] = a.x, t[1] = a.y, t[2] = a.z, t[3] = a.w;
      }
    }
    const int key[4] = {c.x, c.y, c.z, c.w};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      if constexpr (WARPC) {
        warp_combine(act, key[k], fb * t[k], [](T x, T y) { return x + y; },
                     [&](int v, T tot) { red_add(gu + v, tot); });
      } else if (act) {
        red_add(gu + key[k], fb * t[k]);
      }
    }
  }
}

// FP32 kernels without shared-memory staging: no ring, no CTA barrier per
// tile, and more loads in flight per warp than the staged kernel at the same
// four CTAs of 256 threads per SM.  Each thread takes two elements per step:
// their conn (int4) and G (three float4) are streamed with no L1 allocation
// and all of their loads and u (and v) gathers are issued before any is used.
// Lanes of a warp hold consecutive elements; the scatter combines equal
// vertices of a warp by key groups (warp_combine_groups).  Modes as the staged
// kernel: forward, gradient (warp-combined or plain atomics), tape, Hessian-
// vector product.
struct DirectArgs {
  const int4* conn;
  const float4* G;
  const float* u;
  const float* v;
  int64_t ne;
  const float* seed;
  float* gu;
  float* tape;
  double* fpart;
  unsigned* counter;
  float* f;
};

template <int MODE, bool WARPC>
__global__ void __launch_bounds__(256) tet_direct_f32_kernel(DirectArgs a) {
  __shared__ double red[32];
  constexpr bool REV = MODE == TS_GRAD || MODE == TS_HVP;
  const int lane = threadIdx.x & 31;
  const float fb = REV ? load_seed(a.seed) : 1.f;
  float fa = 0.f, fc = 0.f;  // TwoSum-compensated float sum of f_e
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  // warp-uniform trip count: the loop runs on the warp's first element
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < a.ne;
       base += 2 * stride) {
    int4 c[2];
    float4 g[2][3];
    bool act[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int64_t e = base + lane + h * stride;
      act[h] = e < a.ne;
      c[h] = act[h] ? __ldcs(a.conn + e) : make_int4(0, 0, 0, 0);
#pragma unroll
      for (int q = 0; q < 3; ++q) g[h][q] = act[h] ? __ldcs(a.G + e * 3 + q) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    float uv[2][4], vv[2][4];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      uv[h][0] = __ldg(a.u + c[h].x);  // vertex 0 for inactive lanes (N_v >= 1)
      uv[h][1] = __ldg(a.u + c[h].y);
      uv[h][2] = __ldg(a.u + c[h].z);
      uv[h][3] = __ldg(a.u + c[h].w);
      if constexpr (MODE == TS_HVP) {
        vv[h][0] = __ldg(a.v + c[h].x);
        vv[h][1] = __ldg(a.v + c[h].y);
        vv[h][2] = __ldg(a.v + c[h].z);
        vv[h][3] = __ldg(a.v + c[h].w);
      }
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      float gg[3], gd[3];
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        gg[q] = g[h][q].x * uv[h][0] + g[h][q].y * uv[h][1] + g[h][q].z * uv[h][2] + g[h][q].w * uv[h][3];
        if constexpr (MODE == TS_HVP)
          gd[q] = g[h][q].x * vv[h][0] + g[h][q].y * vv[h][1] + g[h][q].z * vv[h][2] + g[h][q].w * vv[h][3];
      }
      const float sq = gg[0] * gg[0] + gg[1] * gg[1] + gg[2] * gg[2];
      float hq[3];  // the vector that G^T maps to the element's four contributions
      if constexpr (MODE != TS_HVP) {
        if (act[h]) {
          float t, r;
          two_sum(fa, log1pf(sq), t, r);
          fa = t;
          fc += r;
        }
        const float w = 2.f * fb / (1.f + sq);
#pragma unroll
        for (int q = 0; q < 3; ++q) hq[q] = w * gg[q];
      } else {
        const float t1 = 1.f + sq;
        const float w = 2.f * fb / t1;
        const float sd = 2.f * (gg[0] * gd[0] + gg[1] * gd[1] + gg[2] * gd[2]);
        const float wd = -w * sd / t1;
#pragma unroll
        for (int q = 0; q < 3; ++q) hq[q] = wd * gg[q] + w * gd[q];
      }
      if constexpr (MODE != TS_EVAL) {
        float cv[4];
        cv[0] = g[h][0].x * hq[0] + g[h][1].x * hq[1] + g[h][2].x * hq[2];
        cv[1] = g[h][0].y * hq[0] + g[h][1].y * hq[1] + g[h][2].y * hq[2];
        cv[2] = g[h][0].z * hq[0] + g[h][1].z * hq[1] + g[h][2].z * hq[2];
        cv[3] = g[h][0].w * hq[0] + g[h][1].w * hq[1] + g[h][2].w * hq[2];
        const int key[4] = {c[h].x, c[h].y, c[h].z, c[h].w};
        if constexpr (MODE == TS_TAPE) {
          if (act[h])
            reinterpret_cast<float4*>(a.tape)[base + lane + h * stride] =
                make_float4(cv[0], cv[1], cv[2], cv[3]);
        } else {
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            if constexpr (WARPC) {
              warp_combine_groups(act[h], key[k], cv[k], a.gu);
            } else if (act[h]) {
              red_add(a.gu + key[k], cv[k]);
            }
          }
        }
      }
    }
  }
  finish_sum<float>(block_sum((double)fa + (double)fc, red), a.fpart, a.counter, a.f, 0, red);
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
    inc[pos] = (int)i;  // tets: i = 4 e + k = (e << 2) | k
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
  const bool auto_strategy = p->strategy == KG_STRATEGY_AUTO;
  if (auto_strategy) p->strategy = KG_STRATEGY_WARP;  // TILE where it applies, decided below
  if (p->strategy != KG_STRATEGY_ATOMIC && p->strategy != KG_STRATEGY_CSR &&
      p->strategy != KG_STRATEGY_SHARED && p->strategy != KG_STRATEGY_WARP &&
      p->strategy != KG_STRATEGY_TILE)
    return fail(KG_ERR_UNSUPPORTED, "TETENERGY: strategy must be ATOMIC, SHARED, WARP, TILE or CSR");
  const size_t tape_bytes = p->esize * 4 * (size_t)p->m;
  size_t budget = p->opt.tape_budget_bytes ? p->opt.tape_budget_bytes : (size_t(1) << 30);
  p->tet_block = p->opt.block ? p->opt.block : 256;
  if (p->tet_block != 256) return fail(KG_ERR_UNSUPPORTED, "TETENERGY: block must be 256");
  p->tet_grid = tet_staged_grid(p);
  kg_status rc = ws_common(p, p->tet_grid, s);
  if (rc != KG_OK) return rc;
  // FP64 arithmetic: float pairs when G is within the pair range (u is checked per call)
  if (p->dtype == KG_F32) {
    p->arith = KG_ARITH_NATIVE;
  } else if (p->arith != KG_ARITH_NATIVE) {
    bool in_range = false;
    if ((rc = pair_range_ok(p, static_cast<const double*>(p->data1), 12 * p->m, s, &in_range)) != KG_OK)
      return rc;
    if (!in_range && p->arith == KG_ARITH_PAIR)
      return fail(KG_ERR_UNSUPPORTED, "TETENERGY PAIR arithmetic: G has entries outside "
                                      "0 or [2^-60, 2^40) in magnitude");
    p->arith = in_range ? KG_ARITH_PAIR : KG_ARITH_NATIVE;
  }
  // Pair arithmetic: G split into float pairs once (same bytes) when it fits the
  // budget; the kernels then stream that copy and skip 12 splits per element.
  const size_t gprep_bytes = 12 * sizeof(double) * (size_t)p->m;
  if (p->arith == KG_ARITH_PAIR && gprep_bytes <= budget) {
    if ((rc = ws_alloc(p, &p->aprep, gprep_bytes, "prepared G (float pairs)")) != KG_OK) return rc;
    if ((rc = pair_prepare(static_cast<const double*>(p->data1), p->aprep, 12 * p->m, s)) != KG_OK)
      return rc;
    budget -= gprep_bytes;
  }
  // AUTO: the tiled scatter for FP32 data (measured 109 -> 87 us on the 6e6-tet mesh); for
  // float pairs the warp combine stays (199 against 206 us: their arithmetic dominates)
  if (auto_strategy && p->dtype == KG_F32 && tet_tile_supported(p)) p->strategy = KG_STRATEGY_TILE;
  if (p->strategy == KG_STRATEGY_TILE && !tet_tile_supported(p))
    return fail(KG_ERR_UNSUPPORTED, "TETENERGY TILE strategy: needs FP64 data in PAIR arithmetic "
                                    "with the prepared G (within tape_budget_bytes) and check = 0");
  if (p->mode == KG_MODE_AUTO) p->mode = tape_bytes <= budget ? KG_MODE_TAPE : KG_MODE_RECOMPUTE;
  // the CSR strategy goes through the tape where no tile kernel computes the elements
  if (p->mode == KG_MODE_TAPE || (p->strategy == KG_STRATEGY_CSR && !tet_tile_supported(p))) {
    if ((rc = ws_alloc(p, &p->tape, tape_bytes, "tape c_e")) != KG_OK) return rc;
  }
  if ((rc = tet_staged_setup(p)) != KG_OK) return rc;
  const int64_t n4 = 4 * p->m;
  const int* conn = static_cast<const int*>(p->data0);
  tet_validate_kernel<<<grid_for(n4, 256, 8), 256, 0, s>>>(conn, n4, (int)p->n, p->err);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "validate connectivity");
  if (p->strategy == KG_STRATEGY_CSR || p->strategy == KG_STRATEGY_TILE) {
    // the connectivity must be in range before it is used as an index
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_fail(e, "validate connectivity");
    unsigned h = 0;
    if ((e = cudaMemcpy(&h, p->err, sizeof(h), cudaMemcpyDeviceToHost)) != cudaSuccess)
      return cuda_fail(e, "read error word");
    if (h & ERRBIT_BOUNDS) return fail(KG_ERR_BOUNDS, "kg_create: connectivity entry outside [0, N_v)");
  }
  if (p->strategy == KG_STRATEGY_TILE) return tet_tile_setup(p, s);
  if (p->strategy == KG_STRATEGY_CSR) return tet_tile_csr_setup(p, s);
  return KG_OK;
}

void scan_exclusive(int* data, int n, cudaStream_t s) { csr_scan_kernel<<<1, 1024, 0, s>>>(data, n); }

// Buckets of the positions of keys[0..count) by key value (keys in [0, nbins)):
// binptr[k] .. binptr[k+1] delimit, in perm, the positions i with keys[i] == k,
// in ascending order.  Device kernels on s (count, scan, fill, per-bucket
// sort); synchronises s.
kg_status build_buckets(const int* keys, int64_t count, int nbins, int* binptr, int* perm,
                        cudaStream_t s) {
  int* cursor = nullptr;
  cudaError_t e;
  if ((e = dev_alloc((void**)&cursor, sizeof(int) * (size_t)std::max(nbins, 1))) != cudaSuccess)
    return fail(KG_ERR_OOM, "bucket build cursor allocation failed");
  bool ok = cudaMemsetAsync(binptr, 0, sizeof(int) * (size_t)(nbins + 1), s) == cudaSuccess;
  if (ok && count > 0) {
    csr_degree_kernel<<<grid_for(count, 256, 8), 256, 0, s>>>(keys, count, binptr);
    csr_scan_kernel<<<1, 1024, 0, s>>>(binptr, nbins);
    ok = cudaMemcpyAsync(cursor, binptr, sizeof(int) * (size_t)nbins, cudaMemcpyDeviceToDevice, s) ==
         cudaSuccess;
    if (ok) {
      csr_fill_kernel<<<grid_for(count, 256, 8), 256, 0, s>>>(keys, count, cursor, perm);
      csr_sort_kernel<<<grid_for(nbins, 256, 8), 256, 0, s>>>(binptr, nbins, perm);
    }
  }
  e = cudaGetLastError();
  cudaError_t e2 = cudaStreamSynchronize(s);
  cudaFree(cursor);
  if (!ok || e != cudaSuccess || e2 != cudaSuccess)
    return cuda_fail(e != cudaSuccess ? e : e2, "bucket build");
  return KG_OK;
}

// FP32 problems without bounds checks run the direct kernels, except the
// shared-memory-table strategy, which needs the staged tiles.
static bool use_direct(const kg_problem* p) {
  return p->dtype == KG_F32 && !p->opt.check && p->strategy != KG_STRATEGY_SHARED;
}

// One wave: the resident CTAs of this instantiation on every SM (queried once),
// within the f partials sized at kg_create.
template <int MODE, bool WARPC>
static void launch_direct(const kg_problem* p, const DirectArgs& a, cudaStream_t s) {
  static int occ = 0;
  if (occ < 1) {
    int o = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, tet_direct_f32_kernel<MODE, WARPC>, 256, 0) !=
        cudaSuccess)
      o = 1;
    occ = std::max(o, 1);
  }
  const int64_t g = std::min<int64_t>({(p->m + 511) / 512, (int64_t)num_sms() * occ,
                                       (int64_t)p->fpart_len});
  tet_direct_f32_kernel<MODE, WARPC><<<(int)std::max<int64_t>(g, 1), 256, 0, s>>>(a);
}

static kg_status tet_direct(kg_problem* p, int mode, const void* x, const void* v, void* f,
                            void* gx, const void* seed, cudaStream_t s) {
  DirectArgs a{};
  a.conn = static_cast<const int4*>(p->data0);
  a.G = static_cast<const float4*>(p->data1);
  a.u = static_cast<const float*>(x);
  a.v = static_cast<const float*>(v);
  a.ne = p->m;
  a.seed = static_cast<const float*>(seed);
  a.gu = static_cast<float*>(gx);
  a.tape = static_cast<float*>(p->tape);
  a.fpart = p->fpart;
  a.counter = p->counter;
  a.f = static_cast<float*>(f);
  const bool warp = p->strategy == KG_STRATEGY_WARP;
  static const char* names[4] = {"tet_direct_f32_kernel<eval>", "tet_direct_f32_kernel<grad>",
                                 "tet_direct_f32_kernel<tape>", "tet_direct_f32_kernel<hvp>"};
  prof_begin(s, names[mode]);
  switch (mode) {
    case TS_EVAL: launch_direct<TS_EVAL, false>(p, a, s); break;
    case TS_TAPE: launch_direct<TS_TAPE, false>(p, a, s); break;
    case TS_GRAD:
      if (warp) launch_direct<TS_GRAD, true>(p, a, s);
      else launch_direct<TS_GRAD, false>(p, a, s);
      break;
    default:
      if (warp) launch_direct<TS_HVP, true>(p, a, s);
      else launch_direct<TS_HVP, false>(p, a, s);
      break;
  }
  prof_end(s);
  count_launch();
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? KG_OK : cuda_fail(e, names[mode]);
}

kg_status tet_eval(kg_problem* p, const void* x, void* f, bool tape, cudaStream_t s) {
  kg_status rc = use_direct(p) ? tet_direct(p, tape ? TS_TAPE : TS_EVAL, x, nullptr, f, nullptr, nullptr, s)
                               : tet_staged(p, tape ? 2 : 0, x, f, nullptr, nullptr, s);
  if (rc == KG_OK && tape) {
    p->tape_valid = true;
    p->tape_gen += 1;
  }
  return rc;
}

template <typename T>
static kg_status tet_scatter_t(kg_problem* p, void* gx, const void* seed, int accumulate,
                               cudaStream_t s) {
  cudaError_t e;
  if (p->strategy == KG_STRATEGY_CSR || p->strategy == KG_STRATEGY_TILE) {
    return tet_tile_from_tape(p, gx, seed, accumulate, s);
  } else {
    if (!accumulate) {
      if ((e = cudaMemsetAsync(gx, 0, sizeof(T) * (size_t)p->n, s)) != cudaSuccess)
        return cuda_fail(e, "zero gu");
      count_launch();
    }
    prof_begin(s, "tet_tape_scatter_kernel");
    // FP64 tape values would be combined with FP64 adds, which cost more here than the
    // atomics they save (measured): the warp combine is used for FP32 tapes only
    auto kern = p->strategy == KG_STRATEGY_WARP && sizeof(T) == 4 ? tet_tape_scatter_kernel<T, true>
                                                                  : tet_tape_scatter_kernel<T, false>;
    kern<<<p->tet_grid, 256, 0, s>>>(static_cast<const int4*>(p->data0),
                                     static_cast<const T*>(p->tape), p->m,
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
    // reproducible: tile partials in fixed order, then the vertex gather in fixed order;
    // through the tape where no tile kernel computes the elements
    kg_status rc;
    if (!tet_tile_supported(p)) {
      if ((rc = tet_eval(p, x, f, true, s)) != KG_OK) return rc;
      return tet_tile_from_tape(p, gx, seed, accumulate, s);
    }
    if (sizeof(T) == 4) {
      rc = tet_tile_run_f32(p, TS_GRAD, x, nullptr, f, gx, seed, s);
    } else {
      const float2 *us = nullptr, *vs = nullptr;
      if ((rc = tet_split_vertex_values(p, x, nullptr, gx, false, &us, &vs, s)) != KG_OK) return rc;
      rc = tet_tile_run(p, TS_GRAD, us, nullptr, f, gx, seed, s);
    }
    return rc == KG_OK ? tet_tile_gather(p, gx, accumulate, s) : rc;
  }
  // pair arithmetic: the kernel that splits u also zeroes gu (one launch for both)
  const bool fold_zero = p->arith == KG_ARITH_PAIR && sizeof(T) == 8;
  if (p->strategy == KG_STRATEGY_TILE) {
    if (sizeof(T) == 4) {
      if (!accumulate) {
        cudaError_t e = cudaMemsetAsync(gx, 0, sizeof(T) * (size_t)p->n, s);
        if (e != cudaSuccess) return cuda_fail(e, "zero gu");
        count_launch();
      }
      return tet_tile_run_f32(p, TS_GRAD, x, nullptr, f, gx, seed, s);
    }
    const float2 *us = nullptr, *vs = nullptr;
    kg_status rc = tet_split_vertex_values(p, x, nullptr, gx, !accumulate, &us, &vs, s);
    if (rc != KG_OK) return rc;
    return tet_tile_run(p, TS_GRAD, us, nullptr, f, gx, seed, s);
  }
  cudaError_t e;
  if (!accumulate && !fold_zero) {
    if ((e = cudaMemsetAsync(gx, 0, sizeof(T) * (size_t)p->n, s)) != cudaSuccess)
      return cuda_fail(e, "zero gu");
    count_launch();
  }
  if (use_direct(p)) return tet_direct(p, TS_GRAD, x, nullptr, f, gx, seed, s);
  return tet_staged(p, 1, x, f, gx, seed, s, nullptr, fold_zero && !accumulate);
}

kg_status tet_grad(kg_problem* p, const void* x, void* f, void* gx, const void* seed,
                   int accumulate, cudaStream_t s) {
  return p->dtype == KG_F64 ? tet_grad_t<double>(p, x, f, gx, seed, accumulate, s)
                            : tet_grad_t<float>(p, x, f, gx, seed, accumulate, s);
}

kg_status tet_hvp(kg_problem* p, const void* x, const void* v, void* hv, const void* seed,
                  int accumulate, cudaStream_t s) {
  const bool fold_zero = p->arith == KG_ARITH_PAIR && p->dtype == KG_F64;
  if (p->strategy == KG_STRATEGY_CSR && tet_tile_supported(p)) {  // reproducible, as the gradient
    kg_status rc;
    if (p->dtype == KG_F32) {
      rc = tet_tile_run_f32(p, TS_HVP, x, v, nullptr, hv, seed, s);
    } else {
      const float2 *us = nullptr, *vs = nullptr;
      if ((rc = tet_split_vertex_values(p, x, v, hv, false, &us, &vs, s)) != KG_OK) return rc;
      rc = tet_tile_run(p, TS_HVP, us, vs, nullptr, hv, seed, s);
    }
    return rc == KG_OK ? tet_tile_gather(p, hv, accumulate, s) : rc;
  }
  if (p->strategy == KG_STRATEGY_TILE) {
    if (p->dtype == KG_F32) {
      if (!accumulate) {
        cudaError_t e = cudaMemsetAsync(hv, 0, p->esize * (size_t)p->n, s);
        if (e != cudaSuccess) return cuda_fail(e, "zero hv");
        count_launch();
      }
      return tet_tile_run_f32(p, TS_HVP, x, v, nullptr, hv, seed, s);
    }
    const float2 *us = nullptr, *vs = nullptr;
    kg_status rc = tet_split_vertex_values(p, x, v, hv, !accumulate, &us, &vs, s);
    if (rc != KG_OK) return rc;
    return tet_tile_run(p, TS_HVP, us, vs, nullptr, hv, seed, s);
  }
  if (!accumulate && !fold_zero) {
    cudaError_t e = cudaMemsetAsync(hv, 0, p->esize * (size_t)p->n, s);
    if (e != cudaSuccess) return cuda_fail(e, "zero hv");
    count_launch();
  }
  if (use_direct(p)) return tet_direct(p, TS_HVP, x, v, nullptr, hv, seed, s);
  return tet_staged(p, 3, x, nullptr, hv, seed, s, v, fold_zero && !accumulate);
}

kg_status tet_grad_from_tape(kg_problem* p, void* gx, const void* seed, int accumulate,
                             cudaStream_t s) {
  return p->dtype == KG_F64 ? tet_scatter_t<double>(p, gx, seed, accumulate, s)
                            : tet_scatter_t<float>(p, gx, seed, accumulate, s);
}

}  // namespace kg
