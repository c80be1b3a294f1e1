// Dense ||A x||^2 value-and-gradient for FP32 data, streamed through shared
// memory with TMA.
//
// Same schedule as the float-pair FP64 kernel (quadform_pair.cu): one pass
// over A, rows in a two-stage shared-memory ring filled by cp.async.bulk with
// mbarrier transaction counts, warps release a stage through an "empty"
// mbarrier and thread 0 refills it with the row two ahead.  Thread t owns the
// column quads jq = t + 512 k (4 columns, one 16-byte shared load); the row
// dot y_i uses four independent FMA chains, ybar_i = 2 fbar y_i is broadcast
// and xbar_j += ybar_i A_ij accumulates in registers.  Two CTAs per SM.  The
// CTA partials are summed in a fixed order in the kernel's tail, after a grid
// barrier (a cooperative launch), or by a second small kernel when the grid
// cannot be resident at once; both give the same bits.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdlib>

#include "kg_device.cuh"
#include "kg_internal.h"
#include "kg_pair.cuh"

namespace kg {

constexpr int QF_CW = 16;
constexpr int QF_CT = QF_CW * 32;
constexpr int QF_BAR = 1;

struct Qf32Args {
  const float* A;
  const float* x;
  int64_t m;
  int n;  // multiple of 4
  int band;
  const float* seed;
  float4* partials;  // [grid][n/4]
  double* fpart;
  unsigned* counter;
  float* f;  // EVAL: last CTA; fused reduction: CTA 0
  unsigned* err;
  float* gx;       // fused reduction (GRIDRED): the gradient
  int accumulate;  // fused reduction: 1 adds to gx
};

// Fixed-order sum of the CTA partials over quads [j0, j1) by a CTA of 512
// threads: thread (cx, py) adds partials py, py + 32, ... of quad cx of each
// block of 16 (twelve loads in flight: one round for up to 384 partials), then
// the 32 sums are added in py order (and gx's old value last when
// accumulating).  The order depends on neither the CTA nor the range: the fused
// tail and the reduce kernel give the same bits.  A block of 16 holds a column
// CTA's share of the quads in the tail (n / 4 over 303 CTAs) for n <= 19392.
constexpr int F32R_CX = 16, F32R_PY = 32, F32R_LOADS = 12;

__device__ __forceinline__ void reduce_quads(const float4* partials, int nparts, int nq, int j0, int j1,
                                             float* gx, int accumulate, float4 (*red)[F32R_CX]) {
  const int cx = threadIdx.x % F32R_CX, py = threadIdx.x / F32R_CX;
  for (int jb = j0; jb < j1; jb += F32R_CX) {
    const int jq = jb + cx;
    float4 s = make_float4(0.f, 0.f, 0.f, 0.f);
    if (jq < j1) {
      for (int c = py; c < nparts; c += F32R_LOADS * F32R_PY) {
        float4 v[F32R_LOADS];
#pragma unroll
        for (int u = 0; u < F32R_LOADS; ++u)
          if (c + F32R_PY * u < nparts) v[u] = __ldcg(partials + (int64_t)(c + F32R_PY * u) * nq + jq);
#pragma unroll
        for (int u = 0; u < F32R_LOADS; ++u)
          if (c + F32R_PY * u < nparts) {
            s.x += v[u].x;
            s.y += v[u].y;
            s.z += v[u].z;
            s.w += v[u].w;
          }
      }
    }
    red[py][cx] = s;
    __syncthreads();
    if (py == 0 && jq < j1) {
      float4 t = red[0][cx];
#pragma unroll
      for (int i = 1; i < F32R_PY; ++i) {
        t.x += red[i][cx].x;
        t.y += red[i][cx].y;
        t.z += red[i][cx].z;
        t.w += red[i][cx].w;
      }
      float4* o = reinterpret_cast<float4*>(gx) + jq;
      if (accumulate) {
        const float4 v = *o;
        t.x += v.x;
        t.y += v.y;
        t.z += v.z;
        t.w += v.w;
      }
      *o = t;
    }
    __syncthreads();
  }
}

__device__ __forceinline__ void reduce_f32_fparts(const double* fpart, int nparts, float* f, double* scratch) {
  double fs = 0.0;
  for (int i = threadIdx.x; i < nparts; i += blockDim.x) fs += __ldcg(fpart + i);
  fs = block_sum(fs, scratch);
  if (threadIdx.x == 0) *f = (float)fs;
}

// The reduction as the fused kernel's tail: a grid barrier, then with more than
// one CTA, CTA 0 sums the f partials while CTAs 1 .. grid - 1 sum their shares
// of the quads; the last CTA out resets the barrier's counters.
__device__ __forceinline__ void f32_grid_reduce(const Qf32Args& a, int nq) {
  static_assert(QF_CT == F32R_CX * F32R_PY, "reduce_quads takes 512 threads");
  __shared__ float4 red[F32R_PY][F32R_CX];
  __shared__ double fred[32];
  __shared__ int go;
  if (threadIdx.x == 0) go = grid_arrive_and_wait(a.counter + 2, a.err, ERRBIT_TIMEOUT);
  __syncthreads();
  if (go) {
    const int nparts = gridDim.x;
    const int cols = nparts > 1 ? nparts - 1 : 1, b = nparts > 1 ? (int)blockIdx.x - 1 : 0;
    if (b >= 0) {
      const int j0 = (int)((int64_t)b * nq / cols), j1 = (int)((int64_t)(b + 1) * nq / cols);
      reduce_quads(a.partials, nparts, nq, j0, j1, a.gx, a.accumulate, red);
    }
    if (blockIdx.x == 0 && a.f) reduce_f32_fparts(a.fpart, nparts, a.f, fred);
  }
  if (threadIdx.x == 0) grid_depart(a.counter + 2, a.counter + 3);
}

template <int QPT, bool FUSED, bool GRIDRED>
__global__ void __launch_bounds__(QF_CT, 2) qf_f32_kernel(Qf32Args a) {
  extern __shared__ __align__(128) unsigned char smem[];
  const int n = a.n, nq = n >> 2;
  float* stage0 = reinterpret_cast<float*>(smem);
  float* stage1 = stage0 + n;
  uint64_t* full = reinterpret_cast<uint64_t*>(stage1 + n);
  uint64_t* empty = full + 2;
  float* red = reinterpret_cast<float*>(empty + 2);  // [2][QF_CW]
  volatile int* abort_flag = reinterpret_cast<volatile int*>(red + 2 * QF_CW);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, t = threadIdx.x;
  const int64_t r0 = (int64_t)blockIdx.x * a.band;
  const int64_t r1 = r0 + a.band < a.m ? r0 + a.band : a.m;
  const int nrows = r1 > r0 ? (int)(r1 - r0) : 0;
  const uint32_t row_bytes = (uint32_t)n * 4u;

  if (t == 0) {
    mbar_init(&full[0], 1);
    mbar_init(&full[1], 1);
    mbar_init(&empty[0], QF_CW);
    mbar_init(&empty[1], QF_CW);
    *abort_flag = 0;
    fence_barrier_init();
  }
  __syncthreads();
  int issued = 0;
  if (t == 0) {
    for (int it = 0; it < 2 && it < nrows; ++it) {
      const float* src = a.A + (r0 + it) * (int64_t)n;
      mbar_arrive_expect_tx(&full[it], row_bytes);
      tma_load_1d(it ? stage1 : stage0, src, row_bytes, &full[it]);
      ++issued;
      if (it + 2 < nrows) prefetch_l2_bulk(src + 2 * (int64_t)n, row_bytes);
    }
  }

  float4 xv[QPT];
#pragma unroll
  for (int k = 0; k < QPT; ++k) {
    const int jq = t + QF_CT * k;
    xv[k] = jq < nq ? reinterpret_cast<const float4*>(a.x)[jq] : make_float4(0.f, 0.f, 0.f, 0.f);
  }
  const float fb2 = 2.0f * (a.seed ? *a.seed : 1.0f);
  float4 xb[QPT];
#pragma unroll
  for (int k = 0; k < QPT; ++k) xb[k] = make_float4(0.f, 0.f, 0.f, 0.f);
  FSum<float> fsum;

  for (int it = 0; it < nrows; ++it) {
    const int s = it & 1;
    const bool ok = mbar_wait_bounded(&full[s], (it >> 1) & 1);
    const float4* row = reinterpret_cast<const float4*>(s ? stage1 : stage0);
    float d0 = 0.f, d1 = 0.f, d2 = 0.f, d3 = 0.f;
    if (ok) {
#pragma unroll
      for (int k = 0; k < QPT; ++k) {
        const int jq = t + QF_CT * k;
        if (jq < nq) {
          const float4 v = row[jq];
          d0 = fmaf(v.x, xv[k].x, d0);
          d1 = fmaf(v.y, xv[k].y, d1);
          d2 = fmaf(v.z, xv[k].z, d2);
          d3 = fmaf(v.w, xv[k].w, d3);
        }
      }
    }
    float yv = warp_sum((d0 + d1) + (d2 + d3));
    if (lane == 0) red[(it & 1) * QF_CW + warp] = yv;
    if (named_barrier_or(QF_BAR, QF_CT, !ok)) {
      if (t == 0) set_error(a.err, ERRBIT_TIMEOUT);
      *abort_flag = 1;
      break;
    }
    float y = 0.f;
#pragma unroll
    for (int q = 0; q < QF_CW; ++q) y += red[(it & 1) * QF_CW + q];
    if (t == 0) fsum.add(y);
    if (FUSED) {
      const float yb = fb2 * y;
#pragma unroll
      for (int k = 0; k < QPT; ++k) {
        const int jq = t + QF_CT * k;
        if (jq < nq) {
          const float4 v = row[jq];
          xb[k].x = fmaf(yb, v.x, xb[k].x);
          xb[k].y = fmaf(yb, v.y, xb[k].y);
          xb[k].z = fmaf(yb, v.z, xb[k].z);
          xb[k].w = fmaf(yb, v.w, xb[k].w);
        }
      }
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty[s]);
    if (t == 0 && it + 2 < nrows && !*abort_flag) {
      if (!mbar_wait_bounded(&empty[s], (it >> 1) & 1)) {
        set_error(a.err, ERRBIT_TIMEOUT);
        *abort_flag = 1;
      } else {
        const float* src = a.A + (r0 + it + 2) * (int64_t)n;
        mbar_arrive_expect_tx(&full[s], row_bytes);
        tma_load_1d(s ? stage1 : stage0, src, row_bytes, &full[s]);
        ++issued;
        if (it + 4 < nrows) prefetch_l2_bulk(src + 2 * (int64_t)n, row_bytes);
      }
    }
    __syncwarp();
  }
  if (t == 0) {  // no copy into this CTA's shared memory may still be in flight
    for (int st = 0; st < 2; ++st) {
      const int last = issued - 1 - ((issued - 1 - st) & 1);
      if (last >= 0) mbar_wait_bounded(&full[st], (last >> 1) & 1);
    }
  }
  if (FUSED) {
    float4* out = a.partials + (int64_t)blockIdx.x * nq;
#pragma unroll
    for (int k = 0; k < QPT; ++k) {
      const int jq = t + QF_CT * k;
      if (jq < nq) out[jq] = xb[k];
    }
    if (t == 0) a.fpart[blockIdx.x] = fsum.get();
    if constexpr (GRIDRED) {
      __syncthreads();
      f32_grid_reduce(a, nq);
    }
  } else if (t == 0) {
    a.fpart[blockIdx.x] = fsum.get();
    __threadfence();
    if (atomicAdd(a.counter, 1u) == gridDim.x - 1) {
      __threadfence();
      double tot = 0.0;
      for (int i = 0; i < (int)gridDim.x; ++i) tot += __ldcg(&a.fpart[i]);
      *a.f = (float)tot;
      *a.counter = 0u;
    }
  }
}

// The same reduction as a separate kernel: block b sums quads [16 b, 16 b + 16);
// block 0 also writes f.  Launched as a programmatic dependent of the fused kernel.
__global__ void __launch_bounds__(512) qf_f32_reduce_kernel(const float4* __restrict__ partials,
                                                            int nparts, int nq,
                                                            const double* __restrict__ fpart,
                                                            float* gx, float* f, int accumulate) {
  __shared__ float4 red[F32R_PY][F32R_CX];
  __shared__ double fred[32];
  grid_dependency_wait();  // the fused kernel has completed and its partials are visible
  const int j0 = blockIdx.x * F32R_CX;
  reduce_quads(partials, nparts, nq, j0, min(j0 + F32R_CX, nq), gx, accumulate, red);
  if (blockIdx.x == 0 && f) reduce_f32_fparts(fpart, nparts, f, fred);
}

// ---------------------------------------------------------------- host ----
static int f32_qpt(int64_t n) {
  const int64_t need = (n / 4 + QF_CT - 1) / QF_CT;
  for (int q : {1, 2, 3, 4, 5, 6})
    if (need <= q) return q;
  return -1;
}

bool qf_f32_supported(const kg_problem* p) {
  return p->dtype == KG_F32 && (p->n % 4) == 0 && p->n >= 1024 && f32_qpt(p->n) > 0 &&
         (p->strategy == KG_STRATEGY_FUSED || p->strategy == KG_STRATEGY_AUTO) && p->opt.team == 0;
}

int qf_f32_grid(const kg_problem* p, int* band) {
  const int64_t g = std::min<int64_t>(p->m, 2 * (int64_t)num_sms());
  const int64_t b = (p->m + g - 1) / g;
  *band = (int)b;
  return (int)((p->m + b - 1) / b);
}

static size_t f32_smem(int n) { return (size_t)2 * n * 4 + 4 * 8 + 2 * QF_CW * 4 + 16; }

// GRIDRED: the fused kernel with the reduction in its tail, as a cooperative
// launch (refused when the grid cannot be resident at once).
template <int QPT, bool FUSED, bool GRIDRED>
static cudaError_t launch_f32(int grid, size_t smem, cudaStream_t s, const Qf32Args& a) {
  auto kern = qf_f32_kernel<QPT, FUSED, GRIDRED>;
  cudaError_t e = set_smem_once(kern, smem);
  if (e != cudaSuccess) return e;
  if constexpr (GRIDRED) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(QF_CT);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, a);
  }
  kern<<<grid, QF_CT, smem, s>>>(a);
  return cudaGetLastError();
}

template <bool FUSED, bool GRIDRED = false>
static cudaError_t dispatch_f32(int qpt, int grid, size_t smem, cudaStream_t s, const Qf32Args& a) {
  switch (qpt) {
    case 1: return launch_f32<1, FUSED, GRIDRED>(grid, smem, s, a);
    case 2: return launch_f32<2, FUSED, GRIDRED>(grid, smem, s, a);
    case 3: return launch_f32<3, FUSED, GRIDRED>(grid, smem, s, a);
    case 4: return launch_f32<4, FUSED, GRIDRED>(grid, smem, s, a);
    case 5: return launch_f32<5, FUSED, GRIDRED>(grid, smem, s, a);
    case 6: return launch_f32<6, FUSED, GRIDRED>(grid, smem, s, a);
  }
  return cudaErrorInvalidValue;
}

template <int QPT>
static bool f32_coop_fits_q(int grid, size_t smem) {
  int dev = 0, coop = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess || !coop)
    return false;
  auto kern = qf_f32_kernel<QPT, true, true>;
  if (set_smem_once(kern, smem) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, QF_CT, smem) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return (int64_t)per_sm * num_sms() >= grid;
}

bool qf_f32_coop_fits(const kg_problem* p) {
  if (const char* env = std::getenv("KG_TEST_NO_COOP"))
    if (std::atoi(env) == 1) return false;
  const size_t smem = f32_smem((int)p->n);
  switch (f32_qpt(p->n)) {
    case 1: return f32_coop_fits_q<1>(p->qf.grid, smem);
    case 2: return f32_coop_fits_q<2>(p->qf.grid, smem);
    case 3: return f32_coop_fits_q<3>(p->qf.grid, smem);
    case 4: return f32_coop_fits_q<4>(p->qf.grid, smem);
    case 5: return f32_coop_fits_q<5>(p->qf.grid, smem);
    case 6: return f32_coop_fits_q<6>(p->qf.grid, smem);
  }
  return false;
}

static Qf32Args f32_args(kg_problem* p, const void* x, const void* seed) {
  Qf32Args a{};
  a.A = static_cast<const float*>(p->data0);
  a.x = static_cast<const float*>(x);
  a.m = p->m;
  a.n = (int)p->n;
  a.band = p->qf.rows_per_cta;
  a.seed = static_cast<const float*>(seed);
  a.partials = static_cast<float4*>(p->partials);
  a.fpart = p->fpart;
  a.counter = p->counter;
  a.err = p->err;
  return a;
}

kg_status qf_f32_eval(kg_problem* p, const void* x, void* f, cudaStream_t s) {
  if ((reinterpret_cast<uintptr_t>(x) & 15u) != 0)
    return fail(KG_ERR_INVALID_ARG, "QUADFORM FP32 streamed kernels need a 16-byte aligned x");
  Qf32Args a = f32_args(p, x, nullptr);
  a.f = static_cast<float*>(f);
  prof_begin(s, "qf_f32_kernel<eval>");
  cudaError_t e = dispatch_f32<false>(f32_qpt(p->n), p->qf.grid, f32_smem((int)p->n), s, a);
  prof_end(s);
  count_launch();
  return e == cudaSuccess ? KG_OK : cuda_fail(e, "qf f32 forward kernel");
}

kg_status qf_f32_grad(kg_problem* p, const void* x, void* f, void* gx, const void* seed,
                      int accumulate, cudaStream_t s) {
  if ((reinterpret_cast<uintptr_t>(x) & 15u) != 0 || (reinterpret_cast<uintptr_t>(gx) & 15u) != 0)
    return fail(KG_ERR_INVALID_ARG, "QUADFORM FP32 streamed kernels need 16-byte aligned x and gx");
  Qf32Args a = f32_args(p, x, seed);
  cudaError_t e;
  if (p->qf.coop) {
    // one launch: the partials' reduction in the kernel's tail
    a.gx = static_cast<float*>(gx);
    a.f = static_cast<float*>(f);
    a.accumulate = accumulate;
    prof_begin(s, "qf_f32_kernel<fused, grid reduction>");
    e = dispatch_f32<true, true>(f32_qpt(p->n), p->qf.grid, f32_smem((int)p->n), s, a);
    prof_end(s);
    count_launch();
    if (e == cudaSuccess) return KG_OK;
    if (e != cudaErrorCooperativeLaunchTooLarge) return cuda_fail(e, "qf f32 fused kernel");
    cudaGetLastError();  // the grid is not resident at once here: two launches from now on
    p->qf.coop = 0;
    a.gx = nullptr;
    a.f = nullptr;
  }
  prof_begin(s, "qf_f32_kernel<fused>");
  e = dispatch_f32<true>(f32_qpt(p->n), p->qf.grid, f32_smem((int)p->n), s, a);
  prof_end(s);
  count_launch();
  if (e != cudaSuccess) return cuda_fail(e, "qf f32 fused kernel");
  const int nq = (int)(p->n / 4);
  // programmatic dependent launch: it waits for the fused kernel's completion
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((nq + F32R_CX - 1) / F32R_CX);
  cfg.blockDim = dim3(512);
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  e = cudaLaunchKernelEx(&cfg, qf_f32_reduce_kernel, static_cast<const float4*>(p->partials),
                         p->qf.grid, nq, static_cast<const double*>(p->fpart), static_cast<float*>(gx),
                         static_cast<float*>(f), accumulate);
  count_launch();
  if (e != cudaSuccess) return cuda_fail(e, "qf f32 reduce kernel");
  return KG_OK;
}

}  // namespace kg
