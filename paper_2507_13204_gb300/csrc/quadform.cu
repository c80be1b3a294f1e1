// Dense quadratic form f(x; A) = ||A x||^2 (A m x n, row-major) and its
// reverse-mode gradient.
//
// Forward (the primal): a team of threads per row computes y_i = A_i,: . x
// (a team-nested parallel_reduce), then f = sum_i y_i^2 (a parallel_sum
// reduction).  Reverse: the reduction's adjoint is broadcast,
// ybar_i = 2 fbar y_i (Sec. 3.2), and every read A_ij x_j of the row loop
// becomes xbar_j += A_ij ybar_i and Abar_ij += x_j ybar_i (Sec. 3.1 rule).
// Because x_j is read by every row, the paper's race detection makes the
// xbar update atomic when the reverse reuses the forward schedule (Sec. 3.3);
// that is KG_STRATEGY_ATOMIC here.  KG_STRATEGY_TRANSPOSE reschedules the
// reverse by columns and KG_STRATEGY_FUSED keeps one pass over A with
// per-CTA private partials (the paper's Sec. 5 proposals: rescheduling,
// on-chip temporaries, kernel fusion).
#include <cuda_runtime.h>

#include <algorithm>
#include <string>

#include "kg_device.cuh"
#include "kg_internal.h"

namespace kg {

template <typename T>
struct QfArgs {
  const T* A;
  const T* x;
  int64_t m;
  int n;
  int cpt;           // columns per team thread actually used (<= CPT_MAX)
  int rows_per_cta;  // contiguous band of rows per CTA
  const T* seed;     // nullable device scalar (fbar)
  T* partials;       // FUSED: [gridDim.x][n] private xbar partials
  double* fpart;     // per-CTA f partials
  unsigned* counter; // arrival counter for the last-CTA reduction
  T* y;              // nullable: forward row values
  T* f;              // EVAL: output
  T* gA;             // FUSED, nullable: gradient w.r.t. A
  int accumulate;
};

enum { QF_EVAL = 0, QF_FUSED = 1 };

// Sum over a team of TEAM threads; every thread of the CTA calls it in the same
// iteration.  red: shared [2][nteams][TEAM/32], double-buffered by `par`.
template <typename T, int TEAM>
__device__ __forceinline__ T team_sum(T v, T* red, int par) {
  v = warp_sum(v);
  if constexpr (TEAM == 32) {
    return v;
  } else {
    constexpr int W = TEAM / 32;
    const int team = threadIdx.x / TEAM, w = (threadIdx.x % TEAM) >> 5;
    const int nteams = blockDim.x / TEAM;
    T* r = red + (par * nteams + team) * W;
    if ((threadIdx.x & 31) == 0) r[w] = v;
    __syncthreads();
    // lane l takes warp l mod W's sum, and a butterfly over W lanes gives every lane the
    // same total: log2(W) adds a thread instead of W (FP64 adds are scarce on GB300)
    T s = r[(threadIdx.x & 31) % W];
#pragma unroll
    for (int o = W / 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    return s;
  }
}

// Team-per-row kernel.  Team thread lt owns columns j = lt + k*TEAM, k < cpt.
// EVAL: y_i and f.  FUSED: additionally ybar_i = 2 fbar y_i and the private
// partial xbar_j += ybar_i A_ij (and Abar_ij when gA is given), with the
// row's A values still in registers: A is read once.
template <typename T, int TEAM, int CPT_MAX, int MODE>
__global__ void __launch_bounds__(512) qf_team_kernel(QfArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int n = a.n;
  const int nteams = blockDim.x / TEAM;
  const int team = threadIdx.x / TEAM, lt = threadIdx.x % TEAM;
  T* xs = reinterpret_cast<T*>(smem_raw);                  // CPT_MAX*TEAM (x, later xbar)
  T* red = xs + CPT_MAX * TEAM;                            // 2*nteams*(TEAM/32)
  double* fs = reinterpret_cast<double*>(red + 2 * nteams * (TEAM / 32) + 2);  // nteams + 32
  fs = reinterpret_cast<double*>((reinterpret_cast<uintptr_t>(fs) + 7) & ~uintptr_t(7));

  for (int j = threadIdx.x; j < CPT_MAX * TEAM; j += blockDim.x) xs[j] = j < n ? a.x[j] : T(0);
  __syncthreads();

  const T fb = MODE == QF_FUSED ? load_seed(a.seed) : T(1);
  T xb[CPT_MAX];
#pragma unroll
  for (int k = 0; k < CPT_MAX; ++k) xb[k] = T(0);
  FSum<T> fsum;

  const int64_t r0 = (int64_t)blockIdx.x * a.rows_per_cta;
  const int64_t r1 = r0 + a.rows_per_cta < a.m ? r0 + a.rows_per_cta : a.m;
  const int iters = r1 > r0 ? (int)((r1 - r0 + nteams - 1) / nteams) : 0;
  for (int it = 0; it < iters; ++it) {
    const int64_t row = r0 + (int64_t)it * nteams + team;
    const bool valid = row < r1;
    const T* Ar = a.A + (valid ? row : r0) * (int64_t)n;
    T av[CPT_MAX];
#pragma unroll
    for (int k = 0; k < CPT_MAX; ++k) {
      const int j = lt + k * TEAM;
      av[k] = (k < a.cpt && valid && j < n) ? ld_stream(Ar + j) : T(0);
    }
    T d = T(0);
#pragma unroll
    for (int k = 0; k < CPT_MAX; ++k)
      if (k < a.cpt) d = fma(av[k], xs[lt + k * TEAM], d);
    const T yv = team_sum<T, TEAM>(d, red, it & 1);
    if (valid) {
      if (lt == 0) {
        fsum.add(yv);
        if (a.y) a.y[row] = yv;
      }
      if constexpr (MODE == QF_FUSED) {
        const T yb = T(2) * fb * yv;
#pragma unroll
        for (int k = 0; k < CPT_MAX; ++k)
          if (k < a.cpt) xb[k] = fma(yb, av[k], xb[k]);
        if (a.gA) {
          T* gr = a.gA + row * (int64_t)n;
#pragma unroll
          for (int k = 0; k < CPT_MAX; ++k) {
            const int j = lt + k * TEAM;
            if (k < a.cpt && j < n) {
              const T v = yb * xs[j];
              gr[j] = a.accumulate ? gr[j] + v : v;
            }
          }
        }
      }
    }
  }

  // CTA's f partial: team leaders in team order.
  __syncthreads();
  if (lt == 0) fs[team] = fsum.get();
  __syncthreads();
  double fcta = 0.0;
  for (int t = 0; t < nteams; ++t) fcta += fs[t];

  if constexpr (MODE == QF_EVAL) {
    finish_sum<T>(fcta, a.fpart, a.counter, a.f, 0, fs + nteams);
  } else {
    if (threadIdx.x == 0) a.fpart[blockIdx.x] = fcta;
    // combine the teams' private xbar in team order, then store this CTA's partial
    T* out = a.partials + (int64_t)blockIdx.x * n;
    if (nteams == 1) {
#pragma unroll
      for (int k = 0; k < CPT_MAX; ++k) {
        const int j = lt + k * TEAM;
        if (k < a.cpt && j < n) out[j] = xb[k];
      }
    } else {
      for (int t = 0; t < nteams; ++t) {
        if (team == t) {
#pragma unroll
          for (int k = 0; k < CPT_MAX; ++k) {
            const int j = lt + k * TEAM;
            if (k < a.cpt) xs[j] = t == 0 ? xb[k] : xs[j] + xb[k];
          }
        }
        __syncthreads();
      }
      for (int j = threadIdx.x; j < n; j += blockDim.x) out[j] = xs[j];
    }
  }
}

// Reverse with the forward schedule (the paper's atomic scatter): each team
// re-reads its row and adds ybar_i A_ij into gx[j] (a global red); ybar_i comes from
// the y the forward kernel stored.
template <typename T, int TEAM, int CPT_MAX>
__global__ void __launch_bounds__(512) qf_atomic_adjoint_kernel(QfArgs<T> a, T* gx) {
  const int n = a.n;
  const int nteams = blockDim.x / TEAM;
  const int team = threadIdx.x / TEAM, lt = threadIdx.x % TEAM;
  const T fb = load_seed(a.seed);
  const int64_t r0 = (int64_t)blockIdx.x * a.rows_per_cta;
  const int64_t r1 = r0 + a.rows_per_cta < a.m ? r0 + a.rows_per_cta : a.m;
  for (int64_t row = r0 + team; row < r1; row += nteams) {
    const T yb = T(2) * fb * a.y[row];
    const T* Ar = a.A + row * (int64_t)n;
#pragma unroll
    for (int k = 0; k < CPT_MAX; ++k) {
      const int j = lt + k * TEAM;
      if (k < a.cpt && j < n) red_add(gx + j, yb * ld_stream(Ar + j));
    }
  }
}

// Reverse rescheduled by columns: thread per column j, rows split into chunks
// (blockIdx.y); partial[chunk][j] = sum_{i in chunk} A_ij ybar_i.  Reads A a
// second time, coalesced across j.
template <typename T>
__global__ void __launch_bounds__(256) qf_transpose_kernel(const T* __restrict__ A,
                                                           const T* __restrict__ y, int64_t m,
                                                           int n, int rows_per_chunk,
                                                           const T* seed, T* partials) {
  __shared__ T yb_s[256];
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t r0 = (int64_t)blockIdx.y * rows_per_chunk;
  const int64_t r1 = r0 + rows_per_chunk < m ? r0 + rows_per_chunk : m;
  const T fb = load_seed(seed);
  T s = T(0);
  for (int64_t rb = r0; rb < r1; rb += 256) {
    const int cnt = (int)((r1 - rb) < 256 ? (r1 - rb) : 256);
    __syncthreads();
    if (threadIdx.x < cnt) yb_s[threadIdx.x] = T(2) * fb * y[rb + threadIdx.x];
    __syncthreads();
    if (j < n) {
      const T* Ac = A + rb * (int64_t)n + j;
#pragma unroll 8
      for (int i = 0; i < cnt; ++i) s = fma(ld_stream(Ac + (int64_t)i * n), yb_s[i], s);
    }
  }
  if (j < n) partials[(int64_t)blockIdx.y * n + j] = s;
}

// Sum of the private partials in a fixed order: thread (cx, py) sums partials
// py, py+PY, ... of column cx; the PY sums are then added in py order.
// Block 0 also sums the per-CTA f partials into *f.
template <typename T>
__global__ void __launch_bounds__(512) qf_reduce_kernel(const T* __restrict__ partials, int nparts,
                                                        int n, const double* __restrict__ fpart,
                                                        int nf, T* gx, T* f, int accumulate) {
  constexpr int CX = 32, PY = 16;
  __shared__ T red[PY][CX + 1];
  __shared__ double fred[32];
  const int cx = threadIdx.x % CX, py = threadIdx.x / CX;
  const int j = blockIdx.x * CX + cx;
  T s = T(0);
  if (j < n)
    for (int c = py; c < nparts; c += PY) s += partials[(int64_t)c * n + j];
  red[py][cx] = s;
  __syncthreads();
  if (py == 0 && j < n) {
    T t = red[0][cx];
#pragma unroll
    for (int i = 1; i < PY; ++i) t += red[i][cx];
    gx[j] = accumulate ? gx[j] + t : t;
  }
  if (blockIdx.x == 0 && f) {
    double fs = 0.0;
    for (int i = threadIdx.x; i < nf; i += blockDim.x) fs += fpart[i];
    fs = block_sum(fs, fred);
    if (threadIdx.x == 0) *f = (T)fs;
  }
}

// ---------------------------------------------------------------- host ----
// Variants: (TEAM, CPT_MAX, block).  Team thread count x CPT_MAX bounds n.
struct QfVariant {
  int team, cpt_max, block;
};
static const QfVariant kVariants[] = {
    {32, 4, 256},    // n <= 128: warp per row, 8 rows in flight per CTA
    {128, 8, 256},   // n <= 1024
    {256, 8, 256},   // n <= 2048
    {512, 20, 512},  // n <= 10240: the whole CTA is one row team (n = 1e4: no idle column slot)
    {512, 24, 512},  // n <= 12288
};
constexpr int kNumVariants = (int)(sizeof(kVariants) / sizeof(kVariants[0]));

static int pick_variant(int64_t n, int team_hint) {
  for (int v = 0; v < kNumVariants; ++v) {
    if (team_hint && kVariants[v].team != team_hint) continue;
    if (n <= (int64_t)kVariants[v].team * kVariants[v].cpt_max) return v;
  }
  return -1;
}

template <typename T>
static size_t qf_smem_bytes(const QfVariant& v) {
  const int nteams = v.block / v.team;
  return sizeof(T) * ((size_t)v.cpt_max * v.team + 2 * nteams * (v.team / 32) + 2) + 8 +
         sizeof(double) * (nteams + 32);
}

template <typename T, int MODE>
static cudaError_t launch_team(int var, dim3 grid, cudaStream_t s, const QfArgs<T>& a) {
  const QfVariant& v = kVariants[var];
  const size_t smem = qf_smem_bytes<T>(v);
  cudaError_t e = cudaSuccess;
  auto go = [&](auto kern) {
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) {
      prof_begin(s, MODE == QF_FUSED ? "qf_team_kernel<fused>" : "qf_team_kernel<eval>");
      kern<<<grid, v.block, smem, s>>>(a);
      prof_end(s);
      e = cudaGetLastError();
    }
  };
  switch (var) {
    case 0: go(qf_team_kernel<T, 32, 4, MODE>); break;
    case 1: go(qf_team_kernel<T, 128, 8, MODE>); break;
    case 2: go(qf_team_kernel<T, 256, 8, MODE>); break;
    case 3: go(qf_team_kernel<T, 512, 20, MODE>); break;
    case 4: go(qf_team_kernel<T, 512, 24, MODE>); break;
    default: e = cudaErrorInvalidValue;
  }
  count_launch();
  return e;
}

template <typename T>
static cudaError_t launch_atomic(int var, dim3 grid, cudaStream_t s, const QfArgs<T>& a, T* gx) {
  const QfVariant& v = kVariants[var];
  prof_begin(s, "qf_atomic_adjoint_kernel");
  struct End { cudaStream_t s; ~End() { prof_end(s); } } end{s};
  switch (var) {
    case 0: qf_atomic_adjoint_kernel<T, 32, 4><<<grid, v.block, 0, s>>>(a, gx); break;
    case 1: qf_atomic_adjoint_kernel<T, 128, 8><<<grid, v.block, 0, s>>>(a, gx); break;
    case 2: qf_atomic_adjoint_kernel<T, 256, 8><<<grid, v.block, 0, s>>>(a, gx); break;
    case 3: qf_atomic_adjoint_kernel<T, 512, 20><<<grid, v.block, 0, s>>>(a, gx); break;
    case 4: qf_atomic_adjoint_kernel<T, 512, 24><<<grid, v.block, 0, s>>>(a, gx); break;
    default: return cudaErrorInvalidValue;
  }
  count_launch();
  return cudaGetLastError();
}

static int transpose_chunks(const kg_problem* p) {
  const int col_blocks = (int)((p->n + 255) / 256);
  int chunks = std::max(1, (4 * num_sms() + col_blocks - 1) / col_blocks);
  chunks = (int)std::min<int64_t>(chunks, p->m);
  return std::min(chunks, 1024);
}

kg_status qf_setup(kg_problem* p, cudaStream_t s) {
  int var = pick_variant(p->n, p->opt.team);
  if (p->strategy == KG_STRATEGY_CSR)
    return fail(KG_ERR_UNSUPPORTED, "QUADFORM: the CSR strategy is for index-map gathers (TETENERGY)");
  if (p->mode == KG_MODE_TAPE)
    return fail(KG_ERR_UNSUPPORTED, "QUADFORM: the reverse pass needs only y; no tape mode");
  p->mode = KG_MODE_RECOMPUTE;

  // FP64 arithmetic: float pairs on the FP32 units when the kernel and the data allow
  bool pair = false;
  if (p->dtype == KG_F64 && p->arith != KG_ARITH_NATIVE) {
    const bool shape_ok = qf_pair_supported(p) && p->n >= 1024 && p->opt.team == 0;
    if (!shape_ok && p->arith == KG_ARITH_PAIR)
      return fail(KG_ERR_UNSUPPORTED, "QUADFORM PAIR arithmetic needs the FUSED strategy, even n "
                                      "and 1024 <= n <= 12288");
    if (shape_ok) {
      kg_status rc = ws_common(p, num_sms(), s);
      if (rc != KG_OK) return rc;
      bool in_range = false;
      if ((rc = qf_pair_range_ok(p, s, &in_range)) != KG_OK) return rc;
      if (!in_range && p->arith == KG_ARITH_PAIR)
        return fail(KG_ERR_UNSUPPORTED, "QUADFORM PAIR arithmetic: A has entries outside "
                                        "0 or [2^-60, 2^40) in magnitude");
      pair = in_range;
    }
  }
  if (pair) {
    p->arith = KG_ARITH_PAIR;
    p->strategy = KG_STRATEGY_FUSED;
    QfConfig& c = p->qf;
    c.grid = qf_pair_grid(p, &c.rows_per_cta);
    c.team = c.block = 512;
    kg_status rc = ws_alloc(p, &p->partials, 8 * (size_t)c.grid * p->n, "xbar partials (pairs)");
    if (rc == KG_OK) rc = qf_pair_prepare(p, s);
    if (rc == KG_OK) c.coop = qf_pair_coop_fits(p) ? 1 : 0;
    return rc;
  }
  if (p->arith == KG_ARITH_AUTO || p->dtype == KG_F32) p->arith = KG_ARITH_NATIVE;
  if (qf_f32_supported(p)) {  // FP32: rows streamed through shared memory by TMA
    p->strategy = KG_STRATEGY_FUSED;
    QfConfig& c = p->qf;
    c.streamed = 1;
    c.grid = qf_f32_grid(p, &c.rows_per_cta);
    c.team = c.block = 512;
    kg_status rc = ws_common(p, c.grid, s);
    if (rc == KG_OK) rc = ws_alloc(p, &p->partials, 4 * (size_t)c.grid * p->n, "xbar partials (FP32)");
    if (rc == KG_OK) c.coop = qf_f32_coop_fits(p) ? 1 : 0;
    return rc;
  }
  if (p->strategy == KG_STRATEGY_AUTO) p->strategy = var >= 0 ? KG_STRATEGY_FUSED : KG_STRATEGY_TRANSPOSE;
  if (var < 0) {
    if (p->strategy != KG_STRATEGY_TRANSPOSE)
      return fail(KG_ERR_UNSUPPORTED, "QUADFORM: n = " + std::to_string(p->n) +
                                          " exceeds the row-team variants (n <= 12288); use TRANSPOSE");
    return fail(KG_ERR_UNSUPPORTED, "QUADFORM: n > 12288 is not supported by the forward kernel");
  }
  const QfVariant& v = kVariants[var];
  QfConfig& c = p->qf;
  c.team = v.team;
  c.block = v.block;
  c.cpt = (int)((p->n + v.team - 1) / v.team);
  const int nteams = v.block / v.team;
  const int resident = v.block >= 512 ? 1 : 2;
  int64_t target = (int64_t)num_sms() * resident;
  int64_t rows = std::max<int64_t>(nteams, (p->m + target - 1) / target);
  if (p->opt.tile > 0) rows = p->opt.tile;
  c.rows_per_cta = (int)rows;
  c.grid = (int)((p->m + rows - 1) / rows);
  int fp = std::max(c.grid, transpose_chunks(p));
  kg_status rc = ws_common(p, fp, s);
  if (rc != KG_OK) return rc;
  if (p->strategy == KG_STRATEGY_FUSED || p->strategy == KG_STRATEGY_TRANSPOSE) {
    int parts = p->strategy == KG_STRATEGY_FUSED ? c.grid : transpose_chunks(p);
    rc = ws_alloc(p, &p->partials, p->esize * (size_t)parts * p->n, "xbar partials");
    if (rc != KG_OK) return rc;
  }
  if (p->strategy != KG_STRATEGY_FUSED) {
    rc = ws_alloc(p, &p->y, p->esize * (size_t)p->m, "y");
    if (rc != KG_OK) return rc;
  }
  return KG_OK;
}

template <typename T>
static QfArgs<T> make_args(kg_problem* p, const void* x, const void* seed) {
  QfArgs<T> a{};
  a.A = static_cast<const T*>(p->data0);
  a.x = static_cast<const T*>(x);
  a.m = p->m;
  a.n = (int)p->n;
  a.cpt = p->qf.cpt;
  a.rows_per_cta = p->qf.rows_per_cta;
  a.seed = static_cast<const T*>(seed);
  a.partials = static_cast<T*>(p->partials);
  a.fpart = p->fpart;
  a.counter = p->counter;
  return a;
}

template <typename T>
static kg_status qf_eval_t(kg_problem* p, const void* x, void* f, T* y, cudaStream_t s) {
  QfArgs<T> a = make_args<T>(p, x, nullptr);
  a.f = static_cast<T*>(f);
  a.y = y;
  const int var = pick_variant(p->n, p->qf.team);
  cudaError_t e = launch_team<T, QF_EVAL>(var, dim3(p->qf.grid), s, a);
  if (e != cudaSuccess) return cuda_fail(e, "qf forward kernel");
  return KG_OK;
}

kg_status qf_eval(kg_problem* p, const void* x, void* f, cudaStream_t s) {
  if (p->arith == KG_ARITH_PAIR) return qf_pair_eval(p, x, f, s);
  if (p->qf.streamed) return qf_f32_eval(p, x, f, s);
  return p->dtype == KG_F64 ? qf_eval_t<double>(p, x, f, nullptr, s)
                            : qf_eval_t<float>(p, x, f, nullptr, s);
}

template <typename T>
static kg_status qf_grad_t(kg_problem* p, const void* x, void* f, void* gx, void* gA,
                           const void* seed, int accumulate, cudaStream_t s) {
  const int var = pick_variant(p->n, p->qf.team);
  const int n = (int)p->n;
  cudaError_t e;
  if (p->strategy == KG_STRATEGY_FUSED) {
    QfArgs<T> a = make_args<T>(p, x, seed);
    a.gA = static_cast<T*>(gA);
    a.accumulate = accumulate;
    e = launch_team<T, QF_FUSED>(var, dim3(p->qf.grid), s, a);
    if (e != cudaSuccess) return cuda_fail(e, "qf fused kernel");
    qf_reduce_kernel<T><<<(n + 31) / 32, 512, 0, s>>>(static_cast<const T*>(p->partials), p->qf.grid,
                                                      n, p->fpart, p->qf.grid, static_cast<T*>(gx),
                                                      static_cast<T*>(f), accumulate);
    count_launch();
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "qf reduce kernel");
    return KG_OK;
  }
  if (gA) return fail(KG_ERR_UNSUPPORTED, "QUADFORM: gradient w.r.t. A needs the FUSED strategy");
  // forward with y stored (f written by the last CTA)
  kg_status rc = qf_eval_t<T>(p, x, f, static_cast<T*>(p->y), s);
  if (rc != KG_OK) return rc;
  if (p->strategy == KG_STRATEGY_ATOMIC) {
    if (!accumulate) {
      e = cudaMemsetAsync(gx, 0, sizeof(T) * (size_t)n, s);
      count_launch();
      if (e != cudaSuccess) return cuda_fail(e, "zero gx");
    }
    QfArgs<T> a = make_args<T>(p, x, seed);
    a.y = static_cast<T*>(p->y);
    e = launch_atomic<T>(var, dim3(p->qf.grid), s, a, static_cast<T*>(gx));
    if (e != cudaSuccess) return cuda_fail(e, "qf atomic adjoint kernel");
    return KG_OK;
  }
  // TRANSPOSE
  const int chunks = transpose_chunks(p);
  const int rpc = (int)((p->m + chunks - 1) / chunks);
  const int used = (int)((p->m + rpc - 1) / rpc);
  prof_begin(s, "qf_transpose_kernel");
  qf_transpose_kernel<T><<<dim3((n + 255) / 256, used), 256, 0, s>>>(
      static_cast<const T*>(p->data0), static_cast<const T*>(p->y), p->m, n, rpc,
      static_cast<const T*>(seed), static_cast<T*>(p->partials));
  prof_end(s);
  count_launch();
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "qf transpose kernel");
  qf_reduce_kernel<T><<<(n + 31) / 32, 512, 0, s>>>(static_cast<const T*>(p->partials), used, n,
                                                    p->fpart, 0, static_cast<T*>(gx), nullptr,
                                                    accumulate);
  count_launch();
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "qf reduce kernel");
  return KG_OK;
}

// Native FP64 fused value-and-gradient with every workspace taken from
// `scratch` (partials: grid * n doubles, then grid f partials).  The fused
// kernel writes all of them before the reduce kernel reads them, so the
// scratch needs no clearing.  The grid is capped at scratch_doubles / (n + 1)
// CTAs (more rows per CTA instead), so any m fits once that cap is >= 1;
// KG_ERR_INVALID_ARG otherwise.
kg_status qf_native_fused_on_scratch(const double* A, int64_t m, int64_t n, const double* x,
                                     double* f, double* gx, double* scratch,
                                     size_t scratch_doubles, cudaStream_t s) {
  const int var = pick_variant(n, 0);
  if (var < 0) return fail(KG_ERR_INVALID_ARG, "n must be <= 12288");
  const QfVariant& v = kVariants[var];
  const int nteams = v.block / v.team;
  const int resident = v.block >= 512 ? 1 : 2;
  const int64_t target = (int64_t)num_sms() * resident;
  const int64_t max_grid = (int64_t)(scratch_doubles / ((size_t)n + 1));
  if (max_grid < 1)
    return fail(KG_ERR_INVALID_ARG, "scratch of " + std::to_string(scratch_doubles) +
                                        " doubles is too small for n = " + std::to_string(n));
  const int64_t rows = std::max<int64_t>({(int64_t)nteams, (m + target - 1) / target,
                                          (m + max_grid - 1) / max_grid});
  const int grid = (int)((m + rows - 1) / rows);
  const size_t need = (size_t)grid * (size_t)n + (size_t)grid;
  if (need > scratch_doubles)
    return fail(KG_ERR_INVALID_ARG, "problem needs " + std::to_string(need) +
                                        " scratch doubles, more than the " +
                                        std::to_string(scratch_doubles) + " available");
  QfArgs<double> a{};
  a.A = A;
  a.x = x;
  a.m = m;
  a.n = (int)n;
  a.cpt = (int)((n + v.team - 1) / v.team);
  a.rows_per_cta = (int)rows;
  a.partials = scratch;
  a.fpart = scratch + (size_t)grid * n;
  cudaError_t e = launch_team<double, QF_FUSED>(var, dim3(grid), s, a);
  if (e != cudaSuccess) return cuda_fail(e, "qf fused kernel");
  qf_reduce_kernel<double><<<(int)((n + 31) / 32), 512, 0, s>>>(scratch, grid, (int)n, a.fpart, grid,
                                                               gx, f, 0);
  count_launch();
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "qf reduce kernel");
  return KG_OK;
}

kg_status qf_grad(kg_problem* p, const void* x, void* f, void* gx, void* gA, const void* seed,
                  int accumulate, cudaStream_t s) {
  if (p->arith == KG_ARITH_PAIR) {
    if (gA)
      return fail(KG_ERR_UNSUPPORTED, "QUADFORM: the gradient w.r.t. A is produced by the native "
                                      "kernels (create the problem with KG_ARITH_NATIVE)");
    return qf_pair_grad(p, x, f, gx, seed, accumulate, s);
  }
  if (p->qf.streamed) {
    if (gA)
      return fail(KG_ERR_UNSUPPORTED, "QUADFORM: the gradient w.r.t. A is produced by the register "
                                      "team kernels (pass team=block size)");
    return qf_f32_grad(p, x, f, gx, seed, accumulate, s);
  }
  return p->dtype == KG_F64 ? qf_grad_t<double>(p, x, f, gx, gA, seed, accumulate, s)
                            : qf_grad_t<float>(p, x, f, gx, gA, seed, accumulate, s);
}

}  // namespace kg
