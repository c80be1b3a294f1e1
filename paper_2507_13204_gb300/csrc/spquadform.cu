// Sparse ||A x||^2 with A in compressed sparse rows (KG_SPQUADFORM).
//
// Forward (team-nested parallel_reduce over the stored entries of a row, then
// a sum reduction): y_i = sum_{p in row i} val[p] x[col[p]], f = sum_i y_i^2.
// Reverse: ybar_i = 2 fbar y_i (broadcast of the reduction adjoint); the read
// of x through the index map col becomes a scatter-add xbar[col[p]] += val[p]
// ybar_i (Sec. 3.3), and valbar[p] = x[col[p]] ybar_i.
//
// A team of TW lanes works on one row (32 / TW rows per warp, grid-stride over
// row groups so that every lane of a warp runs the same iterations); the team
// reduces its row sum with xor shuffles, a fixed order.
//
// Strategies for the scatter:
//   ATOMIC     the forward schedule (as generated code would run it): one
//              fused kernel, the team adds val[p] ybar_i into xbar with
//              atomics right after its row sum.
//   TRANSPOSE  rescheduled, atomic-free (Sec. 5, first restriction): the row
//              kernel stores y; a column kernel gathers over the transpose
//              (CSC, built once at kg_create with the values copied into
//              column order): xbar_j = 2 fbar sum_{q in col j} valT[q] y[rowT[q]],
//              in ascending row order.  Bitwise reproducible.
//
// Arithmetic: FP32 for FP32 problems.  FP64 problems use float pairs (as the
// dense and tet kernels do) when the stored values are in the pair range: the
// values are split once at kg_create into a float-pair copy (same 8 bytes),
// x is split per gather, y is kept as pairs, and the only FP64 instruction
// left is the pair -> double add that feeds each atomic (ATOMIC) or each
// gradient entry (TRANSPOSE); otherwise native FP64.
#include <cuda_runtime.h>

#include <algorithm>
#include <string>

#include "kg_device.cuh"
#include "kg_internal.h"
#include "kg_pair.cuh"

namespace kg {

constexpr int SQ_THREADS = 256;

enum { SQ_EVAL = 0, SQ_ATOMIC = 1, SQ_ROWPASS = 2 };

template <typename T>
struct SqArgs {
  const int* rowptr;
  const int* col;
  const T* val;
  const T* x;
  int64_t m;
  const T* seed;
  T* gx;    // ATOMIC: the scatter target (zeroed or accumulated by the caller)
  T* gval;  // nullable: gradient w.r.t. the stored values
  T* y;     // ROWPASS: the row sums
  int accumulate;
  double* fpart;
  unsigned* counter;
  T* f;
};

template <typename T>
__device__ __forceinline__ T team_sum(T v, int tw) {
  for (int o = tw >> 1; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Entries a lane handles per step: all their loads are issued before any use,
// so that a lane keeps SQ_U index loads, then SQ_U gathers, in flight.
constexpr int SQ_U = 4;

template <typename T, int TW, int MODE>
__global__ void __launch_bounds__(SQ_THREADS) spq_row_kernel(SqArgs<T> a) {
  __shared__ double red[32];
  constexpr int RPW = 32 / TW;  // rows per warp and iteration
  const int lane = threadIdx.x & 31, tl = lane & (TW - 1);
  const int64_t warp = ((int64_t)blockIdx.x * SQ_THREADS + threadIdx.x) >> 5;
  const int64_t nwarps = (int64_t)gridDim.x * (SQ_THREADS / 32);
  const T fb2 = MODE == SQ_EVAL ? T(0) : T(2) * load_seed(a.seed);
  FSum<T> fl;
  for (int64_t base = warp * RPW; base < a.m; base += nwarps * RPW) {
    const int64_t i = base + lane / TW;
    const bool act = i < a.m;
    const int p0 = act ? __ldg(a.rowptr + i) : 0, p1 = act ? __ldg(a.rowptr + i + 1) : 0;
    // first step kept in registers for the reverse pass
    int c[SQ_U];
    T v[SQ_U], xv[SQ_U];
#pragma unroll
    for (int u = 0; u < SQ_U; ++u) {
      const int p = p0 + tl + u * TW;
      c[u] = p < p1 ? __ldg(a.col + p) : 0;
      v[u] = p < p1 ? __ldg(a.val + p) : T(0);
    }
#pragma unroll
    for (int u = 0; u < SQ_U; ++u) xv[u] = __ldg(a.x + c[u]);  // column 0 for padding (n >= 1)
    T yp = T(0);
#pragma unroll
    for (int u = 0; u < SQ_U; ++u) yp = fma(v[u], xv[u], yp);
    for (int pb = p0 + SQ_U * TW; pb < p1; pb += SQ_U * TW) {  // rows longer than one step
      int cc[SQ_U];
      T vv[SQ_U];
#pragma unroll
      for (int u = 0; u < SQ_U; ++u) {
        const int p = pb + tl + u * TW;
        cc[u] = p < p1 ? __ldg(a.col + p) : 0;
        vv[u] = p < p1 ? __ldg(a.val + p) : T(0);
      }
#pragma unroll
      for (int u = 0; u < SQ_U; ++u) yp = fma(vv[u], __ldg(a.x + cc[u]), yp);
    }
    const T y = team_sum(yp, TW);
    if (act && tl == 0) fl.add(y);
    if constexpr (MODE == SQ_ROWPASS) {
      if (act && tl == 0) a.y[i] = y;
    }
    if constexpr (MODE != SQ_EVAL) {
      const T yb = fb2 * y;
#pragma unroll
      for (int u = 0; u < SQ_U; ++u) {
        const int p = p0 + tl + u * TW;
        if (p < p1) {
          if constexpr (MODE == SQ_ATOMIC) red_add(a.gx + c[u], v[u] * yb);
          if (a.gval) {
            const T g = xv[u] * yb;
            a.gval[p] = a.accumulate ? a.gval[p] + g : g;
          }
        }
      }
      for (int p = p0 + SQ_U * TW + tl; p < p1; p += TW) {
        const int cp = __ldg(a.col + p);
        if constexpr (MODE == SQ_ATOMIC) red_add(a.gx + cp, __ldg(a.val + p) * yb);
        if (a.gval) {
          const T g = __ldg(a.x + cp) * yb;
          a.gval[p] = a.accumulate ? a.gval[p] + g : g;
        }
      }
    }
  }
  finish_sum<T>(block_sum(fl.get(), red), a.fpart, a.counter, a.f, 0, red);
}

// xbar_j = 2 fbar sum_{q in col j} valT[q] y[rowT[q]]: a team per column of
// the transpose, ascending rows, fixed reduction order.
template <typename T, int TW>
__global__ void __launch_bounds__(SQ_THREADS) spq_col_kernel(const int* __restrict__ colptr,
                                                             const int* __restrict__ rowT,
                                                             const T* __restrict__ valT,
                                                             const T* __restrict__ y, int64_t n,
                                                             const T* seed, T* gx, int accumulate) {
  constexpr int CPW = 32 / TW;
  const int lane = threadIdx.x & 31, tl = lane & (TW - 1);
  const int64_t warp = ((int64_t)blockIdx.x * SQ_THREADS + threadIdx.x) >> 5;
  const int64_t nwarps = (int64_t)gridDim.x * (SQ_THREADS / 32);
  const T fb2 = T(2) * load_seed(seed);
  for (int64_t base = warp * CPW; base < n; base += nwarps * CPW) {
    const int64_t j = base + lane / TW;
    const bool act = j < n;
    const int q0 = act ? __ldg(colptr + j) : 0, q1 = act ? __ldg(colptr + j + 1) : 0;
    T s = T(0);
    for (int qb = q0; qb < q1; qb += SQ_U * TW) {
      int r[SQ_U];
      T v[SQ_U];
#pragma unroll
      for (int u = 0; u < SQ_U; ++u) {
        const int q = qb + tl + u * TW;
        r[u] = q < q1 ? __ldg(rowT + q) : 0;
        v[u] = q < q1 ? __ldg(valT + q) : T(0);
      }
#pragma unroll
      for (int u = 0; u < SQ_U; ++u) s = fma(v[u], __ldg(y + r[u]), s);  // row 0 for padding
    }
    s = team_sum(s, TW);
    if (act && tl == 0) {
      const T g = fb2 * s;
      gx[j] = accumulate ? gx[j] + g : g;
    }
  }
}

// ---------------------------------------------------------- float pairs ----
struct SqPairArgs {
  const int* rowptr;
  const int* col;
  const float2* valp;  // prepared (h, l) of every stored value
  const double* x;
  int64_t m;
  const double* seed;
  double* gx;
  double* gval;
  float2* yp;  // ROWPASS: y as pairs
  int accumulate;
  double* fpart;
  unsigned* counter;
  double* f;
  unsigned* err;
};

__device__ __forceinline__ Acc team_sum_acc(Acc v, int tw) {
  for (int o = tw >> 1; o > 0; o >>= 1) {
    Acc b;
    b.s = __shfl_xor_sync(0xffffffffu, v.s, o);
    b.l = __shfl_xor_sync(0xffffffffu, v.l, o);
    v = acc_add(v, b);
  }
  return v;
}

template <int TW, int MODE>
__global__ void __launch_bounds__(SQ_THREADS) spq_row_pair_kernel(SqPairArgs a) {
  __shared__ double red[32];
  constexpr int RPW = 32 / TW;
  const int lane = threadIdx.x & 31, tl = lane & (TW - 1);
  const int64_t warp = ((int64_t)blockIdx.x * SQ_THREADS + threadIdx.x) >> 5;
  const int64_t nwarps = (int64_t)gridDim.x * (SQ_THREADS / 32);
  bool bad = false;
  Pair fb2{0.f, 0.f};
  if constexpr (MODE != SQ_EVAL) {
    const double fb = load_seed(a.seed);
    bad |= !pair_in_range(2.0 * fb);
    fb2 = split_f64(2.0 * fb);
  }
  Acc fa = acc_zero();
  int nrows = 0;
  for (int64_t base = warp * RPW; base < a.m; base += nwarps * RPW) {
    const int64_t i = base + lane / TW;
    const bool act = i < a.m;
    const int p0 = act ? __ldg(a.rowptr + i) : 0, p1 = act ? __ldg(a.rowptr + i + 1) : 0;
    Acc ya = acc_zero();
    for (int pb = p0; pb < p1; pb += SQ_U * TW) {
      int c[SQ_U];
      float2 v[SQ_U];
#pragma unroll
      for (int u = 0; u < SQ_U; ++u) {
        const int p = pb + tl + u * TW;
        c[u] = p < p1 ? __ldg(a.col + p) : 0;
        v[u] = p < p1 ? __ldg(a.valp + p) : make_float2(0.f, 0.f);
      }
#pragma unroll
      for (int u = 0; u < SQ_U; ++u) {
        const double xd = __ldg(a.x + c[u]);  // column 0 for padding (n >= 1)
        bad |= !pair_in_range(xd);
        const Pair xp = split_f64(xd);
        acc_fma(ya, v[u].x, v[u].y, xp.h, xp.l);
      }
    }
    const Pair y = acc_pair(team_sum_acc(ya, TW));
    if (act && tl == 0) {
      const Pair y2 = pair_mul(y, y);
      fa = acc_add(fa, Acc{y2.h, y2.l});
      if ((++nrows & 31) == 0) acc_renorm(fa);
      if constexpr (MODE == SQ_ROWPASS) a.yp[i] = make_float2(y.h, y.l);
    }
    if constexpr (MODE != SQ_EVAL) {
      const Pair yb = pair_mul(fb2, y);
      if (MODE == SQ_ATOMIC || a.gval) {
        for (int p = p0 + tl; p < p1; p += TW) {
          const int cp = __ldg(a.col + p);
          if constexpr (MODE == SQ_ATOMIC) {
            const float2 v = __ldg(a.valp + p);
            red_add(a.gx + cp, pair_to_double_fast(pair_mul(Pair{v.x, v.y}, yb)));
          }
          if (a.gval) {
            const double g = pair_to_double_fast(pair_mul(split_f64(__ldg(a.x + cp)), yb));
            a.gval[p] = a.accumulate ? a.gval[p] + g : g;
          }
        }
      }
    }
  }
  if (bad) set_error(a.err, ERRBIT_RANGE);
  finish_sum<double>(block_sum(acc_to_double(fa), red), a.fpart, a.counter, a.f, 0, red);
}

template <int TW>
__global__ void __launch_bounds__(SQ_THREADS) spq_col_pair_kernel(const int* __restrict__ colptr,
                                                                  const int* __restrict__ rowT,
                                                                  const float2* __restrict__ valTp,
                                                                  const float2* __restrict__ yp,
                                                                  int64_t n, const double* seed,
                                                                  double* gx, int accumulate) {
  constexpr int CPW = 32 / TW;
  const int lane = threadIdx.x & 31, tl = lane & (TW - 1);
  const int64_t warp = ((int64_t)blockIdx.x * SQ_THREADS + threadIdx.x) >> 5;
  const int64_t nwarps = (int64_t)gridDim.x * (SQ_THREADS / 32);
  const Pair fb2 = split_f64(2.0 * load_seed(seed));  // range checked by the row kernel
  for (int64_t base = warp * CPW; base < n; base += nwarps * CPW) {
    const int64_t j = base + lane / TW;
    const bool act = j < n;
    const int q0 = act ? __ldg(colptr + j) : 0, q1 = act ? __ldg(colptr + j + 1) : 0;
    Acc sa = acc_zero();
    for (int qb = q0; qb < q1; qb += SQ_U * TW) {
      int r[SQ_U];
      float2 v[SQ_U];
#pragma unroll
      for (int u = 0; u < SQ_U; ++u) {
        const int q = qb + tl + u * TW;
        r[u] = q < q1 ? __ldg(rowT + q) : 0;
        v[u] = q < q1 ? __ldg(valTp + q) : make_float2(0.f, 0.f);
      }
#pragma unroll
      for (int u = 0; u < SQ_U; ++u) {
        const float2 yr = __ldg(yp + r[u]);  // row 0 for padding
        acc_fma(sa, v[u].x, v[u].y, yr.x, yr.y);
      }
    }
    const Pair sum = acc_pair(team_sum_acc(sa, TW));
    if (act && tl == 0) {
      const double g = pair_to_double_fast(pair_mul(fb2, sum));
      gx[j] = accumulate ? gx[j] + g : g;
    }
  }
}

// Set-up for pair arithmetic: range of every stored value (ERRBIT_RANGE), and
// the float-pair copy out[i] = (h, l) of v[perm ? perm[i] : i].
__global__ void spq_range_kernel(const double* __restrict__ v, int64_t n, unsigned* err) {
  bool bad = false;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
    bad |= !pair_in_range(v[i]);
  if (bad) set_error(err, ERRBIT_RANGE);
}

__global__ void spq_split_kernel(const double* __restrict__ v, const int* __restrict__ perm,
                                 int64_t n, float2* out) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const Pair p = split_f64(v[perm ? perm[i] : i]);
    out[i] = make_float2(p.h, p.l);
  }
}

// Structure check at kg_create: rowptr[0] = 0, rowptr[m] = nnz, non-decreasing,
// every column in [0, n).  Sets ERRBIT_BOUNDS.
__global__ void spq_validate_kernel(const int* __restrict__ rowptr, int64_t m,
                                    const int* __restrict__ col, int64_t nnz, int64_t n,
                                    unsigned* err) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  bool bad = false;
  if (t0 == 0) bad |= rowptr[0] != 0 || rowptr[m] != (int)nnz;
  for (int64_t i = t0; i < m; i += stride) bad |= rowptr[i + 1] < rowptr[i];
  for (int64_t p = t0; p < nnz; p += stride) bad |= (unsigned)col[p] >= (unsigned)n;
  if (bad) set_error(err, ERRBIT_BOUNDS);
}

// Row index of every stored entry (set-up only).
__global__ void spq_rowid_kernel(const int* __restrict__ rowptr, int64_t m, int* rowid) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += stride)
    for (int p = rowptr[i]; p < rowptr[i + 1]; ++p) rowid[p] = (int)i;
}

// rowT[q] = rowid[perm[q]], valT[q] = val[perm[q]] (set-up only).
template <typename T>
__global__ void spq_permute_kernel(const int* __restrict__ perm, const int* __restrict__ rowid,
                                   const T* __restrict__ val, int64_t nnz, int* rowT, T* valT) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < nnz; q += stride) {
    const int pq = perm[q];
    rowT[q] = rowid[pq];
    valT[q] = val[pq];
  }
}

// ---------------------------------------------------------------- host ----
static int sq_grid(int64_t work_rows, int tw) {
  const int64_t rows_per_block = (int64_t)(SQ_THREADS / 32) * (32 / tw);
  const int64_t g = (work_rows + rows_per_block - 1) / rows_per_block;
  return (int)std::max<int64_t>(1, std::min<int64_t>(g, (int64_t)num_sms() * 8));
}

// Lanes per row (or column) team: the smallest power of two (2..32) whose
// SQ_U-entry steps cover `cover` x the average length in one step.  Measured on
// the 2^20-row matrix with 8..24 entries a row: FP64 (float pairs) is fastest
// at 8 lanes (cover 1.5: 185 us against 218 at 4 lanes); FP32 at 2 lanes (cover
// 0.5: 168.6 / 167.0 us for the atomic / CSC gradient, against 175.2 / 208.1 at
// 8): its cheaper arithmetic leaves the loads the bound, and narrower teams keep
// more rows' gathers in flight.
static int team_for(double avg, int requested, double cover) {
  if (requested) return requested;
  int tw = 2;
  while (tw < 32 && (double)(tw * SQ_U) < cover * avg) tw *= 2;
  return tw;
}

kg_status spq_setup(kg_problem* p, cudaStream_t s) {
  // AUTO: the atomic scatter measured faster on the 2^20-row, 16-per-row workload
  if (p->strategy == KG_STRATEGY_AUTO) p->strategy = KG_STRATEGY_ATOMIC;
  if (p->strategy != KG_STRATEGY_ATOMIC && p->strategy != KG_STRATEGY_TRANSPOSE)
    return fail(KG_ERR_UNSUPPORTED, "SPQUADFORM: strategy must be ATOMIC or TRANSPOSE");
  if (p->mode == KG_MODE_TAPE)
    return fail(KG_ERR_UNSUPPORTED, "SPQUADFORM: the reverse pass needs only y; no tape mode");
  p->mode = KG_MODE_RECOMPUTE;
  if (p->dtype == KG_F32) {
    if (p->arith == KG_ARITH_PAIR) return fail(KG_ERR_UNSUPPORTED, "SPQUADFORM: PAIR is for FP64 data");
    p->arith = KG_ARITH_NATIVE;
  }
  const int t = p->opt.team;
  if (t && t != 2 && t != 4 && t != 8 && t != 16 && t != 32)
    return fail(KG_ERR_UNSUPPORTED, "SPQUADFORM: team must be 2, 4, 8, 16 or 32");
  const double cover = p->dtype == KG_F32 ? 0.5 : 1.5;
  p->sq_team = team_for((double)p->nnz / (double)p->m, t, cover);
  p->sq_col_team = team_for((double)p->nnz / (double)p->n, t, cover);
  const int grid = sq_grid(p->m, p->sq_team);
  kg_status rc = ws_common(p, grid, s);
  if (rc != KG_OK) return rc;
  const int* rowptr = static_cast<const int*>(p->data0);
  const int* col = static_cast<const int*>(p->data1);
  const int g = (int)std::max<int64_t>(1, std::min<int64_t>((std::max(p->m, p->nnz) + 255) / 256,
                                                           (int64_t)num_sms() * 8));
  spq_validate_kernel<<<g, 256, 0, s>>>(rowptr, p->m, col, p->nnz, p->n, p->err);
  // FP64: float pairs when every stored value is in the pair range and the copy fits
  const bool try_pair = p->dtype == KG_F64 && p->arith != KG_ARITH_NATIVE;
  if (try_pair && p->nnz > 0)
    spq_range_kernel<<<g, 256, 0, s>>>(static_cast<const double*>(p->data2), p->nnz, p->err);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "validate CSR");
  // the structure must be valid before it is used as an index
  if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_fail(e, "validate CSR");
  unsigned h = 0;
  if ((e = cudaMemcpy(&h, p->err, sizeof(h), cudaMemcpyDeviceToHost)) != cudaSuccess)
    return cuda_fail(e, "read error word");
  if (h & ERRBIT_BOUNDS) return fail(KG_ERR_BOUNDS, "kg_create: CSR structure invalid");
  if ((e = cudaMemsetAsync(p->err, 0, sizeof(unsigned), s)) != cudaSuccess)
    return cuda_fail(e, "clear error word");
  if (try_pair) {
    const size_t budget = p->opt.tape_budget_bytes ? p->opt.tape_budget_bytes : (size_t(1) << 30);
    const bool in_range = (h & ERRBIT_RANGE) == 0;
    if (p->arith == KG_ARITH_PAIR && !in_range)
      return fail(KG_ERR_UNSUPPORTED, "SPQUADFORM PAIR arithmetic: a stored value is outside "
                                      "0 or [2^-60, 2^40) in magnitude");
    const bool fits = 8 * (size_t)p->nnz <= budget || p->arith == KG_ARITH_PAIR;
    p->arith = in_range && fits ? KG_ARITH_PAIR : KG_ARITH_NATIVE;
  }
  const bool pair = p->arith == KG_ARITH_PAIR;
  const size_t nz = (size_t)std::max<int64_t>(p->nnz, 1);
  if (pair) {
    if ((rc = ws_alloc(p, &p->aprep, 8 * nz, "prepared values (float pairs)")) != KG_OK) return rc;
    if (p->nnz > 0)
      spq_split_kernel<<<g, 256, 0, s>>>(static_cast<const double*>(p->data2), nullptr, p->nnz,
                                         static_cast<float2*>(p->aprep));
  }
  if (p->strategy == KG_STRATEGY_ATOMIC) {
    e = cudaGetLastError();
    return e == cudaSuccess ? KG_OK : cuda_fail(e, "prepare values");
  }
  if ((rc = ws_alloc(p, &p->y, p->esize * (size_t)p->m, "y")) != KG_OK) return rc;
  if ((rc = ws_alloc(p, (void**)&p->rowptr, sizeof(int) * (size_t)(p->n + 1), "CSC colptr")) != KG_OK)
    return rc;
  if ((rc = ws_alloc(p, (void**)&p->inc, sizeof(int) * nz, "CSC rows")) != KG_OK) return rc;
  if ((rc = ws_alloc(p, &p->valT, p->esize * nz, "CSC values")) != KG_OK) return rc;
  int *perm = nullptr, *rowid = nullptr;
  if (dev_alloc((void**)&perm, sizeof(int) * nz) != cudaSuccess ||
      dev_alloc((void**)&rowid, sizeof(int) * nz) != cudaSuccess) {
    cudaFree(perm);
    return fail(KG_ERR_OOM, "CSC build scratch allocation failed");
  }
  rc = build_buckets(col, p->nnz, (int)p->n, p->rowptr, perm, s);
  if (rc == KG_OK && p->nnz > 0) {
    spq_rowid_kernel<<<g, 256, 0, s>>>(rowptr, p->m, rowid);
    if (p->dtype == KG_F64)
      spq_permute_kernel<double><<<g, 256, 0, s>>>(perm, rowid, static_cast<const double*>(p->data2),
                                                   p->nnz, p->inc, static_cast<double*>(p->valT));
    else
      spq_permute_kernel<float><<<g, 256, 0, s>>>(perm, rowid, static_cast<const float*>(p->data2),
                                                  p->nnz, p->inc, static_cast<float*>(p->valT));
    if (pair)  // in place: each entry's 8 bytes become its float pair
      spq_split_kernel<<<g, 256, 0, s>>>(static_cast<const double*>(p->valT), nullptr, p->nnz,
                                         static_cast<float2*>(p->valT));
    e = cudaGetLastError();
    cudaError_t e2 = cudaStreamSynchronize(s);
    if (e != cudaSuccess || e2 != cudaSuccess) rc = cuda_fail(e != cudaSuccess ? e : e2, "CSC build");
  }
  cudaFree(perm);
  cudaFree(rowid);
  return rc;
}

template <typename T, int MODE>
static cudaError_t launch_row(const kg_problem* p, const SqArgs<T>& a, cudaStream_t s) {
  const int g = sq_grid(p->m, p->sq_team);
  switch (p->sq_team) {
    case 2: spq_row_kernel<T, 2, MODE><<<g, SQ_THREADS, 0, s>>>(a); break;
    case 4: spq_row_kernel<T, 4, MODE><<<g, SQ_THREADS, 0, s>>>(a); break;
    case 8: spq_row_kernel<T, 8, MODE><<<g, SQ_THREADS, 0, s>>>(a); break;
    case 16: spq_row_kernel<T, 16, MODE><<<g, SQ_THREADS, 0, s>>>(a); break;
    default: spq_row_kernel<T, 32, MODE><<<g, SQ_THREADS, 0, s>>>(a); break;
  }
  return cudaGetLastError();
}

template <typename T>
static cudaError_t launch_col(const kg_problem* p, const T* y, const T* seed, T* gx, int acc,
                              cudaStream_t s) {
  const int g = sq_grid(p->n, p->sq_col_team);
  const int* cp = p->rowptr;
  const int* rt = p->inc;
  const T* vt = static_cast<const T*>(p->valT);
  switch (p->sq_col_team) {
    case 2: spq_col_kernel<T, 2><<<g, SQ_THREADS, 0, s>>>(cp, rt, vt, y, p->n, seed, gx, acc); break;
    case 4: spq_col_kernel<T, 4><<<g, SQ_THREADS, 0, s>>>(cp, rt, vt, y, p->n, seed, gx, acc); break;
    case 8: spq_col_kernel<T, 8><<<g, SQ_THREADS, 0, s>>>(cp, rt, vt, y, p->n, seed, gx, acc); break;
    case 16: spq_col_kernel<T, 16><<<g, SQ_THREADS, 0, s>>>(cp, rt, vt, y, p->n, seed, gx, acc); break;
    default: spq_col_kernel<T, 32><<<g, SQ_THREADS, 0, s>>>(cp, rt, vt, y, p->n, seed, gx, acc); break;
  }
  return cudaGetLastError();
}

template <int MODE>
static cudaError_t launch_row_pair(const kg_problem* p, const SqPairArgs& a, cudaStream_t s) {
  const int g = sq_grid(p->m, p->sq_team);
  switch (p->sq_team) {
    case 2: spq_row_pair_kernel<2, MODE><<<g, SQ_THREADS, 0, s>>>(a); break;
    case 4: spq_row_pair_kernel<4, MODE><<<g, SQ_THREADS, 0, s>>>(a); break;
    case 8: spq_row_pair_kernel<8, MODE><<<g, SQ_THREADS, 0, s>>>(a); break;
    case 16: spq_row_pair_kernel<16, MODE><<<g, SQ_THREADS, 0, s>>>(a); break;
    default: spq_row_pair_kernel<32, MODE><<<g, SQ_THREADS, 0, s>>>(a); break;
  }
  return cudaGetLastError();
}

static cudaError_t launch_col_pair(const kg_problem* p, const double* seed, double* gx, int acc,
                                   cudaStream_t s) {
  const int g = sq_grid(p->n, p->sq_col_team);
  const int* cp = p->rowptr;
  const int* rt = p->inc;
  const float2* vt = static_cast<const float2*>(p->valT);
  const float2* y = static_cast<const float2*>(p->y);
  switch (p->sq_col_team) {
    case 2: spq_col_pair_kernel<2><<<g, SQ_THREADS, 0, s>>>(cp, rt, vt, y, p->n, seed, gx, acc); break;
    case 4: spq_col_pair_kernel<4><<<g, SQ_THREADS, 0, s>>>(cp, rt, vt, y, p->n, seed, gx, acc); break;
    case 8: spq_col_pair_kernel<8><<<g, SQ_THREADS, 0, s>>>(cp, rt, vt, y, p->n, seed, gx, acc); break;
    case 16: spq_col_pair_kernel<16><<<g, SQ_THREADS, 0, s>>>(cp, rt, vt, y, p->n, seed, gx, acc); break;
    default: spq_col_pair_kernel<32><<<g, SQ_THREADS, 0, s>>>(cp, rt, vt, y, p->n, seed, gx, acc); break;
  }
  return cudaGetLastError();
}

static SqPairArgs sq_pair_args(kg_problem* p, const void* x, void* f, const void* seed) {
  SqPairArgs a{};
  a.rowptr = static_cast<const int*>(p->data0);
  a.col = static_cast<const int*>(p->data1);
  a.valp = static_cast<const float2*>(p->aprep);
  a.x = static_cast<const double*>(x);
  a.m = p->m;
  a.seed = static_cast<const double*>(seed);
  a.fpart = p->fpart;
  a.counter = p->counter;
  a.f = static_cast<double*>(f);
  a.err = p->err;
  return a;
}

static kg_status spq_pair_eval(kg_problem* p, const void* x, void* f, cudaStream_t s) {
  SqPairArgs a = sq_pair_args(p, x, f, nullptr);
  prof_begin(s, "spq_row_pair_kernel<eval>");
  cudaError_t e = launch_row_pair<SQ_EVAL>(p, a, s);
  prof_end(s);
  count_launch();
  return e == cudaSuccess ? KG_OK : cuda_fail(e, "spq pair forward kernel");
}

static kg_status spq_pair_grad(kg_problem* p, const void* x, void* f, void* gx, void* gval,
                               const void* seed, int accumulate, cudaStream_t s) {
  SqPairArgs a = sq_pair_args(p, x, f, seed);
  a.gval = static_cast<double*>(gval);
  a.accumulate = accumulate;
  cudaError_t e;
  if (p->strategy == KG_STRATEGY_ATOMIC) {
    if (!accumulate) {
      if ((e = cudaMemsetAsync(gx, 0, sizeof(double) * (size_t)p->n, s)) != cudaSuccess)
        return cuda_fail(e, "zero gx");
      count_launch();
    }
    a.gx = static_cast<double*>(gx);
    prof_begin(s, "spq_row_pair_kernel<atomic>");
    e = launch_row_pair<SQ_ATOMIC>(p, a, s);
    prof_end(s);
    count_launch();
    return e == cudaSuccess ? KG_OK : cuda_fail(e, "spq pair atomic kernel");
  }
  a.yp = static_cast<float2*>(p->y);
  if ((e = launch_row_pair<SQ_ROWPASS>(p, a, s)) != cudaSuccess) return cuda_fail(e, "spq pair row kernel");
  count_launch();
  prof_begin(s, "spq_col_pair_kernel");
  e = launch_col_pair(p, static_cast<const double*>(seed), static_cast<double*>(gx), accumulate, s);
  prof_end(s);
  count_launch();
  return e == cudaSuccess ? KG_OK : cuda_fail(e, "spq pair column kernel");
}

template <typename T>
static SqArgs<T> sq_args(kg_problem* p, const void* x, void* f, const void* seed) {
  SqArgs<T> a{};
  a.rowptr = static_cast<const int*>(p->data0);
  a.col = static_cast<const int*>(p->data1);
  a.val = static_cast<const T*>(p->data2);
  a.x = static_cast<const T*>(x);
  a.m = p->m;
  a.seed = static_cast<const T*>(seed);
  a.fpart = p->fpart;
  a.counter = p->counter;
  a.f = static_cast<T*>(f);
  return a;
}

template <typename T>
static kg_status spq_eval_t(kg_problem* p, const void* x, void* f, cudaStream_t s) {
  SqArgs<T> a = sq_args<T>(p, x, f, nullptr);
  prof_begin(s, "spq_row_kernel<eval>");
  cudaError_t e = launch_row<T, SQ_EVAL>(p, a, s);
  prof_end(s);
  count_launch();
  return e == cudaSuccess ? KG_OK : cuda_fail(e, "spq forward kernel");
}

template <typename T>
static kg_status spq_grad_t(kg_problem* p, const void* x, void* f, void* gx, void* gval,
                            const void* seed, int accumulate, cudaStream_t s) {
  SqArgs<T> a = sq_args<T>(p, x, f, seed);
  a.gval = static_cast<T*>(gval);
  a.accumulate = accumulate;
  cudaError_t e;
  if (p->strategy == KG_STRATEGY_ATOMIC) {
    if (!accumulate) {
      if ((e = cudaMemsetAsync(gx, 0, sizeof(T) * (size_t)p->n, s)) != cudaSuccess)
        return cuda_fail(e, "zero gx");
      count_launch();
    }
    a.gx = static_cast<T*>(gx);
    prof_begin(s, "spq_row_kernel<atomic>");
    e = launch_row<T, SQ_ATOMIC>(p, a, s);
    prof_end(s);
    count_launch();
    return e == cudaSuccess ? KG_OK : cuda_fail(e, "spq atomic kernel");
  }
  a.y = static_cast<T*>(p->y);
  if ((e = launch_row<T, SQ_ROWPASS>(p, a, s)) != cudaSuccess) return cuda_fail(e, "spq row kernel");
  count_launch();
  prof_begin(s, "spq_col_kernel");
  e = launch_col<T>(p, static_cast<const T*>(p->y), static_cast<const T*>(seed), static_cast<T*>(gx),
                    accumulate, s);
  prof_end(s);
  count_launch();
  return e == cudaSuccess ? KG_OK : cuda_fail(e, "spq column kernel");
}

kg_status spq_eval(kg_problem* p, const void* x, void* f, cudaStream_t s) {
  if (p->arith == KG_ARITH_PAIR) return spq_pair_eval(p, x, f, s);
  return p->dtype == KG_F64 ? spq_eval_t<double>(p, x, f, s) : spq_eval_t<float>(p, x, f, s);
}

kg_status spq_grad(kg_problem* p, const void* x, void* f, void* gx, void* gval, const void* seed,
                   int accumulate, cudaStream_t s) {
  if (p->arith == KG_ARITH_PAIR) return spq_pair_grad(p, x, f, gx, gval, seed, accumulate, s);
  return p->dtype == KG_F64 ? spq_grad_t<double>(p, x, f, gx, gval, seed, accumulate, s)
                            : spq_grad_t<float>(p, x, f, gx, gval, seed, accumulate, s);
}

}  // namespace kg
