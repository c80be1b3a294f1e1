// Dense ||A x||^2 value-and-gradient for FP64 data with float-pair arithmetic.
//
// Same method as quadform.cu (forward row dot products y_i, broadcast of the
// reduction adjoint ybar_i = 2 fbar y_i, reverse xbar_j += A_ij ybar_i with
// one pass over A), laid out for GB300:
//   - one CTA of 16 warps per SM;
//   - whole rows of A stream into a two-stage shared-memory ring through TMA
//     bulk copies (cp.async.bulk + mbarrier transaction counts), the rows two
//     ahead are prefetched into L2; warps release a stage through an "empty"
//     mbarrier and thread 0, once every warp has released it, issues the copy
//     of the row two ahead into it;
//   - consumer thread t owns the column pairs jp = t + 512 k; it splits A's
//     doubles into float pairs (integer instructions), writes the split values
//     back in place so the reverse pass does not split again, and accumulates
//     with FMA two-product / TwoSum on the FP32 units;
//   - PREP: when the problem holds A already split into float pairs (made once
//     by kg_create, same 8 bytes per entry), rows of that copy stream instead
//     and no split or write-back runs in the row loop (about a fifth of the
//     instructions per entry);
//   - the private xbar partials (float pairs) of each CTA go to a workspace that
//     a second kernel sums in a fixed order: bitwise reproducible.
// For 2048 < n <= 10240 on the prepared A the fused pass runs qf_pair_ws_kernel
// instead, with dot-product, update and copy roles in separate warps (described
// at the kernel); the forward and all other shapes use qf_pair_kernel.
// All waits are bounded (about one second) and report KG_ERR_TIMEOUT.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdlib>
#include <string>

#include "kg_device.cuh"
#include "kg_internal.h"
#include "kg_pair.cuh"

namespace kg {

constexpr int QP_CW = 16;                    // warps
constexpr int QP_CT = QP_CW * 32;            // threads
constexpr int QP_THREADS = QP_CT;
constexpr int QP_BAR = 1;                    // named barrier id

struct QpArgs {
  const double* A;   // FP64 rows, or (PREP) rows of float pairs (h0, l0, h1, l1, ...)
  const double* x;
  int64_t m;
  int n;  // even
  int band;
  const double* seed;
  float4* partials;  // [grid][n/2] of (h0, l0, h1, l1)
  double* fpart;
  unsigned* counter;
  double* f;  // EVAL: written by the last CTA; fused reduction: by CTA 0
  unsigned* err;
  double* gx;      // fused reduction (qf_pair_ws_kernel<KP, true>): the gradient
  int accumulate;  // fused reduction: 1 adds to gx
};

__device__ __forceinline__ Acc shfl_xor_acc(Acc a, int o) {
  Acc b;
  b.s = __shfl_xor_sync(0xffffffffu, a.s, o);
  b.l = __shfl_xor_sync(0xffffffffu, a.l, o);
  return b;
}

template <int PPT, bool FUSED, bool PREP>
__global__ void __launch_bounds__(QP_THREADS, 1) qf_pair_kernel(QpArgs a) {
  extern __shared__ __align__(128) unsigned char smem[];
  const int n = a.n, npairs = n >> 1;
  double* stage0 = reinterpret_cast<double*>(smem);
  double* stage1 = stage0 + n;
  uint64_t* full = reinterpret_cast<uint64_t*>(stage1 + n);
  uint64_t* empty = full + 2;
  Acc* red = reinterpret_cast<Acc*>(empty + 2);  // [2][QP_CW]
  volatile int* abort_flag = reinterpret_cast<volatile int*>(red + 2 * QP_CW);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t r0 = (int64_t)blockIdx.x * a.band;
  const int64_t r1 = r0 + a.band < a.m ? r0 + a.band : a.m;
  const int nrows = r1 > r0 ? (int)(r1 - r0) : 0;
  const uint32_t row_bytes = (uint32_t)n * 8u;

  if (threadIdx.x == 0) {
    mbar_init(&full[0], 1);
    mbar_init(&full[1], 1);
    mbar_init(&empty[0], QP_CW);
    mbar_init(&empty[1], QP_CW);
    *abort_flag = 0;
    fence_barrier_init();
  }
  __syncthreads();
  // thread 0 issues the copies: rows 0 and 1 now, row it+2 once stage it&1 is released
  int issued = 0;
  if (threadIdx.x == 0) {
    for (int it = 0; it < 2 && it < nrows; ++it) {
      const double* src = a.A + (r0 + it) * (int64_t)n;
      mbar_arrive_expect_tx(&full[it], row_bytes);
      tma_load_1d(it ? stage1 : stage0, src, row_bytes, &full[it]);
      ++issued;
      if (it + 2 < nrows) prefetch_l2_bulk(src + 2 * (int64_t)n, row_bytes);
    }
  }

  // ------------------------------------------------------------ consumers
  const int t = threadIdx.x;
  float xh[PPT][2], xl[PPT][2];
  bool bad = false;
#pragma unroll
  for (int k = 0; k < PPT; ++k) {
    const int jp = t + QP_CT * k;
    double2 xv = make_double2(0.0, 0.0);
    if (jp < npairs) xv = reinterpret_cast<const double2*>(a.x)[jp];
    bad |= !pair_in_range(xv.x) || !pair_in_range(xv.y);
    const Pair p0 = split_f64(xv.x), p1 = split_f64(xv.y);
    xh[k][0] = p0.h;
    xl[k][0] = p0.l;
    xh[k][1] = p1.h;
    xl[k][1] = p1.l;
  }
  const double fb = a.seed ? *a.seed : 1.0;
  if (FUSED) bad |= !pair_in_range(2.0 * fb);
  if (bad) set_error(a.err, ERRBIT_RANGE);
  const Pair fb2 = split_f64(2.0 * fb);

  Acc xb[PPT][2];
#pragma unroll
  for (int k = 0; k < PPT; ++k) xb[k][0] = xb[k][1] = acc_zero();
  Acc facc = acc_zero();

  for (int it = 0; it < nrows; ++it) {
    const int s = it & 1;
    const bool ok = mbar_wait_bounded(&full[s], (it >> 1) & 1);
    double2* rowd = reinterpret_cast<double2*>(s ? stage1 : stage0);
    float4* rowf = reinterpret_cast<float4*>(rowd);
    Acc yc[4] = {acc_zero(), acc_zero(), acc_zero(), acc_zero()};  // independent chains
    if (ok) {
#pragma unroll
      for (int k = 0; k < PPT; ++k) {
        const int jp = t + QP_CT * k;
        if (jp < npairs) {
          Pair p0, p1;
          if (PREP) {
            const float4 q = rowf[jp];
            p0 = Pair{q.x, q.y};
            p1 = Pair{q.z, q.w};
          } else {
            const double2 v = rowd[jp];
            p0 = split_f64(v.x);
            p1 = split_f64(v.y);
            if (FUSED) rowf[jp] = make_float4(p0.h, p0.l, p1.h, p1.l);
          }
          acc_fma(yc[2 * (k & 1)], p0.h, p0.l, xh[k][0], xl[k][0]);
          acc_fma(yc[2 * (k & 1) + 1], p1.h, p1.l, xh[k][1], xl[k][1]);
        }
      }
    }
    Acc yv = acc_add(acc_add(yc[0], yc[1]), acc_add(yc[2], yc[3]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) yv = acc_add(yv, shfl_xor_acc(yv, o));
    if (lane == 0) red[(it & 1) * QP_CW + warp] = yv;
    // all consumers: partials written; the OR tells everyone whether a wait gave up
    if (named_barrier_or(QP_BAR, QP_CT, !ok)) {
      if (lane == 0 && warp == 0) set_error(a.err, ERRBIT_TIMEOUT);
      *abort_flag = 1;
      break;
    }
    Acc ya = lane < QP_CW ? red[(it & 1) * QP_CW + lane] : acc_zero();
#pragma unroll
    for (int o = QP_CW / 2; o > 0; o >>= 1) ya = acc_add(ya, shfl_xor_acc(ya, o));
    // lanes 0..15 now hold the row total; give it to the whole warp
    ya.s = __shfl_sync(0xffffffffu, ya.s, 0);
    ya.l = __shfl_sync(0xffffffffu, ya.l, 0);
    const Pair y = acc_pair(ya);
    if (t == 0) {  // f in pair arithmetic: no FP64 instruction in the row loop
      const Pair y2 = pair_mul(y, y);
      facc = acc_add(facc, Acc{y2.h, y2.l});
    }
    if (FUSED) {
      const Pair yb = pair_mul(fb2, y);
#pragma unroll
      for (int k = 0; k < PPT; ++k) {
        const int jp = t + QP_CT * k;
        if (jp < npairs) {
          const float4 q = rowf[jp];
          acc_fma(xb[k][0], q.x, q.y, yb.h, yb.l);
          acc_fma(xb[k][1], q.z, q.w, yb.h, yb.l);
        }
      }
      if ((it & 15) == 15) {
#pragma unroll
        for (int k = 0; k < PPT; ++k) {
          acc_renorm(xb[k][0]);
          acc_renorm(xb[k][1]);
        }
      }
      if (!PREP) fence_proxy_async_smem();  // split values were written with generic stores
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty[s]);
    if (threadIdx.x == 0 && it + 2 < nrows && !*abort_flag) {
      if (!mbar_wait_bounded(&empty[s], (it >> 1) & 1)) {
        set_error(a.err, ERRBIT_TIMEOUT);
        *abort_flag = 1;
      } else {
        const double* src = a.A + (r0 + it + 2) * (int64_t)n;
        mbar_arrive_expect_tx(&full[s], row_bytes);
        tma_load_1d(s ? stage1 : stage0, src, row_bytes, &full[s]);
        ++issued;
        if (it + 4 < nrows) prefetch_l2_bulk(src + 2 * (int64_t)n, row_bytes);
      }
    }
    __syncwarp();
  }
  // do not leave with a copy into this CTA's shared memory in flight
  if (threadIdx.x == 0) {
    for (int st = 0; st < 2; ++st) {
      const int last = issued - 1 - ((issued - 1 - st) & 1);  // last row copied into stage st
      if (last >= 0) mbar_wait_bounded(&full[st], (last >> 1) & 1);
    }
  }

  if (FUSED) {
    float4* out = a.partials + (int64_t)blockIdx.x * npairs;
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
      const int jp = t + QP_CT * k;
      if (jp < npairs) {
        const Pair p0 = acc_pair(xb[k][0]), p1 = acc_pair(xb[k][1]);
        out[jp] = make_float4(p0.h, p0.l, p1.h, p1.l);
      }
    }
    if (t == 0) a.fpart[blockIdx.x] = acc_to_double(facc);
  } else if (t == 0) {
    // last CTA to arrive sums the f partials in CTA order
    a.fpart[blockIdx.x] = acc_to_double(facc);
    __threadfence();
    const unsigned arrived = atomicAdd(a.counter, 1u);
    if (arrived == gridDim.x - 1) {
      __threadfence();
      double tot = 0.0;
      for (int i = 0; i < (int)gridDim.x; ++i) tot += __ldcg(&a.fpart[i]);
      *a.f = tot;
      *a.counter = 0u;
    }
  }
}

// Warp-specialized fused value+gradient on the prepared A, for 2048 < n <= 10240.
// All warps of qf_pair_kernel meet at the per-row barrier and then run the
// row's latency-bound reduction together; here the work is split by role so
// that one role's reduction overlaps the other's streaming FMAs:
//   - warps 0..6 (dot): hold x as float pairs, column pairs jp = t + 224 k
//     (k < KPD); each warp's partial of y_i goes to a two-row buffer and a
//     y-ready mbarrier;
//   - warps 7..14 (update): hold xbar, column pairs jp = t + 256 k (k < KP);
//     for row i they sum the 7 partials in warp order, then accumulate
//     xbar_j += 2 fbar y_i A_ij chunk by chunk and release each chunk;
//   - warp 15 (lane 0): issues the TMA copies.
// Rows stream in two chunks, pairs [0, H) and [H, n/2) with H = 128 KP, through a
// ring of WS_SLOTS chunk slots: the row being updated, the row being reduced
// and the next copy fit in shared memory.  From the ring depth (5 slots, 2
// chunks a row): the dot warps reach row i + 2 only after the slot of row i's
// first chunk was refilled, i.e. after the update warps read row i's partials,
// so the two-row partial buffer and each y-ready barrier are never more than
// one phase ahead.  All waits are bounded and report KG_ERR_TIMEOUT.
// The ring starts zeroed and a copy fills only the first n/2 - H pairs of a
// row's second chunk, so every slot holds zeros or finite entries of A beyond
// the row's end: the loops read there without a bounds test (x is zero there,
// and the xbar entries past the row's end are never stored).  Only the dot
// warps' last column pair can reach past the second chunk's slot; it keeps its
// test.
constexpr int WS_DW = 7, WS_UW = 8;             // dot and update warps
constexpr int WS_THREADS = (WS_DW + WS_UW + 1) * 32;
constexpr int WS_SLOTS = 5;

// Fixed-order sum of the per-CTA float-pair partials over column pairs
// [j0, j1), by a CTA of 512 threads: thread (cx, py), py < 15, adds partials
// py, py + 15, ... of column pair cx of each block of 34 (twelve loads in
// flight); the 15 sums are added in py order and converted to double once per
// column.  Threads 510 and 511 only join the barriers.  The order depends on
// neither the CTA nor the range, so the fused kernel's tail and the separate
// reduce kernel give the same bits.
constexpr int RED_CX = 34, RED_PY = 15, RED_LOADS = 12;

__device__ __forceinline__ void reduce_pair_columns(const float4* partials, int nparts, int npairs,
                                                    int j0, int j1, double* gx, int accumulate,
                                                    Acc (*red)[RED_CX][2]) {
  const int cx = threadIdx.x % RED_CX, py = threadIdx.x / RED_CX;
  for (int jb = j0; jb < j1; jb += RED_CX) {
    const int jp = jb + cx;
    Acc s0 = acc_zero(), s1 = acc_zero();
    if (py < RED_PY && jp < j1) {
      for (int c = py; c < nparts; c += RED_LOADS * RED_PY) {
        float4 v[RED_LOADS];
#pragma unroll
        for (int u = 0; u < RED_LOADS; ++u)
          if (c + RED_PY * u < nparts) v[u] = __ldcg(partials + (int64_t)(c + RED_PY * u) * npairs + jp);
#pragma unroll
        for (int u = 0; u < RED_LOADS; ++u)
          if (c + RED_PY * u < nparts) {
            s0 = acc_add(s0, Acc{v[u].x, v[u].y});
            s1 = acc_add(s1, Acc{v[u].z, v[u].w});
          }
      }
    }
    if (py < RED_PY) {
      red[py][cx][0] = s0;
      red[py][cx][1] = s1;
    }
    __syncthreads();
    if (py == 0 && jp < j1) {
      Acc t0 = red[0][cx][0], t1 = red[0][cx][1];
#pragma unroll
      for (int g = 1; g < RED_PY; ++g) {
        t0 = acc_add(t0, red[g][cx][0]);
        t1 = acc_add(t1, red[g][cx][1]);
      }
      const double g0 = pair_to_double(acc_pair(t0)), g1 = pair_to_double(acc_pair(t1));
      double2* o = reinterpret_cast<double2*>(gx) + jp;
      if (accumulate) {
        const double2 old = *o;
        *o = make_double2(old.x + g0, old.y + g1);
      } else {
        *o = make_double2(g0, g1);
      }
    }
    __syncthreads();
  }
}

// The f partials' sum, by all threads of a CTA (the same order in both paths).
__device__ __forceinline__ void reduce_f_partials(const double* fpart, int nparts, double* f, double* scratch) {
  double fs = 0.0;
  for (int i = threadIdx.x; i < nparts; i += blockDim.x) fs += __ldcg(fpart + i);
  fs = block_sum(fs, scratch);
  if (threadIdx.x == 0) *f = fs;
}

// The partials' reduction as the tail of the fused kernel (a cooperative
// launch: every CTA is resident).  Each CTA counts itself in (a.counter[2])
// once its partials and f partial are written and waits, bounded, until all
// have.  With more than one CTA, CTA 0 sums the f partials while CTAs 1 ..
// grid - 1 sum their shares of the column pairs, [(b - 1) npairs / (grid - 1),
// b npairs / (grid - 1)) (at most 34 pairs, one block, for n <= 10336 on 152
// CTAs); a single CTA does both.  The last CTA to count itself out
// (a.counter[3]) resets both counters for the next launch.
__device__ __forceinline__ void ws_grid_reduce(const QpArgs& a, int npairs) {
  static_assert(WS_THREADS == 512, "reduce_pair_columns takes 512 threads");
  __shared__ Acc red[RED_PY][RED_CX][2];
  __shared__ double fred[32];
  __shared__ int go;
  if (threadIdx.x == 0) go = grid_arrive_and_wait(a.counter + 2, a.err, ERRBIT_TIMEOUT);
  __syncthreads();
  if (go) {
    const int nparts = gridDim.x;
    const int cols = nparts > 1 ? nparts - 1 : 1, b = nparts > 1 ? (int)blockIdx.x - 1 : 0;
    if (b >= 0) {
      const int j0 = (int)((int64_t)b * npairs / cols), j1 = (int)((int64_t)(b + 1) * npairs / cols);
      reduce_pair_columns(a.partials, nparts, npairs, j0, j1, a.gx, a.accumulate, red);
    }
    if (blockIdx.x == 0 && a.f) reduce_f_partials(a.fpart, nparts, a.f, fred);
  }
  if (threadIdx.x == 0) grid_depart(a.counter + 2, a.counter + 3);
}

template <int KP, bool GRIDRED>
__global__ void __launch_bounds__(WS_THREADS, 1) qf_pair_ws_kernel(QpArgs a) {
  extern __shared__ __align__(128) unsigned char smem[];
  constexpr int H = 128 * KP;                       // column pairs of a chunk slot
  constexpr int TD = WS_DW * 32, TU = WS_UW * 32;   // 224 and 256 threads
  constexpr int KPD = (KP * TU + TD - 1) / TD;      // dot pairs per thread
  const int n = a.n, npairs = n >> 1;
  float4* slots = reinterpret_cast<float4*>(smem);
  uint64_t* full = reinterpret_cast<uint64_t*>(slots + WS_SLOTS * H);
  uint64_t* empty = full + WS_SLOTS;
  uint64_t* yready = empty + WS_SLOTS;                      // [2]
  Acc* dpart = reinterpret_cast<Acc*>(yready + 2);         // [2][8]
  volatile int* abort_flag = reinterpret_cast<volatile int*>(dpart + 16);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t r0 = (int64_t)blockIdx.x * a.band;
  const int64_t r1 = r0 + a.band < a.m ? r0 + a.band : a.m;
  const int nrows = r1 > r0 ? (int)(r1 - r0) : 0;
  const int nchunks = 2 * nrows;

  if (threadIdx.x == 0) {
    for (int i = 0; i < WS_SLOTS; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], WS_UW);
    }
    mbar_init(&yready[0], WS_DW);
    mbar_init(&yready[1], WS_DW);
    *abort_flag = 0;
    fence_barrier_init();
  }
  for (int i = threadIdx.x; i < WS_SLOTS * H; i += WS_THREADS) slots[i] = make_float4(0.f, 0.f, 0.f, 0.f);
  fence_proxy_async_smem();  // the zeros are written before any copy lands in the ring
  __syncthreads();

  if (warp < WS_DW) {
    // ------------------------------------------------------------- dot role
    const int t = threadIdx.x;
    float xh[KPD][2], xl[KPD][2];
    bool bad = false;
#pragma unroll
    for (int k = 0; k < KPD; ++k) {
      const int jp = t + TD * k;
      double2 xv = make_double2(0.0, 0.0);
      if (jp < npairs) xv = reinterpret_cast<const double2*>(a.x)[jp];
      bad |= !pair_in_range(xv.x) || !pair_in_range(xv.y);
      const Pair p0 = split_f64(xv.x), p1 = split_f64(xv.y);
      xh[k][0] = p0.h;
      xl[k][0] = p0.l;
      xh[k][1] = p1.h;
      xl[k][1] = p1.l;
    }
    if (bad) set_error(a.err, ERRBIT_RANGE);
    for (int r = 0; r < nrows; ++r) {
      if (*abort_flag) break;
      const int s0 = (2 * r) % WS_SLOTS, s1 = (2 * r + 1) % WS_SLOTS;
      bool ok = mbar_wait_bounded(&full[s0], (uint32_t)((2 * r) / WS_SLOTS) & 1u);
      ok = ok && mbar_wait_bounded(&full[s1], (uint32_t)((2 * r + 1) / WS_SLOTS) & 1u);
      if (!__all_sync(0xffffffffu, ok)) {
        if (lane == 0) set_error(a.err, ERRBIT_TIMEOUT);
        *abort_flag = 1;
        break;
      }
      const float4* buf0 = slots + s0 * H;
      const float4* buf1 = slots + s1 * H;
      Acc yc[4] = {acc_zero(), acc_zero(), acc_zero(), acc_zero()};
#pragma unroll
      for (int k = 0; k < KPD; ++k) {
        const int jp = t + TD * k;
        if (TD * (k + 1) <= 2 * H || jp < 2 * H) {  // the test is compiled for the last k only
          // which chunk: known at compile time for all k but the one whose
          // threads straddle the chunk boundary
          const float4 q = TD * (k + 1) <= H ? buf0[jp]
                           : TD * k >= H     ? buf1[jp - H]
                                             : (jp < H ? buf0[jp] : buf1[jp - H]);
          acc_fma(yc[2 * (k & 1)], q.x, q.y, xh[k][0], xl[k][0]);
          acc_fma(yc[2 * (k & 1) + 1], q.z, q.w, xh[k][1], xl[k][1]);
        }
      }
      Acc yv = acc_add(acc_add(yc[0], yc[1]), acc_add(yc[2], yc[3]));
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) yv = acc_add(yv, shfl_xor_acc(yv, o));
      if (lane == 0) {
        dpart[(r & 1) * 8 + warp] = yv;
        mbar_arrive(&yready[r & 1]);
      }
      __syncwarp();
    }
  } else if (warp < WS_DW + WS_UW) {
    // ---------------------------------------------------------- update role
    const int t = threadIdx.x - TD;
    const double fb = a.seed ? *a.seed : 1.0;
    if (t == 0 && !pair_in_range(2.0 * fb)) set_error(a.err, ERRBIT_RANGE);
    const Pair fb2 = split_f64(2.0 * fb);
    Acc xb[KP][2];
#pragma unroll
    for (int k = 0; k < KP; ++k) xb[k][0] = xb[k][1] = acc_zero();
    Acc facc = acc_zero();
    for (int r = 0; r < nrows; ++r) {
      if (*abort_flag) break;
      bool ok = mbar_wait_bounded(&yready[r & 1], (uint32_t)(r >> 1) & 1u);
      if (!__all_sync(0xffffffffu, ok)) {
        if (lane == 0) set_error(a.err, ERRBIT_TIMEOUT);
        *abort_flag = 1;
        break;
      }
      Acc ya = dpart[(r & 1) * 8];
#pragma unroll
      for (int w = 1; w < WS_DW; ++w) ya = acc_add(ya, dpart[(r & 1) * 8 + w]);
      const Pair y = acc_pair(ya);
      if (t == 0) {
        const Pair y2 = pair_mul(y, y);
        facc = acc_add(facc, Acc{y2.h, y2.l});
      }
      const Pair yb = pair_mul(fb2, y);
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        const int g = 2 * r + c, slot = g % WS_SLOTS;
        // completed before the dot warps published y_i; the wait orders the copy's data
        ok = ok && mbar_wait_bounded(&full[slot], (uint32_t)(g / WS_SLOTS) & 1u);
        if (ok) {
          const float4* buf = slots + slot * H;
#pragma unroll
          for (int kk = 0; kk < KP / 2; ++kk) {
            const int k = c * (KP / 2) + kk;
            const float4 q = buf[t + TU * kk];
            acc_fma(xb[k][0], q.x, q.y, yb.h, yb.l);
            acc_fma(xb[k][1], q.z, q.w, yb.h, yb.l);
          }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[slot]);
      }
      if (!__all_sync(0xffffffffu, ok)) {
        if (lane == 0) set_error(a.err, ERRBIT_TIMEOUT);
        *abort_flag = 1;
        break;
      }
      if ((r & 15) == 15) {
#pragma unroll
        for (int k = 0; k < KP; ++k) {
          acc_renorm(xb[k][0]);
          acc_renorm(xb[k][1]);
        }
      }
    }
    float4* out = a.partials + (int64_t)blockIdx.x * npairs;
#pragma unroll
    for (int k = 0; k < KP; ++k) {
      const int jp = t + TU * k;
      if (jp < npairs) {
        const Pair p0 = acc_pair(xb[k][0]), p1 = acc_pair(xb[k][1]);
        out[jp] = make_float4(p0.h, p0.l, p1.h, p1.l);
      }
    }
    if (t == 0) a.fpart[blockIdx.x] = acc_to_double(facc);
  } else if (lane == 0) {
    // ----------------------------------------------------- producer (TMA)
    const uint32_t c0 = (uint32_t)H * 16u, c1 = (uint32_t)(npairs - H) * 16u;
    const uint32_t row_bytes = (uint32_t)n * 8u;
    int issued = 0;
    for (int g = 0; g < nchunks; ++g) {
      if (*abort_flag) break;
      const int slot = g % WS_SLOTS;
      if (g >= WS_SLOTS && !mbar_wait_bounded(&empty[slot], (uint32_t)(g / WS_SLOTS - 1) & 1u)) {
        set_error(a.err, ERRBIT_TIMEOUT);
        *abort_flag = 1;
        break;
      }
      const int r = g >> 1, c = g & 1;
      const double* row = a.A + (r0 + r) * (int64_t)n;
      mbar_arrive_expect_tx(&full[slot], c ? c1 : c0);
      tma_load_1d(slots + slot * H, row + (c ? 2 * H : 0), c ? c1 : c0, &full[slot]);
      ++issued;
      if (c == 0 && r + 2 < nrows) prefetch_l2_bulk(row + 2 * (int64_t)n, row_bytes);
    }
    // do not leave with a copy into this CTA's shared memory in flight
    for (int g = issued - WS_SLOTS > 0 ? issued - WS_SLOTS : 0; g < issued; ++g)
      mbar_wait_bounded(&full[g % WS_SLOTS], (uint32_t)(g / WS_SLOTS) & 1u);
  }
  __syncwarp();
  __syncthreads();
  if constexpr (GRIDRED) ws_grid_reduce(a, npairs);
}

// The same reduction as a separate kernel: block b sums column pairs
// [34 b, 34 b + 34); block 0 also writes f.
__global__ void __launch_bounds__(512) qf_pair_reduce_kernel(const float4* __restrict__ partials,
                                                             int nparts, int npairs,
                                                             const double* __restrict__ fpart,
                                                             double* gx, double* f, int accumulate) {
  __shared__ Acc red[RED_PY][RED_CX][2];
  __shared__ double fred[32];
  // launched as a programmatic dependent of the fused kernel: wait until that
  // grid has completed and its partials are visible
  grid_dependency_wait();
  const int j0 = blockIdx.x * RED_CX;
  reduce_pair_columns(partials, nparts, npairs, j0, min(j0 + RED_CX, npairs), gx, accumulate, red);
  if (blockIdx.x == 0 && f) reduce_f_partials(fpart, nparts, f, fred);
}

// The prepared copy of A: every double split into its float pair (h, l).
// count doubles; an odd count's last one is split by thread 0 of block 0.
__global__ void pair_prepare_kernel(const double2* __restrict__ A, float4* __restrict__ out,
                                    int64_t count) {
  const int64_t n2 = count / 2, stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n2; i += stride) {
    const double2 v = __ldcs(A + i);
    const Pair p0 = split_f64(v.x), p1 = split_f64(v.y);
    __stcs(out + i, make_float4(p0.h, p0.l, p1.h, p1.l));
  }
  if ((count & 1) && blockIdx.x == 0 && threadIdx.x == 0) {
    const Pair q = split_f64(reinterpret_cast<const double*>(A)[count - 1]);
    reinterpret_cast<float2*>(out)[count - 1] = make_float2(q.h, q.l);
  }
}

// Sets ERRBIT_RANGE when some entry is outside the pair arithmetic's range.
// count doubles; an odd count's last one is checked by thread 0 of block 0.
__global__ void pair_range_scan_kernel(const double2* __restrict__ p, int64_t count, unsigned* err) {
  bool bad = false;
  const int64_t n2 = count / 2, stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n2; i += stride) {
    const double2 v = __ldcs(p + i);
    bad |= !pair_in_range(v.x) || !pair_in_range(v.y);
  }
  if ((count & 1) && blockIdx.x == 0 && threadIdx.x == 0)
    bad |= !pair_in_range(reinterpret_cast<const double*>(p)[count - 1]);
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) set_error(err, ERRBIT_RANGE);
}

// ---------------------------------------------------------------- host ----
static int pair_ppt(int64_t n) {
  const int64_t need = (n / 2 + QP_CT - 1) / QP_CT;
  for (int p : {1, 2, 4, 6, 8, 10, 12})
    if (need <= p) return p;
  return -1;
}

bool qf_pair_supported(const kg_problem* p) {
  return p->dtype == KG_F64 && (p->n % 2) == 0 && pair_ppt(p->n) > 0 &&
         (p->strategy == KG_STRATEGY_FUSED || p->strategy == KG_STRATEGY_AUTO);
}

static size_t pair_smem(int n) {
  return (size_t)2 * n * 8 + 4 * 8 + 2 * QP_CW * sizeof(Acc) + 16;
}

// Scans `count` doubles once (create time) for values outside the pair range;
// *ok is true if every value is representable.  data: 16-byte aligned.
kg_status pair_range_ok(kg_problem* p, const double* data, int64_t count, cudaStream_t s, bool* ok) {
  const int64_t n2 = (count + 1) / 2;
  cudaError_t e = cudaMemsetAsync(p->err, 0, sizeof(unsigned), s);
  if (e != cudaSuccess) return cuda_fail(e, "pair range scan");
  int grid = (int)std::min<int64_t>((n2 + 255) / 256, (int64_t)num_sms() * 8);
  pair_range_scan_kernel<<<std::max(grid, 1), 256, 0, s>>>(reinterpret_cast<const double2*>(data),
                                                         count, p->err);
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "pair range scan");
  unsigned h = 0;
  if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_fail(e, "pair range scan");
  if ((e = cudaMemcpy(&h, p->err, sizeof(h), cudaMemcpyDeviceToHost)) != cudaSuccess)
    return cuda_fail(e, "pair range scan");
  if ((e = cudaMemsetAsync(p->err, 0, sizeof(unsigned), s)) != cudaSuccess)
    return cuda_fail(e, "pair range scan");
  *ok = (h & ERRBIT_RANGE) == 0;
  return KG_OK;
}

kg_status qf_pair_range_ok(kg_problem* p, cudaStream_t s, bool* ok) {
  return pair_range_ok(p, static_cast<const double*>(p->data0), p->m * p->n, s, ok);
}

int qf_pair_grid(const kg_problem* p, int* band) {
  const int64_t g = std::min<int64_t>(p->m, num_sms());
  const int64_t b = (p->m + g - 1) / g;
  *band = (int)b;
  return (int)((p->m + b - 1) / b);
}

template <int PPT, bool FUSED, bool PREP>
static cudaError_t launch_pair(int grid, size_t smem, cudaStream_t s, const QpArgs& a) {
  auto kern = qf_pair_kernel<PPT, FUSED, PREP>;
  cudaError_t e = set_smem_once(kern, smem);
  if (e != cudaSuccess) return e;
  kern<<<grid, QP_THREADS, smem, s>>>(a);
  return cudaGetLastError();
}

template <bool FUSED, bool PREP>
static cudaError_t dispatch_ppt(int ppt, int grid, size_t smem, cudaStream_t s, const QpArgs& a) {
  switch (ppt) {
    case 1: return launch_pair<1, FUSED, PREP>(grid, smem, s, a);
    case 2: return launch_pair<2, FUSED, PREP>(grid, smem, s, a);
    case 4: return launch_pair<4, FUSED, PREP>(grid, smem, s, a);
    case 6: return launch_pair<6, FUSED, PREP>(grid, smem, s, a);
    case 8: return launch_pair<8, FUSED, PREP>(grid, smem, s, a);
    case 10: return launch_pair<10, FUSED, PREP>(grid, smem, s, a);
    case 12: return launch_pair<12, FUSED, PREP>(grid, smem, s, a);
  }
  return cudaErrorInvalidValue;
}

template <bool FUSED>
static cudaError_t dispatch_pair(bool prep, int ppt, int grid, size_t smem, cudaStream_t s,
                                 const QpArgs& a) {
  return prep ? dispatch_ppt<FUSED, true>(ppt, grid, smem, s, a)
              : dispatch_ppt<FUSED, false>(ppt, grid, smem, s, a);
}

// Prepared copy of A (float pairs, 8 bytes per entry) when it fits the
// problem's workspace budget; later calls stream it instead of A.
kg_status qf_pair_prepare(kg_problem* p, cudaStream_t s) {
  const size_t bytes = 8 * (size_t)p->m * (size_t)p->n;
  const size_t budget = p->opt.tape_budget_bytes ? p->opt.tape_budget_bytes : (size_t(1) << 30);
  if (bytes > budget) return KG_OK;
  kg_status rc = ws_alloc(p, &p->aprep, bytes, "prepared A (float pairs)");
  if (rc != KG_OK) return rc;
  return pair_prepare(static_cast<const double*>(p->data0), p->aprep, (int64_t)p->m * p->n, s);
}

kg_status pair_prepare(const double* src, void* dst, int64_t count, cudaStream_t s) {
  const int64_t n2 = (count + 1) / 2;
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((n2 + 255) / 256, (int64_t)num_sms() * 8));
  pair_prepare_kernel<<<grid, 256, 0, s>>>(reinterpret_cast<const double2*>(src),
                                           static_cast<float4*>(dst), count);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? KG_OK : cuda_fail(e, "prepare float pairs");
}

static QpArgs pair_args(kg_problem* p, const void* x, const void* seed) {
  QpArgs a{};
  a.A = static_cast<const double*>(p->aprep ? p->aprep : p->data0);
  a.x = static_cast<const double*>(x);
  a.m = p->m;
  a.n = (int)p->n;
  a.band = p->qf.rows_per_cta;
  a.seed = static_cast<const double*>(seed);
  a.partials = static_cast<float4*>(p->partials);
  a.fpart = p->fpart;
  a.counter = p->counter;
  a.err = p->err;
  return a;
}

kg_status qf_pair_eval(kg_problem* p, const void* x, void* f, cudaStream_t s) {
  if ((reinterpret_cast<uintptr_t>(x) & 15u) != 0)
    return fail(KG_ERR_INVALID_ARG, "QUADFORM pair kernels need a 16-byte aligned x");
  QpArgs a = pair_args(p, x, nullptr);
  a.f = static_cast<double*>(f);
  prof_begin(s, p->aprep ? "qf_pair_kernel<eval, prepared A>" : "qf_pair_kernel<eval>");
  cudaError_t e = dispatch_pair<false>(p->aprep != nullptr, pair_ppt(p->n), p->qf.grid,
                                       pair_smem((int)p->n), s, a);
  prof_end(s);
  count_launch();
  return e == cudaSuccess ? KG_OK : cuda_fail(e, "qf pair forward kernel");
}

// Column pairs per role thread of qf_pair_ws_kernel (0: not used for this n).
static int ws_kp(const kg_problem* p) {
  if (!p->aprep || p->n <= 2048 || p->n > 10240) return 0;
  return 4 * (int)((p->n / 2 + 1023) / 1024);
}

static size_t ws_smem(int kp) {
  return (size_t)WS_SLOTS * 128 * kp * 16 + (2 * WS_SLOTS + 2) * 8 + 16 * sizeof(Acc) + 16;
}

// fused: the partials' reduction runs in the kernel's tail (ws_grid_reduce),
// which needs every CTA resident at once: a cooperative launch, which the
// runtime refuses when the grid does not fit.
template <int KP>
static cudaError_t launch_ws(int grid, cudaStream_t s, const QpArgs& a, bool fused) {
  const size_t smem = ws_smem(KP);
  cudaError_t e;
  if (fused) {
    auto kern = qf_pair_ws_kernel<KP, true>;
    if ((e = set_smem_once(kern, smem)) != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(WS_THREADS);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, a);
  }
  auto kern = qf_pair_ws_kernel<KP, false>;
  if ((e = set_smem_once(kern, smem)) != cudaSuccess) return e;
  kern<<<grid, WS_THREADS, smem, s>>>(a);
  return cudaGetLastError();
}

static cudaError_t dispatch_ws(int kp, int grid, cudaStream_t s, const QpArgs& a, bool fused) {
  switch (kp) {
    case 8: return launch_ws<8>(grid, s, a, fused);
    case 12: return launch_ws<12>(grid, s, a, fused);
    case 16: return launch_ws<16>(grid, s, a, fused);
    case 20: return launch_ws<20>(grid, s, a, fused);
  }
  return cudaErrorInvalidValue;
}

template <int KP>
static bool ws_coop_fits(int grid) {
  int dev = 0, coop = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess || !coop)
    return false;
  auto kern = qf_pair_ws_kernel<KP, true>;
  if (set_smem_once(kern, ws_smem(KP)) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, WS_THREADS, ws_smem(KP)) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return (int64_t)per_sm * num_sms() >= grid;
}

bool qf_pair_coop_fits(const kg_problem* p) {
  if (const char* env = std::getenv("KG_TEST_NO_COOP"))
    if (std::atoi(env) == 1) return false;
  switch (ws_kp(p)) {
    case 8: return ws_coop_fits<8>(p->qf.grid);
    case 12: return ws_coop_fits<12>(p->qf.grid);
    case 16: return ws_coop_fits<16>(p->qf.grid);
    case 20: return ws_coop_fits<20>(p->qf.grid);
  }
  return false;
}

kg_status qf_pair_grad(kg_problem* p, const void* x, void* f, void* gx, const void* seed,
                       int accumulate, cudaStream_t s) {
  if ((reinterpret_cast<uintptr_t>(x) & 15u) != 0 || (reinterpret_cast<uintptr_t>(gx) & 15u) != 0)
    return fail(KG_ERR_INVALID_ARG, "QUADFORM pair kernels need 16-byte aligned x and gx");
  QpArgs a = pair_args(p, x, seed);
  const int kp = ws_kp(p);
  cudaError_t e;
  if (kp && p->qf.coop) {
    // one launch: the partials' reduction in the kernel's tail
    a.gx = static_cast<double*>(gx);
    a.f = static_cast<double*>(f);
    a.accumulate = accumulate;
    prof_begin(s, "qf_pair_ws_kernel<fused, prepared A, grid reduction>");
    e = dispatch_ws(kp, p->qf.grid, s, a, true);
    prof_end(s);
    count_launch();
    if (e == cudaSuccess) return KG_OK;
    if (e != cudaErrorCooperativeLaunchTooLarge) return cuda_fail(e, "qf pair fused kernel");
    cudaGetLastError();  // the grid is not resident at once here: two launches from now on
    p->qf.coop = 0;
    a.gx = nullptr;
    a.f = nullptr;
  }
  prof_begin(s, kp ? "qf_pair_ws_kernel<fused, prepared A>"
                  : p->aprep ? "qf_pair_kernel<fused, prepared A>" : "qf_pair_kernel<fused>");
  e = kp ? dispatch_ws(kp, p->qf.grid, s, a, false)
         : dispatch_pair<true>(p->aprep != nullptr, pair_ppt(p->n), p->qf.grid,
                               pair_smem((int)p->n), s, a);
  prof_end(s);
  count_launch();
  if (e != cudaSuccess) return cuda_fail(e, "qf pair fused kernel");
  const int npairs = (int)(p->n / 2);
  // programmatic dependent launch: the reduce kernel's launch overlaps the fused
  // kernel's last CTAs; it waits for that grid's completion before reading
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((npairs + RED_CX - 1) / RED_CX);
  cfg.blockDim = dim3(512);
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  e = cudaLaunchKernelEx(&cfg, qf_pair_reduce_kernel, static_cast<const float4*>(p->partials),
                         p->qf.grid, npairs, static_cast<const double*>(p->fpart),
                         static_cast<double*>(gx), static_cast<double*>(f), accumulate);
  count_launch();
  if (e != cudaSuccess) return cuda_fail(e, "qf pair reduce kernel");
  return KG_OK;
}

}  // namespace kg
