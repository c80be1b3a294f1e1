// Tet-mesh energy kernels for FP64 data and the staged variants.
//
// Which kernel runs:
//   - FP64 in float pairs from the prepared G (the default), without bounds
//     checks, any strategy but SHARED: tet_direct_pair_kernel, one element per
//     thread per step with G read straight from global memory (the forward is
//     latency-bound on its gathers; staging would cap occupancy);
//   - FP32 without bounds checks, any strategy but SHARED: the direct FP32
//     kernel in tet.cu;
//   - everything else (native FP64, bounds checks, the SHARED strategy, pair
//     arithmetic without a prepared G): tet_staged_kernel below.
//
// tet_staged_kernel: each CTA walks tiles of 256 elements (tile = blockIdx.x, + gridDim.x, ...).
// Thread 0 streams each tile's connectivity (int4 per element) and G_e
// (12 values per element) into a shared-memory ring (3 stages FP32, 2 FP64) with TMA bulk
// copies (cp.async.bulk, mbarrier transaction counts); warps release a stage
// through an "empty" mbarrier and thread 0 refills it.  Thread i of the CTA
// handles element i of the tile: gathers u_e (4 reads through the index map,
// mostly L2 hits), computes g_e = G_e u_e, f_e = log1p(|g_e|^2) and, in the
// reverse modes, c_e = G_e^T (2 fbar g_e / (1 + |g_e|^2)), which it either
// scatter-adds into gu (FP64/FP32 atomics) or stores to the tape.
//
// KG_STRATEGY_SHARED: the scatter-adds of a tile are first combined per vertex
// in a shared-memory hash table (two tables, used by alternate tiles); after
// one CTA barrier per tile the table is added into gu with one global atomic
// per distinct vertex and emptied.  With elements numbered along the mesh a
// tile of 256 tets of the Kuhn grid touches ~180 distinct vertices for its
// 1024 contributions, so global atomics drop ~5x.
//
// KG_STRATEGY_WARP: the four contributions of each lane stay in registers;
// per local vertex slot k, consecutive lanes holding the same global vertex
// add their values by a segmented scan in float pairs (warp_combine) and the
// first lane of each run issues one global reduction.  No shared memory and
// no CTA barrier; on the Kuhn grid (six consecutive tets share the cube's
// diagonal ends in slots 0 and 3) global reductions drop ~2x.
//
// Arithmetic: FP32 for FP32 problems; for FP64 problems either native FP64
// or float pairs (kg_pair.cuh) with the results converted back to double for
// the atomics / tape (KG_ARITH_PAIR: GB300's FP64 units are ~60x slower than
// its FP32 units).  All waits are bounded.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <mutex>
#include <string>
#include <type_traits>

#include "kg_device.cuh"
#include "kg_internal.h"
#include "kg_pair.cuh"
#include "kg_tet_elem.cuh"

namespace kg {

constexpr int TS_THREADS = 256;  // threads per CTA == elements per tile
constexpr int TS_WARPS = TS_THREADS / 32;
// Shared-memory ring depth: 3 stages for the FP32 forward (16 KB each), else 2.
template <typename T, int MODE>
__host__ __device__ constexpr int ts_stages() { return sizeof(T) == 4 && MODE == TS_EVAL ? 3 : 2; }

// Slots of one shared-memory aggregation table (power of two, > 4 x TS_THREADS).
template <typename T>
__host__ __device__ constexpr int ts_hash_slots() { return 2048; }


template <typename T>
struct TsArgs {
  const int4* conn;
  const T* G;  // N_e x 12 values, or (PREP) N_e x 12 float pairs in the same bytes
  const T* u;
  const T* v;  // TS_HVP: the direction
  int64_t ne;
  int nv;
  const T* seed;
  T* gu;
  T* tape;
  double* fpart;
  unsigned* counter;
  T* f;
  unsigned* err;
  int check;
  const float4* logtab;  // PAIR: 256 entries
  LogConsts K;
};

// Scatter of the reverse pass (GRAD mode).
enum { SC_ATOMIC = 0, SC_SHARED = 1, SC_WARP = 2 };

template <typename T, bool PAIR, int MODE, int SCAT, bool PREP>
__global__ void __launch_bounds__(TS_THREADS) tet_staged_kernel(TsArgs<T> a) {
  constexpr bool SHARED = SCAT == SC_SHARED;
  constexpr bool REV = MODE == TS_GRAD || MODE == TS_HVP;  // scatters into gu
  constexpr bool WARPC = SCAT == SC_WARP && REV;
  constexpr int TS_STAGES = ts_stages<T, MODE>();
  extern __shared__ __align__(128) unsigned char smem[];
  constexpr uint32_t kConnBytes = TS_THREADS * 16u;
  constexpr uint32_t kGBytes = TS_THREADS * 12u * sizeof(T);
  constexpr uint32_t kStage = kConnBytes + kGBytes;
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + TS_STAGES * kStage);
  uint64_t* empty = full + TS_STAGES;
  float4* tab = reinterpret_cast<float4*>(empty + TS_STAGES);  // PAIR only
  double* red = reinterpret_cast<double*>(tab + (PAIR ? kLogTableSize : 0));
  volatile int* abort_flag = reinterpret_cast<volatile int*>(red + 2 * TS_WARPS);
  constexpr int kSlots = ts_hash_slots<T>();
  // SHARED: tables [2][kSlots] of values, then [2][kSlots] of keys
  T* hvals = reinterpret_cast<T*>(red + 2 * TS_WARPS + 2);
  int* hkeys = reinterpret_cast<int*>(hvals + (SHARED ? 2 * kSlots : 0));

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t ntiles = (a.ne + TS_THREADS - 1) / TS_THREADS;
  const int64_t my_tiles = blockIdx.x < ntiles ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;

  if (tid == 0) {
    for (int s = 0; s < TS_STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], TS_WARPS);
    }
    *abort_flag = 0;
    fence_barrier_init();
  }
  if constexpr (PAIR) {
    for (int i = tid; i < kLogTableSize; i += TS_THREADS) tab[i] = a.logtab[i];
  }
  if constexpr (SHARED) {
    for (int i = tid; i < 2 * kSlots; i += TS_THREADS) {
      hkeys[i] = -1;
      hvals[i] = T(0);
    }
  }
  __syncthreads();

  auto issue = [&](int64_t i, int s) {  // tile i of this CTA into stage s
    const int64_t tile = blockIdx.x + i * (int64_t)gridDim.x;
    const int64_t e0 = tile * TS_THREADS;
    const int64_t cnt = a.ne - e0 < TS_THREADS ? a.ne - e0 : TS_THREADS;
    unsigned char* st = smem + s * kStage;
    const uint32_t cb = (uint32_t)cnt * 16u, gb = (uint32_t)cnt * 12u * (uint32_t)sizeof(T);
    mbar_arrive_expect_tx(&full[s], cb + gb);
    tma_load_1d(st, a.conn + e0, cb, &full[s]);
    tma_load_1d(st + kConnBytes, a.G + e0 * 12, gb, &full[s]);
  };
  int64_t issued = 0;
  if (tid == 0) {
    for (int64_t i = 0; i < TS_STAGES && i < my_tiles; ++i) {
      issue(i, (int)i);
      ++issued;
    }
  }

  T facc_n = T(0);
  Acc facc_p = acc_zero();
  bool bad = false;
  const T fb = REV ? load_seed(a.seed) : T(1);
  Pair fb2{2.0f, 0.0f};
  if constexpr (PAIR) {
    if (REV) {
      bad |= !pair_in_range(2.0 * (double)fb);
      fb2 = split_f64(2.0 * (double)fb);
    }
  }

  for (int64_t i = 0; i < my_tiles; ++i) {
    const int s = (int)(i % TS_STAGES);
    const uint32_t par = (uint32_t)((i / TS_STAGES) & 1);
    bool ok = !*abort_flag;
    if (ok && !mbar_wait_bounded(&full[s], par)) {
      set_error(a.err, ERRBIT_TIMEOUT);
      *abort_flag = 1;
      ok = false;
    }
    const int64_t e = (blockIdx.x + i * (int64_t)gridDim.x) * TS_THREADS + tid;
    T wv[4];        // WARPC: this lane's contributions and their vertices
    Pair wp[4];
    int4 wc = make_int4(-1, -1, -1, -1);
    bool wact = false;
    if (ok && e < a.ne) {
      const unsigned char* st = smem + s * kStage;
      const int4 c = reinterpret_cast<const int4*>(st)[tid];
      const T* Gs = reinterpret_cast<const T*>(st + kConnBytes) + tid * 12;
      bool inb = true;
      if (a.check) {
        inb = (unsigned)c.x < (unsigned)a.nv && (unsigned)c.y < (unsigned)a.nv &&
              (unsigned)c.z < (unsigned)a.nv && (unsigned)c.w < (unsigned)a.nv;
        if (!inb) set_error(a.err, ERRBIT_BOUNDS);
      }
      if (inb) {
        const int tb = (int)(i & 1) * kSlots;
        auto run = [&](const auto& sink) {
          if constexpr (MODE == TS_HVP) {
            if constexpr (PAIR)
              elem_pair_hvp<std::decay_t<decltype(sink)>, PREP, true>(
                  c, reinterpret_cast<const double*>(Gs), reinterpret_cast<const double*>(a.u),
                  reinterpret_cast<const double*>(a.v), fb2, sink, bad);
            else
              elem_native_hvp<T>(c, Gs, a.u, a.v, fb, sink);
          } else if constexpr (PAIR) {
            elem_pair<MODE, std::decay_t<decltype(sink)>, PREP, MODE == TS_GRAD>(
                            c, reinterpret_cast<const double*>(Gs),
                            reinterpret_cast<const double*>(a.u), fb2, tab, a.K, facc_p, sink,
                            reinterpret_cast<double*>(a.tape) + e * 4, bad);
            if ((i & 31) == 31) acc_renorm(facc_p);
          } else {
            elem_native<T, MODE>(c, Gs, a.u, fb, facc_n, sink, a.tape + e * 4);
          }
        };
        if constexpr (SHARED) {
          run(HashSink<T, kSlots>{hkeys + tb, hvals + tb, a.gu});
        } else if constexpr (WARPC) {
          run(CollectSink<T>{wv, wp});
          wc = c;
          wact = true;
        } else {
          run(AtomicSink<T>{a.gu});
        }
      }
    }
    if constexpr (WARPC) {  // every lane of the warp, active or not
      const int key[4] = {wc.x, wc.y, wc.z, wc.w};
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        if constexpr (PAIR) {
          warp_combine(wact, key[k], Acc{wp[k].h, wp[k].l},
                       [](Acc x, Acc y) { return acc_add(x, y); },
                       [&](int v, Acc tot) {
                         red_add(reinterpret_cast<double*>(a.gu) + v,
                                   pair_to_double_fast(acc_pair(tot)));
                       });
        } else {
          warp_combine(wact, key[k], wv[k], [](T x, T y) { return x + y; },
                       [&](int v, T tot) { red_add(a.gu + v, tot); });
        }
      }
    }
    if constexpr (SHARED) {  // the tile's insertions are complete: add the table into gu
      __syncthreads();
      const int tb = (int)(i & 1) * kSlots;
      hash_flush<T, kSlots, TS_THREADS>(hkeys + tb, hvals + tb, a.gu, tid);
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty[s]);
    if (tid == 0 && i + TS_STAGES < my_tiles && !*abort_flag) {
      if (!mbar_wait_bounded(&empty[s], par)) {
        set_error(a.err, ERRBIT_TIMEOUT);
        *abort_flag = 1;
      } else {
        issue(i + TS_STAGES, s);
        ++issued;
      }
    }
    __syncwarp();
  }
  if (tid == 0) {  // no copy into this CTA's shared memory may still be in flight
    for (int s = 0; s < TS_STAGES; ++s) {
      int64_t last = -1;
      for (int64_t j = issued - 1; j >= 0 && j >= issued - TS_STAGES; --j)
        if ((int)(j % TS_STAGES) == s) last = j;
      if (last >= 0) mbar_wait_bounded(&full[s], (uint32_t)((last / TS_STAGES) & 1));
    }
  }
  if (bad) set_error(a.err, ERRBIT_RANGE);

  // CTA sum of f (deterministic), then the last CTA sums the CTA partials.
  double fcta;
  if constexpr (PAIR) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) facc_p = acc_add(facc_p, shfl_xor_acc2(facc_p, o));
    Acc* ra = reinterpret_cast<Acc*>(red);
    if (lane == 0) ra[warp] = facc_p;
    __syncthreads();
    Acc tot = acc_zero();
    for (int w = 0; w < TS_WARPS; ++w) tot = acc_add(tot, ra[w]);
    fcta = acc_to_double(tot);
    __syncthreads();
  } else {
    fcta = block_sum((double)facc_n, red);
  }
  finish_sum<T>(fcta, a.fpart, a.counter, a.f, 0, red);
}

// Float pairs of the vertex vector u (and v), once per call for the pair
// gradient and Hessian-vector kernels (which then gather 8-byte pairs instead
// of splitting ~24 gathered doubles per vertex), with the zeroing of the output
// folded in; values outside the pair range set ERRBIT_RANGE.
__global__ void pair_split_vec_kernel(const double* __restrict__ u, const double* __restrict__ v,
                                      int64_t n, float2* us, float2* vs, double* zero,
                                      unsigned* err) {
  bool bad = false;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const double d = __ldg(u + i);
    bad |= !pair_in_range(d);
    const Pair p = split_f64(d);
    us[i] = make_float2(p.h, p.l);
    if (v) {
      const double dv = __ldg(v + i);
      bad |= !pair_in_range(dv);
      const Pair q = split_f64(dv);
      vs[i] = make_float2(q.h, q.l);
    }
    if (zero) zero[i] = 0.0;
  }
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) set_error(err, ERRBIT_RANGE);
}

// FP64 kernels in float pairs without shared-memory staging (the forward is
// latency-bound on its gathers, and the staged tiles cap the SM at 3 CTAs):
// one element per thread per step, G read from its prepared float-pair copy
// in global memory, lanes of a warp on consecutive elements (warp-uniform
// trip count, so the warp combine can run).  GRAD and HVP read u (and v) as
// float pairs split once per call.
template <int MODE, bool WARPC>
__global__ void __launch_bounds__(TS_THREADS) tet_direct_pair_kernel(TsArgs<double> a) {
  __shared__ float4 tab[kLogTableSize];
  __shared__ double red[2 * TS_WARPS];
  constexpr bool REV = MODE == TS_GRAD || MODE == TS_HVP;
  constexpr bool USPLIT = REV;
  for (int i = threadIdx.x; i < kLogTableSize; i += blockDim.x) tab[i] = a.logtab[i];
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  bool bad = false;
  Pair fb2{2.0f, 0.0f};
  if constexpr (REV) {
    const double fb = load_seed(a.seed);
    bad |= !pair_in_range(2.0 * fb);
    fb2 = split_f64(2.0 * fb);
  }
  Acc fa = acc_zero();
  int cnt = 0;
  const double* Gp = reinterpret_cast<const double*>(a.G);
  const double* u = reinterpret_cast<const double*>(a.u);
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < a.ne;
       base += stride, ++cnt) {
    const int64_t e = base + lane;
    const bool act = e < a.ne;
    const int4 c = act ? __ldcs(a.conn + e) : make_int4(-1, -1, -1, -1);
    double wv[4];
    Pair wp[4];
    if (act) {
      auto run = [&](const auto& sink) {
        if constexpr (MODE == TS_HVP)
          elem_pair_hvp<std::decay_t<decltype(sink)>, true, true>(
              c, Gp + e * 12, u, reinterpret_cast<const double*>(a.v), fb2, sink, bad);
        else
          elem_pair<MODE, std::decay_t<decltype(sink)>, true, USPLIT>(
              c, Gp + e * 12, u, fb2, tab, a.K, fa, sink, reinterpret_cast<double*>(a.tape) + e * 4,
              bad);
      };
      if constexpr (WARPC) run(CollectSink<double>{wv, wp});
      else run(AtomicSink<double>{reinterpret_cast<double*>(a.gu)});
    }
    if ((cnt & 31) == 31) acc_renorm(fa);
    if constexpr (WARPC) {
      const int key[4] = {c.x, c.y, c.z, c.w};
#pragma unroll
      for (int k = 0; k < 4; ++k)
        warp_combine(act, key[k], Acc{wp[k].h, wp[k].l}, [](Acc x, Acc y) { return acc_add(x, y); },
                     [&](int vtx, Acc tot) {
                       red_add(reinterpret_cast<double*>(a.gu) + vtx, pair_to_double_fast(acc_pair(tot)));
                     });
    }
  }
  if (bad) set_error(a.err, ERRBIT_RANGE);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) fa = acc_add(fa, shfl_xor_acc2(fa, o));
  Acc* ra = reinterpret_cast<Acc*>(red);
  if (lane == 0) ra[warp] = fa;
  __syncthreads();
  Acc tot = acc_zero();
  for (int w = 0; w < TS_WARPS; ++w) tot = acc_add(tot, ra[w]);
  __syncthreads();
  finish_sum<double>(acc_to_double(tot), a.fpart, a.counter, reinterpret_cast<double*>(a.f), 0, red);
}

template <int MODE, bool WARPC>
static cudaError_t launch_direct_pair(const kg_problem* p, const TsArgs<double>& a, cudaStream_t s) {
  static int occ = 0;
  if (occ < 1) {
    int o = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, tet_direct_pair_kernel<MODE, WARPC>,
                                                      TS_THREADS, 0) != cudaSuccess)
      o = 1;
    occ = std::max(o, 1);
  }
  const int64_t g = std::min<int64_t>({(p->m + TS_THREADS - 1) / TS_THREADS,
                                       (int64_t)num_sms() * occ, (int64_t)p->fpart_len});
  tet_direct_pair_kernel<MODE, WARPC><<<(int)std::max<int64_t>(g, 1), TS_THREADS, 0, s>>>(a);
  return cudaGetLastError();
}

static cudaError_t dispatch_direct_pair(const kg_problem* p, int mode, const TsArgs<double>& a,
                                        cudaStream_t s) {
  const bool warp = p->strategy == KG_STRATEGY_WARP;
  switch (mode) {
    case TS_EVAL: return launch_direct_pair<TS_EVAL, false>(p, a, s);
    case TS_TAPE: return launch_direct_pair<TS_TAPE, false>(p, a, s);
    case TS_GRAD: return warp ? launch_direct_pair<TS_GRAD, true>(p, a, s)
                              : launch_direct_pair<TS_GRAD, false>(p, a, s);
    default: return warp ? launch_direct_pair<TS_HVP, true>(p, a, s)
                         : launch_direct_pair<TS_HVP, false>(p, a, s);
  }
}

// ---------------------------------------------------------------- host ----
static float4* g_logtab[64] = {nullptr};
static std::mutex g_logtab_mu;

static void split_ld(long double v, float& h, float& l) {
  h = (float)v;
  l = (float)(v - (long double)h);
}

LogConsts log_consts() {
  LogConsts K;
  split_ld(logl(2.0L), K.ln2_h, K.ln2_l);
  split_ld(1.0L / 3.0L, K.third_h, K.third_l);
  return K;
}

// The 256-entry table (log c_k, 1/c_k) for c_k = 1 + k/256, computed on the
// host in extended precision and uploaded once per device (kept until exit).
kg_status logtab_for_device(const float4** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (dev < 0 || dev >= 64) return fail(KG_ERR_UNSUPPORTED, "device index >= 64");
  std::lock_guard<std::mutex> lk(g_logtab_mu);
  if (!g_logtab[dev]) {
    float4 h[kLogTableSize];
    for (int k = 0; k < kLogTableSize; ++k) {
      const long double c = 1.0L + (long double)k / kLogTableSize;
      split_ld(logl(c), h[k].x, h[k].y);
      split_ld(1.0L / c, h[k].z, h[k].w);
    }
    void* d = nullptr;
    if ((e = dev_alloc(&d, sizeof(h))) != cudaSuccess)
      return fail(KG_ERR_OOM, "log table allocation failed");
    if ((e = cudaMemcpy(d, h, sizeof(h), cudaMemcpyHostToDevice)) != cudaSuccess) {
      cudaFree(d);
      return cuda_fail(e, "log table upload");
    }
    g_logtab[dev] = static_cast<float4*>(d);
  }
  *out = g_logtab[dev];
  return KG_OK;
}

template <typename T, bool PAIR, bool SHARED, int MODE>
static size_t ts_smem() {
  constexpr int TS_STAGES = ts_stages<T, MODE>();
  return (size_t)TS_STAGES * (TS_THREADS * 16 + TS_THREADS * 12 * sizeof(T)) +
         2 * TS_STAGES * sizeof(uint64_t) + (PAIR ? kLogTableSize * sizeof(float4) : 0) +
         (2 * TS_WARPS + 2) * sizeof(double) +
         (SHARED ? 2 * (size_t)ts_hash_slots<T>() * (sizeof(T) + sizeof(int)) : 0);
}

// Upper bound of the staged kernels' grids (the f partials are sized for it):
// up to TS_MAX_PER_SM CTAs per SM.  Each launch takes the occupancy of its own
// kernel (registers, shared memory) within that bound.
constexpr int TS_MAX_PER_SM = 6;

int tet_staged_grid(const kg_problem* p) {
  const int64_t ntiles = (p->m + TS_THREADS - 1) / TS_THREADS;
  return (int)std::max<int64_t>(1, std::min<int64_t>(ntiles, (int64_t)num_sms() * TS_MAX_PER_SM));
}

// `occ` caches the kernel's resident CTAs per SM (queried on first use).
template <typename K>
static int ts_grid_for(const kg_problem* p, K kern, size_t smem, int& occ_cache) {
  if (occ_cache < 1) {
    int o = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, kern, TS_THREADS, smem) != cudaSuccess)
      o = 1;
    occ_cache = std::max(o, 1);
  }
  const int occ = occ_cache;
  const int64_t ntiles = (p->m + TS_THREADS - 1) / TS_THREADS;
  const int64_t g = std::min<int64_t>(ntiles, (int64_t)num_sms() * std::min(occ, TS_MAX_PER_SM));
  return (int)std::max<int64_t>(1, std::min<int64_t>(g, p->tet_grid));
}

kg_status tet_staged_setup(kg_problem* p) {
  if (p->dtype == KG_F64 && p->arith == KG_ARITH_PAIR) {
    const float4* t = nullptr;
    kg_status rc = logtab_for_device(&t);
    if (rc != KG_OK) return rc;
    // u and v as float pairs (16 N_v bytes), split per call
    if ((rc = ws_alloc(p, &p->usplit, 16 * (size_t)p->n, "vertex values as float pairs")) != KG_OK)
      return rc;
  }
  return KG_OK;
}

template <typename T, bool PAIR, int MODE, int SCAT, bool PREP>
static cudaError_t launch_ts_k(const kg_problem* p, const TsArgs<T>& a, cudaStream_t s) {
  auto kern = tet_staged_kernel<T, PAIR, MODE, SCAT, PREP>;
  const size_t smem = ts_smem<T, PAIR, SCAT == SC_SHARED, MODE>();
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  static int occ = 0;
  kern<<<ts_grid_for(p, kern, smem, occ), TS_THREADS, smem, s>>>(a);
  return cudaGetLastError();
}

template <typename T, bool PAIR, int MODE, bool PREP>
static cudaError_t launch_ts_p(const kg_problem* p, const TsArgs<T>& a, cudaStream_t s) {
  if constexpr (MODE == TS_GRAD || MODE == TS_HVP) {
    if (p->strategy == KG_STRATEGY_SHARED) return launch_ts_k<T, PAIR, MODE, SC_SHARED, PREP>(p, a, s);
    if (p->strategy == KG_STRATEGY_WARP) return launch_ts_k<T, PAIR, MODE, SC_WARP, PREP>(p, a, s);
  }
  return launch_ts_k<T, PAIR, MODE, SC_ATOMIC, PREP>(p, a, s);
}

template <typename T, bool PAIR, int MODE>
static cudaError_t launch_ts(const kg_problem* p, const TsArgs<T>& a, cudaStream_t s) {
  if constexpr (PAIR) {
    if (p->aprep) return launch_ts_p<T, PAIR, MODE, true>(p, a, s);
  }
  return launch_ts_p<T, PAIR, MODE, false>(p, a, s);
}

template <typename T>
static cudaError_t dispatch_ts(const kg_problem* p, int mode, const TsArgs<T>& a, cudaStream_t s) {
  const bool pair = sizeof(T) == 8 && p->arith == KG_ARITH_PAIR;
  if (pair) {
    if constexpr (sizeof(T) == 8) {
      if (mode == TS_EVAL) return launch_ts<T, true, TS_EVAL>(p, a, s);
      if (mode == TS_GRAD) return launch_ts<T, true, TS_GRAD>(p, a, s);
      if (mode == TS_HVP) return launch_ts<T, true, TS_HVP>(p, a, s);
      return launch_ts<T, true, TS_TAPE>(p, a, s);
    }
  }
  if (mode == TS_EVAL) return launch_ts<T, false, TS_EVAL>(p, a, s);
  if (mode == TS_GRAD) return launch_ts<T, false, TS_GRAD>(p, a, s);
  if (mode == TS_HVP) return launch_ts<T, false, TS_HVP>(p, a, s);
  return launch_ts<T, false, TS_TAPE>(p, a, s);
}

template <typename T>
static kg_status tet_staged_t(kg_problem* p, int mode, const void* x, void* f, void* gx,
                              const void* seed, const void* v, bool zero_gx, cudaStream_t s) {
  TsArgs<T> a{};
  a.conn = static_cast<const int4*>(p->data0);
  a.G = static_cast<const T*>(p->aprep ? p->aprep : p->data1);
  a.u = static_cast<const T*>(x);
  a.v = static_cast<const T*>(v);
  a.ne = p->m;
  a.nv = (int)p->n;
  a.seed = static_cast<const T*>(seed);
  a.gu = static_cast<T*>(gx);
  a.tape = static_cast<T*>(p->tape);
  a.fpart = p->fpart;
  a.counter = p->counter;
  a.f = static_cast<T*>(f);
  a.err = p->err;
  a.check = p->opt.check;
  a.K = log_consts();
  if (sizeof(T) == 8 && p->arith == KG_ARITH_PAIR) {
    kg_status rc = logtab_for_device(&a.logtab);
    if (rc != KG_OK) return rc;
    if (mode == TS_GRAD || mode == TS_HVP) {  // u (and v) read as float pairs split here
      float2* us = static_cast<float2*>(p->usplit);
      const int g =
          (int)std::max<int64_t>(1, std::min<int64_t>((p->n + 255) / 256, (int64_t)num_sms() * 8));
      pair_split_vec_kernel<<<g, 256, 0, s>>>(static_cast<const double*>(x),
                                              static_cast<const double*>(v), p->n, us, us + p->n,
                                              zero_gx ? static_cast<double*>(gx) : nullptr, p->err);
      count_launch();
      cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) return cuda_fail(e, "split vertex values");
      a.u = reinterpret_cast<const T*>(us);
      a.v = v ? reinterpret_cast<const T*>(us + p->n) : nullptr;
    }
  }
  // float pairs from the prepared G, no bounds checks, any strategy but the shared-memory
  // table: the direct kernels
  if constexpr (sizeof(T) == 8) {
    if (p->arith == KG_ARITH_PAIR && p->aprep && !p->opt.check && p->strategy != KG_STRATEGY_SHARED) {
      static const char* dnames[4] = {"tet_direct_pair_kernel<eval>", "tet_direct_pair_kernel<grad>",
                                      "tet_direct_pair_kernel<tape>", "tet_direct_pair_kernel<hvp>"};
      prof_begin(s, dnames[mode]);
      cudaError_t e = dispatch_direct_pair(p, mode, a, s);
      prof_end(s);
      count_launch();
      return e == cudaSuccess ? KG_OK : cuda_fail(e, dnames[mode]);
    }
  }
  static const char* names[4] = {"tet_staged_kernel<eval>", "tet_staged_kernel<grad>",
                                 "tet_staged_kernel<tape>", "tet_staged_kernel<hvp>"};
  prof_begin(s, names[mode]);
  cudaError_t e = dispatch_ts<T>(p, mode, a, s);
  prof_end(s);
  count_launch();
  return e == cudaSuccess ? KG_OK : cuda_fail(e, names[mode]);
}

kg_status tet_split_vertex_values(kg_problem* p, const void* x, const void* v, void* gx, bool zero_gx,
                                  const float2** us, const float2** vs, cudaStream_t s) {
  float2* u2 = static_cast<float2*>(p->usplit);
  const int g = (int)std::max<int64_t>(1, std::min<int64_t>((p->n + 255) / 256, (int64_t)num_sms() * 8));
  pair_split_vec_kernel<<<g, 256, 0, s>>>(static_cast<const double*>(x), static_cast<const double*>(v),
                                          p->n, u2, u2 + p->n,
                                          zero_gx ? static_cast<double*>(gx) : nullptr, p->err);
  count_launch();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "split vertex values");
  *us = u2;
  *vs = v ? u2 + p->n : nullptr;
  return KG_OK;
}

kg_status tet_staged(kg_problem* p, int mode, const void* x, void* f, void* gx, const void* seed,
                     cudaStream_t s, const void* v, bool zero_gx) {
  return p->dtype == KG_F64 ? tet_staged_t<double>(p, mode, x, f, gx, seed, v, zero_gx, s)
                            : tet_staged_t<float>(p, mode, x, f, gx, seed, v, zero_gx, s);
}

}  // namespace kg
