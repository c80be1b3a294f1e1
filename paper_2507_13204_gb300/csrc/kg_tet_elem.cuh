// Per-element tet-energy arithmetic shared by the staged kernels and the
// batched persistent kernel: native (FP32 / FP64 instructions) and float-pair
// (FP64 data) variants of g_e = G_e u_e, f_e = log1p(|g_e|^2) and the reverse
// c_e = G_e^T (2 fbar g_e / (1 + |g_e|^2)) with its scatter-add or tape store.
//
// The scatter-add goes through a sink: AtomicSink adds straight into gu in
// global memory; HashSink first combines the contributions of a tile of
// elements per vertex in a shared-memory open-addressing table (Sec. 5:
// temporaries kept in shared memory), which hash_flush then adds into gu with one
// global atomic per distinct vertex; CollectSink keeps them in registers for
// warp_combine, which merges equal vertices across the lanes of a warp.
#pragma once

#include <cuda_runtime.h>

#include <type_traits>

#include "kg_device.cuh"
#include "kg_pair.cuh"

namespace kg {

enum { TS_EVAL = 0, TS_GRAD = 1, TS_TAPE = 2, TS_HVP = 3 };

__device__ __forceinline__ Acc shfl_xor_acc2(Acc a, int o) {
  Acc b;
  b.s = __shfl_xor_sync(0xffffffffu, a.s, o);
  b.l = __shfl_xor_sync(0xffffffffu, a.l, o);
  return b;
}

// Shift-down by d lanes of a value of the warp combine's types.
__device__ __forceinline__ float shfl_down_v(float v, int d) {
  return __shfl_down_sync(0xffffffffu, v, d);
}
__device__ __forceinline__ double shfl_down_v(double v, int d) {
  return __shfl_down_sync(0xffffffffu, v, d);
}
__device__ __forceinline__ Acc shfl_down_v(Acc v, int d) {
  return Acc{__shfl_down_sync(0xffffffffu, v.s, d), __shfl_down_sync(0xffffffffu, v.l, d)};
}

// Sinks receive contribution k (0..3, the element's local vertex) for global
// vertex v.  sink_pair gives a sink the float-pair value of the pair kernels;
// by default it is converted to double first.
template <typename T>
struct AtomicSink {
  T* gu;
  __device__ __forceinline__ void operator()(int, int v, T c) const { red_add(gu + v, c); }
};

template <typename Sink>
__device__ __forceinline__ void sink_pair(const Sink& gu, int k, int v, Pair c) {
  gu(k, v, pair_to_double_fast(c));
}

// Keeps the element's four contributions in registers (k is a compile-time
// index after unrolling) for the warp-level combine below.
template <typename T>
struct CollectSink {
  T* vals;    // [4]
  Pair* prs;  // [4], pair kernels
  __device__ __forceinline__ void operator()(int k, int, T c) const { vals[k] = c; }
};

template <typename T>
__device__ __forceinline__ void sink_pair(const CollectSink<T>& gu, int k, int, Pair c) {
  gu.prs[k] = c;
}

// Warp-level combine of one contribution per lane: a run of consecutive lanes
// whose keys (vertices) are equal adds its values with a segmented suffix
// scan (ceil(log2 of the longest run) shift-down steps that stay inside the
// run), and the run's first lane adds the total to gu with one atomic.  Equal
// keys that are not adjacent form separate runs and simply issue separate
// atomics, so the result does not depend on the element order; elements
// numbered along the mesh put the shared vertices of neighbouring elements
// in neighbouring lanes.  Inactive lanes take part in the shuffles only.
// All 32 lanes must call it together.
template <typename V, typename AddF, typename FlushF>
__device__ __forceinline__ void warp_combine(bool active, int key, V val, AddF add, FlushF flush) {
  const int lane = threadIdx.x & 31;
  const int k = active ? key : -1;
  const int up = __shfl_up_sync(0xffffffffu, k, 1);
  const unsigned heads = __ballot_sync(0xffffffffu, lane == 0 || up != k);
  const unsigned above = heads & (0xFFFFFFFEu << lane);  // heads of the runs after this lane's
  const int last = above ? __ffs(above) - 2 : 31;        // last lane of this lane's run
  const int span = (int)__reduce_max_sync(0xffffffffu, (unsigned)(last - lane + 1));
  V acc = val;
  for (int d = 1; d < span; d <<= 1) {
    const V other = shfl_down_v(acc, d);
    if (lane + d <= last) acc = add(acc, other);
  }
  if (active && ((heads >> lane) & 1u)) flush(key, acc);
}

// The same combine by key groups instead of runs, for plain float values:
// lanes with equal keys anywhere in the warp find each other with match.any,
// and every lane walks the group members above it, one shuffle round per
// member (rounds = the largest group's size - 1).  It catches equal keys that
// are not adjacent, so it issues fewer atomics than warp_combine, at the cost
// of the match and of more rounds; it also needs fewer registers, which keeps
// the FP32 direct kernels at four blocks of 256 threads per SM.
__device__ __forceinline__ void warp_combine_groups(bool active, int key, float val,
                                                    float* __restrict__ gu) {
  const int lane = threadIdx.x & 31;
  const unsigned peers = __match_any_sync(0xffffffffu, active ? key : -1);
  unsigned rest = active ? peers & (0xFFFFFFFEu << lane) : 0u;
  const int rounds = (int)__reduce_max_sync(0xffffffffu, (unsigned)__popc(rest));
  float acc = val;
  for (int r = 0; r < rounds; ++r) {
    const int src = rest ? __ffs(rest) - 1 : lane;
    const float other = __shfl_sync(0xffffffffu, val, src);
    if (rest) {
      acc += other;
      rest &= rest - 1u;
    }
  }
  if (active && lane == __ffs(peers) - 1) red_add(gu + key, acc);
}

// Per-tile table of (vertex, partial sum) in shared memory.  keys[] holds -1
// for an empty slot.  Insertion probes linearly from a multiplicative hash;
// a slot is claimed with atomicCAS and the value added with a shared atomic.
// A tile inserts at most 4 x (elements per tile) distinct vertices, fewer than
// SLOTS, so a free slot always exists; the global atomic after the probe loop
// only keeps the sink total if that bound were ever broken.
template <typename T, int SLOTS>
struct HashSink {
  int* keys;
  T* vals;
  T* gu;
  __device__ __forceinline__ void operator()(int, int v, T c) const {
    static_assert((SLOTS & (SLOTS - 1)) == 0, "SLOTS must be a power of two");
    unsigned h = ((unsigned)v * 2654435761u) >> (32 - __builtin_ctz(SLOTS));
    for (int probe = 0; probe < SLOTS; ++probe) {
      int k = reinterpret_cast<volatile int*>(keys)[h];
      if (k == -1) k = atomicCAS(keys + h, -1, v);
      if (k == -1 || k == v) {
        atomicAdd(vals + h, c);
        return;
      }
      h = (h + 1) & (SLOTS - 1);
    }
    red_add(gu + v, c);
  }
};

// Adds every occupied slot into gu and empties the table (all threads of the
// CTA, after a barrier that ends the tile's insertions).
template <typename T, int SLOTS, int THREADS>
__device__ __forceinline__ void hash_flush(int* keys, T* vals, T* gu, int tid) {
#pragma unroll
  for (int j = tid; j < SLOTS; j += THREADS) {
    const int k = keys[j];
    if (k != -1) {
      red_add(gu + k, vals[j]);
      keys[j] = -1;
      vals[j] = T(0);
    }
  }
}

template <typename T>
__device__ __forceinline__ T log1p_nat(T v) {
  if constexpr (sizeof(T) == 8) return log1p(v);
  else return log1pf(v);
}

// One element in native arithmetic (T = float or double).
template <typename T, int MODE, typename Sink>
__device__ __forceinline__ void elem_native(const int4 c, const T* __restrict__ Gs,
                                            const T* __restrict__ u, T fb, T& facc, const Sink& gu,
                                            T* tape_e) {
  T G[12];  // Gs is 16-byte aligned (48 or 96 bytes per element): vector loads
  if constexpr (sizeof(T) == 4) {
#pragma unroll
    for (int i = 0; i < 12; i += 4) {
      const float4 q = *reinterpret_cast<const float4*>(Gs + i);
      G[i] = q.x, G[i + 1] = q.y, G[i + 2] = q.z, G[i + 3] = q.w;
    }
  } else {
#pragma unroll
    for (int i = 0; i < 12; i += 2) {
      const double2 q = *reinterpret_cast<const double2*>(Gs + i);
      G[i] = q.x, G[i + 1] = q.y;
    }
  }
  const T u0 = __ldg(u + c.x), u1 = __ldg(u + c.y), u2 = __ldg(u + c.z), u3 = __ldg(u + c.w);
  const T g0 = G[0] * u0 + G[1] * u1 + G[2] * u2 + G[3] * u3;
  const T g1 = G[4] * u0 + G[5] * u1 + G[6] * u2 + G[7] * u3;
  const T g2 = G[8] * u0 + G[9] * u1 + G[10] * u2 + G[11] * u3;
  const T s = g0 * g0 + g1 * g1 + g2 * g2;
  facc += log1p_nat(s);
  if constexpr (MODE != TS_EVAL) {
    const T w = T(2) * fb / (T(1) + s);
    const T w0 = w * g0, w1 = w * g1, w2 = w * g2;
    const T c0 = G[0] * w0 + G[4] * w1 + G[8] * w2;
    const T c1 = G[1] * w0 + G[5] * w1 + G[9] * w2;
    const T c2 = G[2] * w0 + G[6] * w1 + G[10] * w2;
    const T c3 = G[3] * w0 + G[7] * w1 + G[11] * w2;
    if constexpr (MODE == TS_GRAD) {
      gu(0, c.x, c0);
      gu(1, c.y, c1);
      gu(2, c.z, c2);
      gu(3, c.w, c3);
    } else {
      tape_e[0] = c0;
      tape_e[1] = c1;
      tape_e[2] = c2;
      tape_e[3] = c3;
    }
  }
}

// The arithmetic of one element in float pairs, from its G_e (12 pairs) and
// gathered vertex values U (4 pairs): g = G_e u_e, f_e = log1p(|g|^2) added to
// facc, and (MODE != TS_EVAL) the element adjoint
// cp[k] = (G_e^T (2 fbar g / (1 + |g|^2)))_k, with fb2 = 2 fbar as a pair.
template <int MODE>
__device__ __forceinline__ void elem_pair_core(const Pair (&G)[12], const Pair (&U)[4], Pair fb2,
                                               const float4* __restrict__ tab, const LogConsts& K,
                                               Acc& facc, Pair (&cp)[4]) {
  Pair g[3];
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    Acc a = acc_prod(G[4 * r].h, G[4 * r].l, U[0].h, U[0].l);
#pragma unroll
    for (int k = 1; k < 4; ++k) acc_fma(a, G[4 * r + k].h, G[4 * r + k].l, U[k].h, U[k].l);
    g[r] = acc_pair(a);
  }
  Acc sa = acc_prod(g[0].h, g[0].l, g[0].h, g[0].l);
#pragma unroll
  for (int r = 1; r < 3; ++r) acc_fma(sa, g[r].h, g[r].l, g[r].h, g[r].l);
  const Pair s = acc_pair(sa);
  Pair t;
  const Pair lf = pair_log1p(s, tab, K, t);
  facc = acc_add(facc, Acc{lf.h, lf.l});
  if constexpr (MODE != TS_EVAL) {
    const Pair w = pair_mul(fb2, pair_recip(t));
    Pair wg[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) wg[r] = pair_mul(w, g[r]);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      Acc a = acc_prod(G[k].h, G[k].l, wg[0].h, wg[0].l);
#pragma unroll
      for (int r = 1; r < 3; ++r) acc_fma(a, G[4 * r + k].h, G[4 * r + k].l, wg[r].h, wg[r].l);
      cp[k] = acc_pair(a);
    }
  }
}

// One element in float-pair arithmetic (FP64 data).  Gs points at the
// element's 12 doubles, or (PREP) at its 12 float pairs (h, l) prepared once.
// USPLIT: u points at float pairs of the vertex values, split (and range
// checked) once per call by pair_split_vec instead of once per gather.
template <int MODE, typename Sink, bool PREP = false, bool USPLIT = false>
__device__ __forceinline__ void elem_pair(const int4 c, const double* __restrict__ Gs,
                                          const double* __restrict__ u, Pair fb2,
                                          const float4* __restrict__ tab, const LogConsts& K,
                                          Acc& facc, const Sink& gu, double* tape_e, bool& bad) {
  Pair G[12];
#pragma unroll
  for (int i = 0; i < 12; i += 2) {
    if constexpr (PREP) {
      const float4 q = *reinterpret_cast<const float4*>(Gs + i);
      G[i] = Pair{q.x, q.y};
      G[i + 1] = Pair{q.z, q.w};
    } else {
      const double2 v = *reinterpret_cast<const double2*>(Gs + i);
      G[i] = split_f64(v.x);
      G[i + 1] = split_f64(v.y);
    }
  }
  Pair U[4];
  if constexpr (USPLIT) {
    const float2* up = reinterpret_cast<const float2*>(u);
    const float2 q0 = __ldg(up + c.x), q1 = __ldg(up + c.y), q2 = __ldg(up + c.z), q3 = __ldg(up + c.w);
    U[0] = Pair{q0.x, q0.y};
    U[1] = Pair{q1.x, q1.y};
    U[2] = Pair{q2.x, q2.y};
    U[3] = Pair{q3.x, q3.y};
  } else {
    const double ud[4] = {__ldg(u + c.x), __ldg(u + c.y), __ldg(u + c.z), __ldg(u + c.w)};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      bad |= !pair_in_range(ud[k]);
      U[k] = split_f64(ud[k]);
    }
  }
  Pair cp[4];
  elem_pair_core<MODE>(G, U, fb2, tab, K, facc, cp);
  if constexpr (MODE != TS_EVAL) {
    if constexpr (MODE == TS_GRAD) {
      sink_pair(gu, 0, c.x, cp[0]);
      sink_pair(gu, 1, c.y, cp[1]);
      sink_pair(gu, 2, c.z, cp[2]);
      sink_pair(gu, 3, c.w, cp[3]);
    } else {
      double cd[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) cd[k] = pair_to_double_fast(cp[k]);
      reinterpret_cast<double2*>(tape_e)[0] = make_double2(cd[0], cd[1]);
      reinterpret_cast<double2*>(tape_e)[1] = make_double2(cd[2], cd[3]);
    }
  }
}

// Hessian-vector product of one element (forward-mode tangent, direction v,
// of the reverse pass): with g = G u_e, gd = G v_e, s = |g|^2, t = 1 + s,
// w = 2 fbar / t, sd = 2 g . gd and wd = -w sd / t, the element adds
// G^T (wd g + w gd) at its four vertices.  Native arithmetic.
template <typename T, typename Sink>
__device__ __forceinline__ void elem_native_hvp(const int4 c, const T* __restrict__ Gs,
                                                const T* __restrict__ u, const T* __restrict__ v,
                                                T fb, const Sink& gu) {
  T G[12];
#pragma unroll
  for (int i = 0; i < 12; ++i) G[i] = Gs[i];
  const T u0 = __ldg(u + c.x), u1 = __ldg(u + c.y), u2 = __ldg(u + c.z), u3 = __ldg(u + c.w);
  const T v0 = __ldg(v + c.x), v1 = __ldg(v + c.y), v2 = __ldg(v + c.z), v3 = __ldg(v + c.w);
  T g[3], gd[3];
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    g[r] = G[4 * r] * u0 + G[4 * r + 1] * u1 + G[4 * r + 2] * u2 + G[4 * r + 3] * u3;
    gd[r] = G[4 * r] * v0 + G[4 * r + 1] * v1 + G[4 * r + 2] * v2 + G[4 * r + 3] * v3;
  }
  const T s = g[0] * g[0] + g[1] * g[1] + g[2] * g[2];
  const T sd = T(2) * (g[0] * gd[0] + g[1] * gd[1] + g[2] * gd[2]);
  const T t = T(1) + s;
  const T w = T(2) * fb / t;
  const T wd = -w * sd / t;
  T h[3];
#pragma unroll
  for (int r = 0; r < 3; ++r) h[r] = wd * g[r] + w * gd[r];
  gu(0, c.x, G[0] * h[0] + G[4] * h[1] + G[8] * h[2]);
  gu(1, c.y, G[1] * h[0] + G[5] * h[1] + G[9] * h[2]);
  gu(2, c.z, G[2] * h[0] + G[6] * h[1] + G[10] * h[2]);
  gu(3, c.w, G[3] * h[0] + G[7] * h[1] + G[11] * h[2]);
}

// The Hessian-vector arithmetic of one element in float pairs, from its G_e
// and the gathered U (point) and V (direction): hc[k] = (G_e^T (wd g + w gd))_k.
__device__ __forceinline__ void elem_pair_hvp_core(const Pair (&G)[12], const Pair (&U)[4],
                                                   const Pair (&V)[4], Pair fb2, Pair (&hc)[4]) {
  Pair g[3], gd[3];
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    Acc a = acc_prod(G[4 * r].h, G[4 * r].l, U[0].h, U[0].l);
    Acc b = acc_prod(G[4 * r].h, G[4 * r].l, V[0].h, V[0].l);
#pragma unroll
    for (int k = 1; k < 4; ++k) {
      acc_fma(a, G[4 * r + k].h, G[4 * r + k].l, U[k].h, U[k].l);
      acc_fma(b, G[4 * r + k].h, G[4 * r + k].l, V[k].h, V[k].l);
    }
    g[r] = acc_pair(a);
    gd[r] = acc_pair(b);
  }
  Acc sa = acc_prod(g[0].h, g[0].l, g[0].h, g[0].l);
  Acc sda = acc_prod(g[0].h, g[0].l, gd[0].h, gd[0].l);
#pragma unroll
  for (int r = 1; r < 3; ++r) {
    acc_fma(sa, g[r].h, g[r].l, g[r].h, g[r].l);
    acc_fma(sda, g[r].h, g[r].l, gd[r].h, gd[r].l);
  }
  const Pair s = acc_pair(sa);
  Pair sd = acc_pair(sda);
  sd.h *= 2.0f;  // exact
  sd.l *= 2.0f;
  const Pair rt = pair_recip(pair_add(Pair{1.0f, 0.0f}, s));
  const Pair w = pair_mul(fb2, rt);
  Pair wd = pair_mul(pair_mul(w, sd), rt);
  wd.h = -wd.h;
  wd.l = -wd.l;
  Pair h[3];
#pragma unroll
  for (int r = 0; r < 3; ++r) h[r] = pair_add(pair_mul(wd, g[r]), pair_mul(w, gd[r]));
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    Acc a = acc_prod(G[k].h, G[k].l, h[0].h, h[0].l);
#pragma unroll
    for (int r = 1; r < 3; ++r) acc_fma(a, G[4 * r + k].h, G[4 * r + k].l, h[r].h, h[r].l);
    hc[k] = acc_pair(a);
  }
}

// The same in float-pair arithmetic (FP64 data); fb2 = 2 fbar as a pair.
template <typename Sink, bool PREP = false, bool USPLIT = false>
__device__ __forceinline__ void elem_pair_hvp(const int4 c, const double* __restrict__ Gs,
                                              const double* __restrict__ u,
                                              const double* __restrict__ v, Pair fb2,
                                              const Sink& gu, bool& bad) {
  Pair G[12];
#pragma unroll
  for (int i = 0; i < 12; i += 2) {
    if constexpr (PREP) {
      const float4 q = *reinterpret_cast<const float4*>(Gs + i);
      G[i] = Pair{q.x, q.y};
      G[i + 1] = Pair{q.z, q.w};
    } else {
      const double2 q = *reinterpret_cast<const double2*>(Gs + i);
      G[i] = split_f64(q.x);
      G[i + 1] = split_f64(q.y);
    }
  }
  const int idx[4] = {c.x, c.y, c.z, c.w};
  Pair U[4], V[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    if constexpr (USPLIT) {
      const float2 qu = __ldg(reinterpret_cast<const float2*>(u) + idx[k]);
      const float2 qv = __ldg(reinterpret_cast<const float2*>(v) + idx[k]);
      U[k] = Pair{qu.x, qu.y};
      V[k] = Pair{qv.x, qv.y};
    } else {
      const double uk = __ldg(u + idx[k]), vk = __ldg(v + idx[k]);
      bad |= !pair_in_range(uk) || !pair_in_range(vk);
      U[k] = split_f64(uk);
      V[k] = split_f64(vk);
    }
  }
  Pair hc[4];
  elem_pair_hvp_core(G, U, V, fb2, hc);
#pragma unroll
  for (int k = 0; k < 4; ++k) sink_pair(gu, k, idx[k], hc[k]);
}

}  // namespace kg
