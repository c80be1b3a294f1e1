// Tiled reverse pass of the tet energy (KG_STRATEGY_TILE): the rescheduling of
// the reverse pass that Sec. 5 proposes, done per tile of elements.
//
// The forward gathers u through the index map conn, so the reverse pass
// scatters each element's adjoint c_e[k] into gu[conn[e][k]] (Sec. 3.3).  With
// the forward schedule that is 4 N_e global reductions; combining equal
// vertices across a warp's lanes first (KG_STRATEGY_WARP) halves them on the
// Kuhn mesh but costs a segmented scan per local slot.  Here kg_create cuts the
// elements into tiles of TL_E = 32 consecutive elements (a warp's step of the
// gradient kernel) and, per tile, sorts the tile's 128 incidences by vertex
// (tile_build_kernel), which gives the tile's transposed connectivity:
//   - vlist: the tile's distinct vertices (V_t of them, ascending);
//   - vptr / inc: for each tile vertex, its incidences (e_local * 4 + k, one
//     byte) in ascending order.
// The gradient kernel keeps the direct kernel's schedule (a warp on 32
// consecutive elements per step, G and u read from global memory), stores the
// element adjoints in the warp's slice of shared memory, and after a
// __syncwarp lets lane j add the incidences of tile vertices j, j + 32, ... in
// ascending order and issue one global reduction per tile vertex.  On the
// 100^3 Kuhn mesh a tile has about 25 distinct vertices, so global reductions
// drop from 4 to about 0.8 per element, with no combine and no CTA barrier.
// The sum is the same in another order: a vertex shared by several tiles
// still receives one reduction per tile, in no fixed order (the CSR strategy
// is the reproducible one).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <string>
#include <type_traits>

#include "kg_device.cuh"
#include "kg_internal.h"
#include "kg_pair.cuh"
#include "kg_tet_elem.cuh"

namespace kg {

constexpr int TL_E = 32;            // elements per tile: one warp's step
constexpr int TL_C = 4 * TL_E;      // incidences per tile (< 2^8: uint8 positions)
constexpr int TL_VPTR = TL_C + 8;   // stride of a tile's vertex pointers (uint8, 8-byte rows)
constexpr int TL_THREADS = 256;     // threads of the gradient kernel's CTA
constexpr int TL_BUILD = TL_C / 2;  // threads of the build kernel's CTA: two entries each

// ---------------------------------------------------------------- build ----
// One CTA per tile: bitonic sort of the tile's incidences by (vertex, position),
// then a scan of the vertex boundaries.  Outputs, for tile t:
//   tile_nv[t] = V_t; vlist[t * TL_C + j] (j < V_t); vptr[t * TL_VPTR + j]
//   (j <= V_t, vptr[V_t] = 4 n_t); inc[t * TL_C + i] (i < 4 n_t), the
//   incidences grouped by vertex.  conn must be in [0, N_v).
__global__ void __launch_bounds__(TL_BUILD) tile_build_kernel(const int* __restrict__ conn, int64_t ne,
                                                             int* __restrict__ tile_nv,
                                                             int* __restrict__ vlist,
                                                             uint8_t* __restrict__ vptr,
                                                             uint8_t* __restrict__ inc) {
  constexpr int PB = 8;  // bits of the position in the sort key (TL_C <= 256)
  __shared__ unsigned long long key[TL_C];
  __shared__ int wsum[32];
  const int t = blockIdx.x;
  const int64_t e0 = (int64_t)t * TL_E;
  const int nt = (int)min((int64_t)TL_E, ne - e0);
  const int n4 = 4 * nt;
  for (int i = threadIdx.x; i < TL_C; i += TL_BUILD)
    key[i] = i < n4 ? ((unsigned long long)(unsigned)conn[e0 * 4 + i] << PB) | (unsigned)i : ~0ull;
  __syncthreads();
  for (int k = 2; k <= TL_C; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = threadIdx.x; i < TL_C; i += TL_BUILD) {
        const int ixj = i ^ j;
        if (ixj > i) {
          const unsigned long long a = key[i], b = key[ixj];
          if ((a > b) == ((i & k) == 0)) {
            key[i] = b;
            key[ixj] = a;
          }
        }
      }
      __syncthreads();
    }
  }
  // thread t owns sorted entries 2t and 2t + 1; a head starts a new vertex
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int i0 = 2 * threadIdx.x, i1 = i0 + 1;
  const unsigned v0 = (unsigned)(key[i0] >> PB), v1 = (unsigned)(key[i1] >> PB);
  const int h0 = i0 < n4 && (i0 == 0 || v0 != (unsigned)(key[i0 - 1] >> PB));
  const int h1 = i1 < n4 && v1 != v0;
  const int sum = h0 + h1;
  int incl = sum;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) wsum[w] = incl;
  __syncthreads();
  if (w == 0) {
    const int ws = lane < TL_BUILD / 32 ? wsum[lane] : 0;
    int wi = ws;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, wi, o);
      if (lane >= o) wi += y;
    }
    if (lane < TL_BUILD / 32) wsum[lane] = wi - ws;  // heads in the warps before
  }
  __syncthreads();
  const int vid0 = wsum[w] + incl - sum + h0 - 1;  // local vertex of entry i0
  const int vid1 = vid0 + h1;
  int* vl = vlist + (int64_t)t * TL_C;
  uint8_t* vp = vptr + (int64_t)t * TL_VPTR;
  uint8_t* ic = inc + (int64_t)t * TL_C;
  const unsigned pmask = (1u << PB) - 1u;
  if (i0 < n4) {
    ic[i0] = (uint8_t)(key[i0] & pmask);
    if (h0) {
      vl[vid0] = (int)v0;
      vp[vid0] = (uint8_t)i0;
    }
    if (i0 == n4 - 1) {
      vp[vid0 + 1] = (uint8_t)min(n4, 255);  // n4 = 128 at most
      tile_nv[t] = vid0 + 1;
    }
  }
  if (i1 < n4) {
    ic[i1] = (uint8_t)(key[i1] & pmask);
    if (h1) {
      vl[vid1] = (int)v1;
      vp[vid1] = (uint8_t)i1;
    }
    if (i1 == n4 - 1) {
      vp[vid1 + 1] = (uint8_t)min(n4, 255);
      tile_nv[t] = vid1 + 1;
    }
  }
}

// ------------------------------------------------------------- gradient ----
struct TileArgs {
  const int4* conn;
  const double* G;          // prepared G: [N_e][12] float pairs in the bytes of 12 doubles
  const double* u;          // u as float pairs (split this call)
  const double* v;          // HVP: v as float pairs
  int64_t ne;
  const int* tile_nv;
  const int* vlist;
  const uint8_t* vptr;
  const uint8_t* inc;
  const double* seed;
  double* gu;
  float2* part;             // STORE: the tile vertex sums (float pairs), [tile][TL_C]
  double* fpart;
  unsigned* counter;
  double* f;
  unsigned* err;
  const float4* logtab;
  LogConsts K;
};

// The direct float-pair kernel's schedule (lanes of a warp on consecutive
// elements, one element per lane and step, G and u gathered from global
// memory) with the tiled scatter: a warp's 32 elements are one tile; their
// adjoints go to the warp's slice of shared memory, and after a __syncwarp
// lane j takes tile vertices j, j + 32, ...: it adds the vertex's incidences
// in ascending order and issues one global reduction -- or, STORE (the
// reproducible CSR strategy), writes the sum to the tile's partials instead.
template <int MODE, bool STORE>
__global__ void __launch_bounds__(TL_THREADS, 4) tet_tile_pair_kernel(TileArgs a) {
  __shared__ float4 tab[kLogTableSize];
  __shared__ __align__(16) float2 c_s[TL_THREADS / 32][TL_C];  // float4 stores
  __shared__ double red[2 * (TL_THREADS / 32)];
  constexpr bool GRAD = MODE == TS_GRAD;
  for (int i = threadIdx.x; i < kLogTableSize; i += blockDim.x) tab[i] = a.logtab[i];
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const double fb = load_seed(a.seed);
  bool bad = !pair_in_range(2.0 * fb);
  const Pair fb2 = split_f64(2.0 * fb);
  Acc fa = acc_zero();
  int cnt = 0;
  float2* cw = c_s[warp];
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < a.ne;
       base += stride, ++cnt) {
    const int64_t e = base + lane;
    // the tile's transposed connectivity, loaded before the element arithmetic so
    // that its latency overlaps it: lane l holds incidence bytes 4l .. 4l + 3 and
    // the pointers and vertex of tile vertex l
    const int64_t t = base / TL_E;
    const int V = __ldg(a.tile_nv + t);
    const uint8_t* vp = a.vptr + t * TL_VPTR;
    const uint8_t* ic = a.inc + t * TL_C;
    const unsigned incw = __ldg(reinterpret_cast<const unsigned*>(ic) + lane);
    const int p0 = lane < V ? __ldg(vp + lane) : 0, p1 = lane < V ? __ldg(vp + lane + 1) : 0;
    const int vg = lane < V ? __ldg(a.vlist + t * TL_C + lane) : 0;
    if (e < a.ne) {
      const int4 c = __ldcs(a.conn + e);
      double wv[4];
      Pair wp[4];
      if constexpr (GRAD)
        elem_pair<TS_GRAD, CollectSink<double>, true, true>(c, a.G + e * 12, a.u, fb2, tab, a.K, fa,
                                                             CollectSink<double>{wv, wp}, nullptr, bad);
      else
        elem_pair_hvp<CollectSink<double>, true, true>(c, a.G + e * 12, a.u, a.v, fb2,
                                                       CollectSink<double>{wv, wp}, bad);
      float4* cs = reinterpret_cast<float4*>(cw + 4 * lane);
      cs[0] = make_float4(wp[0].h, wp[0].l, wp[1].h, wp[1].l);
      cs[1] = make_float4(wp[2].h, wp[2].l, wp[3].h, wp[3].l);
    }
    if ((cnt & 31) == 31) acc_renorm(fa);
    __syncwarp();
    {  // tile vertex `lane`: incidence bytes from the lanes' registers
      const int rounds = (int)__reduce_max_sync(0xffffffffu, (unsigned)(p1 - p0));
      Acc s = acc_zero();
      for (int r = 0; r < rounds; ++r) {
        const int q = p0 + r;
        const unsigned w = __shfl_sync(0xffffffffu, incw, (q >> 2) & 31);
        if (q < p1) {
          const float2 cv = cw[(w >> (8 * (q & 3))) & 0xFFu];
          s = acc_add(s, Acc{cv.x, cv.y});
        }
      }
      if (lane < V) {
        const Pair pr = acc_pair(s);
        if constexpr (STORE) a.part[t * TL_C + lane] = make_float2(pr.h, pr.l);
        else red_add(a.gu + vg, pair_to_double_fast(pr));
      }
    }
    for (int j = lane + 32; j < V; j += 32) {  // tiles of more than 32 distinct vertices
      const int q0 = __ldg(vp + j), q1 = __ldg(vp + j + 1);
      Acc s = acc_zero();
      for (int q = q0; q < q1; ++q) {
        const float2 cv = cw[__ldg(ic + q)];
        s = acc_add(s, Acc{cv.x, cv.y});
      }
      const Pair pr = acc_pair(s);
      if constexpr (STORE) a.part[t * TL_C + j] = make_float2(pr.h, pr.l);
      else red_add(a.gu + __ldg(a.vlist + t * TL_C + j), pair_to_double_fast(pr));
    }
    __syncwarp();
  }
  if (bad) set_error(a.err, ERRBIT_RANGE);
  if constexpr (GRAD) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) fa = acc_add(fa, shfl_xor_acc2(fa, o));
    Acc* ra = reinterpret_cast<Acc*>(red);
    if (lane == 0) ra[warp] = fa;
    __syncthreads();
    Acc tot = acc_zero();
    for (int w = 0; w < TL_THREADS / 32; ++w) tot = acc_add(tot, ra[w]);
    __syncthreads();
    finish_sum<double>(acc_to_double(tot), a.fpart, a.counter, a.f, 0, red);
  }
}

// FP32 data: the direct FP32 kernel's arithmetic with the tiled scatter.  A
// warp's step covers two tiles (elements base + lane and base + 32 + lane, so
// that each lane has two elements' loads in flight); their adjoints go to the
// warp's shared memory and lane j sums the incidences of vertex j of each tile
// in ascending order (float adds, one reduction per tile vertex).
struct TileArgs32 {
  const int4* conn;
  const float4* G;  // [N_e][3] float4
  const float* u;
  const float* v;   // HVP: the direction
  int64_t ne;
  const int* tile_nv;
  const int* vlist;
  const uint8_t* vptr;
  const uint8_t* inc;
  const float* seed;
  float* gu;
  float* part;      // STORE: the tile vertex sums, [tile][TL_C]
  double* fpart;
  unsigned* counter;
  float* f;
};

template <int MODE, bool STORE>
__global__ void __launch_bounds__(TL_THREADS, MODE == TS_HVP ? 3 : 4) tet_tile_f32_kernel(TileArgs32 a) {
  __shared__ __align__(16) float c_s[TL_THREADS / 32][2][TL_C];  // float4 stores
  __shared__ double red[32];
  constexpr bool HVP = MODE == TS_HVP;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const float fb = load_seed(a.seed);
  float fa = 0.f, fc = 0.f;  // TwoSum-compensated float sum of f_e
  const int64_t stride = (int64_t)gridDim.x * blockDim.x * 2;
  for (int64_t base = ((int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31)) * 2; base < a.ne;
       base += stride) {
    int4 c[2];
    float4 g[2][3];
    bool act[2];
    int V[2], p0[2], p1[2], vg[2];
    unsigned incw[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int64_t e = base + h * 32 + lane;
      act[h] = e < a.ne;
      c[h] = act[h] ? __ldcs(a.conn + e) : make_int4(0, 0, 0, 0);
#pragma unroll
      for (int q = 0; q < 3; ++q) g[h][q] = act[h] ? __ldcs(a.G + e * 3 + q) : make_float4(0.f, 0.f, 0.f, 0.f);
      const int64_t t = base / TL_E + h;  // may be past the last tile when the mesh ends here
      const bool tv = t * TL_E < a.ne;
      V[h] = tv ? __ldg(a.tile_nv + t) : 0;
      incw[h] = tv ? __ldg(reinterpret_cast<const unsigned*>(a.inc + t * TL_C) + lane) : 0u;
      p0[h] = lane < V[h] ? __ldg(a.vptr + t * TL_VPTR + lane) : 0;
      p1[h] = lane < V[h] ? __ldg(a.vptr + t * TL_VPTR + lane + 1) : 0;
      vg[h] = lane < V[h] ? __ldg(a.vlist + t * TL_C + lane) : 0;
    }
    float uv[2][4], vv[2][4];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      uv[h][0] = __ldg(a.u + c[h].x);  // vertex 0 for inactive lanes (N_v >= 1)
      uv[h][1] = __ldg(a.u + c[h].y);
      uv[h][2] = __ldg(a.u + c[h].z);
      uv[h][3] = __ldg(a.u + c[h].w);
      if constexpr (HVP) {
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
        if constexpr (HVP)
          gd[q] = g[h][q].x * vv[h][0] + g[h][q].y * vv[h][1] + g[h][q].z * vv[h][2] + g[h][q].w * vv[h][3];
      }
      const float sq = gg[0] * gg[0] + gg[1] * gg[1] + gg[2] * gg[2];
      float hq[3];
      if constexpr (!HVP) {
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
      if (act[h]) {
        reinterpret_cast<float4*>(c_s[warp][h])[lane] =
            make_float4(g[h][0].x * hq[0] + g[h][1].x * hq[1] + g[h][2].x * hq[2],
                        g[h][0].y * hq[0] + g[h][1].y * hq[1] + g[h][2].y * hq[2],
                        g[h][0].z * hq[0] + g[h][1].z * hq[1] + g[h][2].z * hq[2],
                        g[h][0].w * hq[0] + g[h][1].w * hq[1] + g[h][2].w * hq[2]);
      }
    }
    __syncwarp();
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int rounds = (int)__reduce_max_sync(0xffffffffu, (unsigned)(p1[h] - p0[h]));
      float sum = 0.f;
      for (int r = 0; r < rounds; ++r) {
        const int q = p0[h] + r;
        const unsigned w = __shfl_sync(0xffffffffu, incw[h], (q >> 2) & 31);
        if (q < p1[h]) sum += c_s[warp][h][(w >> (8 * (q & 3))) & 0xFFu];
      }
      const int64_t t = base / TL_E + h;
      if (lane < V[h]) {
        if constexpr (STORE) a.part[t * TL_C + lane] = sum;
        else red_add(a.gu + vg[h], sum);
      }
      for (int j = lane + 32; j < V[h]; j += 32) {  // tiles of more than 32 distinct vertices
        const int q0 = __ldg(a.vptr + t * TL_VPTR + j), q1 = __ldg(a.vptr + t * TL_VPTR + j + 1);
        float s2 = 0.f;
        for (int q = q0; q < q1; ++q) s2 += c_s[warp][h][__ldg(a.inc + t * TL_C + q)];
        if constexpr (STORE) a.part[t * TL_C + j] = s2;
        else red_add(a.gu + __ldg(a.vlist + t * TL_C + j), s2);
      }
    }
    __syncwarp();
  }
  if constexpr (!HVP) finish_sum<float>(block_sum((double)fa + (double)fc, red), a.fpart, a.counter, a.f, 0, red);
}

// ------------------------------------------------------ from the tape ----
// The reverse pass from the tape c_e (N_e x 4 values, written by the taping
// forward): a tile's 128 tape entries are contiguous, so each warp reads its
// tile's with coalesced loads into shared memory and sums, per tile vertex,
// the incidences in ascending order; the sum times fbar is stored to the
// tile's partials (STORE) or added to gu with one reduction.  VT: 0 FP32
// values, 1 FP64 tape summed in float pairs (FP64 problems in PAIR
// arithmetic), 2 FP64 tape summed in FP64.
template <int VT> struct TileVal;
template <> struct TileVal<0> { using tape_t = float; using part_t = float; };
template <> struct TileVal<1> { using tape_t = double; using part_t = float2; };
template <> struct TileVal<2> { using tape_t = double; using part_t = double; };

template <int VT, bool STORE>
__global__ void __launch_bounds__(TL_THREADS) tet_tile_tape_kernel(
    const typename TileVal<VT>::tape_t* __restrict__ tape, int ntiles, const int* __restrict__ tile_nv,
    const int* __restrict__ vlist, const uint8_t* __restrict__ vptr, const uint8_t* __restrict__ inc,
    const typename TileVal<VT>::tape_t* seed, typename TileVal<VT>::tape_t* gu,
    typename TileVal<VT>::part_t* part) {
  using T = typename TileVal<VT>::tape_t;
  using S = std::conditional_t<VT == 1, Acc, T>;
  __shared__ __align__(16) S c_s[TL_THREADS / 32][TL_C];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const T fb = load_seed(seed);
  const Pair fbp = split_f64((double)fb);
  S* cw = c_s[warp];
  const int nwarps = gridDim.x * (TL_THREADS / 32);
  for (int t = blockIdx.x * (TL_THREADS / 32) + warp; t < ntiles; t += nwarps) {
    const int V = __ldg(tile_nv + t);
    const int n4 = V ? __ldg(vptr + (int64_t)t * TL_VPTR + V) : 0;  // 4 n_t
    const unsigned incw = __ldg(reinterpret_cast<const unsigned*>(inc + (int64_t)t * TL_C) + lane);
    const int p0 = lane < V ? __ldg(vptr + (int64_t)t * TL_VPTR + lane) : 0;
    const int p1 = lane < V ? __ldg(vptr + (int64_t)t * TL_VPTR + lane + 1) : 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int q = 4 * lane + k;
      if (q < n4) {
        const T c = __ldcs(tape + (int64_t)t * TL_C + q);
        if constexpr (VT == 1) {
          const Pair pc = split_f64(c);
          cw[q] = Acc{pc.h, pc.l};
        } else {
          cw[q] = c;
        }
      }
    }
    __syncwarp();
    const int rounds = (int)__reduce_max_sync(0xffffffffu, (unsigned)(p1 - p0));
    S sum{};
    for (int r = 0; r < rounds; ++r) {
      const int q = p0 + r;
      const unsigned w = __shfl_sync(0xffffffffu, incw, (q >> 2) & 31);
      if (q < p1) {
        const S cv = cw[(w >> (8 * (q & 3))) & 0xFFu];
        if constexpr (VT == 1) sum = acc_add(sum, cv);
        else sum += cv;
      }
    }
    auto finish = [&](int j, S sv) {
      if constexpr (VT == 1) {
        const Pair pr = pair_mul(acc_pair(sv), fbp);
        if constexpr (STORE) part[(int64_t)t * TL_C + j] = make_float2(pr.h, pr.l);
        else red_add(gu + __ldg(vlist + (int64_t)t * TL_C + j), pair_to_double_fast(pr));
      } else {
        if constexpr (STORE) part[(int64_t)t * TL_C + j] = fb * sv;
        else red_add(gu + __ldg(vlist + (int64_t)t * TL_C + j), fb * sv);
      }
    };
    if (lane < V) finish(lane, sum);
    for (int j = lane + 32; j < V; j += 32) {  // tiles of more than 32 distinct vertices
      const int q0 = __ldg(vptr + (int64_t)t * TL_VPTR + j), q1 = __ldg(vptr + (int64_t)t * TL_VPTR + j + 1);
      S s2{};
      for (int q = q0; q < q1; ++q) {
        const S cv = cw[__ldg(inc + (int64_t)t * TL_C + q)];
        if constexpr (VT == 1) s2 = acc_add(s2, cv);
        else s2 += cv;
      }
      finish(j, s2);
    }
    __syncwarp();
  }
}

// Second pass of the reproducible CSR strategy: vertex v adds the partials of
// its tiles in ascending tile order, perm[rowptr[v] .. rowptr[v+1]) listing
// the slots (tile * TL_C + local vertex) of v (built at kg_create).
template <int VT>
__global__ void __launch_bounds__(256) tet_tile_gather_kernel(const int* __restrict__ rowptr,
                                                              const int* __restrict__ perm,
                                                              const typename TileVal<VT>::part_t* __restrict__ part,
                                                              int nv, typename TileVal<VT>::tape_t* gu,
                                                              int accumulate) {
  using T = typename TileVal<VT>::tape_t;
  const int stride = gridDim.x * blockDim.x;
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < nv; v += stride) {
    const int q0 = __ldg(rowptr + v), q1 = __ldg(rowptr + v + 1);
    T r;
    if constexpr (VT == 1) {
      Acc s = acc_zero();
      for (int q = q0; q < q1; ++q) {
        const float2 c = __ldg(part + __ldg(perm + q));
        s = acc_add(s, Acc{c.x, c.y});
      }
      r = pair_to_double(acc_pair(s));
    } else {
      T s = T(0);
      for (int q = q0; q < q1; ++q) s += __ldg(part + __ldg(perm + q));
      r = s;
    }
    gu[v] = accumulate ? gu[v] + r : r;
  }
}

// The valid tile slots (tile t, local vertex j < V_t), compacted: slot
// toff[t] + j gets key vlist[t][j] (its vertex) and id t * TL_C + j.  toff is
// the exclusive scan of tile_nv.
__global__ void tile_slot_compact_kernel(const int* __restrict__ tile_nv, const int* __restrict__ toff,
                                         const int* __restrict__ vlist, int ntiles, int* keys, int* ids) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < (int64_t)ntiles * TL_C; i += stride) {
    const int t = (int)(i / TL_C), j = (int)(i % TL_C);
    if (j < __ldg(tile_nv + t)) {
      const int c = __ldg(toff + t) + j;
      keys[c] = __ldg(vlist + i);
      ids[c] = (int)i;
    }
  }
}

// perm[q] <- ids[perm[q]]: bucket positions (compact slots, ascending) to slot ids
// (also ascending, as the compaction keeps the slot order).
__global__ void tile_slot_ids_kernel(const int* __restrict__ ids, int n, int* perm) {
  const int stride = gridDim.x * blockDim.x;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < n; q += stride) perm[q] = __ldg(ids + perm[q]);
}

// ---------------------------------------------------------------- host ----
bool tet_tile_supported(const kg_problem* p) {
  if (p->opt.check) return false;
  if (p->dtype == KG_F32) return true;
  return p->arith == KG_ARITH_PAIR && p->aprep != nullptr;
}

kg_status tet_tile_setup(kg_problem* p, cudaStream_t s) {
  static_assert(TL_C <= 128 && TL_VPTR % 8 == 0, "tile positions and pointers are bytes");
  const int64_t ntiles = (p->m + TL_E - 1) / TL_E;
  kg_status rc;
  if ((rc = ws_alloc(p, (void**)&p->tile_nv, sizeof(int) * (size_t)ntiles, "tile vertex counts")) != KG_OK ||
      (rc = ws_alloc(p, (void**)&p->tile_vlist, sizeof(int) * (size_t)ntiles * TL_C, "tile vertices")) != KG_OK ||
      (rc = ws_alloc(p, (void**)&p->tile_vptr, (size_t)ntiles * TL_VPTR, "tile vertex pointers")) != KG_OK ||
      (rc = ws_alloc(p, (void**)&p->tile_inc, (size_t)ntiles * TL_C, "tile incidences")) != KG_OK)
    return rc;
  p->ntiles = (int)ntiles;
  tile_build_kernel<<<(int)ntiles, TL_BUILD, 0, s>>>(static_cast<const int*>(p->data0), p->m, p->tile_nv,
                                                     p->tile_vlist, p->tile_vptr, p->tile_inc);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? KG_OK : cuda_fail(e, "tile build");
}

template <int MODE, bool STORE>
static cudaError_t launch_tile(const kg_problem* p, const TileArgs& a, cudaStream_t s) {
  auto kern = tet_tile_pair_kernel<MODE, STORE>;
  static int occ = 0;
  if (occ < 1) {
    int o = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, kern, TL_THREADS, 0) != cudaSuccess) o = 1;
    occ = std::max(o, 1);
  }
  const int64_t g = std::min<int64_t>({(p->m + TL_THREADS - 1) / TL_THREADS, (int64_t)num_sms() * occ,
                                       (int64_t)p->fpart_len});
  kern<<<(int)std::max<int64_t>(g, 1), TL_THREADS, 0, s>>>(a);
  return cudaGetLastError();
}

// us, vs: the float pairs of u (and v) split this call; gx zeroed (or holding
// the values to accumulate onto).
kg_status tet_tile_run(kg_problem* p, int mode, const float2* us, const float2* vs, void* f, void* gx,
                       const void* seed, cudaStream_t s) {
  TileArgs a{};
  a.conn = static_cast<const int4*>(p->data0);
  a.G = static_cast<const double*>(p->aprep);
  a.u = reinterpret_cast<const double*>(us);
  a.v = reinterpret_cast<const double*>(vs);
  a.ne = p->m;
  a.tile_nv = p->tile_nv;
  a.vlist = p->tile_vlist;
  a.vptr = p->tile_vptr;
  a.inc = p->tile_inc;
  a.seed = static_cast<const double*>(seed);
  a.gu = static_cast<double*>(gx);
  a.fpart = p->fpart;
  a.counter = p->counter;
  a.f = static_cast<double*>(f);
  a.err = p->err;
  a.K = log_consts();
  kg_status rc = logtab_for_device(&a.logtab);
  if (rc != KG_OK) return rc;
  const bool store = p->strategy == KG_STRATEGY_CSR;
  a.part = static_cast<float2*>(p->tile_part);
  const char* name = mode == TS_HVP ? (store ? "tet_tile_pair_kernel<hvp, partials>" : "tet_tile_pair_kernel<hvp>")
                                    : (store ? "tet_tile_pair_kernel<grad, partials>" : "tet_tile_pair_kernel<grad>");
  prof_begin(s, name);
  cudaError_t e = mode == TS_HVP ? (store ? launch_tile<TS_HVP, true>(p, a, s) : launch_tile<TS_HVP, false>(p, a, s))
                                 : (store ? launch_tile<TS_GRAD, true>(p, a, s) : launch_tile<TS_GRAD, false>(p, a, s));
  prof_end(s);
  count_launch();
  return e == cudaSuccess ? KG_OK : cuda_fail(e, name);
}

template <int MODE, bool STORE>
static cudaError_t launch_tile32(const kg_problem* p, const TileArgs32& a, cudaStream_t s) {
  auto kern = tet_tile_f32_kernel<MODE, STORE>;
  static int occ = 0;
  if (occ < 1) {
    int o = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, kern, TL_THREADS, 0) != cudaSuccess) o = 1;
    occ = std::max(o, 1);
  }
  const int64_t g = std::min<int64_t>({(p->m + 2 * TL_THREADS - 1) / (2 * TL_THREADS),
                                       (int64_t)num_sms() * occ, (int64_t)p->fpart_len});
  kern<<<(int)std::max<int64_t>(g, 1), TL_THREADS, 0, s>>>(a);
  return cudaGetLastError();
}

// FP32: u (and v) read directly; gx zeroed by the caller (or accumulated onto).
kg_status tet_tile_run_f32(kg_problem* p, int mode, const void* x, const void* v, void* f, void* gx,
                           const void* seed, cudaStream_t s) {
  TileArgs32 a{};
  a.conn = static_cast<const int4*>(p->data0);
  a.G = static_cast<const float4*>(p->data1);
  a.u = static_cast<const float*>(x);
  a.v = static_cast<const float*>(v);
  a.ne = p->m;
  a.tile_nv = p->tile_nv;
  a.vlist = p->tile_vlist;
  a.vptr = p->tile_vptr;
  a.inc = p->tile_inc;
  a.seed = static_cast<const float*>(seed);
  a.gu = static_cast<float*>(gx);
  a.fpart = p->fpart;
  a.counter = p->counter;
  a.f = static_cast<float*>(f);
  const bool store = p->strategy == KG_STRATEGY_CSR;
  a.part = static_cast<float*>(p->tile_part);
  const char* name = mode == TS_HVP ? (store ? "tet_tile_f32_kernel<hvp, partials>" : "tet_tile_f32_kernel<hvp>")
                                    : (store ? "tet_tile_f32_kernel<grad, partials>" : "tet_tile_f32_kernel<grad>");
  prof_begin(s, name);
  cudaError_t e = mode == TS_HVP ? (store ? launch_tile32<TS_HVP, true>(p, a, s) : launch_tile32<TS_HVP, false>(p, a, s))
                                 : (store ? launch_tile32<TS_GRAD, true>(p, a, s) : launch_tile32<TS_GRAD, false>(p, a, s));
  prof_end(s);
  count_launch();
  return e == cudaSuccess ? KG_OK : cuda_fail(e, name);
}

// Value type of the tile partials / tape sums of this problem.
static int tile_vt(const kg_problem* p) {
  return p->dtype == KG_F32 ? 0 : p->arith == KG_ARITH_PAIR ? 1 : 2;
}

// The reproducible CSR strategy's set-up: the tiles, the partials buffer and
// the vertex -> slot buckets (ascending slots per vertex), over the valid
// slots only.  Synchronises s.
kg_status tet_tile_csr_setup(kg_problem* p, cudaStream_t s) {
  kg_status rc = tet_tile_setup(p, s);
  if (rc != KG_OK) return rc;
  const int64_t nslots = (int64_t)p->ntiles * TL_C;
  if (nslots >= (int64_t(1) << 31)) return fail(KG_ERR_INVALID_ARG, "TETENERGY CSR: too many tiles");
  const size_t vsz = tile_vt(p) == 0 ? sizeof(float) : tile_vt(p) == 1 ? sizeof(float2) : sizeof(double);
  if ((rc = ws_alloc(p, &p->tile_part, vsz * (size_t)nslots, "tile partials")) != KG_OK ||
      (rc = ws_alloc(p, (void**)&p->rowptr, sizeof(int) * (size_t)(p->n + 1), "vertex -> slot pointers")) != KG_OK)
    return rc;
  // exclusive scan of the tiles' vertex counts: the compact slot offsets
  int* toff = nullptr;
  if (dev_alloc((void**)&toff, sizeof(int) * ((size_t)p->ntiles + 1)) != cudaSuccess)
    return fail(KG_ERR_OOM, "tile offsets allocation failed");
  cudaError_t e = cudaMemcpyAsync(toff, p->tile_nv, sizeof(int) * (size_t)p->ntiles, cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess) {
    scan_exclusive(toff, p->ntiles, s);
    e = cudaGetLastError();
  }
  int nvalid = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&nvalid, toff + p->ntiles, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    cudaFree(toff);
    return cuda_fail(e, "tile slot offsets");
  }
  int *keys = nullptr, *ids = nullptr;
  rc = ws_alloc(p, (void**)&p->inc, sizeof(int) * (size_t)std::max(nvalid, 1), "vertex -> slot lists");
  if (rc == KG_OK && (dev_alloc((void**)&keys, sizeof(int) * (size_t)std::max(nvalid, 1)) != cudaSuccess ||
                      dev_alloc((void**)&ids, sizeof(int) * (size_t)std::max(nvalid, 1)) != cudaSuccess))
    rc = fail(KG_ERR_OOM, "tile slot keys allocation failed");
  if (rc == KG_OK) {
    const int g = (int)std::max<int64_t>(1, std::min<int64_t>((nslots + 255) / 256, (int64_t)num_sms() * 8));
    tile_slot_compact_kernel<<<g, 256, 0, s>>>(p->tile_nv, toff, p->tile_vlist, p->ntiles, keys, ids);
    e = cudaGetLastError();
    rc = e == cudaSuccess ? build_buckets(keys, nvalid, (int)p->n, p->rowptr, p->inc, s)
                          : cuda_fail(e, "tile slot compaction");
  }
  if (rc == KG_OK && nvalid > 0) {
    const int g = (int)std::max<int64_t>(1, std::min<int64_t>((nvalid + 255) / 256, (int64_t)num_sms() * 8));
    tile_slot_ids_kernel<<<g, 256, 0, s>>>(ids, nvalid, p->inc);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) rc = cuda_fail(e, "tile slot ids");
  }
  cudaFree(keys);
  cudaFree(ids);
  cudaFree(toff);
  return rc;
}

// Second pass of the CSR strategy: gx[v] (+)= the sum of v's tile partials.
kg_status tet_tile_gather(kg_problem* p, void* gx, int accumulate, cudaStream_t s) {
  const int g = (int)std::max<int64_t>(1, std::min<int64_t>((p->n + 255) / 256, (int64_t)num_sms() * 8));
  // a second-stage sum like the dense partials reduction: not bracketed by the profiling events
  switch (tile_vt(p)) {
    case 0:
      tet_tile_gather_kernel<0><<<g, 256, 0, s>>>(p->rowptr, p->inc, static_cast<const float*>(p->tile_part),
                                                  (int)p->n, static_cast<float*>(gx), accumulate);
      break;
    case 1:
      tet_tile_gather_kernel<1><<<g, 256, 0, s>>>(p->rowptr, p->inc, static_cast<const float2*>(p->tile_part),
                                                  (int)p->n, static_cast<double*>(gx), accumulate);
      break;
    default:
      tet_tile_gather_kernel<2><<<g, 256, 0, s>>>(p->rowptr, p->inc, static_cast<const double*>(p->tile_part),
                                                  (int)p->n, static_cast<double*>(gx), accumulate);
  }
  count_launch();
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? KG_OK : cuda_fail(e, "tile gather");
}

template <int VT, bool STORE>
static void launch_tape_pass(const kg_problem* p, const void* seed, void* gx, cudaStream_t s) {
  using T = typename TileVal<VT>::tape_t;
  using PT = typename TileVal<VT>::part_t;
  const int64_t g = std::max<int64_t>(1, std::min<int64_t>(((int64_t)p->ntiles + 7) / 8, (int64_t)num_sms() * 8));
  tet_tile_tape_kernel<VT, STORE><<<(int)g, TL_THREADS, 0, s>>>(
      static_cast<const T*>(p->tape), p->ntiles, p->tile_nv, p->tile_vlist, p->tile_vptr, p->tile_inc,
      static_cast<const T*>(seed), static_cast<T*>(gx), static_cast<PT*>(p->tile_part));
}

// The reverse pass from the tape: CSR strategy, the tile partials then the
// vertex gather (reproducible); TILE strategy, one reduction per tile vertex
// into gx (zeroed here unless accumulating).
kg_status tet_tile_from_tape(kg_problem* p, void* gx, const void* seed, int accumulate, cudaStream_t s) {
  const bool store = p->strategy == KG_STRATEGY_CSR;
  cudaError_t e;
  if (!store && !accumulate) {
    if ((e = cudaMemsetAsync(gx, 0, p->esize * (size_t)p->n, s)) != cudaSuccess) return cuda_fail(e, "zero gu");
    count_launch();
  }
  prof_begin(s, store ? "tet_tile_tape_kernel<partials>" : "tet_tile_tape_kernel");
  switch (tile_vt(p) * 2 + (store ? 1 : 0)) {
    case 0: launch_tape_pass<0, false>(p, seed, gx, s); break;
    case 1: launch_tape_pass<0, true>(p, seed, gx, s); break;
    case 2: launch_tape_pass<1, false>(p, seed, gx, s); break;
    case 3: launch_tape_pass<1, true>(p, seed, gx, s); break;
    case 4: launch_tape_pass<2, false>(p, seed, gx, s); break;
    default: launch_tape_pass<2, true>(p, seed, gx, s); break;
  }
  prof_end(s);
  count_launch();
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "tile tape pass");
  return store ? tet_tile_gather(p, gx, accumulate, s) : KG_OK;
}

}  // namespace kg
