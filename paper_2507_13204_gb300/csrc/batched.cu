// Batched value-and-gradient of many independent problems in ONE persistent
// kernel launch, replayed from a CUDA graph (the paper's Sec. 5 second
// restriction: the generated gradient doubles the kernel launches and host
// synchronisation points; here a whole batch of gradients is one launch).
//
// Work: every instance is cut into tiles -- row tiles for the dense quadratic
// form, element tiles for the tet energy -- and the (instance, tile) items are
// sorted longest-first into a device work table.  Each CTA of the persistent
// grid claims items from a device queue head (one atomicAdd per item) until
// the table is exhausted.
//   dense tile:  rows [r0, r0 + R): y_i by a row team (4 .. 256 threads,
//                about 8 columns a thread), ybar_i = 2 y_i, private xbar
//                partial of the tile written to the instance's partial buffer;
//                on float-pair copies (pair batches) the rows arrive by bulk
//                copies into a shared-memory ring, otherwise by plain loads;
//   tet tile:    elements [e0, e0 + T): f_e and the scatter of c_e into gu (zeroed
//                by a small kernel earlier in the graph): one global reduction per
//                contribution, or warp-combined first with the WARP strategy.
// The CTA that finishes an instance's last tile (a per-instance arrival
// counter; nobody waits) sums the instance's partials in tile order into gx
// and f, and resets the counter.  The last CTA to leave resets the queue head,
// so the graph can be replayed as is.
//
// Tile sizes R and T are chosen per (kind, size bucket) by an autotuner that
// times candidates on the instances of the batch at kg_batch_create and keeps
// the choices in a JSON cache keyed by GPU name, kind, dtype and bucket.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <map>
#include <mutex>
#include <new>
#include <sstream>
#include <string>
#include <vector>

#include <sys/stat.h>

#include "kg_device.cuh"
#include "kg_internal.h"
#include "kg_pair.cuh"
#include "kg_tet_elem.cuh"

namespace kg {

enum { BK_DENSE = 1, BK_TET = 2 };
constexpr int BT = 256;   // threads per CTA
constexpr int BW = BT / 32;
constexpr int B_CPT = 8;  // dense: columns per team thread (n <= 8 * team)
constexpr int B_MAXN = 2048;

struct BInst {
  int kind;
  int n;      // dense: columns; tet: vertices
  int64_t m;  // dense: rows; tet: elements
  int ntiles;
  int team;   // dense: 32 or 256
  int prep;   // pair batches: d0 (dense A) or d1 (tet G) is the prepared float-pair copy
  const void* d0;
  const void* d1;
  const void* x;
  void* f;
  void* gx;
  void* partials;  // dense: [ntiles][n]  (pair: Acc; native: T)
  double* fpart;   // [ntiles]
  unsigned* done;
};

struct BItem {
  int inst, tile;
  int64_t start;
  int count;
};

struct BArgs {
  const BInst* insts;
  const BItem* items;
  int nitems;
  unsigned* head;  // [0] queue head, [1] CTAs that left
  unsigned* err;
  const float4* logtab;
  LogConsts K;
  int warpc;  // tet tiles: warp-combined atomics (else one per contribution)
};

// ------------------------------------------------------------- device ----
// L2 prefetch of the whole 16-byte units inside [p, p + bytes) (never beyond).
__device__ __forceinline__ void prefetch_range_l2(const void* p, size_t bytes) {
  uintptr_t a = (reinterpret_cast<uintptr_t>(p) + 15) & ~uintptr_t(15);
  const uintptr_t b = (reinterpret_cast<uintptr_t>(p) + bytes) & ~uintptr_t(15);
  while (a < b) {
    const uint32_t chunk = (uint32_t)((b - a) < (uintptr_t(1) << 16) ? (b - a) : (uintptr_t(1) << 16));
    prefetch_l2_bulk(reinterpret_cast<const void*>(a), chunk);
    a += chunk;
  }
}

// The float pair (h, l) of v for pair arithmetic (zeros otherwise).
template <bool PAIR, typename T>
__device__ __forceinline__ void b_split(T v, float& h, float& l) {
  if constexpr (PAIR) {
    const Pair p = split_f64((double)v);
    h = p.h;
    l = p.l;
  } else {
    h = 0.f;
    l = 0.f;
  }
}

// Barrier over the TEAM threads of one row team: the whole CTA for TEAM = BT,
// otherwise hardware barrier 1 + team (TEAM = 64 or 128).
template <int TEAM>
__device__ __forceinline__ void team_barrier(int team) {
  if constexpr (TEAM == BT) __syncthreads();
  else named_barrier(1 + team, TEAM);
}

// The team's sum of its TW warps' row sums ra[q * 2 + upper] (q < TW), for a
// team wider than a warp: lane l takes warp l mod TW's and a butterfly over TW
// lanes (inside the lane's half-warp, so over one row) gives every lane the
// same total, with log2(TW) pair additions a thread instead of TW - 1.
template <int TW>
__device__ __forceinline__ Acc team_warps_sum(const Acc* ra, int lane, bool upper) {
  Acc k = ra[(lane & (TW - 1)) * 2 + (upper ? 1 : 0)];
#pragma unroll
  for (int o = TW / 2; o > 0; o >>= 1) k = acc_add(k, shfl_xor_acc2(k, o));
  return k;
}

// Rows [w.start, w.start + w.count) of a dense instance on its FP64 or FP32
// data (pair batches: split on every load); returns the tile's f.
template <typename T, bool PAIR, int TEAM>
__device__ double dense_tile(const BInst& I, const BItem& w, unsigned char* wsp, double* red,
                             bool& bad) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int n = I.n;
  const T* __restrict__ A = static_cast<const T*>(I.d0);
  const T* __restrict__ x = static_cast<const T*>(I.x);
  constexpr int NT = BT / TEAM;
  const int lt = tid % TEAM, team = tid / TEAM;
  const int cpt = (n + TEAM - 1) / TEAM;  // <= B_CPT, uniform over the item
  float xh[B_CPT], xl[B_CPT];
  T xv[B_CPT];
  Acc xbp[B_CPT];
  T xbn[B_CPT];
#pragma unroll
  for (int k = 0; k < B_CPT; ++k) {
    const int j = lt + k * TEAM;
    xv[k] = (k < cpt && j < n) ? x[j] : T(0);
    if constexpr (PAIR) {
      bad |= !pair_in_range((double)xv[k]);
      b_split<PAIR>(xv[k], xh[k], xl[k]);
    }
    xbp[k] = acc_zero();
    xbn[k] = T(0);
  }
  Acc fp = acc_zero();
  FSum<T> fn;
  const int64_t r1 = w.start + w.count;
  if constexpr (PAIR) {
    // Two rows per team and iteration, rows r and r + NT: their loads are issued
    // together, and one transposed butterfly reduces both dot products (the
    // first exchange hands each half of the team one row), so the reduction
    // and, for teams wider than a warp, the barrier are paid once per two rows.
    constexpr int W = TEAM < 32 ? TEAM : 32;  // lanes of the team inside one warp
    const bool upper = (lane & (W / 2)) != 0;  // keeps the second row
    const int iters2 = (w.count + 2 * NT - 1) / (2 * NT);
    for (int itr = 0; itr < iters2; ++itr) {
      const int64_t rr[2] = {w.start + (int64_t)itr * 2 * NT + team,
                             w.start + (int64_t)itr * 2 * NT + NT + team};
      const bool vr[2] = {rr[0] < r1, rr[1] < r1};
      float ah[2][B_CPT], al[2][B_CPT];
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const T* Ar = A + (vr[q] ? rr[q] : w.start) * (int64_t)n;
#pragma unroll
        for (int k = 0; k < B_CPT; ++k) {
          const int j = lt + k * TEAM;
          const T v = (k < cpt && vr[q] && j < n) ? __ldcs(Ar + j) : T(0);
          b_split<PAIR, T>(v, ah[q][k], al[q][k]);
        }
      }
      Acc y[2] = {acc_zero(), acc_zero()};
#pragma unroll
      for (int k = 0; k < B_CPT; ++k) {
        if (k < cpt) {
          acc_fma(y[0], ah[0][k], al[0][k], xh[k], xl[k]);
          acc_fma(y[1], ah[1][k], al[1][k], xh[k], xl[k]);
        }
      }
      Acc keep = upper ? y[1] : y[0];
      keep = acc_add(keep, shfl_xor_acc2(upper ? y[0] : y[1], W / 2));
#pragma unroll
      for (int o = W / 4; o > 0; o >>= 1) keep = acc_add(keep, shfl_xor_acc2(keep, o));
      if constexpr (TEAM > 32) {  // warps of the team exchange through shared memory
        constexpr int TW = TEAM / 32;
        Acc* ra = reinterpret_cast<Acc*>(red) + (itr & 1) * 2 * BW + team * 2 * TW;  // [TW][2]
        if ((lane & (W / 2 - 1)) == 0) ra[(warp % TW) * 2 + (upper ? 1 : 0)] = keep;
        team_barrier<TEAM>(team);
        keep = team_warps_sum<TW>(ra, lane, upper);
      }
      const Acc other = shfl_xor_acc2(keep, W / 2);
      const Acc yt[2] = {upper ? other : keep, upper ? keep : other};
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        if (vr[q]) {
          const Pair yq = acc_pair(yt[q]);
          const Pair y2 = pair_mul(yq, yq);
          fp = acc_add(fp, Acc{y2.h, y2.l});
          const Pair yb{2.0f * yq.h, 2.0f * yq.l};  // exact
#pragma unroll
          for (int k = 0; k < B_CPT; ++k)
            if (k < cpt) acc_fma(xbp[k], ah[q][k], al[q][k], yb.h, yb.l);
        }
      }
      if ((itr & 7) == 7) {
#pragma unroll
        for (int k = 0; k < B_CPT; ++k) acc_renorm(xbp[k]);
      }
    }
  } else {
    const int iters = (w.count + NT - 1) / NT;
    // software pipeline: the next row's loads are in flight while this row computes
    T an[B_CPT];
    auto load_row = [&](int itr_, T* dst) {
      const int64_t r = w.start + (int64_t)itr_ * NT + team;
      const bool v = itr_ < iters && r < r1;
      const T* Ar = A + (v ? r : w.start) * (int64_t)n;
#pragma unroll
      for (int k = 0; k < B_CPT; ++k) {
        const int j = lt + k * TEAM;
        dst[k] = (k < cpt && v && j < n) ? __ldcs(Ar + j) : T(0);
      }
    };
    load_row(0, an);
    for (int itr = 0; itr < iters; ++itr) {
      const int64_t r = w.start + (int64_t)itr * NT + team;
      const bool valid = r < r1;
      T av[B_CPT];
#pragma unroll
      for (int k = 0; k < B_CPT; ++k) av[k] = an[k];
      load_row(itr + 1, an);
      {
        T d = T(0);
#pragma unroll
        for (int k = 0; k < B_CPT; ++k)
          if (k < cpt) d = fma(av[k], xv[k], d);
#pragma unroll
        for (int o = (TEAM < 32 ? TEAM : 32) / 2; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
        if constexpr (TEAM > 32) {
          constexpr int TW = TEAM / 32;
          T* rt = reinterpret_cast<T*>(red) + (itr & 1) * BW + team * TW;
          if (lane == 0) rt[warp % TW] = d;
          team_barrier<TEAM>(team);
          d = rt[0];
#pragma unroll
          for (int q = 1; q < TW; ++q) d += rt[q];
        }
        if (valid) {
          fn.add(d);
          const T yb = T(2) * d;
#pragma unroll
          for (int k = 0; k < B_CPT; ++k)
            if (k < cpt) xbn[k] = fma(yb, av[k], xbn[k]);
        }
      }
    }
  }
  // combine the teams' partials in team order and store the tile's partial
  __syncthreads();
  if constexpr (PAIR) {
    Acc* out = static_cast<Acc*>(I.partials) + (int64_t)w.tile * n;
    if constexpr (NT == 1) {
#pragma unroll
      for (int k = 0; k < B_CPT; ++k) {
        const int j = lt + k * TEAM;
        if (j < n) out[j] = xbp[k];
      }
    } else {
      Acc* ws = reinterpret_cast<Acc*>(wsp);  // [NT][TEAM * B_CPT]
#pragma unroll
      for (int k = 0; k < B_CPT; ++k) ws[team * TEAM * B_CPT + lt + k * TEAM] = xbp[k];
      __syncthreads();
      for (int j = tid; j < n; j += BT) {
        Acc s = ws[j];
        for (int t2 = 1; t2 < NT; ++t2) s = acc_add(s, ws[t2 * TEAM * B_CPT + j]);
        out[j] = s;
      }
    }
    // in a pair batch wsp lies in the ring: order these generic accesses before
    // the copies that will land there
    fence_proxy_async_smem();
    // f of the tile: team leaders in team order
    Acc* ra = reinterpret_cast<Acc*>(red);
    __syncthreads();
    if (lt == 0) ra[team] = fp;
    __syncthreads();
    Acc tot = ra[0];
    for (int t2 = 1; t2 < NT; ++t2) tot = acc_add(tot, ra[t2]);
    __syncthreads();
    return acc_to_double(tot);
  } else {
    T* out = static_cast<T*>(I.partials) + (int64_t)w.tile * n;
    if constexpr (NT == 1) {
#pragma unroll
      for (int k = 0; k < B_CPT; ++k) {
        const int j = lt + k * TEAM;
        if (j < n) out[j] = xbn[k];
      }
    } else {
      T* ws = reinterpret_cast<T*>(wsp);
#pragma unroll
      for (int k = 0; k < B_CPT; ++k) ws[team * TEAM * B_CPT + lt + k * TEAM] = xbn[k];
      __syncthreads();
      for (int j = tid; j < n; j += BT) {
        T s = ws[j];
        for (int t2 = 1; t2 < NT; ++t2) s += ws[t2 * TEAM * B_CPT + j];
        out[j] = s;
      }
    }
    __syncthreads();
    if (lt == 0) red[team] = fn.get();
    __syncthreads();
    double tot = 0.0;
    for (int t2 = 0; t2 < NT; ++t2) tot += red[t2];
    __syncthreads();
    return tot;
  }
}

// ---- dense tiles of pair batches on float-pair copies: rows staged by bulk copies ----
// A tile's rows are contiguous, so its data arrives by 1-D bulk copies (TMA)
// into a ring of RING_S shared-memory slots, one iteration group (the 2 NT rows
// one iteration of the teams takes, at most 32 KB: about B_CPT columns per
// team thread) a slot, while the teams compute on the slot before: bytes in
// flight without registers.  A copy covers the 16-byte aligned span around its
// rows (a row starts 8 bytes off the boundary when n is odd; those copies are
// the batch's own, allocated 16 bytes longer), and the rows sit `off` bytes into
// the slot.  All threads count the chunks the CTA has consumed (g), which
// gives each slot's barrier phase across tiles; thread 0, the only one that
// issues, counts the chunks issued (iss).  When a tile has no chunk left to
// issue, the slots it frees take the first chunks of the CTA's next item
// (claimed when this one started) if that is a ring tile too, so the copies
// run on across the tile boundary.
constexpr int RING_S = 3;
constexpr int RING_SLOT = 32768 + 128;

struct Ring {
  unsigned char* slots;  // RING_S * RING_SLOT bytes
  uint64_t* full;        // RING_S barriers: a slot's copy has landed
};

// The CTA's next item as ring chunks (thread 0 only); nchunks 0: not a ring tile.
struct RingNext {
  const double* src;   // its first row
  int64_t chunk;       // entries a chunk (2 NT n)
  int64_t total;       // entries of the item (count n)
  int nchunks;
};

constexpr int RING_WS = 1024;  // Acc entries of the team combine's buffer (8 KB)

__device__ __forceinline__ uint32_t ring_issue(const Ring& R, uint32_t g, const void* src, size_t bytes) {
  const uintptr_t lo = reinterpret_cast<uintptr_t>(src) & ~uintptr_t(15);
  const uintptr_t hi = (reinterpret_cast<uintptr_t>(src) + bytes + 15) & ~uintptr_t(15);
  const int slot = (int)(g % RING_S);
  mbar_arrive_expect_tx(&R.full[slot], (uint32_t)(hi - lo));
  tma_load_1d(R.slots + slot * RING_SLOT, reinterpret_cast<const void*>(lo), (uint32_t)(hi - lo),
              &R.full[slot]);
  return (uint32_t)(reinterpret_cast<uintptr_t>(src) - lo);
}

// The dense_tile pair path on a prepared copy, reading its rows from the ring.
// Returns the tile's f; sets `failed` (on all threads) when a copy did not land
// within the wait limit, after waiting for the CTA's other copies in flight.
// CPT > 0: the columns per team thread, ceil(n / TEAM), fixed at compile time
// (no per-column tests but the last column's j < n); 0: at run time.
template <int TEAM, int CPT>
__device__ double dense_tile_ring(const BInst& I, const BItem& w, const Ring& R, uint32_t& g,
                                  uint32_t& iss, const RingNext& nx, unsigned char* wsp, double* red,
                                  bool& bad, bool& failed) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int n = I.n;
  const double* __restrict__ A = static_cast<const double*>(I.d0);  // float pairs, 8 bytes an entry
  const double* __restrict__ x = static_cast<const double*>(I.x);
  constexpr int NT = BT / TEAM;
  constexpr int W = TEAM < 32 ? TEAM : 32;  // lanes of the team inside one warp
  const int lt = tid % TEAM, team = tid / TEAM;
  constexpr int KM = CPT ? CPT : B_CPT;
  const int cpt = CPT ? CPT : (n + TEAM - 1) / TEAM;
  // column k of this thread is in the row: compile-time true below the last one
  auto col_in = [&](int k, int j) { return (CPT && k < CPT - 1) || (k < cpt && j < n); };
  float xh[KM], xl[KM];
  Acc xbp[KM];
#pragma unroll
  for (int k = 0; k < KM; ++k) {
    const int j = lt + k * TEAM;
    const double xv = col_in(k, j) ? x[j] : 0.0;
    bad |= !pair_in_range(xv);
    b_split<true>(xv, xh[k], xl[k]);
    xbp[k] = acc_zero();
  }
  Acc fp = acc_zero();
  const int64_t r1 = w.start + w.count;
  const int nchunks = (w.count + 2 * NT - 1) / (2 * NT);
  auto chunk_src = [&](int c) { return A + (w.start + (int64_t)c * 2 * NT) * n; };
  auto chunk_bytes = [&](int c) {
    const int64_t left = r1 - (w.start + (int64_t)c * 2 * NT);
    return (size_t)(left < 2 * NT ? left : 2 * NT) * n * 8;
  };
  const uint32_t off = (uint32_t)(reinterpret_cast<uintptr_t>(chunk_src(0)) & 15u);
  // chunk row starts are n * 16 bytes apart: every chunk has the same offset
  const uint32_t g0 = g;  // this tile's chunk c is the CTA's chunk g0 + c
  if (tid == 0)  // (the first ones may have been issued by the tile before)
    for (; (int)(iss - g0) < nchunks && iss - g0 < (uint32_t)RING_S; ++iss)
      ring_issue(R, iss, chunk_src((int)(iss - g0)), chunk_bytes((int)(iss - g0)));
  const bool upper = (lane & (W / 2)) != 0;  // keeps the second row
  for (int c = 0; c < nchunks; ++c) {
    const int slot = (int)(g % RING_S);
    const bool ok = mbar_wait_bounded(&R.full[slot], (g / RING_S) & 1u);
    const unsigned char* buf = R.slots + slot * RING_SLOT + off;
    const int64_t row0 = w.start + (int64_t)c * 2 * NT;
    const int64_t rr[2] = {row0 + team, row0 + NT + team};
    const bool vr[2] = {ok && rr[0] < r1, ok && rr[1] < r1};
    float ah[2][KM], al[2][KM];
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const float2* Ar = reinterpret_cast<const float2*>(buf) + (int64_t)(q * NT + team) * n;
#pragma unroll
      for (int k = 0; k < KM; ++k) {
        const int j = lt + k * TEAM;
        const float2 v = (vr[q] && col_in(k, j)) ? Ar[j] : make_float2(0.f, 0.f);
        ah[q][k] = v.x;
        al[q][k] = v.y;
      }
    }
    Acc y[2] = {acc_zero(), acc_zero()};
#pragma unroll
    for (int k = 0; k < KM; ++k) {
      if (CPT || k < cpt) {
        acc_fma(y[0], ah[0][k], al[0][k], xh[k], xl[k]);
        acc_fma(y[1], ah[1][k], al[1][k], xh[k], xl[k]);
      }
    }
    Acc keep = upper ? y[1] : y[0];
    keep = acc_add(keep, shfl_xor_acc2(upper ? y[0] : y[1], W / 2));
#pragma unroll
    for (int o = W / 4; o > 0; o >>= 1) keep = acc_add(keep, shfl_xor_acc2(keep, o));
    // teams wider than a warp exchange their warps' sums through shared memory
    // (two buffers: chunk c + 1 writes the other while chunk c's are read)
    constexpr int TW = TEAM > 32 ? TEAM / 32 : 1;
    Acc* ra = reinterpret_cast<Acc*>(red) + (c & 1) * 2 * BW + team * 2 * TW;  // [TW][2]
    if constexpr (TEAM > 32)
      if ((lane & (W / 2 - 1)) == 0) ra[(warp % TW) * 2 + (upper ? 1 : 0)] = keep;
    // one CTA barrier a chunk: the slot's entries are in registers now, so the
    // slot is refilled here; it also publishes the warps' sums
    if (__syncthreads_or(!ok)) {
      if (tid == 0)  // do not go on with a copy into this CTA's shared memory in flight
        for (uint32_t h = g; h < iss; ++h) mbar_wait_bounded(&R.full[h % RING_S], (h / RING_S) & 1u);
      failed = true;
      __syncthreads();
      return 0.0;
    }
    if (tid == 0 && iss - g0 < (uint32_t)(nchunks + nx.nchunks)) {
      const int k = (int)(iss - g0);
      if (k < nchunks) {
        ring_issue(R, iss, chunk_src(k), chunk_bytes(k));
      } else {  // the next item's chunk k - nchunks
        const int64_t e0 = (int64_t)(k - nchunks) * nx.chunk, left = nx.total - e0;
        ring_issue(R, iss, nx.src + e0, (size_t)(left < nx.chunk ? left : nx.chunk) * 8);
      }
      ++iss;
    }
    ++g;
    if constexpr (TEAM > 32) {
      keep = team_warps_sum<TW>(ra, lane, upper);
    }
    const Acc other = shfl_xor_acc2(keep, W / 2);
    const Acc yt[2] = {upper ? other : keep, upper ? keep : other};
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      if (vr[q]) {
        const Pair yq = acc_pair(yt[q]);
        const Pair y2 = pair_mul(yq, yq);
        fp = acc_add(fp, Acc{y2.h, y2.l});
        const Pair yb{2.0f * yq.h, 2.0f * yq.l};  // exact
#pragma unroll
        for (int k = 0; k < KM; ++k)
          if (CPT || k < cpt) acc_fma(xbp[k], ah[q][k], al[q][k], yb.h, yb.l);
      }
    }
    if ((c & 7) == 7) {
#pragma unroll
      for (int k = 0; k < KM; ++k) acc_renorm(xbp[k]);
    }
  }
  // combine the teams' partials in team order and store the tile's partial, in
  // two halves of the columns through RING_WS entries (outside the ring, into
  // which the next item's copies may be landing)
  Acc* out = static_cast<Acc*>(I.partials) + (int64_t)w.tile * n;
  if constexpr (NT == 1) {
#pragma unroll
    for (int k = 0; k < KM; ++k) {
      const int j = lt + k * TEAM;
      if (j < n) out[j] = xbp[k];
    }
  } else {
    constexpr int H = B_CPT / 2;
    static_assert(BT * H <= RING_WS, "the combine buffer holds half the columns of all teams");
    Acc* ws = reinterpret_cast<Acc*>(wsp);  // [NT][TEAM * H]
#pragma unroll
    for (int half = 0; half < 2; ++half) {
#pragma unroll
      for (int kk = 0; kk < H; ++kk)  // columns k >= KM are past the row's end: not read
        if (half * H + kk < KM) ws[team * TEAM * H + lt + kk * TEAM] = xbp[half * H + kk < KM ? half * H + kk : 0];
      __syncthreads();
      for (int jj = tid; jj < TEAM * H; jj += BT) {
        const int j = jj % TEAM + (half * H + jj / TEAM) * TEAM;
        if (j < n) {
          Acc s = ws[jj];
          for (int t2 = 1; t2 < NT; ++t2) s = acc_add(s, ws[t2 * TEAM * H + jj]);
          out[j] = s;
        }
      }
      __syncthreads();
    }
  }
  Acc* ra = reinterpret_cast<Acc*>(red);
  __syncthreads();
  if (lt == 0) ra[team] = fp;
  __syncthreads();
  Acc tot = ra[0];
  for (int t2 = 1; t2 < NT; ++t2) tot = acc_add(tot, ra[t2]);
  __syncthreads();
  return acc_to_double(tot);
}

// Elements [w.start, w.start + w.count) of a tet instance; returns the tile's f.
template <typename T, bool PAIR, bool WARPC, bool PREP>
__device__ double tet_tile(const BInst& I, const BItem& w, const float4* tab, const LogConsts& K,
                           double* red, bool& bad) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int4* conn = static_cast<const int4*>(I.d0);
  const T* G = static_cast<const T*>(I.d1);
  const T* u = static_cast<const T*>(I.x);
  T* gu = static_cast<T*>(I.gx);
  Acc fp = acc_zero();
  T fn = T(0);
  const int64_t e1 = w.start + w.count;
  int cnt = 0;
  if constexpr (!WARPC) {  // one atomic per contribution
    for (int64_t e = w.start + tid; e < e1; e += BT, ++cnt) {
      const int4 c = __ldcs(conn + e);
      if constexpr (PAIR) {
        elem_pair<TS_GRAD, AtomicSink<double>, PREP>(
            c, reinterpret_cast<const double*>(G) + e * 12, reinterpret_cast<const double*>(u),
            Pair{2.0f, 0.0f}, tab, K, fp, AtomicSink<double>{reinterpret_cast<double*>(gu)}, nullptr,
            bad);
        if ((cnt & 31) == 31) acc_renorm(fp);
      } else {
        elem_native<T, TS_GRAD>(c, G + e * 12, u, T(1), fn, AtomicSink<T>{gu}, nullptr);
      }
    }
  }
  // WARPC: block-uniform loop, so that every lane reaches the warp-level combine
  for (int64_t e0 = w.start; WARPC && e0 < e1; e0 += BT, ++cnt) {
    const int64_t e = e0 + tid;
    const bool act = e < e1;
    T cv[4];
    Pair cpr[4];
    int4 c = make_int4(-1, -1, -1, -1);
    if (act) {
      c = __ldcs(conn + e);
      if constexpr (PAIR) {
        elem_pair<TS_GRAD, CollectSink<T>, PREP>(
            c, reinterpret_cast<const double*>(G) + e * 12, reinterpret_cast<const double*>(u),
            Pair{2.0f, 0.0f}, tab, K, fp, CollectSink<T>{cv, cpr}, nullptr, bad);
        if ((cnt & 31) == 31) acc_renorm(fp);
      } else {
        elem_native<T, TS_GRAD>(c, G + e * 12, u, T(1), fn, CollectSink<T>{cv, cpr}, nullptr);
      }
    }
    const int key[4] = {c.x, c.y, c.z, c.w};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      if constexpr (PAIR) {
        warp_combine(act, key[k], Acc{cpr[k].h, cpr[k].l},
                     [](Acc x, Acc y) { return acc_add(x, y); },
                     [&](int v, Acc tot) {
                       red_add(reinterpret_cast<double*>(gu) + v, pair_to_double_fast(acc_pair(tot)));
                     });
      } else {
        warp_combine(act, key[k], cv[k], [](T x, T y) { return x + y; },
                     [&](int v, T tot) { red_add(gu + v, tot); });
      }
    }
  }
  __syncthreads();
  if constexpr (PAIR) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) fp = acc_add(fp, shfl_xor_acc2(fp, o));
    Acc* ra = reinterpret_cast<Acc*>(red);
    if (lane == 0) ra[warp] = fp;
    __syncthreads();
    Acc tot = ra[0];
    for (int q = 1; q < BW; ++q) tot = acc_add(tot, ra[q]);
    __syncthreads();
    return acc_to_double(tot);
  } else {
    const double t = block_sum((double)fn, red);
    __syncthreads();
    return t;
  }
}

template <typename T, bool PAIR>
__device__ __forceinline__ double dense_dispatch(const BInst& I, const BItem& w, unsigned char* wsp,
                                                 double* red, bool& bad) {
  switch (I.team) {
    case 4: return dense_tile<T, PAIR, 4>(I, w, wsp, red, bad);
    case 8: return dense_tile<T, PAIR, 8>(I, w, wsp, red, bad);
    case 16: return dense_tile<T, PAIR, 16>(I, w, wsp, red, bad);
    case 32: return dense_tile<T, PAIR, 32>(I, w, wsp, red, bad);
    case 64: return dense_tile<T, PAIR, 64>(I, w, wsp, red, bad);
    case 128: return dense_tile<T, PAIR, 128>(I, w, wsp, red, bad);
    default: return dense_tile<T, PAIR, BT>(I, w, wsp, red, bad);
  }
}

// The team is the smallest power of two (>= 4) with 8 columns a thread, so
// above 4 threads a team thread has 5 to 8 columns.
template <int TEAM>
__device__ __forceinline__ double dense_ring_cpt(const BInst& I, const BItem& w, const Ring& R, uint32_t& g,
                                                 uint32_t& iss, const RingNext& nx, unsigned char* wsp,
                                                 double* red, bool& bad, bool& failed) {
  switch ((I.n + TEAM - 1) / TEAM) {
    case 5: return dense_tile_ring<TEAM, 5>(I, w, R, g, iss, nx, wsp, red, bad, failed);
    case 6: return dense_tile_ring<TEAM, 6>(I, w, R, g, iss, nx, wsp, red, bad, failed);
    case 7: return dense_tile_ring<TEAM, 7>(I, w, R, g, iss, nx, wsp, red, bad, failed);
    case 8: return dense_tile_ring<TEAM, 8>(I, w, R, g, iss, nx, wsp, red, bad, failed);
    default: return dense_tile_ring<TEAM, 0>(I, w, R, g, iss, nx, wsp, red, bad, failed);
  }
}

__device__ __forceinline__ double dense_ring_dispatch(const BInst& I, const BItem& w, const Ring& R,
                                                      uint32_t& g, uint32_t& iss, const RingNext& nx,
                                                      unsigned char* wsp, double* red, bool& bad,
                                                      bool& failed) {
  switch (I.team) {
    case 4: return dense_tile_ring<4, 0>(I, w, R, g, iss, nx, wsp, red, bad, failed);
    case 8: return dense_ring_cpt<8>(I, w, R, g, iss, nx, wsp, red, bad, failed);
    case 16: return dense_ring_cpt<16>(I, w, R, g, iss, nx, wsp, red, bad, failed);
    case 32: return dense_ring_cpt<32>(I, w, R, g, iss, nx, wsp, red, bad, failed);
    case 64: return dense_ring_cpt<64>(I, w, R, g, iss, nx, wsp, red, bad, failed);
    case 128: return dense_ring_cpt<128>(I, w, R, g, iss, nx, wsp, red, bad, failed);
    default: return dense_ring_cpt<BT>(I, w, R, g, iss, nx, wsp, red, bad, failed);
  }
}

// Last tile of an instance: sum the tile partials in tile order.
template <typename T, bool PAIR>
__device__ void finalize(const BInst& I, double* red) {
  const int tid = threadIdx.x;
  if (I.kind == BK_DENSE) {
    const int n = I.n;
    for (int j = tid; j < n; j += BT) {
      if constexpr (PAIR) {
        const Acc* P = static_cast<const Acc*>(I.partials);
        Acc s = acc_zero();
        for (int t = 0; t < I.ntiles; ++t) {
          const float2 v = __ldcg(reinterpret_cast<const float2*>(P + (int64_t)t * n + j));
          s = acc_add(s, Acc{v.x, v.y});
          if ((t & 31) == 31) acc_renorm(s);
        }
        static_cast<double*>(I.gx)[j] = pair_to_double_fast(acc_pair(s));
      } else {
        const T* P = static_cast<const T*>(I.partials);
        T s = T(0);
        for (int t = 0; t < I.ntiles; ++t) s += __ldcg(P + (int64_t)t * n + j);
        static_cast<T*>(I.gx)[j] = s;
      }
    }
  }
  if (tid == 0 && I.f) {
    double fs = 0.0;
    for (int t = 0; t < I.ntiles; ++t) fs += __ldcg(I.fpart + t);
    *static_cast<T*>(I.f) = (T)fs;
  }
}

template <typename T, bool PAIR>
__global__ void __launch_bounds__(BT, 2) batched_kernel(BArgs a) {
  // PAIR: [log table][ring: RING_S slots][ring combine buffer][red][ring barriers];
  // the other dense tiles of a pair batch combine inside the ring (idle then).
  // Otherwise [wsp][red].
  extern __shared__ __align__(16) unsigned char smem[];
  float4* tab = reinterpret_cast<float4*>(smem);
  unsigned char* wsp = smem + (PAIR ? kLogTableSize * sizeof(float4) : 0);
  unsigned char* rws = wsp + (PAIR ? (size_t)RING_S * RING_SLOT : 0);
  double* red = reinterpret_cast<double*>(PAIR ? rws + RING_WS * sizeof(Acc) : wsp + (size_t)BT * B_CPT * 8);
  Ring R{wsp, reinterpret_cast<uint64_t*>(red + 64)};
  uint32_t g = 0, iss = 0;  // ring chunks consumed by this CTA; issued (thread 0)
  __shared__ int s_item, s_last;
  const int tid = threadIdx.x;
  if constexpr (PAIR) {
    for (int i = tid; i < kLogTableSize; i += BT) tab[i] = a.logtab[i];
    if (tid == 0) {
      for (int i = 0; i < RING_S; ++i) mbar_init(&R.full[i], 1);
      fence_barrier_init();
    }
  }
  bool bad = false, failed = false;
  // items are claimed one ahead: the next one's first copies can be issued
  // during this one (pair batches)
  if (tid == 0) s_item = (int)atomicAdd(&a.head[0], 1u);
  __syncthreads();
  int it = s_item;
  for (;;) {
    __syncthreads();  // every thread has read s_item
    if (it >= a.nitems) break;
    RingNext nx{nullptr, 0, 0, 0};
    if (tid == 0) {
      const int nit = (int)atomicAdd(&a.head[0], 1u);
      s_item = nit;
      if (PAIR && nit < a.nitems) {
        const BItem wn = a.items[nit];
        const BInst& In = a.insts[wn.inst];
        if (In.kind == BK_DENSE && In.prep) {
          const int64_t rows = 2 * (BT / In.team);
          nx.src = static_cast<const double*>(In.d0) + wn.start * (int64_t)In.n;
          nx.chunk = rows * In.n;
          nx.total = (int64_t)wn.count * In.n;
          nx.nchunks = (int)((wn.count + rows - 1) / rows);
        }
      }
    }
    const BItem w = a.items[it];
    const BInst I = a.insts[w.inst];
    // the tile's contiguous data into L2 while the first loads are in flight (not
    // for the ring's tiles: their copies stream it, and whole-tile prefetches of
    // every CTA exceed L2 and are evicted before use)
    if (tid == 0) {
      if (I.kind == BK_DENSE) {
        if (!(PAIR && I.prep))
          prefetch_range_l2(static_cast<const T*>(I.d0) + w.start * (int64_t)I.n,
                            (size_t)w.count * I.n * sizeof(T));
      } else {
        prefetch_range_l2(static_cast<const int4*>(I.d0) + w.start, (size_t)w.count * 16);
        prefetch_range_l2(static_cast<const T*>(I.d1) + w.start * 12, (size_t)w.count * 12 * sizeof(T));
      }
    }
    double ft;
    const bool prep = PAIR && I.prep;
    if (I.kind == BK_DENSE) {
      if constexpr (PAIR) {
        ft = prep ? dense_ring_dispatch(I, w, R, g, iss, nx, rws, red, bad, failed)
                  : dense_dispatch<T, PAIR>(I, w, wsp, red, bad);
        if (failed) {  // a copy did not land: this CTA leaves the queue
          if (tid == 0) set_error(a.err, ERRBIT_TIMEOUT);
          break;
        }
      } else {
        ft = dense_dispatch<T, PAIR>(I, w, wsp, red, bad);
      }
    } else {
      if (a.warpc)
        ft = prep ? tet_tile<T, PAIR, true, true>(I, w, tab, a.K, red, bad)
                  : tet_tile<T, PAIR, true, false>(I, w, tab, a.K, red, bad);
      else
        ft = prep ? tet_tile<T, PAIR, false, true>(I, w, tab, a.K, red, bad)
                  : tet_tile<T, PAIR, false, false>(I, w, tab, a.K, red, bad);
    }
    if (tid == 0) I.fpart[w.tile] = ft;
    __threadfence();
    __syncthreads();
    if (tid == 0) s_last = atomicAdd(I.done, 1u) == (unsigned)I.ntiles - 1u;
    __syncthreads();
    if (s_last) {
      __threadfence();
      finalize<T, PAIR>(I, red);
      if (tid == 0) *I.done = 0u;
    }
    it = s_item;  // written by thread 0 before the barriers above
  }
  if (bad) set_error(a.err, ERRBIT_RANGE);
  if (tid == 0) {  // the last CTA to leave resets the queue for the next replay
    __threadfence();
    if (atomicAdd(&a.head[1], 1u) == gridDim.x - 1) {
      a.head[0] = 0u;
      a.head[1] = 0u;
      __threadfence();
    }
  }
}

template <typename T>
__global__ void batched_zero_kernel(const BInst* __restrict__ insts, const int* __restrict__ ids,
                                    int count) {
  for (int k = blockIdx.x; k < count; k += gridDim.x) {
    const BInst I = insts[ids[k]];
    T* g = static_cast<T*>(I.gx);
    for (int j = threadIdx.x; j < I.n; j += blockDim.x) g[j] = T(0);
  }
}

}  // namespace kg

// ------------------------------------------------------------------ host --
using namespace kg;

namespace {

size_t batched_smem(bool pair) {
  if (pair)
    return kLogTableSize * sizeof(float4) + (size_t)RING_S * RING_SLOT + RING_WS * sizeof(Acc) +
           64 * sizeof(double) + RING_S * sizeof(uint64_t);
  return (size_t)BT * B_CPT * 8 + 64 * sizeof(double);
}

int bucket_of(int64_t v) {
  int b = 0;
  while ((int64_t(1) << (b + 1)) <= v) ++b;
  return b;
}

// ---- tuning cache: one JSON object of "key": value lines ----
std::mutex g_tune_mu;

std::string cache_path() {
  if (const char* p = std::getenv("KG_TUNE_CACHE")) return p;
  const char* home = std::getenv("HOME");
  return std::string(home ? home : ".") + "/.cache/kg_tune.json";
}

std::map<std::string, int> cache_read() {
  std::map<std::string, int> m;
  std::ifstream in(cache_path());
  std::string line;
  while (std::getline(in, line)) {
    const size_t q1 = line.find('"'), q2 = line.find('"', q1 + 1), c = line.find(':', q2 + 1);
    if (q1 == std::string::npos || q2 == std::string::npos || c == std::string::npos) continue;
    m[line.substr(q1 + 1, q2 - q1 - 1)] = std::atoi(line.c_str() + c + 1);
  }
  return m;
}

void cache_write(const std::map<std::string, int>& m) {
  const std::string path = cache_path();
  const size_t slash = path.rfind('/');
  if (slash != std::string::npos) {  // create the parent directories
    const std::string dir = path.substr(0, slash);
    for (size_t i = 1; i <= dir.size(); ++i)
      if (i == dir.size() || dir[i] == '/') mkdir(dir.substr(0, i).c_str(), 0755);
  }
  const std::string tmp = path + ".tmp";
  std::ofstream out(tmp);
  if (!out) return;
  out << "{\n";
  size_t i = 0;
  for (const auto& kv : m) out << "  \"" << kv.first << "\": " << kv.second << (++i < m.size() ? ",\n" : "\n");
  out << "}\n";
  out.close();
  std::rename(tmp.c_str(), path.c_str());
}

}  // namespace

namespace {

// ---- plans: instances cut into tiles ----
struct Plan {
  std::vector<BInst> insts;
  std::vector<BItem> items;
  std::vector<int> tet_ids;
  std::vector<size_t> part_off;  // byte offset of each dense instance's partials
  std::vector<size_t> fpart_off; // index of each instance's first f partial
  size_t part_bytes = 0, fparts = 0;
};

struct Tuning {
  std::map<int, int> dense_rows;   // bucket -> rows per item
  std::map<int, int> tet_elems;    // bucket -> elements per item
};

int default_rows(int n) { return n <= 64 ? 128 : n <= 256 ? 64 : (n <= 1024 ? 16 : 8); }
int default_elems(int64_t) { return 4096; }

// prep[i]: the float-pair copy of problem i's A (dense) or G (tet) that the
// batch streams, or NULL (the FP64 data, split per load).
Plan make_plan(const std::vector<kg_problem*>& probs, const std::vector<const void*>& prep,
               const std::vector<int>& ids, const Tuning& tu, bool pair, size_t es) {
  Plan P;
  struct Cost {
    double c;
    BItem it;
  };
  std::vector<Cost> all;
  for (int idx = 0; idx < (int)ids.size(); ++idx) {
    const kg_problem* p = probs[ids[idx]];
    BInst I{};
    I.kind = p->kind == KG_QUADFORM ? BK_DENSE : BK_TET;
    I.n = (int)p->n;
    I.m = p->m;
    I.d0 = p->data0;
    I.d1 = p->data1;
    if (pair && prep[ids[idx]]) {  // stream the prepared float pairs
      I.prep = 1;
      if (p->kind == KG_QUADFORM) I.d0 = prep[ids[idx]];
      else I.d1 = prep[ids[idx]];
    }
    int64_t per;
    if (I.kind == BK_DENSE) {
      auto f = tu.dense_rows.find(bucket_of(p->n));
      per = f != tu.dense_rows.end() ? f->second : default_rows((int)p->n);
      // row team: about B_CPT columns per thread (4 .. 256 threads)
      I.team = 4;
      while (I.team < BT && (int64_t)I.team * B_CPT < p->n) I.team *= 2;
    } else {
      auto f = tu.tet_elems.find(bucket_of(p->m));
      per = f != tu.tet_elems.end() ? f->second : default_elems(p->m);
      I.team = 0;
      P.tet_ids.push_back(idx);
    }
    I.ntiles = (int)((I.m + per - 1) / per);
    P.fpart_off.push_back(P.fparts);
    P.fparts += I.ntiles;
    P.part_off.push_back(P.part_bytes);
    if (I.kind == BK_DENSE) {
      const size_t b = (size_t)I.ntiles * I.n * (pair ? sizeof(Acc) : es);
      P.part_bytes += (b + 255) & ~size_t(255);
    }
    for (int t = 0; t < I.ntiles; ++t) {
      BItem it{idx, t, (int64_t)t * per, (int)std::min<int64_t>(per, I.m - (int64_t)t * per)};
      const double bytes = I.kind == BK_DENSE ? (double)it.count * I.n * es
                                              : (double)it.count * (16.0 + 12.0 * es);
      all.push_back({bytes, it});
    }
    P.insts.push_back(I);
  }
  std::stable_sort(all.begin(), all.end(), [](const Cost& a, const Cost& b) { return a.c > b.c; });
  for (const auto& c : all) P.items.push_back(c.it);
  return P;
}

// Device copy of a plan with its workspaces; x/f/gx filled per call.
struct DevPlan {
  BInst* insts = nullptr;
  BItem* items = nullptr;
  int* tet_ids = nullptr;
  unsigned* head = nullptr;
  unsigned* done = nullptr;
  unsigned char* parts = nullptr;
  double* fpart = nullptr;
  int nitems = 0, ntet = 0, ninst = 0;
  std::vector<void*> allocs;
  void release() {
    for (void* p : allocs) cudaFree(p);
    allocs.clear();
  }
};

kg_status devplan_alloc(DevPlan& D, Plan& P, cudaStream_t s) {
  auto al = [&](void** ptr, size_t bytes, const char* what) -> kg_status {
    cudaError_t e = dev_alloc(ptr, bytes);
    if (e != cudaSuccess) return fail(KG_ERR_OOM, std::string("batch workspace: ") + what);
    D.allocs.push_back(*ptr);
    return KG_OK;
  };
  kg_status rc;
  D.ninst = (int)P.insts.size();
  D.nitems = (int)P.items.size();
  D.ntet = (int)P.tet_ids.size();
  if ((rc = al((void**)&D.insts, sizeof(BInst) * P.insts.size(), "descriptors")) != KG_OK) return rc;
  if ((rc = al((void**)&D.items, sizeof(BItem) * P.items.size(), "work table")) != KG_OK) return rc;
  if ((rc = al((void**)&D.tet_ids, sizeof(int) * std::max<size_t>(1, P.tet_ids.size()), "tet ids")) != KG_OK) return rc;
  if ((rc = al((void**)&D.head, 16, "queue head")) != KG_OK) return rc;
  if ((rc = al((void**)&D.done, sizeof(unsigned) * P.insts.size(), "arrival counters")) != KG_OK) return rc;
  if ((rc = al((void**)&D.parts, std::max<size_t>(256, P.part_bytes), "partials")) != KG_OK) return rc;
  if ((rc = al((void**)&D.fpart, sizeof(double) * std::max<size_t>(1, P.fparts), "f partials")) != KG_OK) return rc;
  for (int i = 0; i < D.ninst; ++i) {
    P.insts[i].partials = D.parts + P.part_off[i];
    P.insts[i].fpart = D.fpart + P.fpart_off[i];
    P.insts[i].done = D.done + i;
  }
  cudaError_t e;
  if ((e = cudaMemsetAsync(D.head, 0, 16, s)) != cudaSuccess) return cuda_fail(e, "batch set-up");
  if ((e = cudaMemsetAsync(D.done, 0, sizeof(unsigned) * P.insts.size(), s)) != cudaSuccess)
    return cuda_fail(e, "batch set-up");
  if ((e = cudaMemcpyAsync(D.items, P.items.data(), sizeof(BItem) * P.items.size(),
                           cudaMemcpyHostToDevice, s)) != cudaSuccess)
    return cuda_fail(e, "batch set-up");
  if (!P.tet_ids.empty() &&
      (e = cudaMemcpyAsync(D.tet_ids, P.tet_ids.data(), sizeof(int) * P.tet_ids.size(),
                           cudaMemcpyHostToDevice, s)) != cudaSuccess)
    return cuda_fail(e, "batch set-up");
  return KG_OK;
}

// The pair kernels' shared memory (the ring) is above the 48 KB default: raise
// their limit before the first occupancy query or launch.
cudaError_t batched_smem_attrs() {
  return cudaFuncSetAttribute(batched_kernel<double, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)batched_smem(true));
}

int batched_grid(bool pair) {
  int per = 0, dev = 0;
  cudaGetDevice(&dev);
  const size_t smem = batched_smem(pair);
  cudaError_t e;
  if (pair)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, batched_kernel<double, true>, BT, smem);
  else
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, batched_kernel<double, false>, BT, smem);
  if (e != cudaSuccess || per < 1) per = 2;
  return num_sms() * std::min(per, 4);
}

// Launches the zero kernel (tet gradients) and the persistent kernel on s.
static void launch_batched(int dtype, bool pair, int grid, size_t smem, cudaStream_t s, const BArgs& a) {
  if (dtype == KG_F64) {
    if (pair) batched_kernel<double, true><<<grid, BT, smem, s>>>(a);
    else batched_kernel<double, false><<<grid, BT, smem, s>>>(a);
  } else {
    batched_kernel<float, false><<<grid, BT, smem, s>>>(a);
  }
}

kg_status launch_plan(const DevPlan& D, int dtype, bool pair, bool warp, unsigned* err,
                      cudaStream_t s, int grid) {
  cudaError_t e = cudaSuccess;
  if (D.ntet > 0) {
    const int zg = std::min(D.ntet, num_sms() * 4);
    if (dtype == KG_F64) batched_zero_kernel<double><<<zg, 256, 0, s>>>(D.insts, D.tet_ids, D.ntet);
    else batched_zero_kernel<float><<<zg, 256, 0, s>>>(D.insts, D.tet_ids, D.ntet);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "batched zero kernel");
  }
  BArgs a{};
  a.insts = D.insts;
  a.items = D.items;
  a.nitems = D.nitems;
  a.head = D.head;
  a.err = err;
  a.K = log_consts();
  if (pair) {
    kg_status rc = logtab_for_device(&a.logtab);
    if (rc != KG_OK) return rc;
  }
  a.warpc = warp ? 1 : 0;
  launch_batched(dtype, pair, grid, batched_smem(pair), s, a);
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "batched kernel");
  return KG_OK;
}

}  // namespace

struct kg_batch {
  std::vector<kg_problem*> probs;
  std::vector<const void*> prep;  // per problem: the float-pair copy streamed, or NULL
  std::vector<void*> own_preps;   // the copies the batch made itself
  int dtype = KG_F64;
  bool pair = false;
  bool warp = false;  // tet scatter: warp-combined atomics (false: one atomic per contribution)
  size_t es = 8;
  Plan plan;
  DevPlan dev;
  unsigned* err = nullptr;
  int grid = 0;
  Tuning tune;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  std::vector<const void*> last_x, last_f, last_gx;
  bool ptrs_valid = false;
  cudaStream_t last_stream = nullptr;
  std::string gpu;
};

namespace {

std::string gpu_name() {
  int dev = 0;
  cudaDeviceProp pr{};
  if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&pr, dev) != cudaSuccess)
    return "unknown";
  std::string s = pr.name;
  for (char& c : s)
    if (c == '"' || c == '|') c = '_';
  return s;
}

// Times the persistent kernel on the instances `ids` with tuning `tu`.
kg_status time_plan(kg_batch* b, const std::vector<int>& ids, const Tuning& tu, cudaStream_t s,
                    void* xbuf, void* gbuf, float* ms) {
  Plan P = make_plan(b->probs, b->prep, ids, tu, b->pair, b->es);
  DevPlan D;
  kg_status rc = devplan_alloc(D, P, s);
  if (rc == KG_OK) {
    size_t off = 0;
    for (auto& I : P.insts) {
      I.x = static_cast<unsigned char*>(xbuf) + off;
      I.gx = static_cast<unsigned char*>(gbuf) + off;
      I.f = nullptr;
      off += ((size_t)I.n * b->es + 255) & ~size_t(255);
    }
    cudaError_t e = cudaMemcpyAsync(D.insts, P.insts.data(), sizeof(BInst) * P.insts.size(),
                                    cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) rc = cuda_fail(e, "autotune");
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (rc == KG_OK && (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess))
      rc = fail(KG_ERR_CUDA, "autotune events");
    float best = 1e30f;
    for (int r = 0; rc == KG_OK && r < 4; ++r) {
      cudaEventRecord(e0, s);
      rc = launch_plan(D, b->dtype, b->pair, b->warp, b->err, s, b->grid);
      cudaEventRecord(e1, s);
      if (rc == KG_OK && (e = cudaEventSynchronize(e1)) != cudaSuccess) rc = cuda_fail(e, "autotune");
      float t = 0.f;
      if (rc == KG_OK && r > 0 && cudaEventElapsedTime(&t, e0, e1) == cudaSuccess) best = std::min(best, t);
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    *ms = best;
  }
  cudaStreamSynchronize(s);
  D.release();
  return rc;
}

// Chooses rows (dense) / elements (tet) per item for every size bucket of the
// batch: each candidate runs on a sample of the bucket's instances large
// enough that the largest candidate still gives four items per CTA of the
// persistent grid (or on all of them); the fastest wins.  A smaller sample
// would favour small tiles for want of parallelism that the whole batch has.
// Choices are cached by GPU name, kind, dtype, arithmetic and bucket.
kg_status autotune(kg_batch* b, cudaStream_t s) {
  std::map<std::pair<int, int>, std::vector<int>> groups;  // (kind, bucket) -> instance ids
  for (int i = 0; i < (int)b->probs.size(); ++i) {
    const kg_problem* p = b->probs[i];
    const int kind = p->kind == KG_QUADFORM ? BK_DENSE : BK_TET;
    groups[{kind, bucket_of(kind == BK_DENSE ? p->n : p->m)}].push_back(i);
  }
  std::lock_guard<std::mutex> lk(g_tune_mu);
  std::map<std::string, int> cache = cache_read();
  bool dirty = false;
  // "k3": dense tiles of pair batches stream float-pair copies through a ring; larger samples
  const std::string prefix = b->gpu + "|k3|" + (b->dtype == KG_F64 ? "f64" : "f32") + "|" +
                             (b->pair ? "pair" : "native") + "|";
  const std::vector<int> dense_cands{4, 8, 16, 32, 64, 128, 256}, tet_cands{1024, 2048, 4096, 8192, 16384};
  std::map<std::pair<int, int>, std::vector<int>> sample;
  for (auto& g : groups) {
    const int64_t biggest = g.first.first == BK_DENSE ? dense_cands.back() : tet_cands.back();
    std::vector<int>& ids = sample[g.first];
    int64_t items = 0;
    for (int i : g.second) {
      ids.push_back(i);
      items += (b->probs[i]->m + biggest - 1) / biggest;
      if (items >= 4 * (int64_t)b->grid) break;
    }
  }
  // scratch x / gx for the timing runs (zeros are valid inputs for both kinds)
  size_t need = 0;
  for (auto& g : sample) {
    size_t sz = 0;
    for (int i : g.second) sz += ((size_t)b->probs[i]->n * b->es + 255) & ~size_t(255);
    need = std::max(need, sz);
  }
  void *xbuf = nullptr, *gbuf = nullptr;
  if (dev_alloc(&xbuf, need) != cudaSuccess || dev_alloc(&gbuf, need) != cudaSuccess) {
    cudaFree(xbuf);
    return fail(KG_ERR_OOM, "autotune scratch");
  }
  cudaMemsetAsync(xbuf, 0, need, s);
  kg_status rc = KG_OK;
  for (auto& g : groups) {
    const int kind = g.first.first, bucket = g.first.second;
    const std::string key = prefix + (kind == BK_DENSE ? "dense|" : "tet|") + std::to_string(bucket);
    auto hit = cache.find(key);
    if (hit != cache.end()) {
      (kind == BK_DENSE ? b->tune.dense_rows : b->tune.tet_elems)[bucket] = hit->second;
      continue;
    }
    const std::vector<int>& ids = sample[g.first];
    const std::vector<int>& cands = kind == BK_DENSE ? dense_cands : tet_cands;
    int best = cands[0];
    float best_ms = 1e30f;
    for (int c : cands) {
      Tuning tu;
      (kind == BK_DENSE ? tu.dense_rows : tu.tet_elems)[bucket] = c;
      float ms = 0.f;
      if ((rc = time_plan(b, ids, tu, s, xbuf, gbuf, &ms)) != KG_OK) break;
      if (ms < best_ms) {
        best_ms = ms;
        best = c;
      }
    }
    if (rc != KG_OK) break;
    (kind == BK_DENSE ? b->tune.dense_rows : b->tune.tet_elems)[bucket] = best;
    cache[key] = best;
    dirty = true;
  }
  cudaFree(xbuf);
  cudaFree(gbuf);
  if (rc == KG_OK && dirty) cache_write(cache);
  return rc;
}

void batch_free(kg_batch* b) {
  if (!b) return;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->dev.release();
  for (void* q : b->own_preps) cudaFree(q);
  if (b->err) cudaFree(b->err);
  delete b;
}

}  // namespace

extern "C" {

kg_status kg_batch_create(kg_batch** out, kg_problem* const* probs, int count,
                          const kg_options* opt, kg_stream stream) {
  if (!out) return fail(KG_ERR_INVALID_ARG, "kg_batch_create: out is NULL");
  *out = nullptr;
  if (!probs || count < 1) return fail(KG_ERR_INVALID_ARG, "kg_batch_create: no problems");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  kg_batch* b = new (std::nothrow) kg_batch();
  if (!b) return fail(KG_ERR_OOM, "kg_batch_create: host allocation");
  b->probs.assign(probs, probs + count);
  b->dtype = b->probs[0] ? b->probs[0]->dtype : KG_F64;
  b->es = b->dtype == KG_F64 ? 8 : 4;
  kg_status rc = KG_OK;
  const int strat = opt ? opt->strategy : KG_STRATEGY_AUTO;
  if (strat != KG_STRATEGY_AUTO && strat != KG_STRATEGY_WARP && strat != KG_STRATEGY_ATOMIC)
    rc = fail(KG_ERR_UNSUPPORTED, "kg_batch_create: strategy must be AUTO, WARP or ATOMIC");
  b->warp = strat == KG_STRATEGY_WARP;  // AUTO: plain atomics (measured ~3% faster here)
  for (kg_problem* p : b->probs) {
    if (rc != KG_OK) break;
    if (!p) rc = fail(KG_ERR_INVALID_ARG, "kg_batch_create: NULL problem");
    else if (p->dtype != b->dtype) rc = fail(KG_ERR_INVALID_ARG, "kg_batch_create: mixed dtypes");
    else if (p->kind == KG_QUADFORM && p->n > B_MAXN)
      rc = fail(KG_ERR_UNSUPPORTED, "kg_batch_create: dense instances need n <= 2048");
    else if (p->kind != KG_QUADFORM && p->kind != KG_TETENERGY)
      rc = fail(KG_ERR_UNSUPPORTED, "kg_batch_create: QUADFORM and TETENERGY only");
    if (rc != KG_OK) break;
  }
  if (rc == KG_OK && dev_alloc((void**)&b->err, 16) != cudaSuccess)
    rc = fail(KG_ERR_OOM, "kg_batch_create: error word");
  if (rc == KG_OK) cudaMemsetAsync(b->err, 0, 16, s);
  // FP64 arithmetic of the batch: pairs when every instance's data is in range
  if (rc == KG_OK && b->dtype == KG_F64) {
    const int want = opt ? opt->arith : KG_ARITH_AUTO;
    bool pair = want != KG_ARITH_NATIVE;
    for (kg_problem* p : b->probs) {
      if (!pair) break;
      if (p->arith == KG_ARITH_PAIR) continue;
      if (p->kind == KG_TETENERGY) {
        pair = false;
        break;
      }
      bool ok = false;
      if ((rc = pair_range_ok(p, static_cast<const double*>(p->data0), p->m * p->n, s, &ok)) != KG_OK)
        break;
      pair = ok;
    }
    if (rc == KG_OK && want == KG_ARITH_PAIR && !pair)
      rc = fail(KG_ERR_UNSUPPORTED, "kg_batch_create: some data is outside the pair range");
    b->pair = pair;
  }
  // the float-pair copies: the instances' own, else (dense instances whose
  // kg_create took none, n < 1024) one the batch makes, largest first, within
  // opt->tape_budget_bytes (0: 1 GiB)
  b->prep.assign(count, nullptr);
  if (rc == KG_OK && b->pair) {
    size_t budget = opt && opt->tape_budget_bytes ? opt->tape_budget_bytes : (size_t(1) << 30);
    std::vector<int> order;
    for (int i = 0; i < count; ++i) {
      kg_problem* p = b->probs[i];
      if (p->aprep && p->arith == KG_ARITH_PAIR) b->prep[i] = p->aprep;
      else if (p->kind == KG_QUADFORM) order.push_back(i);
    }
    std::stable_sort(order.begin(), order.end(), [&](int a, int c) {
      return b->probs[a]->m * b->probs[a]->n > b->probs[c]->m * b->probs[c]->n;
    });
    for (int i : order) {
      kg_problem* p = b->probs[i];
      const size_t bytes = 8 * (size_t)p->m * (size_t)p->n;
      if (bytes > budget) continue;
      void* q = nullptr;
      // 16 bytes beyond the end: the ring's copies read whole 16-byte units
      if (dev_alloc(&q, bytes + 16) != cudaSuccess) {
        rc = fail(KG_ERR_OOM, "kg_batch_create: float-pair copy of A");
        break;
      }
      b->own_preps.push_back(q);
      if ((rc = pair_prepare(static_cast<const double*>(p->data0), q, p->m * p->n, s)) != KG_OK) break;
      b->prep[i] = q;
      budget -= bytes;
    }
  }
  if (rc == KG_OK) {
    cudaError_t e = batched_smem_attrs();
    if (e != cudaSuccess) rc = cuda_fail(e, "kg_batch_create: kernel attributes");
  }
  if (rc == KG_OK) {
    b->gpu = gpu_name();
    b->grid = batched_grid(b->pair);
    if (b->pair) {
      const float4* t = nullptr;
      rc = logtab_for_device(&t);
    }
    const char* no_tune = std::getenv("KG_NO_AUTOTUNE");
    if (rc == KG_OK && !(no_tune && no_tune[0] == '1')) rc = autotune(b, s);
  }
  if (rc == KG_OK) {
    std::vector<int> ids(count);
    for (int i = 0; i < count; ++i) ids[i] = i;
    b->plan = make_plan(b->probs, b->prep, ids, b->tune, b->pair, b->es);
    rc = devplan_alloc(b->dev, b->plan, s);
  }
  if (rc == KG_OK) {
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) rc = cuda_fail(e, "kg_batch_create");
  }
  if (rc != KG_OK) {
    batch_free(b);
    return rc;
  }
  b->last_stream = s;
  *out = b;
  return KG_OK;
}

static kg_status batch_update_ptrs(kg_batch* b, const void* const* x, void* const* f,
                                   void* const* gx, cudaStream_t s) {
  const int n = (int)b->probs.size();
  for (int i = 0; i < n; ++i)
    if (!x[i] || !gx[i]) return fail(KG_ERR_INVALID_ARG, "kg_grad_batched: NULL x or gx entry");
  bool same = b->ptrs_valid;
  for (int i = 0; same && i < n; ++i)
    same = b->last_x[i] == x[i] && b->last_f[i] == f[i] && b->last_gx[i] == gx[i];
  if (same) return KG_OK;
  b->last_x.assign(x, x + n);
  b->last_f.assign(f, f + n);
  b->last_gx.assign(gx, gx + n);
  for (int i = 0; i < n; ++i) {
    b->plan.insts[i].x = x[i];
    b->plan.insts[i].f = f[i];
    b->plan.insts[i].gx = gx[i];
  }
  cudaError_t e = cudaMemcpyAsync(b->dev.insts, b->plan.insts.data(), sizeof(BInst) * n,
                                  cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return cuda_fail(e, "kg_grad_batched: descriptor update");
  b->ptrs_valid = true;
  return KG_OK;
}

kg_status kg_grad_batched(kg_batch* b, const void* const* x, void* const* f, void* const* gx,
                          kg_stream stream) {
  reset_launch_count();
  if (!b || !x || !f || !gx) return fail(KG_ERR_INVALID_ARG, "kg_grad_batched: NULL argument");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  b->last_stream = s;
  kg_status rc = batch_update_ptrs(b, x, f, gx, s);
  if (rc != KG_OK) return rc;
  cudaError_t e;
  if (!b->exec) {  // capture the launch sequence once, replay it afterwards
    cudaStream_t cs = nullptr;
    if ((e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking)) != cudaSuccess)
      return cuda_fail(e, "kg_grad_batched: capture stream");
    e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      rc = launch_plan(b->dev, b->dtype, b->pair, b->warp, b->err, cs, b->grid);
      cudaError_t e2 = cudaStreamEndCapture(cs, &b->graph);
      if (rc == KG_OK && e2 != cudaSuccess) rc = cuda_fail(e2, "kg_grad_batched: end capture");
    } else {
      rc = cuda_fail(e, "kg_grad_batched: begin capture");
    }
    cudaStreamDestroy(cs);
    if (rc != KG_OK) return rc;
    if ((e = cudaGraphInstantiate(&b->exec, b->graph, 0)) != cudaSuccess) {
      b->exec = nullptr;
      return cuda_fail(e, "kg_grad_batched: instantiate");
    }
  }
  prof_begin(s, "batched_kernel (graph)");
  e = cudaGraphLaunch(b->exec, s);
  prof_end(s);
  if (e != cudaSuccess) return cuda_fail(e, "kg_grad_batched: launch");
  count_launch(b->dev.ntet > 0 ? 2 : 1);
  return KG_OK;
}

kg_status kg_grad_batched_loop(kg_batch* b, const void* const* x, void* const* f, void* const* gx,
                               kg_stream stream) {
  if (!b || !x || !f || !gx) return fail(KG_ERR_INVALID_ARG, "kg_grad_batched_loop: NULL argument");
  int launches = 0;
  for (size_t i = 0; i < b->probs.size(); ++i) {
    kg_status rc = kg_grad(b->probs[i], x[i], f[i], gx[i], nullptr, nullptr, 0, stream);
    if (rc != KG_OK) return rc;
    launches += kg_last_launch_count();
  }
  reset_launch_count();
  count_launch(launches);
  return KG_OK;
}

kg_status kg_batch_get_config(const kg_batch* b, int* arith, int* items, int* grid) {
  if (!b) return fail(KG_ERR_INVALID_ARG, "kg_batch_get_config: NULL batch");
  if (arith) *arith = b->pair ? KG_ARITH_PAIR : KG_ARITH_NATIVE;
  if (items) *items = b->dev.nitems;
  if (grid) *grid = b->grid;
  return KG_OK;
}

kg_status kg_batch_sync(kg_batch* b) {
  if (!b) return fail(KG_ERR_INVALID_ARG, "kg_batch_sync: NULL batch");
  cudaError_t e = cudaStreamSynchronize(b->last_stream);
  if (e != cudaSuccess) return cuda_fail(e, "kg_batch_sync");
  unsigned h = 0;
  if ((e = cudaMemcpy(&h, b->err, sizeof(h), cudaMemcpyDeviceToHost)) != cudaSuccess)
    return cuda_fail(e, "kg_batch_sync");
  if (h) cudaMemset(b->err, 0, sizeof(unsigned));
  if (h & ERRBIT_RANGE)
    return fail(KG_ERR_RANGE, "device: an input is outside the float-pair range");
  if (h & ERRBIT_TIMEOUT) return fail(KG_ERR_TIMEOUT, "device: a bounded wait gave up");
  return KG_OK;
}

void kg_batch_destroy(kg_batch* b) {
  if (!b) return;
  cudaStreamSynchronize(b->last_stream);
  batch_free(b);
}

}  // extern "C"
