// Float-pair ("pair") arithmetic for FP64 data on GB300.
//
// GB300 issues about 2 FP64 FMA per clock per SM but 128 FP32 FMA, so the FP64
// kernels keep their data in FP64 memory and compute on pairs of floats
// (hi + lo):
//   - split_f64 turns a double into hi (its leading 24 significant bits,
//     truncated) and lo (the next 23 bits) with integer instructions only;
//     the pair holds the double to within 2^-46 relative for
//     2^-60 <= |d| < 2^40 (pair_in_range) and maps +-0 to +-0; callers check
//     the range of their inputs.
//   - products use the FMA error-free transformation: for floats a, b,
//     p = a*b and fma(a, b, -p) = a*b - p exactly;
//   - sums of the hi parts use Knuth's TwoSum (exact rounding error), so an
//     accumulator (s, l) carries every hi product exactly and the low-order
//     terms in l.
// The result of a dot product of length n is within about 2^-46 * sum|a_j b_j|
// of the exact value.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

namespace kg {

struct Pair {
  float h, l;
};

__host__ __device__ __forceinline__ uint32_t f2u(float f) {
#ifdef __CUDA_ARCH__
  return __float_as_uint(f);
#else
  uint32_t u;
  memcpy(&u, &f, 4);
  return u;
#endif
}
__host__ __device__ __forceinline__ float u2f(uint32_t u) {
#ifdef __CUDA_ARCH__
  return __uint_as_float(u);
#else
  float f;
  memcpy(&f, &u, 4);
  return f;
#endif
}
__host__ __device__ __forceinline__ void d2words(double d, uint32_t& lo, uint32_t& hi) {
#ifdef __CUDA_ARCH__
  lo = (uint32_t)__double2loint(d);
  hi = (uint32_t)__double2hiint(d);
#else
  uint64_t u;
  memcpy(&u, &d, 8);
  lo = (uint32_t)u;
  hi = (uint32_t)(u >> 32);
#endif
}

// (hi << 3) | (lo >> 29): exponent bits 8..0 and the top 23 mantissa bits.
__host__ __device__ __forceinline__ uint32_t fshl3(uint32_t lo, uint32_t hi) {
#ifdef __CUDA_ARCH__
  return __funnelshift_l(lo, hi, 3);
#else
  return (hi << 3) | (lo >> 29);
#endif
}

// Split a double into a float pair with integer instructions.
//   hi: sign | (e - 896) << 23 | m[51:29]   (e = biased FP64 exponent), so
//       hi is d truncated to 24 significant bits.  t = fshl3 holds e mod 512
//       in its top 9 bits and (e - 896) = (e mod 512 + 128) mod 512 for every
//       e in [897, 1150], so adding 2^30 re-biases the field; e = 0 (+-0) is
//       kept as a signed zero by the select.
//   lo: m[28:6] * 2^(E - 46), built as (1.m' * 2^k) - 2^k with 2^k = 2^(E-23)
//       taken from hi's exponent field, so the subtraction is exact.
// For d = +-0 the low word is 0 and lo = s - s = 0.
__host__ __device__ __forceinline__ Pair split_f64(double d) {
  uint32_t lo, hi;
  d2words(d, lo, hi);
  const uint32_t sign = hi & 0x80000000u;
  const uint32_t t = fshl3(lo, hi);
  const uint32_t hb = (hi & 0x7FF00000u) ? ((t + 0x40000000u) | sign) : sign;
  const uint32_t fs = (hb & 0xFF800000u) - (23u << 23);
  const uint32_t lb = fs | ((lo >> 6) & 0x007FFFFFu);
  Pair p;
  p.h = u2f(hb);
  p.l = u2f(lb) - u2f(fs);
  return p;
}

// True when the pair arithmetic represents d (0, or 2^-60 <= |d| < 2^40).
__host__ __device__ __forceinline__ bool pair_in_range(double d) {
  uint32_t lo, hi;
  d2words(d, lo, hi);
  const uint32_t e = (hi >> 20) & 0x7FFu;
  return ((hi & 0x7FFFFFFFu) | lo) == 0u || (e >= 1023u - 60u && e < 1023u + 40u);
}

// Knuth TwoSum: s + e == a + b exactly.
__host__ __device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

// Dekker FastTwoSum (requires |a| >= |b| or a == 0).
__host__ __device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  e = b - (s - a);
}

// Accumulator of a sum of pair products: value s + l.
struct Acc {
  float s, l;
};

__host__ __device__ __forceinline__ Acc acc_zero() { return Acc{0.f, 0.f}; }

// acc += (ah + al) * (bh + bl), dropping al*bl (2^-48 relative).
__host__ __device__ __forceinline__ void acc_fma(Acc& c, float ah, float al, float bh, float bl) {
  const float p = ah * bh;
  float e = fmaf(ah, bh, -p);
  e = fmaf(ah, bl, e);
  e = fmaf(al, bh, e);
  float s, r;
  two_sum(c.s, p, s, r);
  c.s = s;
  c.l += r + e;
}

// The first term of an accumulation: (ah + al) * (bh + bl) as an
// accumulator, the value acc_fma gives on a zero accumulator (up to the sign
// of a zero) without its TwoSum, which the compiler cannot drop because
// 0 + p is not p for p = -0.
__host__ __device__ __forceinline__ Acc acc_prod(float ah, float al, float bh, float bl) {
  const float p = ah * bh;
  float e = fmaf(ah, bh, -p);
  e = fmaf(ah, bl, e);
  e = fmaf(al, bh, e);
  return Acc{p, e};
}

// Renormalise: move l into s so that |l| <= ulp(s)/2 again (TwoSum).  Long
// accumulations call this every few terms; otherwise |l| grows with the
// number of terms and its own float rounding becomes visible (n * 2^-48).
__host__ __device__ __forceinline__ void acc_renorm(Acc& c) {
  float s, e;
  two_sum(c.s, c.l, s, e);
  c.s = s;
  c.l = e;
}

// a + b for two accumulators.
__host__ __device__ __forceinline__ Acc acc_add(Acc a, Acc b) {
  float s, r;
  two_sum(a.s, b.s, s, r);
  Acc c;
  c.s = s;
  c.l = a.l + b.l + r;
  return c;
}

// Sum of the per-row squares y_i^2 that make f: in double for FP64 data; for
// FP32 data a float sum with its exact rounding error (TwoSum), so that FP32
// kernels issue no FP64 instruction per row (one FP64 instruction occupies
// GB300's narrow FP64 unit for the whole warp, however few lanes are active).
template <typename T>
struct FSum {
  double v = 0.0;
  __device__ __forceinline__ void add(T y) { v += (double)y * (double)y; }
  __device__ __forceinline__ double get() const { return v; }
};
template <>
struct FSum<float> {
  float s = 0.f, l = 0.f;
  __device__ __forceinline__ void add(float y) {
    float t, e;
    two_sum(s, y * y, t, e);
    s = t;
    l += e;
  }
  __device__ __forceinline__ double get() const { return (double)s + (double)l; }
};

// Normalised pair (|l| <= ulp(h)/2) of an accumulator.
__host__ __device__ __forceinline__ Pair acc_pair(Acc a) {
  Pair p;
  two_sum(a.s, a.l, p.h, p.l);
  return p;
}

// Pair product (ah + al) * (bh + bl) as a normalised pair.
__host__ __device__ __forceinline__ Pair pair_mul(Pair a, Pair b) {
  const float p = a.h * b.h;
  float e = fmaf(a.h, b.h, -p);
  e = fmaf(a.h, b.l, e);
  e = fmaf(a.l, b.h, e);
  Pair r;
  fast_two_sum(p, e, r.h, r.l);
  return r;
}

__host__ __device__ __forceinline__ double pair_to_double(Pair p) {
  return (double)p.h + (double)p.l;
}
__host__ __device__ __forceinline__ double acc_to_double(Acc a) {
  return (double)a.s + (double)a.l;
}

}  // namespace kg

// ---------------------------------------------------------------------------
// Pair functions for the tet energy: sums, reciprocal, log1p, conversion.
// ---------------------------------------------------------------------------
namespace kg {

// a + b for normalised pairs, normalised result.
__host__ __device__ __forceinline__ Pair pair_add(Pair a, Pair b) {
  float s, e;
  two_sum(a.h, b.h, s, e);
  e += a.l + b.l;
  Pair r;
  fast_two_sum(s, e, r.h, r.l);
  return r;
}

// 1/t for t >= 1 (normalised pair): the correctly rounded float reciprocal r0
// has relative error <= 2^-24; one Newton step r0 (1 + (1 - t r0)) in pair
// form leaves an error of order 2^-48.
__host__ __device__ __forceinline__ Pair pair_recip(Pair t) {
#ifdef __CUDA_ARCH__
  const float r0 = __frcp_rn(t.h);
#else
  const float r0 = 1.0f / t.h;  // IEEE division: also correctly rounded
#endif
  float e = fmaf(-t.h, r0, 1.0f);
  e = fmaf(-t.l, r0, e);
  Pair r;
  fast_two_sum(r0, r0 * e, r.h, r.l);
  return r;
}

// Constants for pair_log1p, computed on the host from their definitions.
struct LogConsts {
  float ln2_h, ln2_l;      // ln 2 = ln2_h + ln2_l (a float pair)
  float third_h, third_l;  // 1/3 as a pair
};

// Table entry k (0..255) for c_k = 1 + k/256: (log c_k as a pair, 1/c_k as a pair).
constexpr int kLogTableSize = 256;

// log1p(s) for s >= 0 given as a normalised pair; also returns t = 1 + s.
// t = 2^E m with m in [1, 2); m = c_k (1 + r) with c_k = 1 + k/256 from the
// top 8 mantissa bits, so |r| < 2^-8; log t = E ln2 + log c_k + log1p(r) with
//   log1p(r) = r + r^2 (-1/2 + r/3) + r^4 (-1/4 + r/5 - r^2/6) + O(r^7),
// the first three terms in pair precision and the rest in float.  Relative
// error about 2^-46 (for s near 0, r = s exactly, so the result stays
// relatively accurate).
__host__ __device__ __forceinline__ Pair pair_log1p(Pair s, const float4* __restrict__ tab,
                                           const LogConsts& K, Pair& t) {
  float th, tl;
  two_sum(1.0f, s.h, th, tl);
  tl += s.l;
  fast_two_sum(th, tl, th, tl);
  t.h = th;
  t.l = tl;
  const uint32_t tb = f2u(th);
  const int E = (int)((tb >> 23) & 0xFFu) - 127;            // t >= 1, so E >= 0
  const float mh = u2f((tb & 0x007FFFFFu) | 0x3F800000u);  // th / 2^E
  const float ml = tl * u2f((uint32_t)(127 - E) << 23);     // tl / 2^E (exact)
  const uint32_t k = (f2u(mh) >> 15) & 0xFFu;
  const float ck = u2f(0x3F800000u | (k << 15));
  const float4 T = tab[k];
  // d = m - c_k.  For t < 2 (E = 0) take it from s itself, d = (1 - c_k) + s,
  // because the pair t = 1 + s drops the low bits of a small s; for t >= 2
  // (s >= 1) d = (mh - c_k) + ml, where mh - c_k is exact (c_k <= mh < 2 c_k).
  Pair d;
  if (E == 0) {
    d = pair_add(Pair{1.0f - ck, 0.0f}, s);
  } else {
    two_sum(mh - ck, ml, d.h, d.l);
  }
  const Pair r = pair_mul(d, Pair{T.z, T.w});
  const Pair r2 = pair_mul(r, r);
  const Pair u = pair_add(Pair{-0.5f, 0.0f}, pair_mul(r, Pair{K.third_h, K.third_l}));
  const Pair v = pair_mul(r2, u);
  const float q = fmaf(r.h, fmaf(-r.h, 0.16666667f, 0.2f), -0.25f);
  const float w4 = (r2.h * r2.h) * q;
  Pair lp = pair_add(r, v);
  lp = pair_add(lp, Pair{w4, 0.0f});
  const float Ef = (float)E;
  const float p1 = Ef * K.ln2_h;                // E ln2_h as an exact pair (p1, e1)
  const float e1 = fmaf(Ef, K.ln2_h, -p1);
  Pair el;
  fast_two_sum(p1, fmaf(Ef, K.ln2_l, e1), el.h, el.l);
  return pair_add(pair_add(el, Pair{T.x, T.y}), lp);
}

__host__ __device__ __forceinline__ double u64_to_f64(uint64_t u) {
#ifdef __CUDA_ARCH__
  return __longlong_as_double((long long)u);
#else
  double d;
  memcpy(&d, &u, 8);
  return d;
#endif
}

// Exact float -> double with integer instructions (normal floats and zero).
__host__ __device__ __forceinline__ double f32_to_f64_int(float f) {
  const uint32_t b = f2u(f);
  const uint32_t mag = b & 0x7FFFFFFFu;
  const uint32_t hi = (b & 0x80000000u) | (mag ? (mag >> 3) + (896u << 20) : 0u);
  return u64_to_f64(((uint64_t)hi << 32) | (uint32_t)(b << 29));
}

// h + l as a double: two exact conversions on the integer units, one FP64 add
// (an all-integer add measured slower in the tet gradient kernel).
__host__ __device__ __forceinline__ double pair_to_double_fast(Pair p) {
  return f32_to_f64_int(p.h) + f32_to_f64_int(p.l);
}

}  // namespace kg
