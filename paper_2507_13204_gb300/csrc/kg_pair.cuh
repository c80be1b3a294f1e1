// Float-pair ("pair") arithmetic for FP64 data on GB300.
//
// GB300 issues about 2 FP64 FMA per clock per SM but 128 FP32 FMA, so the FP64
// kernels keep their data in FP64 memory and compute on pairs of floats
// (hi + lo):
//   - split_f64 turns a double into hi (its leading 24 significant bits,
//     truncated) and lo (the next 23 bits) with integer instructions only;
//     the pair holds the double to within 2^-47 relative for
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
