// Host-side check of the float-pair helpers that the FP64 kernels use
// (kg_pair.cuh compiled as plain C++).  Each check draws seeded random inputs,
// compares with long double arithmetic and prints "name worst_relative_error".
#include "kg_pair.cuh"

#include <cmath>
#include <cstdio>
#include <random>

using kg::Pair;

static void split_ld(long double v, float& h, float& l) {
  h = (float)v;
  l = (float)(v - (long double)h);
}

int main() {
  std::mt19937_64 g(20250717);
  std::uniform_real_distribution<double> U(-1.0, 1.0);
  auto mag = [&](int lo, int hi) { return std::ldexp(1.0, lo + (int)(g() % (uint64_t)(hi - lo))); };

  // split_f64: h + l holds d to 2^-46 relative inside the range 2^-60 .. 2^40
  long double w_split = 0;
  for (int i = 0; i < 1000000; ++i) {
    const double d = U(g) * mag(-60, 40);
    if (d == 0) continue;
    const Pair p = kg::split_f64(d);
    const long double e = std::fabs(((long double)p.h + p.l - d) / d);
    if (e > w_split) w_split = e;
  }
  printf("split_f64 %.6Lg\n", w_split);

  // pair_to_double_fast: within one double ulp of h + l
  long double w_conv = 0;
  for (int i = 0; i < 1000000; ++i) {
    Pair p = kg::split_f64(U(g) * mag(-60, 40));
    if (i % 3 == 1) p.l = (float)(U(g) * mag(-80, -20));
    if (i % 5 == 2) p.l = -p.h * (float)U(g);
    const long double ex = (long double)p.h + p.l;
    const double r = kg::pair_to_double_fast(p);
    const long double e = ex == 0 ? std::fabs((long double)r) : std::fabs((r - ex) / ex);
    if (e > w_conv) w_conv = e;
  }
  printf("pair_to_double_fast %.6Lg\n", w_conv);

  // f32_to_f64_int is exact for normal floats and zero
  long double w_f2d = 0;
  for (int i = 0; i < 100000; ++i) {
    const float f = (float)(U(g) * mag(-100, 100));
    const long double e = std::fabs((long double)kg::f32_to_f64_int(f) - (long double)f);
    if (e > w_f2d) w_f2d = e;
  }
  printf("f32_to_f64_int %.6Lg\n", w_f2d);

  // pair_recip for t >= 1 (a normalised pair)
  long double w_rcp = 0;
  for (int i = 0; i < 1000000; ++i) {
    const double t = 1.0 + std::fabs(U(g)) * mag(-30, 20);
    Pair tp = kg::split_f64(t);
    kg::fast_two_sum(tp.h, tp.l, tp.h, tp.l);  // normalised, as the kernels pass it (t = 1 + s)
    const Pair r = kg::pair_recip(tp);
    const long double ex = 1.0L / ((long double)tp.h + tp.l);
    const long double e = std::fabs(((long double)r.h + r.l - ex) / ex);
    if (e > w_rcp) w_rcp = e;
  }
  printf("pair_recip %.6Lg\n", w_rcp);

  // pair_log1p for s >= 0, with the 256-entry table built here from its definition
  float4 tab[kg::kLogTableSize];
  for (int k = 0; k < kg::kLogTableSize; ++k) {
    const long double c = 1.0L + (long double)k / kg::kLogTableSize;
    split_ld(logl(c), tab[k].x, tab[k].y);
    split_ld(1.0L / c, tab[k].z, tab[k].w);
  }
  kg::LogConsts K;
  split_ld(logl(2.0L), K.ln2_h, K.ln2_l);
  split_ld(1.0L / 3.0L, K.third_h, K.third_l);
  long double w_log = 0, w_t = 0;
  for (int i = 0; i < 1000000; ++i) {
    const double s = std::fabs(U(g)) * mag(-60, 30);
    const Pair sp = kg::split_f64(s);
    Pair t;
    const Pair lf = kg::pair_log1p(sp, tab, K, t);
    const long double sx = (long double)sp.h + sp.l;
    const long double ex = log1pl(sx);
    const long double e = std::fabs(((long double)lf.h + lf.l - ex) / ex);
    if (e > w_log) w_log = e;
    const long double et = std::fabs(((long double)t.h + t.l - (1.0L + sx)) / (1.0L + sx));
    if (et > w_t) w_t = et;
  }
  printf("pair_log1p %.6Lg\n", w_log);
  printf("pair_log1p_t %.6Lg\n", w_t);

  // acc_prod: the same accumulator as acc_fma on a zero accumulator
  long double w_prod = 0;
  for (int i = 0; i < 1000000; ++i) {
    float ah, al, bh, bl;
    split_ld((long double)U(g) * mag(-30, 30), ah, al);
    split_ld((long double)U(g) * mag(-30, 30), bh, bl);
    const kg::Acc p = kg::acc_prod(ah, al, bh, bl);
    kg::Acc q = kg::acc_zero();
    kg::acc_fma(q, ah, al, bh, bl);
    const long double d = std::fabs((long double)p.s - q.s) + std::fabs((long double)p.l - q.l);
    if (d > w_prod) w_prod = d;
  }
  printf("acc_prod_vs_acc_fma %.6Lg\n", w_prod);
  return 0;
}
