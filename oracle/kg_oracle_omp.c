/*
 * The CPU baseline: the oracle's dense and tet value-and-gradient run on all
 * host cores with OpenMP.
 *
 * TEST INFRASTRUCTURE ONLY, like kg_oracle.c: only the benchmark's CPU-baseline
 * leg (and the tests that check this file against kg_oracle.c) load it.  It is
 * the timed baseline, not the parity oracle: parity is always checked against
 * the single-threaded functions of kg_oracle.c, which are pinned to closed
 * forms and invariants.  These functions take the same steps in the same
 * order as those (forward pass over all rows / elements, broadcast of the
 * reduction adjoint, reverse accumulation), with each loop over rows or
 * elements split into one contiguous block per thread:
 *   - f: one compensated partial per thread, summed in thread order;
 *   - the adjoint: a thread-private compensated accumulator array per thread,
 *     then, for each entry, the thread partials summed in thread order.
 * The result therefore depends on the thread count only through the order of
 * compensated sums (differences at the 1e-16 level), and is the same run to
 * run for a given count.  Nothing here is shared with the CUDA path.
 *
 * Method: Liegeois et al., arXiv 2507.13204 -- forward then reverse pass
 * (Sec. 3), reduction adjoint broadcast (Sec. 3.2), index-map reads reversed
 * into scatter-adds (Sec. 3.3).
 */
#include <math.h>
#include <omp.h>
#include <stddef.h>
#include <stdint.h>
#include <stdlib.h>

typedef struct { double s, c; } nsum;

static void nadd(nsum *a, double v) {
  double t = a->s + v;
  if (fabs(a->s) >= fabs(v)) a->c += (a->s - t) + v;
  else a->c += (v - t) + a->s;
  a->s = t;
}
static double nval(const nsum *a) { return a->s + a->c; }

/* Threads an OpenMP parallel region of this library uses. */
int kgo_omp_threads(void) { return omp_get_max_threads(); }

/* Value and gradient of f(x) = ||A x||^2 (A m x n row-major), output adjoint
 * fbar: y_i = sum_j A_ij x_j, f = sum_i y_i^2, ybar_i = 2 fbar y_i,
 * xbar_j = sum_i A_ij ybar_i.  gx (n) is overwritten.  *threads receives the
 * thread count used. */
int kgo_quadform_grad_omp(int64_t m, int64_t n, const double *A, const double *x, double fbar,
                          double *f, double *gx, int *threads) {
  if (m < 0 || n < 0 || (m * n > 0 && (!A || !x)) || (n > 0 && !gx)) return -1;
  const int T = omp_get_max_threads();
  double *y = (double *)malloc((size_t)(m > 0 ? m : 1) * sizeof(double));
  nsum *part = (nsum *)calloc((size_t)T * (size_t)(n > 0 ? n : 1), sizeof(nsum));
  nsum *fpart = (nsum *)calloc((size_t)T, sizeof(nsum));
  if (!y || !part || !fpart) { free(y); free(part); free(fpart); return -2; }
  int used = 1;
#pragma omp parallel num_threads(T)
  {
    const int t = omp_get_thread_num(), nt = omp_get_num_threads();
#pragma omp single
    used = nt;
    const int64_t i0 = m * t / nt, i1 = m * (t + 1) / nt;
    /* forward: row dot products and the thread's part of sum y_i^2 */
    for (int64_t i = i0; i < i1; ++i) {
      nsum yi = {0, 0};
      for (int64_t j = 0; j < n; ++j) nadd(&yi, A[i * n + j] * x[j]);
      y[i] = nval(&yi);
      nadd(&fpart[t], y[i] * y[i]);
    }
    /* reverse: broadcast ybar_i, accumulate the thread's xbar partial */
    nsum *acc = part + (size_t)t * (size_t)n;
    for (int64_t i = i0; i < i1; ++i) {
      const double ybar = 2.0 * y[i] * fbar;
      for (int64_t j = 0; j < n; ++j) nadd(&acc[j], A[i * n + j] * ybar);
    }
#pragma omp barrier
#pragma omp for schedule(static)
    for (int64_t j = 0; j < n; ++j) {
      nsum s = {0, 0};
      for (int tt = 0; tt < nt; ++tt) nadd(&s, nval(&part[(size_t)tt * (size_t)n + j]));
      gx[j] = nval(&s);
    }
  }
  nsum tot = {0, 0};
  for (int t = 0; t < used; ++t) nadd(&tot, nval(&fpart[t]));
  if (f) *f = nval(&tot);
  if (threads) *threads = used;
  free(y);
  free(part);
  free(fpart);
  return 0;
}

/* Value and gradient of f(u) = sum_e log1p(|G_e u_e|^2), u_e = u[conn[e][0..3]]:
 * forward g_e = G_e u_e; reverse sbar = fbar / (1 + |g_e|^2),
 * c_e = G_e^T (2 sbar g_e), scatter-add gu[conn[e][k]] += c_e[k].  gu (nv) is
 * overwritten.  *threads receives the thread count used. */
int kgo_tet_grad_omp(int64_t ne, int64_t nv, const int32_t *conn, const double *G,
                     const double *u, double fbar, double *f, double *gu, int *threads) {
  if (ne < 0 || nv < 0 || (nv > 0 && !gu) || (ne > 0 && (!conn || !G || !u))) return -1;
  for (int64_t i = 0; i < ne * 4; ++i)
    if (conn[i] < 0 || conn[i] >= nv) return -3;
  const int T = omp_get_max_threads();
  double *c = (double *)malloc((size_t)(ne > 0 ? ne : 1) * 4 * sizeof(double));
  nsum *part = (nsum *)calloc((size_t)T * (size_t)(nv > 0 ? nv : 1), sizeof(nsum));
  nsum *fpart = (nsum *)calloc((size_t)T, sizeof(nsum));
  if (!c || !part || !fpart) { free(c); free(part); free(fpart); return -2; }
  int used = 1;
#pragma omp parallel num_threads(T)
  {
    const int t = omp_get_thread_num(), nt = omp_get_num_threads();
#pragma omp single
    used = nt;
    const int64_t e0 = ne * t / nt, e1 = ne * (t + 1) / nt;
    /* forward: the thread's part of sum_e log1p(|g_e|^2) */
    for (int64_t e = e0; e < e1; ++e) {
      double g[3];
      for (int r = 0; r < 3; ++r) {
        double s = 0;
        for (int k = 0; k < 4; ++k) s += G[e * 12 + r * 4 + k] * u[conn[e * 4 + k]];
        g[r] = s;
      }
      nadd(&fpart[t], log1p(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]));
    }
    /* reverse: per-element adjoint c_e, then the scatter-add into the thread's
     * accumulators */
    for (int64_t e = e0; e < e1; ++e) {
      double g[3];
      for (int r = 0; r < 3; ++r) {
        double s = 0;
        for (int k = 0; k < 4; ++k) s += G[e * 12 + r * 4 + k] * u[conn[e * 4 + k]];
        g[r] = s;
      }
      const double sbar = fbar / (1.0 + (g[0] * g[0] + g[1] * g[1] + g[2] * g[2]));
      const double gbar[3] = {2.0 * sbar * g[0], 2.0 * sbar * g[1], 2.0 * sbar * g[2]};
      for (int k = 0; k < 4; ++k)
        c[e * 4 + k] = G[e * 12 + 0 * 4 + k] * gbar[0] + G[e * 12 + 1 * 4 + k] * gbar[1] +
                       G[e * 12 + 2 * 4 + k] * gbar[2];
    }
    nsum *acc = part + (size_t)t * (size_t)nv;
    for (int64_t e = e0; e < e1; ++e)
      for (int k = 0; k < 4; ++k) nadd(&acc[conn[e * 4 + k]], c[e * 4 + k]);
#pragma omp barrier
#pragma omp for schedule(static)
    for (int64_t v = 0; v < nv; ++v) {
      nsum s = {0, 0};
      for (int tt = 0; tt < nt; ++tt) nadd(&s, nval(&part[(size_t)tt * (size_t)nv + v]));
      gu[v] = nval(&s);
    }
  }
  nsum tot = {0, 0};
  for (int t = 0; t < used; ++t) nadd(&tot, nval(&fpart[t]));
  if (f) *f = nval(&tot);
  if (threads) *threads = used;
  free(c);
  free(part);
  free(fpart);
  return 0;
}
