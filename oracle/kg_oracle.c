/*
 * CPU oracle for reverse-mode gradients of data-parallel functions.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this code.  It shares nothing with the
 * CUDA path (no headers, no helpers, no tables) and is deliberately plain and
 * slow: double precision, single thread, loops in the order the method states
 * them, and Neumaier-compensated sums for every long reduction.
 *
 * The method (Liegeois et al., "Performance Portable Gradient Computations
 * Using Source Transformation", arXiv 2507.13204):
 *   - the gradient runs the forward pass, then the reverse pass (Sec. 3,
 *     opening of "Methodology");
 *   - in the reverse pass a read of x becomes an accumulation into the adjoint
 *     of x and the adjoint of a written value is consumed and zeroed
 *     (Sec. 3.1, Fig. "view_accesses"); indices are not differentiated;
 *   - the reverse of a sum reduction is a broadcast of the output adjoint
 *     (Sec. 3.2, Figs. "deep_copy_views"/"deep_copy_scalar" and the
 *     parallel_sum helper);
 *   - a gather through an index map becomes a scatter-add (Sec. 3.3, the two
 *     race-detection rules).
 *
 * Every function returns 0 on success and a negative value on bad arguments.
 * Parity pins (tests/test_oracle.py): closed forms, Euler homogeneity, special
 * cases, forward-mode dual numbers, central differences, exact rational
 * arithmetic on tiny inputs, and mesh invariants.  No function here is
 * "parity unpinned".
 */
#include <math.h>
#include <stddef.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ---------------------------------------------------------------- sums -- */
/* Neumaier's variant of Kahan summation: (s, c) carries the running sum and the
 * accumulated rounding error; the result is s + c. */
typedef struct { double s, c; } nsum;

static void nadd(nsum *a, double v) {
  double t = a->s + v;
  if (fabs(a->s) >= fabs(v)) a->c += (a->s - t) + v;
  else a->c += (v - t) + a->s;
  a->s = t;
}
static double nval(const nsum *a) { return a->s + a->c; }

/* ------------------------------------------------------- ||A x||^2 ------ */
/* Forward pass of f(x, A) = sum_i (sum_j A_ij x_j)^2, A m x n row-major.
 * A row of A dotted with x is a team-nested parallel_reduce; the squares are
 * summed by a parallel_sum reduction (Sec. 4 uses the same reduce). y (length
 * m) receives the row products and may be NULL. */
int kgo_quadform_value(int64_t m, int64_t n, const double *A, const double *x,
                       double *y, double *f) {
  if (m < 0 || n < 0 || (m * n > 0 && (!A || !x)) || !f) return -1;
  nsum tot = {0, 0};
  for (int64_t i = 0; i < m; ++i) {
    nsum yi = {0, 0};
    for (int64_t j = 0; j < n; ++j) nadd(&yi, A[i * n + j] * x[j]);
    double v = nval(&yi);
    if (y) y[i] = v;
    nadd(&tot, v * v);
  }
  *f = nval(&tot);
  return 0;
}

/* Value and gradient of f(x, A) = ||A x||^2 with output adjoint fbar.
 *   forward : y_i = sum_j A_ij x_j ;  f = sum_i y_i^2
 *   reverse : the reduction's adjoint is broadcast, ybar_i = 2 y_i fbar;
 *             every read A_ij * x_j of the forward row loop becomes
 *             xbar_j += A_ij ybar_i and Abar_ij += x_j ybar_i.
 * gx (n) is overwritten; gA (m x n) is overwritten when non-NULL. */
int kgo_quadform_grad(int64_t m, int64_t n, const double *A, const double *x,
                      double fbar, double *f, double *gx, double *gA) {
  if (m < 0 || n < 0 || (m * n > 0 && (!A || !x)) || (n > 0 && !gx)) return -1;
  double *y = (double *)malloc((size_t)(m > 0 ? m : 1) * sizeof(double));
  nsum *acc = (nsum *)calloc((size_t)(n > 0 ? n : 1), sizeof(nsum));
  if (!y || !acc) { free(y); free(acc); return -2; }
  double fv = 0;
  kgo_quadform_value(m, n, A, x, y, &fv);
  if (f) *f = fv;
  for (int64_t i = 0; i < m; ++i) {
    double ybar = 2.0 * y[i] * fbar;
    for (int64_t j = 0; j < n; ++j) {
      nadd(&acc[j], A[i * n + j] * ybar);
      if (gA) gA[i * n + j] = x[j] * ybar;
    }
  }
  for (int64_t j = 0; j < n; ++j) gx[j] = nval(&acc[j]);
  free(y);
  free(acc);
  return 0;
}

/* ------------------------------------------------ sparse ||A x||^2 ------ */
/* A is m x n in compressed sparse rows: the entries of row i are
 * val[p] at column col[p] for rowptr[i] <= p < rowptr[i+1]; a column may repeat
 * within a row (the entries then add).  The forward pass is the same
 * team-nested parallel_reduce as the dense case with the inner loop over the
 * stored entries only: a read of x through the index map col (Sec. 3.3), whose
 * reverse is a scatter-add into xbar. */
static int check_csr(int64_t m, int64_t n, int64_t nnz, const int32_t *rowptr,
                     const int32_t *col) {
  if (m < 0 || n < 0 || nnz < 0 || !rowptr) return -1;
  if (rowptr[0] != 0 || rowptr[m] != nnz) return -3;
  for (int64_t i = 0; i < m; ++i)
    if (rowptr[i + 1] < rowptr[i]) return -3;
  for (int64_t p = 0; p < nnz; ++p)
    if (col[p] < 0 || col[p] >= n) return -3;
  return 0;
}

/* Forward: y_i = sum_{p in row i} val[p] x[col[p]] ; f = sum_i y_i^2.  y may be NULL. */
int kgo_spquadform_value(int64_t m, int64_t n, int64_t nnz, const int32_t *rowptr,
                         const int32_t *col, const double *val, const double *x, double *y,
                         double *f) {
  int rc = check_csr(m, n, nnz, rowptr, col);
  if (rc) return rc;
  if (!f || (nnz > 0 && (!val || !x))) return -1;
  nsum tot = {0, 0};
  for (int64_t i = 0; i < m; ++i) {
    nsum yi = {0, 0};
    for (int64_t p = rowptr[i]; p < rowptr[i + 1]; ++p) nadd(&yi, val[p] * x[col[p]]);
    double v = nval(&yi);
    if (y) y[i] = v;
    nadd(&tot, v * v);
  }
  *f = nval(&tot);
  return 0;
}

/* Value and gradient with output adjoint fbar.  Reverse of the forward above:
 * ybar_i = 2 y_i fbar (broadcast of the reduction adjoint); every read
 * val[p] * x[col[p]] becomes xbar[col[p]] += val[p] ybar_i (the scatter-add of
 * the gathered x) and valbar[p] = x[col[p]] ybar_i.  gx (n) is overwritten;
 * gval (nnz) is overwritten when non-NULL. */
int kgo_spquadform_grad(int64_t m, int64_t n, int64_t nnz, const int32_t *rowptr,
                        const int32_t *col, const double *val, const double *x, double fbar,
                        double *f, double *gx, double *gval) {
  int rc = check_csr(m, n, nnz, rowptr, col);
  if (rc) return rc;
  if (n > 0 && !gx) return -1;
  double *y = (double *)malloc((size_t)(m > 0 ? m : 1) * sizeof(double));
  nsum *acc = (nsum *)calloc((size_t)(n > 0 ? n : 1), sizeof(nsum));
  if (!y || !acc) { free(y); free(acc); return -2; }
  double fv = 0;
  rc = kgo_spquadform_value(m, n, nnz, rowptr, col, val, x, y, &fv);
  if (rc) { free(y); free(acc); return rc; }
  if (f) *f = fv;
  for (int64_t i = 0; i < m; ++i) {
    double ybar = 2.0 * y[i] * fbar;
    for (int64_t p = rowptr[i]; p < rowptr[i + 1]; ++p) {
      nadd(&acc[col[p]], val[p] * ybar);
      if (gval) gval[p] = x[col[p]] * ybar;
    }
  }
  for (int64_t j = 0; j < n; ++j) gx[j] = nval(&acc[j]);
  free(y);
  free(acc);
  return 0;
}

/* ----------------------------------------------------- tet energy ------- */
/* Per-element forward quantities of f(u) = sum_e log1p(|G_e u_e|^2):
 * u_e = (u[conn[e][0..3]]) is a gather through the index map conn, and
 * g_e = G_e u_e with G_e 3x4 row-major (G[e*12 + r*4 + k]). */
static void tet_g(const int32_t *conn, const double *G, const double *u, int64_t e,
                  double g[3]) {
  for (int r = 0; r < 3; ++r) {
    double s = 0;
    for (int k = 0; k < 4; ++k) s += G[e * 12 + r * 4 + k] * u[conn[e * 4 + k]];
    g[r] = s;
  }
}

static int check_conn(int64_t ne, int64_t nv, const int32_t *conn) {
  for (int64_t i = 0; i < ne * 4; ++i)
    if (conn[i] < 0 || conn[i] >= nv) return -3;
  return 0;
}

int kgo_tet_value(int64_t ne, int64_t nv, const int32_t *conn, const double *G,
                  const double *u, double *f) {
  if (ne < 0 || nv < 0 || !f || (ne > 0 && (!conn || !G || !u))) return -1;
  if (check_conn(ne, nv, conn)) return -3;
  nsum tot = {0, 0};
  for (int64_t e = 0; e < ne; ++e) {
    double g[3];
    tet_g(conn, G, u, e, g);
    double s = g[0] * g[0] + g[1] * g[1] + g[2] * g[2];
    nadd(&tot, log1p(s));
  }
  *f = nval(&tot);
  return 0;
}

/* Reverse-pass quantity per element, for output adjoint fbar:
 *   f_e = log1p(s_e), s_e = |g_e|^2  ->  sbar = fbar / (1 + s_e),
 *   gbar_e = 2 sbar g_e,  c_e = G_e^T gbar_e  (the adjoint of u_e).
 * c (ne x 4) receives c_e; it is what a tape of the forward pass would hold. */
int kgo_tet_adjoint_local(int64_t ne, int64_t nv, const int32_t *conn, const double *G,
                          const double *u, double fbar, double *c) {
  if (ne < 0 || nv < 0 || (ne > 0 && (!conn || !G || !u || !c))) return -1;
  if (check_conn(ne, nv, conn)) return -3;
  for (int64_t e = 0; e < ne; ++e) {
    double g[3];
    tet_g(conn, G, u, e, g);
    double s = g[0] * g[0] + g[1] * g[1] + g[2] * g[2];
    double sbar = fbar / (1.0 + s);
    double gbar[3] = {2.0 * sbar * g[0], 2.0 * sbar * g[1], 2.0 * sbar * g[2]};
    for (int k = 0; k < 4; ++k)
      c[e * 4 + k] = G[e * 12 + 0 * 4 + k] * gbar[0] + G[e * 12 + 1 * 4 + k] * gbar[1] +
                     G[e * 12 + 2 * 4 + k] * gbar[2];
  }
  return 0;
}

/* Value and gradient of the tet energy.  The forward gather u[conn[e][k]] is
 * an index-map read, so its reverse is the scatter-add
 * gu[conn[e][k]] += c_e[k] (Sec. 3.3, first race rule), done here serially in
 * element order with a compensated accumulator per vertex.  gu (nv) is
 * overwritten. */
int kgo_tet_grad(int64_t ne, int64_t nv, const int32_t *conn, const double *G,
                 const double *u, double fbar, double *f, double *gu) {
  if (ne < 0 || nv < 0 || (nv > 0 && !gu) || (ne > 0 && (!conn || !G || !u))) return -1;
  if (check_conn(ne, nv, conn)) return -3;
  if (f) {
    int rc = kgo_tet_value(ne, nv, conn, G, u, f);
    if (rc) return rc;
  }
  double *c = (double *)malloc((size_t)(ne > 0 ? ne : 1) * 4 * sizeof(double));
  nsum *acc = (nsum *)calloc((size_t)(nv > 0 ? nv : 1), sizeof(nsum));
  if (!c || !acc) { free(c); free(acc); return -2; }
  kgo_tet_adjoint_local(ne, nv, conn, G, u, fbar, c);
  for (int64_t e = 0; e < ne; ++e)
    for (int k = 0; k < 4; ++k) nadd(&acc[conn[e * 4 + k]], c[e * 4 + k]);
  for (int64_t v = 0; v < nv; ++v) gu[v] = nval(&acc[v]);
  free(c);
  free(acc);
  return 0;
}

/* Hessian-vector product hv = fbar * (d^2 f / du^2)(u) v: the forward-mode
 * tangent (direction v) of the reverse pass above (forward over reverse).
 * Per element, with g = G_e u_e, s = |g|^2, sbar = fbar / (1 + s) and
 * gbar = 2 sbar g, the tangents are gdot = G_e v_e, sdot = 2 g . gdot,
 * sbardot = -fbar sdot / (1 + s)^2, gbardot = 2 (sbardot g + sbar gdot), and
 * the element's contribution G_e^T gbardot is scatter-added like c_e.
 * hv (nv) is overwritten. */
int kgo_tet_hvp(int64_t ne, int64_t nv, const int32_t *conn, const double *G, const double *u,
                const double *v, double fbar, double *hv) {
  if (ne < 0 || nv < 0 || (nv > 0 && !hv) || (ne > 0 && (!conn || !G || !u || !v))) return -1;
  if (check_conn(ne, nv, conn)) return -3;
  nsum *acc = (nsum *)calloc((size_t)(nv > 0 ? nv : 1), sizeof(nsum));
  if (!acc) return -2;
  for (int64_t e = 0; e < ne; ++e) {
    double g[3], gd[3];
    tet_g(conn, G, u, e, g);
    tet_g(conn, G, v, e, gd);
    double s = g[0] * g[0] + g[1] * g[1] + g[2] * g[2];
    double sd = 2.0 * (g[0] * gd[0] + g[1] * gd[1] + g[2] * gd[2]);
    double sbar = fbar / (1.0 + s);
    double sbard = -fbar * sd / ((1.0 + s) * (1.0 + s));
    double gbd[3];
    for (int r = 0; r < 3; ++r) gbd[r] = 2.0 * (sbard * g[r] + sbar * gd[r]);
    for (int k = 0; k < 4; ++k)
      nadd(&acc[conn[e * 4 + k]], G[e * 12 + 0 * 4 + k] * gbd[0] + G[e * 12 + 1 * 4 + k] * gbd[1] +
                                      G[e * 12 + 2 * 4 + k] * gbd[2]);
  }
  for (int64_t i = 0; i < nv; ++i) hv[i] = nval(&acc[i]);
  free(acc);
  return 0;
}

/* Gradient descent u <- u - eta * grad f(u), `steps` times, in place.
 * f_hist (steps + 1, nullable) receives f before each step and after the last. */
int kgo_tet_descent(int64_t ne, int64_t nv, const int32_t *conn, const double *G,
                    double *u, double eta, int steps, double *f_hist) {
  if (steps < 0 || (nv > 0 && !u)) return -1;
  double *gu = (double *)malloc((size_t)(nv > 0 ? nv : 1) * sizeof(double));
  if (!gu) return -2;
  for (int t = 0; t < steps; ++t) {
    double f;
    int rc = kgo_tet_grad(ne, nv, conn, G, u, 1.0, &f, gu);
    if (rc) { free(gu); return rc; }
    if (f_hist) f_hist[t] = f;
    for (int64_t v = 0; v < nv; ++v) u[v] -= eta * gu[v];
  }
  if (f_hist) {
    int rc = kgo_tet_value(ne, nv, conn, G, u, &f_hist[steps]);
    if (rc) { free(gu); return rc; }
  }
  free(gu);
  return 0;
}

/* -------------------------------------------- 1-D Laplacian (Sec. 4) ---- */
/* f(x, b) = ||A (3 x) - b||^2 with A = tridiag(-1, 2, -1), the rows at j = 0
 * and j = n-1 truncated (Sec. 4, Fig. "function_f").  Three kernels: scale
 * x3 = 3 x, the stencil y_j = 2 x3_j - b_j - x3_{j-1} - x3_{j+1} with
 * y2_j = y_j^2, and the reduction f = sum_j y2_j. */
static void lap_forward(int64_t n, const double *x, const double *b, double *x3, double *y,
                        double *y2) {
  for (int64_t j = 0; j < n; ++j) x3[j] = 3.0 * x[j];
  for (int64_t j = 0; j < n; ++j) {
    double v = 2.0 * x3[j] - b[j];
    if (j != 0) v -= x3[j - 1];
    if (j != n - 1) v -= x3[j + 1];
    y[j] = v;
    y2[j] = v * v;
  }
}

int kgo_laplace1d_value(int64_t n, const double *x, const double *b, double *f) {
  if (n < 0 || !f || (n > 0 && (!x || !b))) return -1;
  double *w = (double *)malloc((size_t)(n > 0 ? n : 1) * 3 * sizeof(double));
  if (!w) return -2;
  lap_forward(n, x, b, w, w + n, w + 2 * n);
  nsum s = {0, 0};
  for (int64_t j = 0; j < n; ++j) nadd(&s, w[2 * n + j]);
  *f = nval(&s);
  free(w);
  return 0;
}

/* Reverse pass of the three kernels, last kernel first (Sec. 4, Fig. "grad_f"):
 *   reduction  -> broadcast: y2bar_j = fbar;
 *   square     -> ybar_j = 2 y_j y2bar_j;
 *   stencil    -> each read of x3 becomes an accumulation into x3bar
 *                 (x3bar_j += 2 ybar_j, x3bar_{j-1} -= ybar_j if j != 0,
 *                 x3bar_{j+1} -= ybar_j if j != n-1) and b_j's read gives
 *                 bbar_j -= ybar_j;
 *   scale      -> xbar_j = 3 x3bar_j.
 * The stencil's neighbour updates are the accesses the paper's race detection
 * turns into atomics; serially they are plain adds.  gx and gb (n) are
 * overwritten (both nullable). */
int kgo_laplace1d_grad(int64_t n, const double *x, const double *b, double fbar, double *f,
                       double *gx, double *gb) {
  if (n < 0 || (n > 0 && (!x || !b))) return -1;
  double *w = (double *)malloc((size_t)(n > 0 ? n : 1) * 4 * sizeof(double));
  if (!w) return -2;
  double *x3 = w, *y = w + n, *y2 = w + 2 * n, *x3bar = w + 3 * n;
  lap_forward(n, x, b, x3, y, y2);
  if (f) {
    nsum s = {0, 0};
    for (int64_t j = 0; j < n; ++j) nadd(&s, y2[j]);
    *f = nval(&s);
  }
  for (int64_t j = 0; j < n; ++j) x3bar[j] = 0.0;
  for (int64_t j = 0; j < n; ++j) {
    double y2bar = fbar;
    double ybar = 2.0 * y[j] * y2bar;
    if (j != n - 1) x3bar[j + 1] -= ybar;
    if (j != 0) x3bar[j - 1] -= ybar;
    x3bar[j] += 2.0 * ybar;
    if (gb) gb[j] = -ybar;
  }
  if (gx)
    for (int64_t j = 0; j < n; ++j) gx[j] = 3.0 * x3bar[j];
  free(w);
  return 0;
}

/* Hessian-vector product of the 1-D example: the tangent (direction v) of
 * the forward chain x3 = 3x, y = A x3 - b and of the reverse above; b and x
 * drop out (f is quadratic in x), ydot = A (3 v), ybardot = 2 fbar ydot and
 * hv = 3 A^T ybardot with the same boundary guards.  hv (n) is overwritten. */
int kgo_laplace1d_hvp(int64_t n, const double *v, double fbar, double *hv) {
  if (n < 0 || (n > 0 && (!v || !hv))) return -1;
  double *w = (double *)malloc((size_t)(n > 0 ? n : 1) * 2 * sizeof(double));
  if (!w) return -2;
  double *yd = w, *x3bd = w + n;
  for (int64_t j = 0; j < n; ++j) {
    double t = 2.0 * (3.0 * v[j]);
    if (j != 0) t -= 3.0 * v[j - 1];
    if (j != n - 1) t -= 3.0 * v[j + 1];
    yd[j] = t;
    x3bd[j] = 0.0;
  }
  for (int64_t j = 0; j < n; ++j) {
    double ybd = 2.0 * yd[j] * fbar;
    if (j != n - 1) x3bd[j + 1] -= ybd;
    if (j != 0) x3bd[j - 1] -= ybd;
    x3bd[j] += 2.0 * ybd;
  }
  for (int64_t j = 0; j < n; ++j) hv[j] = 3.0 * x3bd[j];
  free(w);
  return 0;
}
