"""Pins for the CPU oracle: each check is fixed by the mathematics or the paper,
not by the oracle itself (closed forms, special cases, dual numbers, exact
rational arithmetic, central differences, mesh invariants)."""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

from oracle import oracle as O
from paper_2507_13204_gb300 import workloads as W
from tests.dual import Dual, log1p as dlog1p, seed

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def rel(a, b):
    a, b = np.asarray(a, float), np.asarray(b, float)
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


# ------------------------------------------------------------------ dense
def test_quadform_identity_and_diag():
    x = np.random.default_rng(0).uniform(-1, 1, 17)
    f, gx = O.quadform_grad(np.eye(17), x)
    assert f == pytest.approx(float(np.dot(x, x)), rel=1e-15)
    assert np.array_equal(gx, 2 * x)
    d = np.random.default_rng(1).normal(size=17)
    f, gx = O.quadform_grad(np.diag(d), x)
    assert rel(gx, 2 * d * d * x) < 1e-15
    assert f == pytest.approx(float(np.sum((d * x) ** 2)), rel=1e-14)


def test_quadform_single_entry_exact():
    A = np.zeros((5, 7))
    A[3, 2] = 0.75
    x = np.linspace(-1, 1, 7)
    f, gx, gA = O.quadform_grad(A, x, want_gA=True)
    y3 = 0.75 * x[2]
    assert f == y3 * y3
    expect = np.zeros(7)
    expect[2] = 2 * y3 * 0.75
    assert np.array_equal(gx, expect)
    assert gA[3, 2] == 2 * y3 * x[2] and np.count_nonzero(gA[3]) == np.count_nonzero(x)


@pytest.mark.parametrize("m,n", [(64, 64), (33, 70), (1, 1), (100, 3)])
def test_quadform_closed_form(m, n):
    A, x = W.quadform_inputs(n, m=m, seed=7)
    f, gx, gA = O.quadform_grad(A, x, fbar=1.0, want_gA=True)
    y = A @ x  # library GEMV
    assert f == pytest.approx(float(y @ y), rel=1e-13)
    assert rel(gx, 2 * A.T @ y) < 1e-13
    assert rel(gA, 2 * np.outer(y, x)) < 1e-14
    # Euler's theorem: f is homogeneous of degree 2 in x and in A
    assert float(x @ gx) == pytest.approx(2 * f, rel=1e-12)
    assert float(np.sum(A * gA)) == pytest.approx(2 * f, rel=1e-12)
    # linear in the output adjoint
    f2, gx2 = O.quadform_grad(A, x, fbar=-2.5)
    assert f2 == f and rel(gx2, -2.5 * gx) < 1e-15


def test_quadform_dual_numbers():
    A, x = W.quadform_inputs(6, m=5, seed=11)
    _, gx, gA = O.quadform_grad(A, x, want_gA=True)

    def f_dual(Am, xv):
        tot = Dual(0.0)
        for i in range(len(Am)):
            yi = Dual(0.0)
            for j in range(len(xv)):
                yi = yi + Am[i][j] * xv[j]
            tot = tot + yi * yi
        return tot

    for j in range(6):
        assert f_dual(A.tolist(), seed(x, j)).d == pytest.approx(gx[j], rel=1e-13, abs=1e-15)
    for (i, j) in [(0, 0), (4, 5), (2, 3)]:
        Ad = [[Dual(A[r][c], 1.0 if (r, c) == (i, j) else 0.0) for c in range(6)] for r in range(5)]
        assert f_dual(Ad, list(x)).d == pytest.approx(gA[i, j], rel=1e-13, abs=1e-15)


def test_quadform_exact_rational():
    # f is quadratic in x, so a central difference is exact in rational arithmetic.
    rng = np.random.default_rng(3)
    A = rng.integers(-4, 5, (4, 4)).astype(float) / 8
    x = rng.integers(-8, 9, 4).astype(float) / 16
    Af = [[Fraction(v) for v in row] for row in A]
    xf = [Fraction(v) for v in x]

    def f_exact(xv):
        return sum(sum(Af[i][j] * xv[j] for j in range(4)) ** 2 for i in range(4))

    f, gx = O.quadform_grad(A, x)
    assert Fraction(f) == f_exact(xf)  # dyadic inputs: every step is exact in binary
    for j in range(4):
        h = Fraction(1, 3)
        xp = list(xf); xp[j] += h
        xm = list(xf); xm[j] -= h
        assert Fraction(gx[j]) == (f_exact(xp) - f_exact(xm)) / (2 * h)


def test_quadform_central_difference():
    A, x = W.quadform_inputs(12, seed=5)
    f, gx = O.quadform_grad(A, x)
    for j in range(12):
        h = 1e-6 * max(1.0, abs(x[j]))
        xp, xm = x.copy(), x.copy()
        xp[j] += h
        xm[j] -= h
        fd = (O.quadform_value(A, xp) - O.quadform_value(A, xm)) / (2 * h)
        assert fd == pytest.approx(gx[j], rel=1e-6, abs=1e-8)


def test_quadform_empty():
    f, gx = O.quadform_grad(np.zeros((0, 4)), np.ones(4))
    assert f == 0.0 and np.array_equal(gx, np.zeros(4))


# ------------------------------------------------------------------ sparse (CSR)
def _small_csr(seed=11, m=9, n=7):
    A, x = W.spquadform_inputs(m, n, d_lo=0, d_hi=5, seed=seed)
    return A, x


def test_spquadform_closed_form_with_repeats_and_empty_rows():
    # grad = 2 fbar A^T (A x) on the densified matrix (numpy), valbar_p = 2 fbar y_i x_col(p)
    for seed in (11, 12, 13):
        A, x = _small_csr(seed)
        D = A.dense()
        y = D @ x
        f, gx, gval = O.spquadform_grad(A.rowptr, A.col, A.val, x, fbar=0.75, want_gval=True)
        assert f == pytest.approx(float(y @ y), rel=1e-14)
        assert rel(gx, 1.5 * D.T @ y) < 1e-14
        rows = np.repeat(np.arange(A.m), np.diff(A.rowptr))
        assert rel(gval, 1.5 * y[rows] * x[A.col]) < 1e-14


def test_spquadform_repeated_column_adds():
    # a row storing column 2 twice (values a, b) behaves as one entry a + b
    rowptr = np.array([0, 3, 4], np.int32)
    col = np.array([2, 2, 0, 1], np.int32)
    val = np.array([0.5, -2.0, 1.0, 3.0])
    x = np.array([0.25, -1.0, 4.0])
    f, gx = O.spquadform_grad(rowptr, col, val, x)
    D = np.array([[1.0, 0.0, -1.5], [0.0, 3.0, 0.0]])
    assert f == (D @ x) @ (D @ x)
    assert np.array_equal(gx, 2 * D.T @ (D @ x))


def test_spquadform_equals_dense_oracle_on_dense_pattern():
    # every entry stored, in column order: the sparse forward is the dense one entry for entry
    A, x = W.quadform_inputs(6, m=5, seed=2)
    rowptr = np.arange(0, 31, 6, dtype=np.int32)
    col = np.tile(np.arange(6, dtype=np.int32), 5)
    fs, gs = O.spquadform_grad(rowptr, col, A.ravel(), x)
    fd, gd = O.quadform_grad(A, x)
    assert fs == fd and np.array_equal(gs, gd)


def test_spquadform_exact_rational():
    rowptr = np.array([0, 2, 2, 5], np.int32)
    col = np.array([0, 3, 1, 1, 2], np.int32)
    val = np.array([1.0, 2.0, 3.0, -1.0, 0.5])
    x = np.array([1.0, 2.0, 3.0, 4.0])
    f, gx, gval = O.spquadform_grad(rowptr, col, val, x, want_gval=True)
    # y = (1 + 8, 0, 6 - 2 + 1.5) = (9, 0, 5.5); f = 81 + 30.25
    assert f == 111.25
    assert np.array_equal(gx, [18.0, 22.0, 5.5, 36.0])
    assert np.array_equal(gval, [18.0, 72.0, 22.0, 22.0, 33.0])


def test_spquadform_dual_numbers_in_x_and_val():
    A, x = _small_csr(14, m=6, n=5)
    f, gx, gval = O.spquadform_grad(A.rowptr, A.col, A.val, x, want_gval=True)

    def f_dual(val, xv):
        tot = 0.0
        for i in range(A.m):
            yi = 0.0
            for p in range(A.rowptr[i], A.rowptr[i + 1]):
                yi = yi + val[p] * xv[A.col[p]]
            tot = tot + yi * yi
        return tot

    for j in range(A.n):
        assert f_dual(list(A.val), seed(x, j)).d == pytest.approx(gx[j], rel=1e-13, abs=1e-14)
    for p in range(A.nnz):
        assert f_dual(seed(A.val, p), list(x)).d == pytest.approx(gval[p], rel=1e-13, abs=1e-14)


def test_spquadform_empty_and_rejects_bad_structure():
    f, gx = O.spquadform_grad(np.zeros(4, np.int32), np.zeros(0, np.int32), np.zeros(0), np.ones(3))
    assert f == 0.0 and np.array_equal(gx, np.zeros(3))
    with pytest.raises(ValueError):  # column out of range
        O.spquadform_grad(np.array([0, 1], np.int32), np.array([3], np.int32), np.ones(1), np.ones(3))
    with pytest.raises(ValueError):  # decreasing rowptr
        O.spquadform_grad(np.array([0, 2, 1, 2], np.int32), np.array([0, 1], np.int32), np.ones(2),
                          np.ones(3))


# ------------------------------------------------------------------ tets
def _ref_tet():
    rows = [l for l in open(os.path.join(GOLDEN, "single_tet_reference.txt"))
            if l.strip() and not l.startswith("#")]
    G = np.array([[float(v) for v in r.split()] for r in rows]).reshape(1, 12)
    return np.array([[0, 1, 2, 3]], np.int32), G


def test_single_tet_golden_matches_mesh_geometry():
    conn, G = _ref_tet()
    p = np.array([[[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]]], float)
    assert np.array_equal(W.p1_gradients(p), G)


def test_single_tet_closed_form():
    conn, G = _ref_tet()
    u = np.array([0.3, -0.7, 0.25, 0.9])
    g = u[1:] - u[0]
    s = float(g @ g)
    f, gu = O.tet_grad(conn, G, u, fbar=1.0)
    assert f == pytest.approx(math.log1p(s), rel=1e-15)
    d = 2 * g / (1 + s)
    assert rel(gu, np.concatenate([[-d.sum()], d])) < 1e-15
    c = O.tet_adjoint_local(conn, G, u, fbar=3.0)
    assert rel(c[0], 3 * np.concatenate([[-d.sum()], d])) < 1e-15


def test_tet_zero_field():
    mesh = W.tet_mesh(3, jitter_seed=2)
    f, gu = O.tet_grad(mesh.conn, mesh.G, np.zeros(mesh.nv))
    assert f == 0.0 and not gu.any()


def test_tet_linear_field_reproduced():
    mesh = W.tet_mesh(4, perm_seed=9)
    a = np.array([0.3, -0.2, 0.5])
    u = W.linear_field(mesh, a)
    f, gu = O.tet_grad(mesh.conn, mesh.G, u)
    assert f == pytest.approx(mesh.ne * math.log1p(float(a @ a)), rel=1e-13)
    # equal-volume Kuhn tets: sum of incident grad lambda_v vanishes at interior vertices
    gi = np.rint(mesh.coords).astype(int)
    interior = np.all((gi > 0) & (gi < 4), axis=1)
    assert interior.sum() == 27
    assert np.max(np.abs(gu[interior])) < 1e-14
    assert np.max(np.abs(gu[~interior])) > 1e-3


def test_tet_translation_invariance():
    mesh = W.tet_mesh(3, jitter_seed=2)
    u = np.random.default_rng(4).uniform(-1, 1, mesh.nv)
    f, gu = O.tet_grad(mesh.conn, mesh.G, u)
    assert abs(gu.sum()) < 1e-12 * np.abs(gu).sum()
    f2 = O.tet_value(mesh.conn, mesh.G, u + 0.37)
    assert f2 == pytest.approx(f, rel=1e-13)


def test_tet_permutation_equivariance():
    m0 = W.tet_mesh(3, relabel=False)
    m1 = W.tet_mesh(3, perm_seed=5)
    u0 = np.random.default_rng(6).uniform(-1, 1, m0.nv)
    u1 = np.empty_like(u0)
    u1[m1.perm] = u0  # same field, relabelled ids
    f0, g0 = O.tet_grad(m0.conn, m0.G, u0)
    f1, g1 = O.tet_grad(m1.conn, m1.G, u1)
    assert f1 == pytest.approx(f0, rel=1e-14)
    assert rel(g1[m1.perm], g0) < 1e-14


def test_tet_dual_numbers_random_G():
    rng = np.random.default_rng(8)
    mesh = W.tet_mesh(1)  # 6 tets, 8 vertices
    G = rng.normal(size=mesh.G.shape)  # G is per-element data: any values are valid
    u = rng.uniform(-1, 1, mesh.nv)
    f, gu = O.tet_grad(mesh.conn, G, u, fbar=0.7)

    def f_dual(uv):
        tot = Dual(0.0)
        for e in range(mesh.ne):
            s = Dual(0.0)
            for r in range(3):
                g = Dual(0.0)
                for k in range(4):
                    g = g + G[e, r * 4 + k] * uv[mesh.conn[e, k]]
                s = s + g * g
            tot = tot + dlog1p(s)
        return tot * 0.7

    for v in range(mesh.nv):
        fd = f_dual(seed(u, v))
        assert fd.v == pytest.approx(0.7 * f, rel=1e-14)
        assert fd.d == pytest.approx(gu[v], rel=1e-13, abs=1e-15)


def test_tet_central_difference_jittered():
    mesh = W.tet_mesh(2, jitter_seed=2)
    u = np.random.default_rng(10).uniform(-1, 1, mesh.nv)
    _, gu = O.tet_grad(mesh.conn, mesh.G, u)
    for v in range(0, mesh.nv, 3):
        h = 1e-6 * max(1.0, abs(u[v]))
        up, um = u.copy(), u.copy()
        up[v] += h
        um[v] -= h
        fd = (O.tet_value(mesh.conn, mesh.G, up) - O.tet_value(mesh.conn, mesh.G, um)) / (2 * h)
        assert fd == pytest.approx(gu[v], rel=1e-6, abs=1e-8)


def test_tet_adjoint_local_scatters_to_grad():
    mesh = W.tet_mesh(3, jitter_seed=2, perm_seed=3)
    u = np.random.default_rng(12).uniform(-1, 1, mesh.nv)
    c = O.tet_adjoint_local(mesh.conn, mesh.G, u, fbar=1.0)
    acc = np.zeros(mesh.nv)
    np.add.at(acc, mesh.conn.reshape(-1), c.reshape(-1))
    _, gu = O.tet_grad(mesh.conn, mesh.G, u)
    assert rel(acc, gu) < 1e-14


def test_tet_rejects_bad_connectivity():
    conn = np.array([[0, 1, 2, 5]], np.int32)
    with pytest.raises(ValueError):
        O.tet_grad(conn, np.zeros((1, 12)), np.zeros(4))


def test_tet_descent_steps():
    mesh = W.tet_mesh(2, jitter_seed=2)
    u0 = np.random.default_rng(13).uniform(-1, 1, mesh.nv)
    u1, hist = O.tet_descent(mesh.conn, mesh.G, u0, 0.05, 1)
    f0, g0 = O.tet_grad(mesh.conn, mesh.G, u0)
    assert hist[0] == f0
    assert rel(u1, u0 - 0.05 * g0) < 1e-15
    # f is L-smooth with L = 2 * lambda_max(sum_e P_e^T G_e^T G_e P_e) (about 144 on the
    # unit Kuhn grid, more when jittered), so any eta < 2/L decreases f at every step.
    u20, hist20 = O.tet_descent(mesh.conn, mesh.G, u0, 0.005, 20)
    assert np.all(np.diff(hist20) < 0)


# ------------------------------------------------------------------ 1-D Laplacian
def _lap_matrix(n):
    return 2 * np.eye(n) - np.eye(n, k=1) - np.eye(n, k=-1)


def test_laplace1d_n1():
    x, b = np.array([0.4]), np.array([-0.3])
    f, gx, gb = O.laplace1d_grad(x, b)
    r = 6 * 0.4 + 0.3
    assert f == pytest.approx(r * r, rel=1e-15)
    assert gx[0] == pytest.approx(12 * r, rel=1e-15)
    assert gb[0] == pytest.approx(-2 * r, rel=1e-15)


@pytest.mark.parametrize("n", [2, 3, 17, 1000])
def test_laplace1d_closed_form(n):
    x, b = W.laplace1d_inputs(n)
    A = _lap_matrix(n)
    y = A @ (3 * x) - b
    f, gx, gb = O.laplace1d_grad(x, b, fbar=1.5)
    assert f == pytest.approx(float(y @ y), rel=1e-13)
    assert rel(gx, 1.5 * 6 * A @ y) < 1e-13
    assert rel(gb, -1.5 * 2 * y) < 1e-14
    assert O.laplace1d_value(x, b) == f


def test_laplace1d_golden_unit_residual():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "laplace1d_unit_residual_n5.txt"))
            if l.strip() and not l.startswith("#")]
    n = 5
    A = _lap_matrix(n)
    x = np.array([0.25, -0.5, 0.75, 0.125, -1.0])  # dyadic: A(3x) is exact
    for r in rows:
        k = int(r[0])
        expect = np.array([float(v) for v in r[1:]])
        b = A @ (3 * x)
        b[k] -= 1.0  # y = A(3x) - b = e_k
        f, gx, gb = O.laplace1d_grad(x, b)
        assert f == 1.0
        assert np.array_equal(gx, expect)
        assert np.array_equal(gb, -2.0 * np.eye(n)[k])


def test_laplace1d_exact_rational():
    n = 6
    x = [Fraction(k - 2, 8) for k in range(n)]
    b = [Fraction(3 - k, 4) for k in range(n)]

    def f_exact(xv, bv):
        tot = Fraction(0)
        for j in range(n):
            v = 2 * 3 * xv[j] - bv[j]
            if j > 0:
                v -= 3 * xv[j - 1]
            if j < n - 1:
                v -= 3 * xv[j + 1]
            tot += v * v
        return tot

    f, gx, gb = O.laplace1d_grad(np.array([float(v) for v in x]), np.array([float(v) for v in b]))
    assert Fraction(f) == f_exact(x, b)
    h = Fraction(1, 7)
    for j in range(n):
        xp = list(x); xp[j] += h
        xm = list(x); xm[j] -= h
        assert Fraction(gx[j]) == (f_exact(xp, b) - f_exact(xm, b)) / (2 * h)
        bp = list(b); bp[j] += h
        bm = list(b); bm[j] -= h
        assert Fraction(gb[j]) == (f_exact(x, bp) - f_exact(x, bm)) / (2 * h)


def test_laplace1d_dual_numbers():
    x, b = W.laplace1d_inputs(7, seed=9)
    _, gx, gb = O.laplace1d_grad(x, b)

    def f_dual(xv, bv):
        n = len(xv)
        tot = Dual(0.0)
        for j in range(n):
            v = 6 * xv[j] - bv[j]
            if j > 0:
                v = v - 3 * xv[j - 1]
            if j < n - 1:
                v = v - 3 * xv[j + 1]
            tot = tot + v * v
        return tot

    for j in range(7):
        assert f_dual(seed(x, j), list(b)).d == pytest.approx(gx[j], rel=1e-13, abs=1e-14)
        assert f_dual(list(x), seed(b, j)).d == pytest.approx(gb[j], rel=1e-13, abs=1e-14)


# ------------------------------------------------------------------ Hessian-vector products
def test_tet_hvp_central_difference_of_gradient():
    mesh = W.tet_mesh(3, 2, 2, jitter_seed=2, perm_seed=5)
    rng = np.random.default_rng(31)
    u, v = rng.uniform(-1, 1, mesh.nv), rng.uniform(-1, 1, mesh.nv)
    hv = O.tet_hvp(mesh.conn, mesh.G, u, v, fbar=0.7)
    h = 1e-5
    fd = (O.tet_grad(mesh.conn, mesh.G, u + h * v, fbar=0.7)[1]
          - O.tet_grad(mesh.conn, mesh.G, u - h * v, fbar=0.7)[1]) / (2 * h)
    assert rel(hv, fd) < 1e-8


def test_tet_hvp_is_symmetric():
    mesh = W.tet_mesh(3, jitter_seed=4, perm_seed=2)
    rng = np.random.default_rng(32)
    u, v, w = (rng.uniform(-1, 1, mesh.nv) for _ in range(3))
    a = w @ O.tet_hvp(mesh.conn, mesh.G, u, v)
    b = v @ O.tet_hvp(mesh.conn, mesh.G, u, w)
    assert a == pytest.approx(b, rel=1e-12)


def test_tet_hvp_at_zero_is_the_stacked_quadratic_form():
    # at u = 0 every element contributes fbar * 2 G_e^T G_e: the Hessian of
    # fbar * ||B v||^2 with B the 3 N_e x N_v matrix whose rows are G_e placed at conn[e]
    mesh = W.tet_mesh(2, jitter_seed=3, perm_seed=7)
    B = np.zeros((3 * mesh.ne, mesh.nv))
    for e in range(mesh.ne):
        for r in range(3):
            for k in range(4):
                B[3 * e + r, mesh.conn[e, k]] += mesh.G[e, 4 * r + k]
    v = np.random.default_rng(33).uniform(-1, 1, mesh.nv)
    hv = O.tet_hvp(mesh.conn, mesh.G, np.zeros(mesh.nv), v, fbar=1.5)
    assert rel(hv, O.quadform_grad(B, v, fbar=1.5)[1]) < 1e-13


def test_laplace1d_hvp_linearity_and_difference():
    # f is quadratic in x: H v = grad(v, b) - grad(0, b) for any b, and H is symmetric
    for n in (1, 2, 9, 50):
        x, b = W.laplace1d_inputs(n, seed=n)
        v = np.random.default_rng(n).uniform(-1, 1, n)
        hv = O.laplace1d_hvp(v, fbar=0.5)
        g1 = O.laplace1d_grad(v, b, fbar=0.5)[1]
        g0 = O.laplace1d_grad(np.zeros(n), b, fbar=0.5)[1]
        assert rel(hv, g1 - g0) < 1e-13
        w = np.random.default_rng(n + 1).uniform(-1, 1, n)
        assert w @ hv == pytest.approx(v @ O.laplace1d_hvp(w, fbar=0.5), rel=1e-12)


# ------------------------------------------------------------------ mutation check
def test_pins_catch_planted_mistakes(tmp_path):
    """Build oracle copies with one plausible mistake each and check a pin fails."""
    import ctypes
    import subprocess
    src = open(os.path.join(os.path.dirname(O.__file__), "kg_oracle.c")).read()
    mutants = {
        "dropped_factor2": ("double ybar = 2.0 * y[i] * fbar;", "double ybar = y[i] * fbar;"),
        "transposed_A": ("nadd(&acc[j], A[i * n + j] * ybar);", "nadd(&acc[j], A[j * n + i] * ybar);"),
        "tet_wrong_sign": ("double sbar = fbar / (1.0 + s);", "double sbar = fbar / (1.0 - s);"),
        "tet_wrong_col": ("c[e * 4 + k] = G[e * 12 + 0 * 4 + k] * gbar[0]",
                          "c[e * 4 + k] = G[e * 12 + 0 * 4 + (3 - k)] * gbar[0]"),
        "lap_missing_guard": ("if (j != n - 1) x3bar[j + 1] -= ybar;",
                              "if (j + 1 < n) x3bar[j + 1] += ybar;"),
        "sp_scatter_to_row": ("nadd(&acc[col[p]], val[p] * ybar);", "nadd(&acc[i % n], val[p] * ybar);"),
        "sp_gather_first_col": ("nadd(&yi, val[p] * x[col[p]]);", "nadd(&yi, val[p] * x[col[rowptr[i]]]);"),
        "hvp_dropped_curvature": ("double sbard = -fbar * sd / ((1.0 + s) * (1.0 + s));",
                                  "double sbard = 0.0;"),
    }
    for name, (old, new) in mutants.items():
        assert old in src, name
        path = tmp_path / f"{name}.c"
        path.write_text(src.replace(old, new))
        so = tmp_path / f"{name}.so"
        subprocess.run(["gcc", *O.CFLAGS, "-o", str(so), str(path), "-lm"], check=True)
        lib = ctypes.CDLL(str(so))
        p = lambda a: a.ctypes.data_as(ctypes.c_void_p)
        caught = False
        if name in ("dropped_factor2", "transposed_A"):
            A, x = W.quadform_inputs(9, m=7, seed=1)
            A = np.ascontiguousarray(A[:, :7]) if name == "transposed_A" else A
            x = x[:A.shape[1]].copy()
            f, gx = np.zeros(1), np.empty(A.shape[1])
            lib.kgo_quadform_grad(ctypes.c_int64(A.shape[0]), ctypes.c_int64(A.shape[1]), p(A), p(x),
                                  ctypes.c_double(1.0), p(f), p(gx), None)
            caught = rel(gx, 2 * A.T @ (A @ x)) > 1e-6
        elif name.startswith("sp_"):
            A, x = _small_csr(15, m=8, n=6)
            f, gx = np.zeros(1), np.empty(A.n)
            lib.kgo_spquadform_grad(ctypes.c_int64(A.m), ctypes.c_int64(A.n), ctypes.c_int64(A.nnz),
                                    p(A.rowptr), p(A.col), p(A.val), p(x), ctypes.c_double(1.0),
                                    p(f), p(gx), None)
            D = A.dense()
            caught = rel(gx, 2 * D.T @ (D @ x)) > 1e-6
        elif name.startswith("hvp"):
            mesh = W.tet_mesh(2, jitter_seed=3, perm_seed=1)
            rng = np.random.default_rng(34)
            u, v = rng.uniform(-1, 1, mesh.nv), rng.uniform(-1, 1, mesh.nv)
            hv = np.empty(mesh.nv)
            conn, G = np.ascontiguousarray(mesh.conn), np.ascontiguousarray(mesh.G)
            lib.kgo_tet_hvp(ctypes.c_int64(mesh.ne), ctypes.c_int64(mesh.nv), p(conn), p(G), p(u), p(v),
                            ctypes.c_double(1.0), p(hv))
            h = 1e-5
            fd = (O.tet_grad(conn, G, u + h * v)[1] - O.tet_grad(conn, G, u - h * v)[1]) / (2 * h)
            caught = rel(hv, fd) > 1e-6
        elif name.startswith("tet"):
            conn, G = _ref_tet()
            u = np.array([0.3, -0.7, 0.25, 0.9])
            g = u[1:] - u[0]
            d = 2 * g / (1 + g @ g)
            gu, f = np.empty(4), np.zeros(1)
            lib.kgo_tet_grad(ctypes.c_int64(1), ctypes.c_int64(4), p(conn), p(G), p(u),
                             ctypes.c_double(1.0), p(f), p(gu))
            caught = rel(gu, np.concatenate([[-d.sum()], d])) > 1e-6
        else:
            x, b = W.laplace1d_inputs(9)
            f, gx, gb = np.zeros(1), np.empty(9), np.empty(9)
            lib.kgo_laplace1d_grad(ctypes.c_int64(9), p(x), p(b), ctypes.c_double(1.0), p(f), p(gx), p(gb))
            A = _lap_matrix(9)
            caught = rel(gx, 6 * A @ (A @ (3 * x) - b)) > 1e-6
        assert caught, f"planted mistake {name} not caught"
