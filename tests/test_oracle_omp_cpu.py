"""The OpenMP CPU baseline (oracle/kg_oracle_omp.c) computes what the serial
oracle computes: same value and gradient up to the order of compensated sums,
run-to-run identical for a given thread count, and the same argument checks.
It is a timing baseline only; parity tests use the serial oracle."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2507_13204_gb300 import workloads as W


@pytest.mark.parametrize("m,n", [(1, 1), (7, 5), (300, 257), (1000, 64)])
def test_dense_omp_matches_serial_oracle(m, n):
    A, x = W.quadform_inputs(n, m=m, seed=m + n)
    f1, g1 = O.quadform_grad(A, x, fbar=1.5)
    f2, g2, t = O.quadform_grad_omp(A, x, fbar=1.5)
    assert t >= 1
    assert abs(f2 - f1) <= 1e-14 * abs(f1)
    assert np.linalg.norm(g2 - g1) <= 1e-14 * np.linalg.norm(g1)
    f3, g3, _ = O.quadform_grad_omp(A, x, fbar=1.5)
    assert f3 == f2 and np.array_equal(g3, g2)


@pytest.mark.parametrize("a,jitter", [(1, None), (3, 2), (12, None)])
def test_tet_omp_matches_serial_oracle(a, jitter):
    mesh = W.tet_mesh(a, jitter_seed=jitter, perm_seed=5)
    u = np.random.default_rng(a).uniform(-1, 1, mesh.nv)
    f1, g1 = O.tet_grad(mesh.conn, mesh.G, u, fbar=0.5)
    f2, g2, t = O.tet_grad_omp(mesh.conn, mesh.G, u, fbar=0.5)
    assert t >= 1
    assert abs(f2 - f1) <= 1e-14 * abs(f1)
    assert np.linalg.norm(g2 - g1) <= 1e-14 * np.linalg.norm(g1)
    f3, g3, _ = O.tet_grad_omp(mesh.conn, mesh.G, u, fbar=0.5)
    assert f3 == f2 and np.array_equal(g3, g2)


def test_tet_omp_rejects_bad_connectivity():
    mesh = W.tet_mesh(2)
    u = np.zeros(mesh.nv)
    conn = mesh.conn.copy()
    conn[3, 2] = mesh.nv
    with pytest.raises(ValueError):
        O.tet_grad_omp(conn, mesh.G, u)
