"""The seeded input generators follow their stated recipes: shapes, draw order and
determinism, value distributions, the Kuhn mesh's geometry and relabelling, the
CSR structure, and the batched size mixes.  Host only."""
import math

import numpy as np
import pytest

from paper_2507_13204_gb300 import workloads as W


def test_quadform_inputs_recipe():
    A, x = W.quadform_inputs(400, m=300, seed=11)
    A2, x2 = W.quadform_inputs(400, m=300, seed=11)
    assert A.shape == (300, 400) and x.shape == (400,)
    assert np.array_equal(A, A2) and np.array_equal(x, x2)
    # N(0, 1/n): 120000 draws give the variance to about 0.4 %
    assert abs(A.var() * 400 - 1.0) < 0.02 and abs(A.mean()) < 0.01
    assert x.min() >= -1.0 and x.max() <= 1.0
    # A is drawn first, then x: the same generator continued gives x
    rng = np.random.Generator(np.random.PCG64(11))
    rng.standard_normal((300, 400))
    assert np.array_equal(rng.uniform(-1.0, 1.0, 400), x)


@pytest.mark.parametrize("box", [(1, 1, 1), (3, 2, 4)])
def test_kuhn_mesh_geometry(box):
    a, b, c = box
    mesh = W.tet_mesh(a, b, c, perm_seed=5)
    assert mesh.ne == 6 * a * b * c and mesh.nv == (a + 1) * (b + 1) * (c + 1)
    assert mesh.conn.dtype == np.int32 and mesh.conn.min() >= 0 and mesh.conn.max() < mesh.nv
    assert all(len(set(t)) == 4 for t in mesh.conn.tolist())
    p = mesh.coords[mesh.conn]                       # [Ne, 4, 3]
    J = np.stack([p[:, 1] - p[:, 0], p[:, 2] - p[:, 0], p[:, 3] - p[:, 0]], axis=2)
    assert np.allclose(np.abs(np.linalg.det(J)), 1.0)  # unit Kuhn tets: volume 1/6
    G = mesh.G.reshape(-1, 3, 4)                      # column k = grad lambda_k
    assert np.allclose(G.sum(axis=2), 0.0)            # the barycentrics sum to 1
    # grad lambda_k . (p_j - p_0) = delta_kj for k, j = 1..3
    assert np.allclose(np.einsum("erk,erj->ekj", G[:, :, 1:], J), np.eye(3)[None])
    # the six tets of one cube come first and share its diagonal (slots 0 and 3)
    assert len(set(mesh.conn[:6, 0])) == 1 and len(set(mesh.conn[:6, 3])) == 1
    assert len(set(map(tuple, np.sort(mesh.conn[:6], axis=1)))) == 6


def test_relabelling_is_a_permutation_of_the_grid():
    mesh = W.tet_mesh(3, 2, 2, perm_seed=9)
    plain = W.tet_mesh(3, 2, 2, relabel=False)
    assert sorted(mesh.perm.tolist()) == list(range(mesh.nv))
    assert np.array_equal(mesh.conn, mesh.perm[plain.conn])
    assert np.array_equal(mesh.coords[mesh.perm], plain.coords)
    assert np.array_equal(mesh.G, plain.G)


def test_jitter_moves_interior_vertices_only():
    plain = W.tet_mesh(4, relabel=False)
    jit = W.tet_mesh(4, relabel=False, jitter_seed=2)
    d = np.abs(jit.coords - plain.coords).max(axis=1)
    gi = plain.coords
    interior = np.all((gi > 0) & (gi < 4), axis=1)
    assert np.all(d[~interior] == 0.0)
    assert np.all(d[interior] > 0.0) and d.max() <= 0.1


def test_tet_inputs_draw_order():
    mesh, u = W.tet_inputs(3, seed=4)
    rng = np.random.Generator(np.random.PCG64(4))
    assert np.array_equal(rng.permutation(mesh.nv), mesh.perm)
    assert np.array_equal(rng.uniform(-1.0, 1.0, mesh.nv), u)


def test_csr_recipe():
    A, x = W.spquadform_inputs(5000, 3000, d_lo=8, d_hi=24, seed=7)
    deg = np.diff(A.rowptr)
    assert A.rowptr[0] == 0 and A.rowptr[-1] == A.nnz and deg.min() >= 8 and deg.max() <= 24
    assert A.col.dtype == np.int32 and A.col.min() >= 0 and A.col.max() < 3000
    rows = np.repeat(np.arange(5000), deg)
    assert np.all((np.diff(A.col) >= 0) | (np.diff(rows) > 0))  # sorted within each row
    z = A.val * np.sqrt(np.repeat(deg, deg))                     # N(0, 1/d_i) -> N(0, 1)
    assert abs(z.var() - 1.0) < 0.03 and abs(z.mean()) < 0.02
    assert x.shape == (3000,) and x.min() >= -1.0 and x.max() <= 1.0
    B, _ = W.spquadform_inputs(5000, 3000, d_lo=8, d_hi=24, seed=7)
    assert np.array_equal(A.col, B.col) and np.array_equal(A.val, B.val)


def test_csr_allows_empty_rows_and_densifies_with_repeats():
    A, _ = W.spquadform_inputs(200, 5, d_lo=0, d_hi=9, seed=3)
    deg = np.diff(A.rowptr)
    assert (deg == 0).any() and np.isfinite(A.val).all()
    D = A.dense()
    rows = np.repeat(np.arange(200), deg)
    for i in range(200):
        ref = np.zeros(5)
        np.add.at(ref, A.col[rows == i], A.val[rows == i])
        assert np.array_equal(D[i], ref)


def test_laplace1d_inputs():
    x, b = W.laplace1d_inputs(1001)
    assert x.shape == b.shape == (1001,)
    assert x.min() >= -1 and x.max() <= 1 and b.min() >= -1 and b.max() <= 1
    assert np.array_equal(W.laplace1d_inputs(1001)[1], b)


def test_batched_mixes():
    n = W.batched_dense_sizes()
    assert n.shape == (4096,) and n.min() >= 32 and n.max() <= 2048
    # log-uniform: the median of ln n sits at the middle of [ln 32, ln 2048]
    assert abs(np.median(np.log(n)) - 0.5 * (math.log(32) + math.log(2048))) < 0.1
    boxes = W.batched_tet_boxes()
    assert len(boxes) == 512
    T = np.array([6 * a * b * c for a, b, c in boxes])
    assert T.min() >= 6 and T.max() <= 2e5 and all(a == b for a, b, _ in boxes)
    mesh, u = W.batched_tet_instance(3, boxes[3])
    mesh2, u2 = W.batched_tet_instance(3, boxes[3])
    assert np.array_equal(mesh.conn, mesh2.conn) and np.array_equal(u, u2)
    assert mesh.ne == T[3]
