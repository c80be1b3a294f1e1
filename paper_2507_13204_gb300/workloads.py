"""Seeded synthetic inputs for the gradient workloads.

This module only draws and lays out input data.  It holds none of the method's
arithmetic (no energy, no adjoint); both the CUDA path and the CPU oracle take
their inputs from here.

Workloads (all synthetic, seeded with numpy ``Generator(PCG64(seed))``):

* dense quadratic form f(x) = ||A x||^2: A has i.i.d. N(0, 1/n) entries
  (variance 1/n), x is uniform on [-1, 1].  A is drawn first, then x.
* tet-mesh energy f(u) = sum_e log1p(|G_e u_e|^2) on an a x b x c box of unit
  cubes, each cube split into the 6 Kuhn tetrahedra, with a random vertex
  relabelling.  G_e (3 x 4) holds the gradients of the four P1 barycentric
  functions of element e (column k = grad lambda_k); it is input data computed
  from the vertex coordinates, exactly (adjugate / determinant) when the
  coordinates are integers.
* sparse quadratic form f(x) = ||A x||^2 with A in compressed sparse rows: row i
  holds d_i ~ U{d_lo, ..., d_hi} entries at uniformly random columns (sorted
  within the row; a column may repeat, the entries then add), values
  N(0, 1/d_i); x uniform on [-1, 1].  Degrees, then columns, then values, then
  x are drawn in that order.
* the paper's 1-D example (Section 4, Fig. "function_f"): x and b uniform on
  [-1, 1].
* batched mixes: sizes n_k = round(exp(U[ln 32, ln 2048])) (seed 3) and tet
  counts T_k = exp(U[ln 1e3, ln 1e5]) (seed 4), box a = b = floor((T/6)^(1/3)),
  c = max(1, round(T / (6 a^2))).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

# Kuhn split of a unit cube: for each permutation (p0, p1, p2) of the axes, in
# lexicographic order, the tet [c, c+e_p0, c+e_p0+e_p1, c+(1,1,1)].
KUHN_PERMS = ((0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0))


def _rng(seed) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


# --------------------------------------------------------------------------
# dense ||A x||^2
# --------------------------------------------------------------------------
def quadform_inputs(n: int, m: int | None = None, seed: int = 0):
    """A (m x n, row-major, i.i.d. N(0, 1/n)) then x (n, uniform[-1,1]); float64."""
    m = n if m is None else m
    rng = _rng(seed)
    A = rng.standard_normal((m, n)) * math.sqrt(1.0 / n)
    x = rng.uniform(-1.0, 1.0, n)
    return A, x


# --------------------------------------------------------------------------
# tet mesh
# --------------------------------------------------------------------------
@dataclass
class TetMesh:
    conn: np.ndarray    # int32 [Ne, 4], relabelled vertex ids
    G: np.ndarray       # float64 [Ne, 12], row-major 3x4 (G[e, r*4+k] = d lambda_k / d x_r)
    coords: np.ndarray  # float64 [Nv, 3], indexed by relabelled id
    perm: np.ndarray    # int64 [Nv]: relabelled id of grid vertex i + (a+1) j + (a+1)(b+1) k
    shape: tuple        # (a, b, c) cubes per axis

    @property
    def ne(self) -> int:
        return int(self.conn.shape[0])

    @property
    def nv(self) -> int:
        return int(self.coords.shape[0])


@dataclass
class CsrMatrix:
    rowptr: np.ndarray  # int32 [m + 1]
    col: np.ndarray     # int32 [nnz]
    val: np.ndarray     # float64 [nnz]
    m: int
    n: int

    @property
    def nnz(self) -> int:
        return int(self.col.shape[0])

    def dense(self) -> np.ndarray:
        """The m x n matrix (repeated columns add)."""
        A = np.zeros((self.m, self.n))
        rows = np.repeat(np.arange(self.m), np.diff(self.rowptr))
        np.add.at(A, (rows, self.col), self.val)
        return A


def spquadform_inputs(m: int = 1 << 20, n: int | None = None, d_lo: int = 8, d_hi: int = 24,
                      seed: int = 7):
    """Random CSR matrix (see the module docstring) and x; returns (CsrMatrix, x)."""
    n = m if n is None else n
    rng = _rng(seed)
    deg = rng.integers(d_lo, d_hi + 1, m)
    rowptr = np.zeros(m + 1, np.int64)
    np.cumsum(deg, out=rowptr[1:])
    nnz = int(rowptr[-1])
    if nnz >= 2 ** 31:
        raise ValueError("nnz must be < 2^31")
    col = rng.integers(0, n, nnz)
    rows = np.repeat(np.arange(m), deg)
    col = col[np.lexsort((col, rows))]  # sorted within each row
    val = rng.standard_normal(nnz) / np.sqrt(np.repeat(deg, deg))
    x = rng.uniform(-1.0, 1.0, n)
    return CsrMatrix(rowptr.astype(np.int32), col.astype(np.int32), val, m, n), x


def _grid_conn(a: int, b: int, c: int) -> np.ndarray:
    """Unrelabelled connectivity, cube-major (cube id i + a j + a b k), 6 tets per cube."""
    sx, sy, sz = 1, a + 1, (a + 1) * (b + 1)
    ci, cj, ck = np.meshgrid(np.arange(a), np.arange(b), np.arange(c), indexing="ij")
    # cube index i + a*j + a*b*k  ->  order by k, then j, then i
    base = (ci * sx + cj * sy + ck * sz).transpose(2, 1, 0).reshape(-1).astype(np.int64)
    step = (sx, sy, sz)
    tets = np.empty((base.size, 6, 4), dtype=np.int64)
    for t, (p0, p1, _p2) in enumerate(KUHN_PERMS):
        tets[:, t, 0] = base
        tets[:, t, 1] = base + step[p0]
        tets[:, t, 2] = base + step[p0] + step[p1]
        tets[:, t, 3] = base + sx + sy + sz
    return tets.reshape(-1, 4)


def _grid_coords(a: int, b: int, c: int) -> np.ndarray:
    k, j, i = np.meshgrid(np.arange(c + 1), np.arange(b + 1), np.arange(a + 1), indexing="ij")
    return np.stack([i.reshape(-1), j.reshape(-1), k.reshape(-1)], axis=1).astype(np.float64)


def p1_gradients(p: np.ndarray) -> np.ndarray:
    """Barycentric gradients of tets p [Ne, 4, 3] -> G [Ne, 12] (3x4 row-major).

    J = [p1-p0 | p2-p0 | p3-p0]; rows of J^-1 are grad lambda_1..3 and
    grad lambda_0 = -(sum of the others).  J^-1 = adj(J)/det(J), which is exact
    for integer coordinates with det = +-1.
    """
    e1 = p[:, 1] - p[:, 0]
    e2 = p[:, 2] - p[:, 0]
    e3 = p[:, 3] - p[:, 0]
    # J has columns e1, e2, e3; rows of J^-1 are (e2 x e3, e3 x e1, e1 x e2) / det
    r1 = np.cross(e2, e3)
    r2 = np.cross(e3, e1)
    r3 = np.cross(e1, e2)
    det = np.einsum("ij,ij->i", e1, r1)[:, None]
    g1, g2, g3 = r1 / det, r2 / det, r3 / det
    g0 = -(g1 + g2 + g3)
    grads = np.stack([g0, g1, g2, g3], axis=2)  # [Ne, 3 (r), 4 (k)]
    return np.ascontiguousarray(grads.reshape(-1, 12))


def tet_mesh(a: int, b: int | None = None, c: int | None = None, perm_seed=1,
             jitter_seed=None, jitter: float = 0.1, relabel: bool = True) -> TetMesh:
    """Kuhn-split a x b x c box (unit spacing), random relabelling drawn from perm_seed.

    jitter_seed moves every interior vertex by U[-jitter, jitter]^3 so that G_e
    differs per element.
    """
    b = a if b is None else b
    c = a if c is None else c
    conn0 = _grid_conn(a, b, c)
    xyz0 = _grid_coords(a, b, c)
    nv = xyz0.shape[0]
    if jitter_seed is not None:
        jr = _rng(jitter_seed).uniform(-jitter, jitter, (nv, 3))
        gi = xyz0.astype(np.int64)
        interior = ((gi[:, 0] > 0) & (gi[:, 0] < a) & (gi[:, 1] > 0) & (gi[:, 1] < b)
                    & (gi[:, 2] > 0) & (gi[:, 2] < c))
        xyz0 = xyz0 + jr * interior[:, None]
    G = p1_gradients(xyz0[conn0])
    if relabel:
        perm = _rng(perm_seed).permutation(nv)
    else:
        perm = np.arange(nv)
    conn = perm[conn0].astype(np.int32)
    coords = np.empty_like(xyz0)
    coords[perm] = xyz0
    return TetMesh(conn=np.ascontiguousarray(conn), G=G, coords=coords, perm=perm, shape=(a, b, c))


def tet_inputs(a: int = 100, seed: int = 1, jitter_seed=None):
    """The relabelled mesh (permutation drawn first from `seed`) and u ~ U[-1,1] drawn next."""
    b = c = a
    rng = _rng(seed)
    nv = (a + 1) * (b + 1) * (c + 1)
    perm = rng.permutation(nv)
    u = rng.uniform(-1.0, 1.0, nv)
    mesh = tet_mesh(a, b, c, perm_seed=seed, jitter_seed=jitter_seed)
    assert np.array_equal(mesh.perm, perm)
    return mesh, u


def linear_field(mesh: TetMesh, avec) -> np.ndarray:
    """u(p) = a . p at every vertex (P1 elements reproduce it exactly)."""
    return mesh.coords @ np.asarray(avec, dtype=np.float64)


# --------------------------------------------------------------------------
# paper example: 1-D Laplacian (Section 4)
# --------------------------------------------------------------------------
def laplace1d_inputs(n: int, seed: int = 5):
    rng = _rng(seed)
    x = rng.uniform(-1.0, 1.0, n)
    b = rng.uniform(-1.0, 1.0, n)
    return x, b


# --------------------------------------------------------------------------
# batched mixes
# --------------------------------------------------------------------------
def batched_dense_sizes(count: int = 4096, lo: int = 32, hi: int = 2048, seed: int = 3) -> np.ndarray:
    r = _rng(seed).uniform(math.log(lo), math.log(hi), count)
    return np.rint(np.exp(r)).astype(np.int64)


def batched_tet_boxes(count: int = 512, lo: float = 1e3, hi: float = 1e5, seed: int = 4):
    T = np.exp(_rng(seed).uniform(math.log(lo), math.log(hi), count))
    boxes = []
    for t in T:
        a = max(1, int(math.floor((t / 6.0) ** (1.0 / 3.0))))
        c = max(1, int(round(t / (6.0 * a * a))))
        boxes.append((a, a, c))
    return boxes


def batched_tet_instance(k: int, box, seed_base: int = 4000):
    """Instance k of the tet batch: mesh relabelled with seed (seed_base + k), u drawn after."""
    a, b, c = box
    mesh = tet_mesh(a, b, c, perm_seed=seed_base + k)
    rng = _rng(seed_base + k)
    rng.permutation(mesh.nv)  # same draw order as the mesh: permutation first
    u = rng.uniform(-1.0, 1.0, mesh.nv)
    return mesh, u


def batched_dense_instance(k: int, n: int, seed_base: int = 3000):
    """Instance k of the dense batch on the host: A (n x n, N(0,1/n)) then x."""
    return quadform_inputs(n, seed=seed_base + k)


def batched_dense_device(k: int, n: int, device, seed_base: int = 3000):
    """Instance k of the dense batch drawn on the device (16.5 GB of A for the
    4096-instance batch would take minutes on the host): torch's seeded CUDA
    generator (seed_base + k) draws A (n x n, N(0, 1/n)) and then x (U[-1, 1])."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(seed_base + k)
    A = torch.randn((n, n), generator=g, dtype=torch.float64, device=device) * math.sqrt(1.0 / n)
    x = torch.rand(n, generator=g, dtype=torch.float64, device=device) * 2.0 - 1.0
    return A, x
