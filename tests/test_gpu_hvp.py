"""GPU parity: Hessian-vector products (kg_hvp, forward mode over the reverse pass)
vs the CPU oracle, for every kind."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2507_13204_gb300 import workloads as W
from tests.helpers import TOL, f32_round, rel_l2, rel_scalar

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api(cuda_ok):
    from paper_2507_13204_gb300 import build
    build.build()
    from paper_2507_13204_gb300 import api as A
    return A


def _tet(api, mesh, dtype=torch.float64, **kw):
    return api.TetEnergy(torch.tensor(mesh.conn, device="cuda"),
                         torch.tensor(mesh.G, dtype=dtype, device="cuda"), mesh.nv, **kw)


@pytest.mark.parametrize("arith", ["pair", "native"])
@pytest.mark.parametrize("strategy", ["warp", "atomic", "shared", "tile", "csr"])
def test_tet_hvp_f64(api, arith, strategy):
    if strategy == "tile" and arith == "native":
        pytest.skip("the tiled reverse pass is float-pair only")
    mesh = W.tet_mesh(9, 7, 5, jitter_seed=2, perm_seed=3)  # ragged tail of the 256-tet tiles
    rng = np.random.default_rng(41)
    u, v = rng.uniform(-1, 1, mesh.nv), rng.uniform(-1, 1, mesh.nv)
    ref = O.tet_hvp(mesh.conn, mesh.G, u, v, fbar=-0.8)
    p = _tet(api, mesh, arith=arith, strategy=strategy)
    assert p.config[2] == arith
    seed = torch.tensor(-0.8, dtype=torch.float64, device="cuda")
    hv = p.hvp(torch.tensor(u, device="cuda"), torch.tensor(v, device="cuda"), seed=seed)
    p.sync()
    assert rel_l2(hv.cpu().numpy(), ref) <= TOL["f64"]


def test_tet_hvp_f32_and_accumulate(api):
    mesh = W.tet_mesh(12, jitter_seed=5, perm_seed=4)
    rng = np.random.default_rng(42)
    G32 = f32_round(mesh.G)
    u, v = f32_round(rng.uniform(-1, 1, mesh.nv)), f32_round(rng.uniform(-1, 1, mesh.nv))
    ref = O.tet_hvp(mesh.conn, G32, u, v)
    p = api.TetEnergy(torch.tensor(mesh.conn, device="cuda"),
                      torch.tensor(G32, dtype=torch.float32, device="cuda"), mesh.nv)
    hv = torch.full((mesh.nv,), 2.0, dtype=torch.float32, device="cuda")
    p.hvp(torch.tensor(u, dtype=torch.float32, device="cuda"),
          torch.tensor(v, dtype=torch.float32, device="cuda"), hv=hv, accumulate=True)
    p.sync()
    assert rel_l2(hv.cpu().numpy().astype(np.float64) - 2.0, ref) <= TOL["f32"]


@pytest.mark.parametrize("strategy", ["tile", "csr"])
def test_tet_hvp_and_grad_f32_half_scattered_element_order(api, strategy):
    # the first half of the elements in mesh order (tiles of about 25 distinct vertices: u
    # gathered once per tile vertex), the second half in random order (tiles of more than 32
    # distinct vertices: gathered through conn); both in one call
    mesh = W.tet_mesh(10, jitter_seed=5, perm_seed=6)
    h = mesh.ne // 2
    order = np.concatenate([np.arange(h), h + np.random.default_rng(7).permutation(mesh.ne - h)])
    conn = np.ascontiguousarray(mesh.conn[order])
    G32 = f32_round(np.ascontiguousarray(mesh.G[order]))
    rng = np.random.default_rng(43)
    u, v = f32_round(rng.uniform(-1, 1, mesh.nv)), f32_round(rng.uniform(-1, 1, mesh.nv))
    p = api.TetEnergy(torch.tensor(conn, device="cuda"), torch.tensor(G32, dtype=torch.float32, device="cuda"),
                      mesh.nv, strategy=strategy)
    assert p.config[0] == strategy
    ut, vt = torch.tensor(u, dtype=torch.float32, device="cuda"), torch.tensor(v, dtype=torch.float32, device="cuda")
    hv = p.hvp(ut, vt)
    f, g = p.grad(ut)
    p.sync()
    f_ref, g_ref = O.tet_grad(conn, G32, u)
    assert rel_l2(hv.cpu().numpy(), O.tet_hvp(conn, G32, u, v)) <= TOL["f32"]
    assert rel_scalar(f.item(), f_ref) <= TOL["f32"]
    assert rel_l2(g.cpu().numpy(), g_ref) <= TOL["f32"]


def test_tet_hvp_full_mesh_f64(api):
    mesh, u = W.tet_inputs(100)
    v = np.random.default_rng(43).uniform(-1, 1, mesh.nv)
    ref = O.tet_hvp(mesh.conn, mesh.G, u, v)
    p = _tet(api, mesh)
    hv = p.hvp(torch.tensor(u, device="cuda"), torch.tensor(v, device="cuda"))
    p.sync()
    assert rel_l2(hv.cpu().numpy(), ref) <= TOL["f64"]


def test_tet_hvp_range_is_checked_in_pair_mode(api):
    from paper_2507_13204_gb300 import _lib as L
    mesh = W.tet_mesh(3, jitter_seed=2)
    p = _tet(api, mesh)
    assert p.config[2] == "pair"
    u = np.random.default_rng(44).uniform(-1, 1, mesh.nv)
    v = u.copy()
    v[5] = 1e300
    p.hvp(torch.tensor(u, device="cuda"), torch.tensor(v, device="cuda"))
    with pytest.raises(L.KGError) as ei:
        p.sync()
    assert ei.value.status == L.KG_ERR_RANGE


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_quadratic_kinds(api, dtype):
    # dense and sparse ||Ax||^2: H v = 2 fbar A^T A v, the gradient at v; 1-D: 18 fbar A^T A v
    tol = TOL["f64"] if dtype == torch.float64 else TOL["f32"]
    rnd = (lambda a: a) if dtype == torch.float64 else f32_round
    A, _ = W.quadform_inputs(3000, m=700, seed=6)
    A = rnd(A)
    v = rnd(np.random.default_rng(45).uniform(-1, 1, 3000))
    p = api.QuadForm(torch.tensor(A, dtype=dtype, device="cuda"))
    hv = p.hvp(None, torch.tensor(v, dtype=dtype, device="cuda"))
    p.sync()
    assert rel_l2(hv.cpu().numpy(), O.quadform_grad(A, v)[1]) <= tol
    S, _ = W.spquadform_inputs(4000, 3500, seed=12)
    S.val = rnd(S.val)
    vs = rnd(np.random.default_rng(46).uniform(-1, 1, 3500))
    for strategy in ("atomic", "transpose"):
        q = api.SpQuadForm(torch.tensor(S.rowptr, device="cuda"), torch.tensor(S.col, device="cuda"),
                           torch.tensor(S.val, dtype=dtype, device="cuda"), S.n, strategy=strategy)
        hv = q.hvp(None, torch.tensor(vs, dtype=dtype, device="cuda"),
                   seed=torch.tensor(0.5, dtype=dtype, device="cuda"))
        q.sync()
        assert rel_l2(hv.cpu().numpy(), O.spquadform_grad(S.rowptr, S.col, S.val, vs, fbar=0.5)[1]) <= tol
    for n in (1, 2, 1001):
        _, b = W.laplace1d_inputs(n)
        vl = rnd(np.random.default_rng(n).uniform(-1, 1, n))
        r = api.Laplace1D(torch.tensor(rnd(b), dtype=dtype, device="cuda"))
        hv = r.hvp(None, torch.tensor(vl, dtype=dtype, device="cuda"))
        r.sync()
        assert rel_l2(hv.cpu().numpy(), O.laplace1d_hvp(vl)) <= tol
