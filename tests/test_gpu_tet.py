"""GPU parity: tet-mesh energy value and gradient (atomic scatter, shared-memory
and warp aggregated scatters, the tiled reverse pass, CSR gather; recompute and
tape) through the C ABI vs the CPU oracle."""
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


def _problem(api, mesh, dtype, **kw):
    conn = torch.tensor(mesh.conn, device="cuda")
    G = torch.tensor(mesh.G, dtype=dtype, device="cuda")
    return api.TetEnergy(conn, G, mesh.nv, **kw)


MESHES = [(1, None), (3, 2), (7, None), (12, 2), (25, 2)]


@pytest.mark.parametrize("a,jit", MESHES)
@pytest.mark.parametrize("strategy", ["atomic", "shared", "warp", "tile", "csr"])
def test_f64_grad_matches_oracle(api, a, jit, strategy):
    mesh = W.tet_mesh(a, jitter_seed=jit, perm_seed=a)
    u = np.random.default_rng(a).uniform(-1, 1, mesh.nv)
    f_ref, g_ref = O.tet_grad(mesh.conn, mesh.G, u, fbar=1.0)
    p = _problem(api, mesh, torch.float64, strategy=strategy)
    ut = torch.tensor(u, device="cuda")
    f, g = p.grad(ut)
    fe = p.eval(ut)
    p.sync()
    assert rel_scalar(f.item(), f_ref) <= TOL["f64"]
    assert rel_scalar(fe.item(), f_ref) <= TOL["f64"]
    assert rel_l2(g.cpu().numpy(), g_ref) <= TOL["f64"]


@pytest.mark.parametrize("strategy", ["atomic", "shared", "warp", "tile", "csr"])
def test_f32_matches_oracle_on_rounded_inputs(api, strategy):
    mesh = W.tet_mesh(20, jitter_seed=2, perm_seed=3)
    u = np.random.default_rng(5).uniform(-1, 1, mesh.nv)
    G32, u32 = f32_round(mesh.G), f32_round(u)
    f_ref, g_ref = O.tet_grad(mesh.conn, G32, u32)
    conn = torch.tensor(mesh.conn, device="cuda")
    p = api.TetEnergy(conn, torch.tensor(G32, dtype=torch.float32, device="cuda"), mesh.nv,
                      strategy=strategy)
    ut = torch.tensor(u32, dtype=torch.float32, device="cuda")
    f, g = p.grad(ut)
    fe = p.eval(ut)
    p.sync()
    assert rel_scalar(f.item(), f_ref) <= TOL["f32"]
    assert rel_scalar(fe.item(), f_ref) <= TOL["f32"]
    assert rel_l2(g.cpu().numpy(), g_ref) <= TOL["f32"]


@pytest.mark.parametrize("box", [(1, 1, 1), (3, 5, 2), (9, 7, 5), (41, 3, 2)])
def test_f32_forward_ragged_counts(api, box):
    # element counts around and between the forward kernels' 256 / 512 element steps
    mesh = W.tet_mesh(*box, jitter_seed=2, perm_seed=sum(box))
    u = f32_round(np.random.default_rng(sum(box)).uniform(-1, 1, mesh.nv))
    G32 = f32_round(mesh.G)
    p = api.TetEnergy(torch.tensor(mesh.conn, device="cuda"),
                      torch.tensor(G32, dtype=torch.float32, device="cuda"), mesh.nv, mode="recompute")
    fe = p.eval(torch.tensor(u, dtype=torch.float32, device="cuda"))
    p.sync()
    assert rel_scalar(fe.item(), O.tet_value(mesh.conn, G32, u)) <= TOL["f32"]


@pytest.mark.parametrize("strategy", ["atomic", "shared", "warp", "tile", "csr"])
def test_tape_mode_seed_and_accumulate(api, strategy):
    mesh = W.tet_mesh(9, jitter_seed=2, perm_seed=4)
    u = np.random.default_rng(6).uniform(-1, 1, mesh.nv)
    f_ref, g_ref = O.tet_grad(mesh.conn, mesh.G, u, fbar=-0.6)
    p = _problem(api, mesh, torch.float64, strategy=strategy, mode="tape")
    ut = torch.tensor(u, device="cuda")
    f = p.eval_tape(ut)
    seed = torch.tensor(-0.6, dtype=torch.float64, device="cuda")
    g = torch.full((mesh.nv,), 2.0, dtype=torch.float64, device="cuda")
    p.grad_from_tape(gx=g, seed=seed, accumulate=True)
    p.sync()
    assert rel_scalar(f.item(), O.tet_value(mesh.conn, mesh.G, u)) <= TOL["f64"]
    assert rel_l2(g.cpu().numpy() - 2.0, g_ref) <= TOL["f64"]


def test_tape_before_record_is_a_state_error(api):
    from paper_2507_13204_gb300 import _lib as L
    mesh = W.tet_mesh(2)
    p = _problem(api, mesh, torch.float64, mode="tape")
    with pytest.raises(L.KGError) as ei:
        p.grad_from_tape()
    assert ei.value.status == L.KG_ERR_STATE


def test_csr_is_bitwise_reproducible_and_close_to_atomic(api):
    mesh = W.tet_mesh(15, jitter_seed=2, perm_seed=8)
    u = torch.tensor(np.random.default_rng(7).uniform(-1, 1, mesh.nv), device="cuda")
    pc = _problem(api, mesh, torch.float64, strategy="csr")
    pa = _problem(api, mesh, torch.float64, strategy="atomic")
    g1 = pc.grad(u)[1].clone()
    g2 = pc.grad(u)[1].clone()
    ga = pa.grad(u)[1]
    torch.cuda.synchronize()
    assert torch.equal(g1, g2)
    assert rel_l2(ga.cpu().numpy(), g1.cpu().numpy()) <= TOL["f64"]


@pytest.mark.parametrize("arith", ["native", "pair"])
def test_linear_field_interior_gradient_vanishes(api, arith):
    # P1 reproduces linear fields: g_e = a on every element, and the incident
    # gradients cancel at interior vertices (equal tet volumes).  The residual is
    # rounding: ~1e-15 for FP64 instructions, ~2^-46 of the O(1) terms for pairs.
    mesh = W.tet_mesh(6, perm_seed=2)
    a = np.array([0.2, -0.4, 0.1])
    p = _problem(api, mesh, torch.float64, arith=arith)
    f, g = p.grad(torch.tensor(W.linear_field(mesh, a), device="cuda"))
    g = g.cpu().numpy()
    gi = np.rint(mesh.coords).astype(int)
    interior = np.all((gi > 0) & (gi < 6), axis=1)
    assert rel_scalar(f.item(), mesh.ne * np.log1p(a @ a)) <= TOL["f64"]
    bound = 1e-13 if arith == "native" else TOL["f64"] * np.max(np.abs(g))
    assert np.max(np.abs(g[interior])) < bound


def test_full_size_100_cubed_f64(api):
    # the 6e6-tet, 1.03e6-vertex relabelled mesh; every gradient entry checked
    mesh, u = W.tet_inputs(100)
    f_ref, g_ref = O.tet_grad(mesh.conn, mesh.G, u)
    ut = torch.tensor(u, device="cuda")
    for strategy in ("atomic", "shared", "warp", "tile", "csr"):
        p = _problem(api, mesh, torch.float64, strategy=strategy)
        f, g = p.grad(ut)
        fe = p.eval(ut)
        p.sync()
        assert rel_scalar(f.item(), f_ref) <= TOL["f64"], strategy
        assert rel_scalar(fe.item(), f_ref) <= TOL["f64"], strategy
        assert rel_l2(g.cpu().numpy(), g_ref) <= TOL["f64"], strategy
        p.close()


def test_bad_connectivity_rejected_at_create(api):
    from paper_2507_13204_gb300 import _lib as L
    mesh = W.tet_mesh(2)
    conn = mesh.conn.copy()
    conn[5, 2] = mesh.nv + 3
    with pytest.raises(L.KGError) as ei:
        api.TetEnergy(torch.tensor(conn, device="cuda"),
                      torch.tensor(mesh.G, device="cuda"), mesh.nv)
    assert ei.value.status == L.KG_ERR_BOUNDS


def test_checked_kernels_flag_connectivity_changed_after_create(api):
    from paper_2507_13204_gb300 import _lib as L
    mesh = W.tet_mesh(3)
    conn = torch.tensor(mesh.conn, device="cuda")
    p = api.TetEnergy(conn, torch.tensor(mesh.G, device="cuda"), mesh.nv, check=True)
    conn[4, 1] = mesh.nv + 10  # the checked kernel skips the element and records the error
    p.grad(torch.zeros(mesh.nv, dtype=torch.float64, device="cuda"))
    with pytest.raises(L.KGError) as ei:
        p.sync()
    assert ei.value.status == L.KG_ERR_BOUNDS
    p.sync()  # the sticky word was cleared by the read


@pytest.mark.parametrize("arith", ["pair", "native"])
@pytest.mark.parametrize("strategy", ["atomic", "shared", "warp", "tile", "csr"])
def test_pair_and_native_match_oracle_jittered(api, arith, strategy):
    if strategy == "tile" and arith == "native":
        pytest.skip("the tiled reverse pass is float-pair only (test_tile_rules)")
    mesh = W.tet_mesh(18, jitter_seed=2, perm_seed=5)
    u = np.random.default_rng(21).uniform(-1, 1, mesh.nv)
    f_ref, g_ref = O.tet_grad(mesh.conn, mesh.G, u, fbar=1.3)
    p = _problem(api, mesh, torch.float64, strategy=strategy, arith=arith, mode="tape")
    assert p.config[2] == arith
    ut = torch.tensor(u, device="cuda")
    seed = torch.tensor(1.3, dtype=torch.float64, device="cuda")
    f, g = p.grad(ut, seed=seed)
    ft = p.eval_tape(ut)
    gt = p.grad_from_tape(seed=seed)
    p.sync()
    assert rel_scalar(f.item(), f_ref) <= TOL["f64"]
    assert rel_scalar(ft.item(), f_ref) <= TOL["f64"]
    assert rel_l2(g.cpu().numpy(), g_ref) <= TOL["f64"]
    assert rel_l2(gt.cpu().numpy(), g_ref) <= TOL["f64"]


def test_pair_default_and_range_rules(api):
    from paper_2507_13204_gb300 import _lib as L
    mesh = W.tet_mesh(5, jitter_seed=2)
    p = _problem(api, mesh, torch.float64)
    assert p.config == ("warp", "tape", "pair")
    u = np.random.default_rng(1).uniform(-1, 1, mesh.nv)
    u[3] = 1e200  # outside the pair range: reported, not silently wrong
    p.grad(torch.tensor(u, device="cuda"))
    with pytest.raises(L.KGError) as ei:
        p.sync()
    assert ei.value.status == L.KG_ERR_RANGE
    G = mesh.G.copy()
    G[0, 0] = 1e-80  # G outside the range: AUTO picks native FP64, PAIR is refused
    q = api.TetEnergy(torch.tensor(mesh.conn, device="cuda"), torch.tensor(G, device="cuda"), mesh.nv)
    assert q.config[2] == "native"
    with pytest.raises(L.KGError) as ei:
        api.TetEnergy(torch.tensor(mesh.conn, device="cuda"), torch.tensor(G, device="cuda"),
                      mesh.nv, arith="pair")
    assert ei.value.status == L.KG_ERR_UNSUPPORTED


def test_ragged_tiles_and_tiny_meshes(api):
    # element counts that are not multiples of the 256-element tile
    for a, b, c in [(1, 1, 1), (1, 1, 7), (3, 5, 2), (11, 1, 3)]:
        mesh = W.tet_mesh(a, b, c, jitter_seed=None, perm_seed=a + b + c)
        u = np.random.default_rng(a * b * c).uniform(-1, 1, mesh.nv)
        f_ref, g_ref = O.tet_grad(mesh.conn, mesh.G, u)
        for arith in ("pair", "native"):
            for strategy in ("atomic", "shared", "warp") + (("tile",) if arith == "pair" else ()):
                p = _problem(api, mesh, torch.float64, arith=arith, strategy=strategy)
                f, g = p.grad(torch.tensor(u, device="cuda"))
                p.sync()
                assert rel_scalar(f.item(), f_ref) <= TOL["f64"]
                assert rel_l2(g.cpu().numpy(), g_ref) <= TOL["f64"]


@pytest.mark.parametrize("strategy", ["shared", "warp", "tile"])
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_aggregation_with_scattered_element_order(api, dtype, strategy):
    # elements in random order: a 256-tet tile then touches ~1000 distinct vertices, close to
    # the worst case for the shared-memory table (long probe chains, nearly no combining),
    # and lanes of a warp rarely share a vertex
    mesh = W.tet_mesh(14, jitter_seed=2, perm_seed=8)
    order = np.random.default_rng(12).permutation(mesh.ne)
    conn, G = np.ascontiguousarray(mesh.conn[order]), np.ascontiguousarray(mesh.G[order])
    u = np.random.default_rng(13).uniform(-1, 1, mesh.nv)
    if dtype == torch.float32:
        G, u = f32_round(G), f32_round(u)
    f_ref, g_ref = O.tet_grad(conn, G, u)
    p = api.TetEnergy(torch.tensor(conn, device="cuda"), torch.tensor(G, dtype=dtype, device="cuda"),
                      mesh.nv, strategy=strategy)
    assert p.config[0] == strategy
    f, g = p.grad(torch.tensor(u, dtype=dtype, device="cuda"))
    p.sync()
    tol = TOL["f64"] if dtype == torch.float64 else TOL["f32"]
    assert rel_scalar(f.item(), f_ref) <= tol
    assert rel_l2(g.cpu().numpy(), g_ref) <= tol


def test_strategy_defaults(api):
    mesh = W.tet_mesh(3)
    conn = torch.tensor(mesh.conn, device="cuda")
    p64 = api.TetEnergy(conn, torch.tensor(mesh.G, device="cuda"), mesh.nv)
    p32 = api.TetEnergy(conn, torch.tensor(mesh.G, dtype=torch.float32, device="cuda"), mesh.nv)
    assert p64.config[0] == "warp" and p32.config[0] == "tile"
    p32c = api.TetEnergy(conn, torch.tensor(mesh.G, dtype=torch.float32, device="cuda"), mesh.nv,
                         check=True)
    assert p32c.config[0] == "warp"  # bounds-checked kernels: the staged kernel's warp combine


def test_tile_rules(api):
    # the tiled reverse pass runs for FP32 data and for FP64 data in float pairs with the
    # prepared G, without bounds checks
    from paper_2507_13204_gb300 import _lib as L
    mesh = W.tet_mesh(3)
    conn = torch.tensor(mesh.conn, device="cuda")
    G64 = torch.tensor(mesh.G, device="cuda")
    for kw in ({"arith": "native"}, {"check": True}, {"tape_budget_bytes": 96 * mesh.ne - 8}):
        with pytest.raises(L.KGError) as ei:
            api.TetEnergy(conn, G64, mesh.nv, strategy="tile", **kw)
        assert ei.value.status == L.KG_ERR_UNSUPPORTED, kw
    with pytest.raises(L.KGError) as ei:
        api.TetEnergy(conn, G64.float(), mesh.nv, strategy="tile", check=True)
    assert ei.value.status == L.KG_ERR_UNSUPPORTED
    assert api.TetEnergy(conn, G64.float(), mesh.nv, strategy="tile").config[0] == "tile"


@pytest.mark.parametrize("ne", [1, 31, 32, 33, 64, 65, 1537])
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_tile_boundaries_and_a_vertex_shared_by_a_whole_tile(api, ne, dtype):
    # a fan around vertex 0 (every tet has it: a tile's vertex 0 sums all 32 of its
    # elements) with element counts around the 32-element tile and the FP32 kernel's
    # two-tile step; the other vertices are shared by consecutive tets (a strip), in random
    # global numbering; seed and accumulate
    rng = np.random.default_rng(ne)
    nv = ne + 3
    conn = np.zeros((ne, 4), dtype=np.int32)
    for e in range(ne):
        conn[e] = (0, e + 1, e + 2, e + 3)
    perm = rng.permutation(nv).astype(np.int32)
    conn = perm[conn]
    G = rng.uniform(-1, 1, (ne, 12))
    u = rng.uniform(-1, 1, nv)
    if dtype == torch.float32:
        G, u = f32_round(G), f32_round(u)
    f_ref, g_ref = O.tet_grad(conn, G, u, fbar=0.75)
    p = api.TetEnergy(torch.tensor(conn, device="cuda"), torch.tensor(G, dtype=dtype, device="cuda"),
                      nv, strategy="tile")
    seed = torch.tensor(0.75, dtype=dtype, device="cuda")
    g = torch.full((nv,), 1.5, dtype=dtype, device="cuda")
    f, _ = p.grad(torch.tensor(u, dtype=dtype, device="cuda"), gx=g, seed=seed, accumulate=True)
    p.sync()
    tol = TOL["f64"] if dtype == torch.float64 else TOL["f32"]
    assert rel_scalar(f.item(), f_ref) <= tol
    assert rel_l2(g.cpu().numpy().astype(np.float64) - 1.5, g_ref) <= tol


def test_prepared_G_and_on_the_fly_split_agree(api):
    # FP64 pair arithmetic keeps G split into float pairs when 96 N_e bytes fit the workspace
    # budget; below it the kernels split G on every call.  With the CSR strategy the prepared
    # G runs the tile kernel (partials in float pairs), the on-the-fly split goes through the
    # tape (FP64 adjoints summed as pairs): the same sums in another rounding, each bitwise
    # reproducible run to run.
    mesh = W.tet_mesh(10, jitter_seed=3, perm_seed=6)
    u = np.random.default_rng(8).uniform(-1, 1, mesh.nv)
    f_ref, g_ref = O.tet_grad(mesh.conn, mesh.G, u)
    prep = _problem(api, mesh, torch.float64, strategy="csr")
    fly = _problem(api, mesh, torch.float64, strategy="csr", tape_budget_bytes=96 * mesh.ne - 8)
    assert prep.config[2] == fly.config[2] == "pair"
    assert prep.workspace_bytes - fly.workspace_bytes == 96 * mesh.ne
    ut = torch.tensor(u, device="cuda")
    out = []
    for p in (prep, fly):
        f, g = p.grad(ut)
        fe = p.eval(ut)
        p.sync()
        assert rel_scalar(f.item(), f_ref) <= TOL["f64"]
        assert rel_l2(g.cpu().numpy(), g_ref) <= TOL["f64"]
        f2, g2 = p.grad(ut)
        p.sync()
        assert torch.equal(f, f2) and torch.equal(g, g2)
        out.append((f.clone(), g.clone(), fe.clone()))
    (fp, gp, ep), (ff, gf, ef) = out
    assert torch.equal(ep, ef)  # the forward is one kernel for both
    assert rel_scalar(fp.item(), ff.item()) <= 1e-13
    assert rel_l2(gp.cpu().numpy(), gf.cpu().numpy()) <= 1e-13


def test_warp_combine_on_a_mesh_where_every_tet_shares_one_vertex(api):
    # a fan of tets around vertex 0: all 32 lanes of every warp hold vertex 0 in slot 0, the
    # largest possible group (31 shuffle rounds), and the other slots are all distinct
    rng = np.random.default_rng(21)
    ne = 1000
    conn = np.zeros((ne, 4), dtype=np.int32)
    conn[:, 1:] = 1 + np.arange(3 * ne, dtype=np.int32).reshape(ne, 3)
    G = rng.uniform(-1, 1, (ne, 12))
    u = rng.uniform(-1, 1, 3 * ne + 1)
    f_ref, g_ref = O.tet_grad(conn, G, u)
    for dtype in (torch.float64, torch.float32):
        Gd, ud = (G, u) if dtype == torch.float64 else (f32_round(G), f32_round(u))
        if dtype == torch.float32:
            f_ref, g_ref = O.tet_grad(conn, Gd, ud)
        p = api.TetEnergy(torch.tensor(conn, device="cuda"), torch.tensor(Gd, dtype=dtype, device="cuda"),
                          3 * ne + 1, strategy="warp")
        f, g = p.grad(torch.tensor(ud, dtype=dtype, device="cuda"))
        p.sync()
        tol = TOL["f64"] if dtype == torch.float64 else TOL["f32"]
        assert rel_scalar(f.item(), f_ref) <= tol
        assert rel_l2(g.cpu().numpy(), g_ref) <= tol


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_warp_combine_odd_counts_and_repeated_elements(api, dtype):
    # odd element counts around the 32-lane warp (a last warp with only some lanes active)
    # and a mesh where every element appears twice in a row (neighbouring lanes hold the
    # same four vertices: every slot a group or run of two), for the gradient and H v
    mesh = W.tet_mesh(6, 5, 4, jitter_seed=2, perm_seed=5)
    rng = np.random.default_rng(31)
    rnd = (lambda a: a) if dtype == torch.float64 else f32_round
    tol = TOL["f64"] if dtype == torch.float64 else TOL["f32"]
    u, v = rnd(rng.uniform(-1, 1, mesh.nv)), rnd(rng.uniform(-1, 1, mesh.nv))
    cases = [np.arange(ne) for ne in (1, 3, 63, 65, 129, 701)] + [np.repeat(np.arange(333), 2)]
    for rows in cases:
        conn, G = np.ascontiguousarray(mesh.conn[rows]), rnd(np.ascontiguousarray(mesh.G[rows]))
        f_ref, g_ref = O.tet_grad(conn, G, u)
        h_ref = O.tet_hvp(conn, G, u, v)
        p = api.TetEnergy(torch.tensor(conn, device="cuda"), torch.tensor(G, dtype=dtype, device="cuda"),
                          mesh.nv, strategy="warp")
        ut = torch.tensor(u, dtype=dtype, device="cuda")
        f, g = p.grad(ut)
        hv = p.hvp(ut, torch.tensor(v, dtype=dtype, device="cuda"))
        p.sync()
        assert rel_scalar(f.item(), f_ref) <= tol, len(rows)
        assert rel_l2(g.cpu().numpy(), g_ref) <= tol, len(rows)
        assert rel_l2(hv.cpu().numpy(), h_ref) <= tol, len(rows)
