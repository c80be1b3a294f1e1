"""GPU parity: sparse (CSR) ||A x||^2 value and gradients (w.r.t. x and the stored
values), atomic scatter and the atomic-free transpose gather, through the C ABI
vs the CPU oracle."""
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


def _problem(api, A, dtype=torch.float64, **kw):
    dev = "cuda"
    return api.SpQuadForm(torch.tensor(A.rowptr, device=dev), torch.tensor(A.col, device=dev),
                          torch.tensor(A.val, dtype=dtype, device=dev), A.n, **kw)


# (m, n, degree range): ragged rows, empty rows, repeated columns, wide and tall shapes
SHAPES = [(1, 1, (1, 1)), (7, 5, (0, 4)), (300, 200, (0, 9)), (5000, 3000, (8, 24)),
          (1000, 70000, (20, 60)), (40000, 100, (1, 3))]


@pytest.mark.parametrize("m,n,deg", SHAPES)
@pytest.mark.parametrize("strategy", ["atomic", "transpose"])
@pytest.mark.parametrize("arith", ["pair", "native"])
def test_f64_matches_oracle(api, m, n, deg, strategy, arith):
    A, x = W.spquadform_inputs(m, n, d_lo=deg[0], d_hi=deg[1], seed=m + n)
    f_ref, g_ref, gv_ref = O.spquadform_grad(A.rowptr, A.col, A.val, x, fbar=0.5, want_gval=True)
    p = _problem(api, A, strategy=strategy, arith=arith)
    assert p.config[0] == strategy and p.config[2] == arith
    xt = torch.tensor(x, device="cuda")
    gval = torch.empty(A.nnz, dtype=torch.float64, device="cuda")
    f, g = p.grad(xt, gdata=gval, seed=torch.tensor(0.5, dtype=torch.float64, device="cuda"))
    fe = p.eval(xt)
    p.sync()
    assert rel_scalar(f.item(), f_ref) <= TOL["f64"]
    assert rel_scalar(fe.item(), O.spquadform_value(A.rowptr, A.col, A.val, x)) <= TOL["f64"]
    assert rel_l2(g.cpu().numpy(), g_ref) <= TOL["f64"]
    assert rel_l2(gval.cpu().numpy(), gv_ref) <= TOL["f64"]


@pytest.mark.parametrize("strategy", ["atomic", "transpose"])
def test_f32_matches_oracle_on_rounded_inputs(api, strategy):
    A, x = W.spquadform_inputs(20000, 15000, seed=3)
    A.val = f32_round(A.val)
    x = f32_round(x)
    f_ref, g_ref = O.spquadform_grad(A.rowptr, A.col, A.val, x)
    p = _problem(api, A, torch.float32, strategy=strategy)
    f, g = p.grad(torch.tensor(x, dtype=torch.float32, device="cuda"))
    p.sync()
    assert rel_scalar(f.item(), f_ref) <= TOL["f32"]
    assert rel_l2(g.cpu().numpy(), g_ref) <= TOL["f32"]


@pytest.mark.parametrize("strategy", ["atomic", "transpose"])
def test_accumulate_adds_to_both_gradients(api, strategy):
    A, x = W.spquadform_inputs(900, 700, seed=8)
    _, g_ref, gv_ref = O.spquadform_grad(A.rowptr, A.col, A.val, x, want_gval=True)
    p = _problem(api, A, strategy=strategy)
    g = torch.full((A.n,), 1.5, dtype=torch.float64, device="cuda")
    gv = torch.full((A.nnz,), -2.0, dtype=torch.float64, device="cuda")
    p.grad(torch.tensor(x, device="cuda"), gx=g, gdata=gv, accumulate=True)
    p.sync()
    assert rel_l2(g.cpu().numpy() - 1.5, g_ref) <= TOL["f64"]
    assert rel_l2(gv.cpu().numpy() + 2.0, gv_ref) <= TOL["f64"]


def test_transpose_is_bitwise_reproducible_and_close_to_atomic(api):
    A, x = W.spquadform_inputs(30000, 30000, seed=9)
    xt = torch.tensor(x, device="cuda")
    pt = _problem(api, A, strategy="transpose")
    pa = _problem(api, A, strategy="atomic")
    g1 = pt.grad(xt)[1].clone()
    g2 = pt.grad(xt)[1].clone()
    ga = pa.grad(xt)[1]
    torch.cuda.synchronize()
    assert torch.equal(g1, g2)
    assert rel_l2(ga.cpu().numpy(), g1.cpu().numpy()) <= TOL["f64"]


def test_edge_cases(api):
    from paper_2507_13204_gb300 import _lib as L
    dev = "cuda"
    # no stored entries: f = 0, gradient 0
    for strategy in ("atomic", "transpose"):
        p = api.SpQuadForm(torch.zeros(6, dtype=torch.int32, device=dev),
                           torch.zeros(0, dtype=torch.int32, device=dev),
                           torch.zeros(0, dtype=torch.float64, device=dev), 4, strategy=strategy)
        f, g = p.grad(torch.ones(4, dtype=torch.float64, device=dev))
        p.sync()
        assert f.item() == 0.0 and torch.equal(g, torch.zeros(4, dtype=torch.float64, device=dev))
    # one dense row much longer than a team, and one column shared by every row
    rowptr = np.array([0, 3000], np.int32)
    col = np.arange(3000, dtype=np.int32)
    val = np.random.default_rng(1).standard_normal(3000)
    x = np.random.default_rng(2).uniform(-1, 1, 3000)
    A1 = W.CsrMatrix(rowptr, col, val, 1, 3000)
    rowptr2 = np.arange(0, 5001, dtype=np.int32)
    A2 = W.CsrMatrix(rowptr2, np.zeros(5000, np.int32), np.random.default_rng(3).standard_normal(5000),
                     5000, 1)
    for A, xv in ((A1, x), (A2, np.array([0.7]))):
        f_ref, g_ref = O.spquadform_grad(A.rowptr, A.col, A.val, xv)
        for strategy in ("atomic", "transpose"):
            p = _problem(api, A, strategy=strategy)
            f, g = p.grad(torch.tensor(xv, device=dev))
            p.sync()
            assert rel_scalar(f.item(), f_ref) <= TOL["f64"]
            assert rel_l2(g.cpu().numpy(), g_ref) <= TOL["f64"]
    # invalid structures are rejected at create
    bad = [(np.array([0, 2, 1, 3], np.int32), np.array([0, 1, 2], np.int32)),  # decreasing rowptr
           (np.array([0, 1, 3], np.int32), np.array([0, 1, 9], np.int32)),     # column >= n
           (np.array([1, 2, 3], np.int32), np.array([0, 1, 2], np.int32))]     # rowptr[0] != 0
    for rp, cl in bad:
        for strategy in ("atomic", "transpose"):
            with pytest.raises(L.KGError) as ei:
                api.SpQuadForm(torch.tensor(rp, device=dev), torch.tensor(cl, device=dev),
                               torch.ones(cl.shape[0], dtype=torch.float64, device=dev), 4,
                               strategy=strategy)
            assert ei.value.status == L.KG_ERR_BOUNDS
    q = api.SpQuadForm(torch.tensor([0, 1], dtype=torch.int32, device=dev),
                       torch.tensor([0], dtype=torch.int32, device=dev),
                       torch.ones(1, dtype=torch.float64, device=dev), 2)
    assert q.config == ("atomic", "recompute", "pair")
    with pytest.raises(L.KGError) as ei:
        api.SpQuadForm(torch.tensor([0, 1], dtype=torch.int32, device=dev),
                       torch.tensor([0], dtype=torch.int32, device=dev),
                       torch.ones(1, dtype=torch.float64, device=dev), 2, strategy="csr")
    assert ei.value.status == L.KG_ERR_UNSUPPORTED


def test_pair_range_rules(api):
    from paper_2507_13204_gb300 import _lib as L
    A, x = W.spquadform_inputs(2000, 1500, seed=21)
    A.val[17] = 1e-70  # below the pair range: AUTO falls back to native FP64
    p = _problem(api, A)
    assert p.config[2] == "native"
    f, g = p.grad(torch.tensor(x, device="cuda"))
    p.sync()
    assert rel_l2(g.cpu().numpy(), O.spquadform_grad(A.rowptr, A.col, A.val, x)[1]) <= TOL["f64"]
    with pytest.raises(L.KGError) as ei:
        _problem(api, A, arith="pair")
    assert ei.value.status == L.KG_ERR_UNSUPPORTED
    # an x out of range is reported through kg_sync; the next good call is clean
    A.val[17] = 0.5
    q = _problem(api, A, arith="pair")
    xb = x.copy()
    xb[A.col[5]] = 1e300
    q.grad(torch.tensor(xb, device="cuda"))
    with pytest.raises(L.KGError) as ei:
        q.sync()
    assert ei.value.status == L.KG_ERR_RANGE
    q.grad(torch.tensor(x, device="cuda"))
    q.sync()
    # the prepared copy is 8 bytes per stored value; with a smaller budget AUTO stays native
    small = _problem(api, A, tape_budget_bytes=8 * A.nnz - 8)
    assert small.config[2] == "native"


@pytest.mark.parametrize("team", [2, 4, 16, 32])
def test_team_widths(api, team):
    A, x = W.spquadform_inputs(3000, 2500, d_lo=0, d_hi=70, seed=team)
    f_ref, g_ref = O.spquadform_grad(A.rowptr, A.col, A.val, x)
    for strategy in ("atomic", "transpose"):
        p = _problem(api, A, strategy=strategy, team=team)
        f, g = p.grad(torch.tensor(x, device="cuda"))
        p.sync()
        assert rel_scalar(f.item(), f_ref) <= TOL["f64"]
        assert rel_l2(g.cpu().numpy(), g_ref) <= TOL["f64"]


def test_full_size_workload_f64(api):
    A, x = W.spquadform_inputs()  # 2^20 x 2^20, 8..24 entries per row (16.8e6 stored)
    f_ref, g_ref = O.spquadform_grad(A.rowptr, A.col, A.val, x)
    xt = torch.tensor(x, device="cuda")
    for strategy in ("atomic", "transpose"):
        p = _problem(api, A, strategy=strategy)
        f, g = p.grad(xt)
        p.sync()
        assert rel_scalar(f.item(), f_ref) <= TOL["f64"], strategy
        assert rel_l2(g.cpu().numpy(), g_ref) <= TOL["f64"], strategy
        p.close()
