"""GPU parity: dense ||A x||^2 value and gradient through the C ABI vs the CPU oracle."""
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


def _run(api, A, x, dtype, strategy, want_gA=False, seed=None, accumulate=False, **kw):
    dev = torch.device("cuda")
    At = torch.tensor(A, dtype=dtype, device=dev)
    xt = torch.tensor(x, dtype=dtype, device=dev)
    p = api.QuadForm(At, strategy=strategy, **kw)
    gx = torch.full((A.shape[1],), 0.5, dtype=dtype, device=dev)
    gA = torch.full(A.shape, 0.25, dtype=dtype, device=dev) if want_gA else None
    sd = None if seed is None else torch.tensor(seed, dtype=dtype, device=dev)
    f, gx = p.grad(xt, gx=gx, gdata=gA, seed=sd, accumulate=accumulate)
    fe = p.eval(xt)
    torch.cuda.synchronize()
    p.sync()
    out = (f.item(), gx.cpu().numpy(), fe.item(), None if gA is None else gA.cpu().numpy())
    p.close()
    return out


SHAPES = [(64, 64), (1, 1), (1, 37), (257, 1), (1000, 777), (300, 2048), (129, 5000), (40, 12288)]


@pytest.mark.parametrize("m,n", SHAPES)
@pytest.mark.parametrize("strategy", ["fused", "atomic", "transpose"])
def test_f64_matches_oracle(api, m, n, strategy):
    A, x = W.quadform_inputs(n, m=m, seed=m * 7 + n)
    f_ref, g_ref = O.quadform_grad(A, x)
    f, gx, fe, _ = _run(api, A, x, torch.float64, strategy)
    assert rel_scalar(f, f_ref) <= TOL["f64"]
    assert rel_scalar(fe, f_ref) <= TOL["f64"]
    assert rel_l2(gx, g_ref) <= TOL["f64"]


@pytest.mark.parametrize("m,n", [(64, 64), (1000, 777), (129, 5000), (10000, 10000)])
@pytest.mark.parametrize("strategy", ["fused", "transpose"])
def test_f32_matches_oracle_on_rounded_inputs(api, m, n, strategy):
    A, x = W.quadform_inputs(n, m=m, seed=3)
    A32, x32 = f32_round(A), f32_round(x)
    f_ref, g_ref = O.quadform_grad(A32, x32)
    f, gx, fe, _ = _run(api, A32, x32, torch.float32, strategy)
    assert rel_scalar(f, f_ref) <= TOL["f32"]
    assert rel_scalar(fe, f_ref) <= TOL["f32"]
    assert rel_l2(gx, g_ref) <= TOL["f32"]


def test_cfg1_gradient_wrt_A_seed_and_accumulate(api):
    # the 64 x 64 workload: gradient w.r.t. x and A, output adjoint 1.7, accumulate onto
    # the 0.5 / 0.25 prefill (the "_d_x +=" convention)
    A, x = W.quadform_inputs(64, seed=0)
    f_ref, g_ref, gA_ref = O.quadform_grad(A, x, fbar=1.7, want_gA=True)
    f, gx, _, gA = _run(api, A, x, torch.float64, "fused", want_gA=True, seed=1.7, accumulate=True)
    assert rel_scalar(f, f_ref) <= TOL["f64"]
    assert rel_l2(gx - 0.5, g_ref) <= TOL["f64"]
    assert rel_l2(gA - 0.25, gA_ref) <= TOL["f64"]


def test_full_size_n10000_f64(api):
    # the 10000 x 10000 FP64 workload (800 MB), every gradient entry checked
    A, x = W.quadform_inputs(10000, seed=0)
    f_ref, g_ref = O.quadform_grad(A, x)
    for strategy in ("fused", "transpose"):
        f, gx, fe, _ = _run(api, A, x, torch.float64, strategy)
        assert rel_scalar(f, f_ref) <= TOL["f64"], strategy
        assert rel_scalar(fe, f_ref) <= TOL["f64"], strategy
        assert rel_l2(gx, g_ref) <= TOL["f64"], strategy


def test_fused_is_bitwise_reproducible(api):
    A, x = W.quadform_inputs(3000, m=2000, seed=9)
    a = _run(api, A, x, torch.float64, "fused")
    b = _run(api, A, x, torch.float64, "fused")
    assert a[0] == b[0] and np.array_equal(a[1], b[1])


def test_identity_special_case_exact(api):
    x = np.random.default_rng(1).uniform(-1, 1, 500)
    f, gx, _, _ = _run(api, np.eye(500), x, torch.float64, "fused")
    assert np.array_equal(gx, 2 * x)


def test_n_beyond_row_team_is_unsupported_for_fused(api):
    from paper_2507_13204_gb300 import _lib as L
    A = torch.zeros((2, 20000), dtype=torch.float64, device="cuda")
    with pytest.raises(L.KGError) as ei:
        api.QuadForm(A, strategy="fused")
    assert ei.value.status == L.KG_ERR_UNSUPPORTED


@pytest.mark.parametrize("m,n", [(10000, 10000), (333, 1024), (5, 12288), (1000, 4098)])
def test_pair_and_native_arithmetic_both_match(api, m, n):
    A, x = W.quadform_inputs(n, m=m, seed=n + m)
    f_ref, g_ref = O.quadform_grad(A, x, fbar=0.75)
    dev = torch.device("cuda")
    At = torch.tensor(A, device=dev)
    xt = torch.tensor(x, device=dev)
    seed = torch.tensor(0.75, dtype=torch.float64, device=dev)
    for arith in ("pair", "native"):
        p = api.QuadForm(At, arith=arith)
        assert p.config[2] == arith
        f, g = p.grad(xt, seed=seed)
        fe = p.eval(xt)
        p.sync()
        assert rel_scalar(f.item(), f_ref) <= TOL["f64"], arith
        assert rel_scalar(fe.item(), O.quadform_value(A, x)) <= TOL["f64"], arith
        assert rel_l2(g.cpu().numpy(), g_ref) <= TOL["f64"], arith
        p.close()


@pytest.mark.parametrize("m,n", [(10000, 10000), (333, 1024), (5, 12288), (1000, 4098)])
def test_prepared_and_on_the_fly_split_agree(api, m, n):
    # within the workspace budget kg_create keeps A split into float pairs and the kernels
    # stream that copy; a budget below 8 m n bytes makes them split A on every call.  The
    # split is the same function either way, so the forward (one kernel for both) gives
    # bitwise identical results.  The gradient on the prepared copy runs the
    # warp-specialized kernel for 2048 < n <= 10240, whose summation order differs from
    # the on-the-fly kernel's: there the two agree to 1e-13 and each matches the oracle.
    A, x = W.quadform_inputs(n, m=m, seed=n + 2 * m)
    f_ref, g_ref = O.quadform_grad(A, x)
    At, xt = torch.tensor(A, device="cuda"), torch.tensor(x, device="cuda")
    prep = api.QuadForm(At)
    fly = api.QuadForm(At, tape_budget_bytes=8 * m * n - 8)
    assert prep.config[2] == fly.config[2] == "pair"
    assert prep.workspace_bytes - fly.workspace_bytes == 8 * m * n
    out = []
    for p in (prep, fly):
        f, g = p.grad(xt)
        fe = p.eval(xt)
        p.sync()
        assert rel_scalar(f.item(), f_ref) <= TOL["f64"]
        assert rel_scalar(fe.item(), f_ref) <= TOL["f64"]
        assert rel_l2(g.cpu().numpy(), g_ref) <= TOL["f64"]
        out.append((f.clone(), g.clone(), fe.clone()))
    (fp, gp, ep), (ff, gf, ef) = out
    assert torch.equal(ep, ef)
    if 2048 < n <= 10240:
        assert rel_scalar(fp.item(), ff.item()) <= 1e-13
        assert rel_l2(gp.cpu().numpy(), gf.cpu().numpy()) <= 1e-13
    else:
        assert torch.equal(fp, ff) and torch.equal(gp, gf)


def test_pair_is_default_for_f64_and_reproducible(api):
    A, x = W.quadform_inputs(2048, m=700, seed=4)
    p = api.QuadForm(torch.tensor(A, device="cuda"))
    assert p.config == ("fused", "recompute", "pair")
    xt = torch.tensor(x, device="cuda")
    g1 = p.grad(xt)[1].clone()
    g2 = p.grad(xt)[1].clone()
    torch.cuda.synchronize()
    assert torch.equal(g1, g2)


def test_pair_range_rules(api):
    from paper_2507_13204_gb300 import _lib as L
    A, x = W.quadform_inputs(1024, m=64, seed=2)
    A[3, 5] = 1e-70  # below the pair range: AUTO falls back to native FP64
    At = torch.tensor(A, device="cuda")
    p = api.QuadForm(At)
    assert p.config[2] == "native"
    f, g = p.grad(torch.tensor(x, device="cuda"))
    p.sync()
    assert rel_l2(g.cpu().numpy(), O.quadform_grad(A, x)[1]) <= TOL["f64"]
    with pytest.raises(L.KGError) as ei:
        api.QuadForm(At, arith="pair")
    assert ei.value.status == L.KG_ERR_UNSUPPORTED
    # an x out of range is reported by the pair kernel through kg_sync
    A[3, 5] = 0.0
    q = api.QuadForm(torch.tensor(A, device="cuda"), arith="pair")
    xb = x.copy()
    xb[7] = 1e300
    q.grad(torch.tensor(xb, device="cuda"))
    with pytest.raises(L.KGError) as ei:
        q.sync()
    assert ei.value.status == L.KG_ERR_RANGE
    q.grad(torch.tensor(x, device="cuda"))
    q.sync()


def test_pair_exact_cases(api):
    # zeros, identity and signed powers of two are exact in the pair representation
    n = 2048
    x = np.random.default_rng(3).uniform(-1, 1, n)
    p = api.QuadForm(torch.tensor(np.eye(n), device="cuda"), arith="pair")
    f, g = p.grad(torch.tensor(x, device="cuda"))
    assert rel_l2(g.cpu().numpy(), 2 * x) <= 2e-14  # x itself is held to 2^-46
    A = np.zeros((8, n))
    A[2, 100] = -4.0
    A[5, 2047] = 0.5
    q = api.QuadForm(torch.tensor(A, device="cuda"), arith="pair")
    f, g = q.grad(torch.tensor(x, device="cuda"))
    _, g_ref = O.quadform_grad(A, x)
    assert rel_l2(g.cpu().numpy(), g_ref) <= 2e-14


@pytest.mark.parametrize("m,n", [(1, 2050), (77, 4098), (200, 6146), (151, 8194), (500, 10240),
                                 (3000, 4098), (2600, 10000)])
def test_warp_specialized_fused_kernel_shapes(api, m, n):
    # 2048 < n <= 10240 on the prepared A runs the warp-specialized fused kernel: every
    # chunk width (8..20 column pairs per update thread), odd pair counts (the second
    # chunk of a row is shorter than the first), a single row, ragged bands, bands of more
    # than 5 and 32 rows (the chunk ring and the two-row partial buffer wrap around), more
    # CTAs than column-pair blocks of the in-kernel reduction and fewer; a seed, and the
    # same result on a second call
    A, x = W.quadform_inputs(n, m=m, seed=m + n)
    f_ref, g_ref = O.quadform_grad(A, x, fbar=0.5)
    p = api.QuadForm(torch.tensor(A, device="cuda"))
    assert p.config == ("fused", "recompute", "pair")
    xt = torch.tensor(x, device="cuda")
    seed = torch.tensor(0.5, dtype=torch.float64, device="cuda")
    f, g = p.grad(xt, seed=seed)
    f1, g1 = f.clone(), g.clone()
    f, g = p.grad(xt, seed=seed)
    p.sync()
    assert rel_scalar(f1.item(), f_ref) <= TOL["f64"]
    assert rel_l2(g1.cpu().numpy(), g_ref) <= TOL["f64"]
    assert torch.equal(f, f1) and torch.equal(g, g1)
    p.close()


@pytest.mark.parametrize("m,n", [(1, 2050), (151, 8194), (2600, 10000)])
def test_one_launch_and_two_launch_reductions_agree_bitwise(api, m, n, monkeypatch):
    # the partials' reduction in the fused kernel's tail (one cooperative launch) and the
    # separate reduce kernel (two launches; KG_TEST_NO_COOP=1 at create) add the same
    # partials in the same order: same bits, also when accumulating into gx
    from paper_2507_13204_gb300 import _lib as L
    A, x = W.quadform_inputs(n, m=m, seed=3 * m + n)
    f_ref, g_ref = O.quadform_grad(A, x, fbar=-1.5)
    At, xt = torch.tensor(A, device="cuda"), torch.tensor(x, device="cuda")
    seed = torch.tensor(-1.5, dtype=torch.float64, device="cuda")
    out = {}
    for coop in (1, 0):
        if coop:
            monkeypatch.delenv("KG_TEST_NO_COOP", raising=False)
        else:
            monkeypatch.setenv("KG_TEST_NO_COOP", "1")
        p = api.QuadForm(At)
        f, g = p.grad(xt, seed=seed)
        launches = L.kg_last_launch_count()
        g2 = torch.full_like(g, 0.25)
        p.grad(xt, gx=g2, seed=seed, accumulate=True)
        p.sync()
        out[coop] = (f.item(), g.cpu().numpy(), g2.cpu().numpy(), launches)
        p.close()
    (f1, g1, a1, l1), (f0, g0, a0, l0) = out[1], out[0]
    assert (l1, l0) == (1, 2)
    assert rel_scalar(f1, f_ref) <= TOL["f64"] and rel_l2(g1, g_ref) <= TOL["f64"]
    assert f1 == f0 and np.array_equal(g1, g0) and np.array_equal(a1, a0)
    assert np.array_equal(a1, 0.25 + g1)


@pytest.mark.parametrize("m,n", [(1, 1024), (777, 4100), (10000, 10000)])
def test_f32_one_launch_and_two_launch_reductions_agree_bitwise(api, m, n, monkeypatch):
    # FP32 streamed kernel: the reduction in the kernel's tail (one cooperative launch) and the
    # separate reduce kernel (KG_TEST_NO_COOP=1 at create) add the partials in the same order
    from paper_2507_13204_gb300 import _lib as L
    A, x = W.quadform_inputs(n, m=m, seed=5 * m + n)
    A, x = f32_round(A), f32_round(x)
    f_ref, g_ref = O.quadform_grad(A, x, fbar=0.5)
    At = torch.tensor(A, dtype=torch.float32, device="cuda")
    xt = torch.tensor(x, dtype=torch.float32, device="cuda")
    seed = torch.tensor(0.5, dtype=torch.float32, device="cuda")
    out = {}
    for coop in (1, 0):
        if coop:
            monkeypatch.delenv("KG_TEST_NO_COOP", raising=False)
        else:
            monkeypatch.setenv("KG_TEST_NO_COOP", "1")
        p = api.QuadForm(At)
        f, g = p.grad(xt, seed=seed)
        launches = L.kg_last_launch_count()
        g2 = torch.full_like(g, 0.25)
        p.grad(xt, gx=g2, seed=seed, accumulate=True)
        p.sync()
        out[coop] = (f.item(), g.cpu().numpy(), g2.cpu().numpy(), launches)
        p.close()
    (f1, g1, a1, l1), (f0, g0, a0, l0) = out[1], out[0]
    assert (l1, l0) == (1, 2)
    assert rel_scalar(f1, f_ref) <= TOL["f32"] and rel_l2(g1, g_ref) <= TOL["f32"]
    assert f1 == f0 and np.array_equal(g1, g0) and np.array_equal(a1, a0)
    assert np.array_equal(a1, np.float32(0.25) + g1)
