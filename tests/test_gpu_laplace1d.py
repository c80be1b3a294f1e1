"""GPU parity: the paper's 1-D Laplacian example (Sec. 4), the literal
six-kernel atomic gradient and the fused single-kernel gradient, vs the oracle."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2507_13204_gb300 import workloads as W
from tests.helpers import TOL, rel_l2, rel_scalar

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api(cuda_ok):
    from paper_2507_13204_gb300 import build
    build.build()
    from paper_2507_13204_gb300 import api as A
    return A


@pytest.mark.parametrize("n", [1, 2, 3, 100, 1001, 10000, 100003])
@pytest.mark.parametrize("strategy", ["fused", "atomic"])
def test_f64_matches_oracle(api, n, strategy):
    x, b = W.laplace1d_inputs(n)
    f_ref, gx_ref, gb_ref = O.laplace1d_grad(x, b, fbar=1.25)
    bt = torch.tensor(b, device="cuda")
    p = api.Laplace1D(bt, strategy=strategy)
    xt = torch.tensor(x, device="cuda")
    gb = torch.empty(n, dtype=torch.float64, device="cuda")
    seed = torch.tensor(1.25, dtype=torch.float64, device="cuda")
    f, gx = p.grad(xt, gdata=gb, seed=seed)
    fe = p.eval(xt)
    p.sync()
    assert rel_scalar(f.item(), f_ref) <= TOL["f64"]
    assert rel_scalar(fe.item(), f_ref) <= TOL["f64"]
    assert rel_l2(gx.cpu().numpy(), gx_ref) <= TOL["f64"]
    assert rel_l2(gb.cpu().numpy(), gb_ref) <= TOL["f64"]


def test_unit_residual_golden(api):
    # tests/golden/laplace1d_unit_residual_n5.txt: y = e_k gives grad_x = column k of 6A
    import os
    rows = [l.split() for l in open(os.path.join(os.path.dirname(__file__), "golden",
                                                 "laplace1d_unit_residual_n5.txt"))
            if l.strip() and not l.startswith("#")]
    A = 2 * np.eye(5) - np.eye(5, k=1) - np.eye(5, k=-1)
    x = np.array([0.25, -0.5, 0.75, 0.125, -1.0])
    for strategy in ("fused", "atomic"):
        for r in rows:
            k = int(r[0])
            b = A @ (3 * x)
            b[k] -= 1.0
            p = api.Laplace1D(torch.tensor(b, device="cuda"), strategy=strategy)
            f, gx = p.grad(torch.tensor(x, device="cuda"))
            assert f.item() == 1.0
            assert np.array_equal(gx.cpu().numpy(), np.array([float(v) for v in r[1:]]))
            p.close()


def test_f32_and_accumulate(api):
    n = 4097
    x, b = W.laplace1d_inputs(n, seed=8)
    x32, b32 = x.astype(np.float32).astype(np.float64), b.astype(np.float32).astype(np.float64)
    f_ref, gx_ref, _ = O.laplace1d_grad(x32, b32)
    for strategy in ("fused", "atomic"):
        p = api.Laplace1D(torch.tensor(b32, dtype=torch.float32, device="cuda"), strategy=strategy)
        gx = torch.ones(n, dtype=torch.float32, device="cuda")
        f, gx = p.grad(torch.tensor(x32, dtype=torch.float32, device="cuda"), gx=gx, accumulate=True)
        p.sync()
        assert rel_scalar(f.item(), f_ref) <= TOL["f32"]
        assert rel_l2(gx.cpu().numpy() - 1.0, gx_ref) <= TOL["f32"]


@pytest.mark.parametrize("n", [1, 2, 7, 4096, 100003])
def test_tape_mode_chain_from_tape(api, n):
    # the forward records y; the reverse chain runs from the tape alone (x and b are not read:
    # they are overwritten between the two calls)
    from paper_2507_13204_gb300 import _lib as L
    x, b = W.laplace1d_inputs(n, seed=n)
    f_ref, gx_ref, _ = O.laplace1d_grad(x, b, fbar=-0.5)
    bt = torch.tensor(b, device="cuda")
    p = api.Laplace1D(bt, mode="tape")
    assert p.config[1] == "tape"
    xt = torch.tensor(x, device="cuda")
    with pytest.raises(L.KGError) as ei:
        p.grad_from_tape()
    assert ei.value.status == L.KG_ERR_STATE
    f = p.eval_tape(xt)
    xt.fill_(123.0)
    bt.fill_(-7.0)
    seed = torch.tensor(-0.5, dtype=torch.float64, device="cuda")
    g = torch.full((n,), 0.25, dtype=torch.float64, device="cuda")
    p.grad_from_tape(gx=g, seed=seed, accumulate=True)
    p.sync()
    assert rel_scalar(f.item(), f_ref) <= TOL["f64"]
    assert rel_l2(g.cpu().numpy() - 0.25, gx_ref) <= TOL["f64"]
    # the default mode has no tape
    q = api.Laplace1D(torch.tensor(b, device="cuda"))
    assert q.config[1] == "recompute"
    with pytest.raises(L.KGError) as ei:
        q.eval_tape(torch.tensor(x, device="cuda"))
    assert ei.value.status == L.KG_ERR_STATE
