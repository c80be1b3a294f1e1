"""torch.autograd integration: gradcheck, equality with the direct gradient,
gradient-descent trajectories against the oracle, tape invalidation, and
checkpoint / resume of the descent loop."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2507_13204_gb300 import workloads as W
from tests.helpers import TOL, f32_round, rel_l2, rel_scalar

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods(cuda_ok):
    from paper_2507_13204_gb300 import build
    build.build()
    from paper_2507_13204_gb300 import api, autograd
    return api, autograd


def _tet(api, mesh, dtype=torch.float64, **kw):
    return api.TetEnergy(torch.tensor(mesh.conn, device="cuda"),
                         torch.tensor(mesh.G, dtype=dtype, device="cuda"), mesh.nv, **kw)


@pytest.mark.parametrize("policy,mode", [("tape", "tape"), ("recompute", "recompute"), ("auto", "auto")])
@pytest.mark.parametrize("strategy", ["atomic", "warp", "tile", "csr"])
def test_gradcheck_6x4cubed_mesh(mods, policy, mode, strategy):
    api, ag = mods
    mesh = W.tet_mesh(4, perm_seed=3)  # 4x4x4 cubes: 384 tets, 125 vertices
    assert (mesh.ne, mesh.nv) == (384, 125)
    p = _tet(api, mesh, strategy=strategy, mode=mode)
    u = torch.tensor(np.random.default_rng(0).uniform(-1, 1, mesh.nv), device="cuda",
                     requires_grad=True)
    # atomic scatter order varies between runs (differences at rounding level, within the
    # 1e-12 bound), with or without the warp combine; the CSR gather is bitwise reproducible,
    # so its backward must be reentrant
    nondet = 0.0 if strategy == "csr" else 1e-12
    assert torch.autograd.gradcheck(lambda v: ag.KGTetEnergy.apply(v, p, policy), (u,),
                                    eps=1e-6, atol=1e-5, rtol=1e-3, nondet_tol=nondet)


def test_backward_equals_direct_gradient_and_oracle(mods):
    api, ag = mods
    mesh = W.tet_mesh(8, jitter_seed=2, perm_seed=1)
    uh = np.random.default_rng(4).uniform(-1, 1, mesh.nv)
    for mode in ("tape", "recompute"):
        p = _tet(api, mesh, mode=mode)
        u = torch.tensor(uh, device="cuda", requires_grad=True)
        f = ag.KGTetEnergy.apply(u, p)
        (3.0 * f).backward()
        _, g_direct = p.grad(u.detach(), seed=torch.tensor(3.0, dtype=torch.float64, device="cuda"))
        f_ref, g_ref = O.tet_grad(mesh.conn, mesh.G, uh, fbar=3.0)
        assert rel_scalar(f.item(), O.tet_value(mesh.conn, mesh.G, uh)) <= TOL["f64"]
        assert rel_l2(u.grad.cpu().numpy(), g_ref) <= TOL["f64"]
        assert rel_l2(u.grad.cpu().numpy(), g_direct.cpu().numpy()) <= TOL["f64"]


def test_stale_tape_falls_back_to_recompute(mods):
    api, ag = mods
    mesh = W.tet_mesh(5, jitter_seed=2)
    p = _tet(api, mesh, mode="tape")
    rng = np.random.default_rng(9)
    u1 = torch.tensor(rng.uniform(-1, 1, mesh.nv), device="cuda", requires_grad=True)
    u2 = torch.tensor(rng.uniform(-1, 1, mesh.nv), device="cuda", requires_grad=True)
    f1 = ag.KGTetEnergy.apply(u1, p)
    f2 = ag.KGTetEnergy.apply(u2, p)  # overwrites the tape
    (f1 + 2 * f2).backward()
    _, g1 = O.tet_grad(mesh.conn, mesh.G, u1.detach().cpu().numpy())
    _, g2 = O.tet_grad(mesh.conn, mesh.G, u2.detach().cpu().numpy(), fbar=2.0)
    assert rel_l2(u1.grad.cpu().numpy(), g1) <= TOL["f64"]
    assert rel_l2(u2.grad.cpu().numpy(), g2) <= TOL["f64"]


@pytest.mark.parametrize("arith", ["native", "pair"])
def test_csr_gradient_between_tape_forward_and_backward(mods, arith):
    """In native FP64 a CSR-strategy gradient writes the same tape as a taping
    forward (its reverse pass reads it); in float pairs it does not.  A forward
    on the tape path, then a direct gradient and a recompute-policy
    forward/backward at another point, then the first backward: the first
    backward must see whether its tape was overwritten (the library's tape
    generation) and recompute at its own point if it was."""
    api, ag = mods
    mesh = W.tet_mesh(5, jitter_seed=2, perm_seed=4)
    p = _tet(api, mesh, strategy="csr", mode="tape", arith=arith)
    rng = np.random.default_rng(12)
    u1 = torch.tensor(rng.uniform(-1, 1, mesh.nv), device="cuda", requires_grad=True)
    u2 = torch.tensor(rng.uniform(-1, 1, mesh.nv), device="cuda", requires_grad=True)
    g0 = p.tape_generation
    f1 = ag.KGTetEnergy.apply(u1, p)  # tape path: records the tape at u1
    assert p.tape_generation == g0 + 1
    _, gd = p.grad(u2.detach())       # CSR gradient at u2: native FP64 rewrites the tape
    assert p.tape_generation == g0 + (2 if arith == "native" else 1)
    f2 = ag.KGTetEnergy.apply(u2, p, "recompute")
    f2.backward()
    f1.backward()
    _, g1 = O.tet_grad(mesh.conn, mesh.G, u1.detach().cpu().numpy())
    _, g2 = O.tet_grad(mesh.conn, mesh.G, u2.detach().cpu().numpy())
    assert rel_l2(u1.grad.cpu().numpy(), g1) <= TOL["f64"]
    assert rel_l2(u2.grad.cpu().numpy(), g2) <= TOL["f64"]
    assert rel_l2(gd.cpu().numpy(), g2) <= TOL["f64"]


def test_quadform_function_gradcheck(mods):
    api, ag = mods
    A, x = W.quadform_inputs(20, m=13, seed=2)
    p = api.QuadForm(torch.tensor(A, device="cuda"))
    xt = torch.tensor(x, device="cuda", requires_grad=True)
    assert torch.autograd.gradcheck(lambda v: ag.KGQuadForm.apply(v, p), (xt,), eps=1e-6,
                                    atol=1e-5, rtol=1e-3)


ETA = 0.01  # step of the descent workload: f is L-smooth with L ~ 144 on the unit Kuhn grid


@pytest.mark.parametrize("policy", ["tape", "recompute"])
def test_descent_trajectory_matches_oracle_f64(mods, policy):
    api, ag = mods
    mesh, u0 = W.tet_inputs(20)  # 48000 tets
    p = _tet(api, mesh, mode="tape" if policy == "tape" else "recompute")
    u = torch.tensor(u0, device="cuda")
    done = 0
    for target in (1, 10, 200):
        u = ag.gradient_descent(p, u, ETA, target - done, policy=policy)
        done = target
        ref, _ = O.tet_descent(mesh.conn, mesh.G, u0, ETA, target)
        assert rel_l2(u.cpu().numpy(), ref) <= 1e-10, target


def test_descent_f32_decreases_and_tracks_f64(mods):
    api, ag = mods
    mesh, u0 = W.tet_inputs(16)
    p32 = api.TetEnergy(torch.tensor(mesh.conn, device="cuda"),
                        torch.tensor(mesh.G, dtype=torch.float32, device="cuda"), mesh.nv)
    hist = []
    u32 = ag.gradient_descent(p32, torch.tensor(u0, dtype=torch.float32, device="cuda"), ETA, 200,
                              history=hist)
    f32 = np.array([h.item() for h in hist])
    assert np.all(np.diff(f32) < 0)
    _, f64_hist = O.tet_descent(mesh.conn, mesh.G, u0, ETA, 200)
    f_end32 = O.tet_value(mesh.conn, mesh.G, u32.double().cpu().numpy())
    assert rel_scalar(f_end32, f64_hist[-1]) <= 1e-4


def test_checkpoint_resume_reproduces_the_uninterrupted_run(mods, tmp_path):
    api, ag = mods
    mesh, u0 = W.tet_inputs(6)
    p = _tet(api, mesh, strategy="csr", mode="recompute")  # deterministic reverse pass
    ck = str(tmp_path / "descent.pt")
    full = ag.gradient_descent(p, torch.tensor(u0, device="cuda"), ETA, 10)
    ag.gradient_descent(p, torch.tensor(u0, device="cuda"), ETA, 6, checkpoint=ck, every=3)
    resumed = ag.gradient_descent(p, torch.tensor(u0, device="cuda"), ETA, 10, checkpoint=ck,
                                  every=3, resume=True)
    assert torch.equal(full, resumed)
    assert torch.load(ck)["step"] == 9
