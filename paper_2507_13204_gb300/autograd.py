"""torch.autograd.Function wrappers over the C ABI.

KGTetEnergy.apply(u, problem) returns f(u) = sum_e log1p(|G_e u_e|^2) as a 0-d
tensor; its backward is the library's reverse pass with the incoming gradient
as the output adjoint (read from device memory, no host synchronisation).

Tape vs recompute (the paper's Sec. 5 taping restriction): when the problem
was created with a tape (mode "tape", or "auto" and the N_e x 4 tape fits the
memory budget) the forward records c_e = G_e^T (2 g_e / (1 + |g_e|^2)) and the
backward only scatters the tape (no G read, no FP64 math); otherwise the
backward recomputes the forward inside the fused value-and-gradient kernel.
A tape is valid only for the forward that wrote it: the forward keeps the
library's tape generation (kg_tape_generation, counted on the C side for every
launch that writes the tape, including a CSR-strategy gradient, whose reverse
pass goes through the same tape) and the backward recomputes if the count has
moved since.

KGQuadForm.apply(x, problem) does the same for f(x) = ||A x||^2 (recompute
only: the reverse pass needs nothing but y, which the fused kernel rebuilds).
"""
from __future__ import annotations

import os

import torch

from .api import QuadForm, TetEnergy


class KGTetEnergy(torch.autograd.Function):
    @staticmethod
    def forward(ctx, u: torch.Tensor, problem: TetEnergy, policy: str = "auto"):
        u = u.detach().contiguous()
        f = torch.empty((), dtype=u.dtype, device=u.device)
        strategy, mode, arith = problem.config
        use_tape = mode == "tape" and policy in ("auto", "tape")
        if policy == "tape" and mode != "tape":
            raise ValueError("KGTetEnergy: the problem was created without a tape")
        if use_tape:
            problem.eval_tape(u, f)
            ctx.tape_gen = problem.tape_generation
        else:
            problem.eval(u, f)
            ctx.tape_gen = None
        ctx.save_for_backward(u)
        ctx.problem = problem
        return f

    @staticmethod
    def backward(ctx, grad_out: torch.Tensor):
        (u,) = ctx.saved_tensors
        problem = ctx.problem
        seed = grad_out.detach().to(dtype=u.dtype).contiguous()
        if ctx.tape_gen is not None and problem.tape_generation == ctx.tape_gen:
            gu = problem.grad_from_tape(seed=seed)
        else:
            _, gu = problem.grad(u, seed=seed)
        return gu, None, None


class KGQuadForm(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x: torch.Tensor, problem: QuadForm):
        x = x.detach().contiguous()
        f = torch.empty((), dtype=x.dtype, device=x.device)
        problem.eval(x, f)
        ctx.save_for_backward(x)
        ctx.problem = problem
        return f

    @staticmethod
    def backward(ctx, grad_out: torch.Tensor):
        (x,) = ctx.saved_tensors
        seed = grad_out.detach().to(dtype=x.dtype).contiguous()
        _, gx = ctx.problem.grad(x, seed=seed)
        return gx, None


def tet_energy(u: torch.Tensor, problem: TetEnergy, policy: str = "auto") -> torch.Tensor:
    return KGTetEnergy.apply(u, problem, policy)


def quad_form(x: torch.Tensor, problem: QuadForm) -> torch.Tensor:
    return KGQuadForm.apply(x, problem)


def gradient_descent(problem: TetEnergy, u0: torch.Tensor, eta: float, steps: int,
                     policy: str = "auto", checkpoint: str | None = None, every: int = 0,
                     resume: bool = False, history: list | None = None) -> torch.Tensor:
    """u <- u - eta * grad f(u) through torch.autograd, `steps` times.

    With `checkpoint` and `every` > 0, {u, step} is saved every `every` steps
    (atomically: written to a temporary file, then renamed); with `resume`, a
    saved checkpoint is loaded first and the loop continues from its step.
    `history` (a list) receives f before each step.
    """
    u = u0.detach().clone()
    start = 0
    if resume and checkpoint and os.path.exists(checkpoint):
        state = torch.load(checkpoint, map_location=u.device)
        u = state["u"].to(device=u0.device, dtype=u0.dtype).clone()
        start = int(state["step"])
    for t in range(start, steps):
        ut = u.requires_grad_(True)
        f = KGTetEnergy.apply(ut, problem, policy)
        (g,) = torch.autograd.grad(f, ut)
        if history is not None:
            history.append(f.detach())
        u = (ut.detach() - eta * g).detach()
        if checkpoint and every > 0 and (t + 1) % every == 0:
            tmp = checkpoint + ".tmp"
            torch.save({"u": u.cpu(), "step": t + 1}, tmp)
            os.replace(tmp, checkpoint)
    return u
