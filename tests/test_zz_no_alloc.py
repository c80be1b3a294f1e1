"""The allocation-free entry point kg_quadform_grad_noalloc, called through the
C ABI, on two calls in a row: its value and gradient match the FP64 oracle and
the problem-handle entry point kg_grad.  It exists for callers that cannot
allocate device memory (code under a memory manager that owns the device heap,
a loop that must never enter the allocator): it takes its scratch from an
array compiled into the library.

Kept in a file that is collected last, and self-contained, so that it passes
alone in a fresh process as well as after the other tests."""
import ctypes

import pytest
import torch

from oracle import oracle as O
from paper_2507_13204_gb300 import workloads as W
from tests.helpers import TOL, rel_l2, rel_scalar

pytestmark = pytest.mark.gpu

N_MAX = 12288  # the entry point's documented limit on n


@pytest.fixture(scope="module")
def mods(cuda_ok):
    from paper_2507_13204_gb300 import build
    build.build()
    from paper_2507_13204_gb300 import _lib as L
    from paper_2507_13204_gb300 import api as A
    return L, A


def _noalloc(L, A, x):
    m, n = A.shape
    f = torch.empty((), dtype=torch.float64, device="cuda")
    gx = torch.full((n,), 7.0, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    rc = L.lib().kg_quadform_grad_noalloc(A.data_ptr(), ctypes.c_int64(m), ctypes.c_int64(n),
                                          x.data_ptr(), f.data_ptr(), gx.data_ptr(), stream)
    L.check(rc, "kg_quadform_grad_noalloc")
    return f, gx


@pytest.mark.parametrize("cases", [
    [(4000, 10000, 0), (777, 3001, 1)],      # the second call reuses the scratch
    [(3000, N_MAX, 2), (5, 1, 3)],           # the largest n, then a 5 x 1 problem
])
def test_noalloc_matches_oracle_and_kg_grad_on_two_calls_in_a_row(mods, cases):
    L, api = mods
    results = []
    for m, n, seed in cases:
        A, x = W.quadform_inputs(n, m=m, seed=seed)
        At = torch.tensor(A, device="cuda")
        xt = torch.tensor(x, device="cuda")
        results.append((A, x, At, xt, _noalloc(L, At, xt)))
    torch.cuda.synchronize()
    for A, x, At, xt, (f, gx) in results:
        f_or, g_or = O.quadform_grad(A, x)
        assert rel_scalar(f.item(), f_or) <= TOL["f64"]
        assert rel_l2(gx.cpu().numpy(), g_or) <= TOL["f64"]
        p = api.QuadForm(At)
        f_ref, g_ref = p.grad(xt)
        p.sync()
        assert rel_scalar(f.item(), f_ref.item()) <= TOL["f64"]
        assert rel_l2(gx.cpu().numpy(), g_ref.cpu().numpy()) <= TOL["f64"]
        p.close()


def test_noalloc_rejects_n_beyond_its_limit(mods):
    L, _ = mods
    n = N_MAX + 1
    A = torch.zeros((4, n), dtype=torch.float64, device="cuda")
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    with pytest.raises(L.KGError) as ei:
        _noalloc(L, A, x)
    assert ei.value.status == L.KG_ERR_INVALID_ARG
    assert str(N_MAX) in str(ei.value)
