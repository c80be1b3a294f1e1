"""The allocation-free entry point kg_quadform_grad_noalloc, called through the
C ABI, gives the same value and gradient as the problem-handle path (kg_grad)
on two calls in a row.  It exists for callers that cannot allocate device
memory: it takes its scratch from an array compiled into the library.

Kept in a file that is collected last, and self-contained, so that it passes
alone in a fresh process as well as after the other tests."""
import ctypes

import numpy as np
import pytest
import torch

from paper_2507_13204_gb300 import workloads as W
from tests.helpers import TOL, rel_l2, rel_scalar

pytestmark = pytest.mark.gpu


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


def test_noalloc_matches_kg_grad_on_two_calls_in_a_row(mods):
    L, api = mods
    cases = [(4000, 10000, 0), (777, 3001, 1)]  # the second call reuses the scratch
    results = []
    for m, n, seed in cases:
        A, x = W.quadform_inputs(n, m=m, seed=seed)
        At = torch.tensor(A, device="cuda")
        xt = torch.tensor(x, device="cuda")
        results.append((At, xt, _noalloc(L, At, xt)))
    torch.cuda.synchronize()
    for At, xt, (f, gx) in results:
        p = api.QuadForm(At)
        f_ref, g_ref = p.grad(xt)
        p.sync()
        assert rel_scalar(f.item(), f_ref.item()) <= TOL["f64"]
        assert rel_l2(gx.cpu().numpy(), g_ref.cpu().numpy()) <= TOL["f64"]
        p.close()


def test_noalloc_rejects_sizes_beyond_its_scratch(mods):
    L, _ = mods
    A = torch.zeros((4, 20000), dtype=torch.float64, device="cuda")
    x = torch.zeros(20000, dtype=torch.float64, device="cuda")
    with pytest.raises(L.KGError) as ei:
        _noalloc(L, A, x)
    assert ei.value.status == L.KG_ERR_INVALID_ARG
    assert "12288" in str(ei.value)
