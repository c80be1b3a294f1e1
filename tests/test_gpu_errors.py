"""Host-side fault injection and argument errors on a GPU (no device fault is
ever provoked: failures are made on the host or caught by bounds checks)."""
import os

import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods(cuda_ok):
    from paper_2507_13204_gb300 import build
    build.build()
    from paper_2507_13204_gb300 import _lib as L
    from paper_2507_13204_gb300 import api as A
    return L, A


def test_fail_alloc_hook(mods):
    L, A = mods
    import subprocess, sys, textwrap
    code = textwrap.dedent("""
        import os, sys, torch
        sys.path.insert(0, os.getcwd())
        from paper_2507_13204_gb300 import api as A, _lib as L
        x = torch.zeros((64, 64), dtype=torch.float64, device='cuda')
        caught = 0
        for k in range(1, 9):
            os.environ['KG_TEST_FAIL_ALLOC'] = str(k)
            # allocation counter is process-wide: the k-th allocation from process start fails
            try:
                p = A.QuadForm(x)
                p.close()
            except L.KGError as e:
                assert e.status == L.KG_ERR_OOM, e
                caught += 1
        print('caught', caught)
    """)
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "-c", code], cwd=root, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    assert int(r.stdout.split()[-1]) >= 1


def test_unsupported_combinations(mods):
    L, A = mods
    x = torch.zeros((8, 8), dtype=torch.float64, device="cuda")
    with pytest.raises(L.KGError) as ei:
        A.QuadForm(x, strategy="csr")
    assert ei.value.status == L.KG_ERR_UNSUPPORTED
    b = torch.zeros(8, dtype=torch.float64, device="cuda")
    with pytest.raises(L.KGError):
        A.Laplace1D(b, strategy="csr")


def test_misaligned_data_rejected(mods):
    L, A = mods
    buf = torch.zeros(65, dtype=torch.float64, device="cuda")
    import ctypes
    from paper_2507_13204_gb300._lib import kg_create, KG_QUADFORM
    with pytest.raises(L.KGError) as ei:
        kg_create(KG_QUADFORM, [4, 4], [buf.data_ptr() + 8])
    assert ei.value.status == L.KG_ERR_INVALID_ARG


@pytest.mark.parametrize("limit_us", [50, 2000])
def test_bounded_wait_runs_out_and_reports_timeout(mods, limit_us):
    """A device wait whose barrier nothing completes gives up after its limit:
    the kernel records KG_ERR_TIMEOUT and returns, kg_sync reports it (and
    clears it), and the context stays usable for a correct gradient after."""
    import time

    import numpy as np
    from oracle import oracle as O
    from paper_2507_13204_gb300 import workloads as W
    L, A = mods
    Ah, xh = W.quadform_inputs(96, m=40, seed=5)
    p = A.QuadForm(torch.tensor(Ah, device="cuda"))
    p.sync()
    t0 = time.perf_counter()
    L.kg_check_bounded_wait(p.handle, limit_us * 1000)
    with pytest.raises(L.KGError) as ei:
        p.sync()
    elapsed = time.perf_counter() - t0
    assert ei.value.status == L.KG_ERR_TIMEOUT
    assert "gave up" in str(ei.value)
    assert elapsed >= limit_us * 1e-6
    p.sync()  # the read cleared the sticky word
    f, g = p.grad(torch.tensor(xh, device="cuda"))
    p.sync()
    f_ref, g_ref = O.quadform_grad(Ah, xh)
    assert abs(f.item() - f_ref) <= 1e-12 * abs(f_ref)
    assert np.linalg.norm(g.cpu().numpy() - g_ref) <= 1e-12 * np.linalg.norm(g_ref)
    p.close()


def test_bounded_wait_check_rejects_bad_limits(mods):
    L, A = mods
    p = A.QuadForm(torch.zeros((4, 4), dtype=torch.float64, device="cuda"))
    for bad in (0, 3_000_000_000):
        with pytest.raises(L.KGError) as ei:
            L.kg_check_bounded_wait(p.handle, bad)
        assert ei.value.status == L.KG_ERR_INVALID_ARG
    p.close()
