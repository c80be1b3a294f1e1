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
