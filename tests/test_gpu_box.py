"""GPU: the device characterisation that sets the ALU and random-access rooflines
(kg_measure_box) returns positive rates in the ranking the hardware fixes."""
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib(cuda_ok):
    from paper_2507_13204_gb300 import build
    build.build()
    from paper_2507_13204_gb300 import _lib as L
    return L


def test_measure_box_rates(lib):
    r = lib.kg_measure_box()
    props = torch.cuda.get_device_properties(0)
    assert r["sms"] == props.multi_processor_count
    assert r["l2_bytes"] > 0
    for k in ("fp64_fma_tflops", "fp32_fma_tflops", "fp64_red_gops", "fp32_red_gops",
              "fp64_log1p_gops", "fp64_div_gops", "fp64_gather_gops", "fp32_gather_gops"):
        assert r[k] > 0.0, k
    # FP32 FMA is the wide pipe; log1p and division take many FMAs each
    assert r["fp32_fma_tflops"] > 4 * r["fp64_fma_tflops"]
    assert r["fp64_log1p_gops"] < r["fp64_fma_tflops"] * 1e3 / 2
    # random L2 accesses: far below the FP32 FMA rate, of the same order for both widths
    assert r["fp32_gather_gops"] < r["fp32_fma_tflops"] * 1e3 / 2
    assert 0.25 < r["fp64_gather_gops"] / r["fp32_gather_gops"] < 4.0
    assert 0.25 < r["fp64_red_gops"] / r["fp32_red_gops"] < 4.0
