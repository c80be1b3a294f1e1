"""Host logic of bench.py: the recorded DRAM traffic is reported only at the default sizes and
only while the dominant kernel's sources are unchanged since the ncu capture; every
workload's CPU-baseline leg runs on the host data its set-up makes."""
import os
import shutil
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402
from oracle import oracle as O  # noqa: E402


def test_traffic_reported_only_at_default_sizes_and_matching_fingerprint():
    for (wl, dt), (nbytes, files, fp) in bench._TRAFFIC.items():
        same = bench.source_fingerprint(files) == fp
        assert bench.recorded_traffic(wl, dt, True) == (nbytes if same else None)
        assert bench.recorded_traffic(wl, dt, False) is None
    assert bench.recorded_traffic("batched_big", "f64", True) is None  # no capture recorded


def test_fingerprint_matches_when_sources_are_restored(tmp_path, monkeypatch):
    csrc = tmp_path / "csrc"
    shutil.copytree(bench._CSRC, csrc)
    monkeypatch.setattr(bench, "_CSRC", str(csrc))
    nbytes, files, fp = bench._TRAFFIC[("dense", "f64")]
    monkeypatch.setitem(bench._TRAFFIC, ("dense", "f64"), (nbytes, files, bench.source_fingerprint(files)))
    assert bench.recorded_traffic("dense", "f64", True) == nbytes


def test_traffic_is_null_once_a_kernel_source_changes_but_not_for_comments(tmp_path, monkeypatch):
    csrc = tmp_path / "csrc"
    shutil.copytree(bench._CSRC, csrc)
    monkeypatch.setattr(bench, "_CSRC", str(csrc))
    nbytes, files, _ = bench._TRAFFIC[("dense", "f64")]
    monkeypatch.setitem(bench._TRAFFIC, ("dense", "f64"), (nbytes, files, bench.source_fingerprint(files)))
    tb, tf, _ = bench._TRAFFIC[("dense32", "f32")]
    monkeypatch.setitem(bench._TRAFFIC, ("dense32", "f32"), (tb, tf, bench.source_fingerprint(tf)))
    assert bench.recorded_traffic("dense", "f64", True) == nbytes
    with open(csrc / "quadform_pair.cu", "a") as fh:  # comments and blank lines: same code
        fh.write("\n// edited\n/* a block\n   comment */\n\n")
    assert bench.recorded_traffic("dense", "f64", True) == nbytes
    with open(csrc / "quadform_pair.cu", "a") as fh:
        fh.write("\nstatic int edited_code = 1;\n")
    assert bench.recorded_traffic("dense", "f64", True) is None
    assert bench.recorded_traffic("dense32", "f32", True) == tb  # other sources untouched


def _host_workload(name):
    """A workload with only the host-side data its CPU-baseline leg reads (what its GPU
    set-up would also have made), at a small size."""
    import numpy as np
    import torch
    from paper_2507_13204_gb300 import workloads as W
    wl = bench.make_workload(name, "auto", {"dense": 300, "batched": 16, "laplace": 500,
                                            "sparse": 5000}.get(name, 6), 0)
    if name == "dense":
        wl.A_host, wl.x_host = W.quadform_inputs(wl.n, seed=0)
        wl.m = wl.n
    elif name == "sparse":
        wl.A, wl.x_host = W.spquadform_inputs(wl.m)
        wl.n, wl.nnz = wl.A.n, wl.A.nnz
    elif name == "laplace":
        wl.x_host, wl.b_host = W.laplace1d_inputs(wl.n)
    elif name == "batched":
        sizes, boxes = W.batched_dense_sizes(wl.ndense), W.batched_tet_boxes(wl.ntet)
        wl.A = [tuple(torch.from_numpy(v) for v in W.batched_dense_instance(k, int(min(n, 64))))
                for k, n in enumerate(sizes)]
        wl.tets = [W.batched_tet_instance(k, b) + (None, None) for k, b in enumerate(boxes[:2])]
    else:  # tet, hvp, autograd
        wl.mesh, wl.u_host = W.tet_inputs(wl.a)
        wl.ne, wl.nv = wl.mesh.ne, wl.mesh.nv
    return wl


@pytest.mark.parametrize("name", ["dense", "sparse", "laplace", "batched", "tet", "hvp", "autograd"])
def test_cpu_baseline_legs_run_on_host_data(name):
    res = _host_workload(name).oracle_sample(budget_s=0.05)
    if isinstance(res, dict):  # dense and tet: the OpenMP build on all cores, serial beside it
        assert res["value"] > 0 and "oracle" in res["sample"] and res["kind"] == "oracle"
        assert res["cores"] == O.omp_threads() >= 1
        assert res["single_thread"]["cores"] == 1 and res["single_thread"]["value"] > 0
    else:
        value, sample = res
        assert value > 0 and "oracle" in sample


def test_fp64_peak_prefers_the_measured_rate():
    peaks = {"fp64_tflops": 1.258}
    assert bench.fp64_peak(peaks, {"fp64_fma_tflops": 1.19})[0] == 1.19
    assert bench.fp64_peak(peaks, {"error": "x"})[0] == 1.258
    assert bench.fp64_peak(peaks, None)[0] == 1.258


def test_batched_profiling_case_takes_the_full_batchs_instances():
    # batched_big: the first 96 dense instances of the 4096-instance draw with 1024 <= n < 2048,
    # at their indices in that draw (their seeds), and no tets; the full batch keeps everything
    from paper_2507_13204_gb300 import workloads as W
    drawn = W.batched_dense_sizes(4096)
    ks, sizes, boxes = bench.make_workload("batched_big", "auto").instances()
    assert len(ks) == 96 and boxes == []
    assert ks == [k for k, n in enumerate(drawn) if 1024 <= n < 2048][:96]
    assert sizes == [int(drawn[k]) for k in ks]
    ks, sizes, boxes = bench.make_workload("batched", "auto").instances()
    assert ks == list(range(4096)) and len(boxes) == 512


def test_sparse_random_access_record():
    # least time = nnz / gather rate + nnz / (reduction rate, ATOMIC; gather rate, CSC)
    wl = bench.SparseWL(1 << 10, "f64")
    wl.nnz = 1_000_000
    box = {"fp64_gather_gops": 300.0, "fp32_gather_gops": 310.0, "fp64_red_gops": 200.0,
           "fp32_red_gops": 205.0}
    rec = wl.l2_record(0.02, 0.01, "atomic", box)
    least = 1e6 / 300e9 + 1e6 / 200e9
    assert abs(rec["least_ms"] - round(least * 1e3, 5)) < 1e-9
    assert rec["reverse"] == "red" and rec["accesses_per_step"] == 2_000_000
    assert abs(rec["frac_of_step"] - round(least * 1e3 / 0.02, 4)) < 1e-9
    rec = wl.l2_record(0.02, 0.01, "transpose", box)
    assert rec["reverse"] == "gather" and rec["frac_of_kernel"] is None
    assert abs(rec["least_ms"] - round(2e6 / 300e9 * 1e3, 5)) < 1e-9
