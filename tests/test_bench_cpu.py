"""Host logic of bench.py: the recorded DRAM traffic is reported only at the default sizes and
only while the dominant kernel's sources are unchanged since the ncu capture."""
import os
import shutil
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_traffic_recorded_for_current_sources_at_default_sizes():
    for (wl, dt), (nbytes, _, _) in bench._TRAFFIC.items():
        assert bench.recorded_traffic(wl, dt, True) == nbytes
        assert bench.recorded_traffic(wl, dt, False) is None
    assert bench.recorded_traffic("batched", "f64", True) is None


def test_traffic_is_null_once_a_kernel_source_changes(tmp_path, monkeypatch):
    csrc = tmp_path / "csrc"
    shutil.copytree(bench._CSRC, csrc)
    monkeypatch.setattr(bench, "_CSRC", str(csrc))
    assert bench.recorded_traffic("dense", "f64", True) is not None
    with open(csrc / "quadform_pair.cu", "a") as fh:
        fh.write("\n// edited\n")
    assert bench.recorded_traffic("dense", "f64", True) is None
    assert bench.recorded_traffic("tet", "f64", True) is not None  # other sources untouched
