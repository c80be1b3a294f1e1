"""Host logic of bench.py: the recorded DRAM traffic is reported only at the default sizes and
only while the dominant kernel's sources are unchanged since the ncu capture."""
import os
import shutil
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_traffic_reported_only_at_default_sizes_and_matching_fingerprint():
    for (wl, dt), (nbytes, files, fp) in bench._TRAFFIC.items():
        same = bench.source_fingerprint(files) == fp
        assert bench.recorded_traffic(wl, dt, True) == (nbytes if same else None)
        assert bench.recorded_traffic(wl, dt, False) is None
    assert bench.recorded_traffic("batched", "f64", True) is None


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
