"""The validity rule of the ncu counters bench.py carries (DRAM traffic and
executed FP32 operations of the coarse-round scan kernel): they are reported
only while the scan kernel's sources hash to the recorded digest.  The digest
ignores comments, whitespace and other translation units, and changes with any
code edit of the scan kernel's sources or headers."""
import os
import shutil

import bench


def _tree(tmp_path):
    root = tmp_path / "repo"
    shutil.copytree(os.path.join(bench.ROOT, "paper_1908_01949_gb300", "csrc"),
                    root / "paper_1908_01949_gb300" / "csrc")
    shutil.copytree(os.path.join(bench.ROOT, "include"), root / "include")
    return root


def _digest(monkeypatch, root):
    monkeypatch.setattr(bench, "ROOT", str(root))
    return bench.csrc_digest()


def _edit(path, old, new):
    s = path.read_text()
    assert old in s
    path.write_text(s.replace(old, new, 1))


def test_recorded_counters_are_current_or_absent():
    """Every recorded ncu figure was taken on the current scan-kernel sources,
    or none is recorded (the line then reports null)."""
    d = bench.csrc_digest()
    for entry in list(bench.TRAFFIC.values()) + [bench.FP32_COUNTS]:
        assert entry["csrc_sha256"] in (d, None)
        assert bench.recorded(entry) is (entry if entry["csrc_sha256"] == d else None)


def test_stale_records_are_not_reported():
    assert bench.recorded({"bytes": 1, "csrc_sha256": "0" * 64}) is None
    assert bench.recorded(None) is None


def test_comments_whitespace_and_other_units_keep_the_digest(tmp_path, monkeypatch):
    root = _tree(tmp_path)
    d0 = _digest(monkeypatch, root)
    csrc = root / "paper_1908_01949_gb300" / "csrc"
    for p, text in ((csrc / "scan.cu", "// a comment line\n\n   \n"), (csrc / "cdc_dev.cuh", "/* a block\n   comment */\n"),
                    (root / "include" / "cdc.h", "/* header comment */\n")):
        p.write_text(text + p.read_text())
    _edit(csrc / "scan.cu", "__global__", "__global__   /* x */ ")
    _edit(csrc / "refine.cu", "__global__", "__global__ /* x */")
    (csrc / "refine.cu").write_text((csrc / "refine.cu").read_text() + "\nstatic int unrelated_code = 1;\n")
    (csrc / "hough.cu").write_text((csrc / "hough.cu").read_text() + "\nstatic int unrelated_code = 2;\n")
    assert _digest(monkeypatch, root) == d0


def test_code_edits_of_the_scan_kernel_sources_void_the_digest(tmp_path, monkeypatch):
    root = _tree(tmp_path)
    d0 = _digest(monkeypatch, root)
    for rel in ("paper_1908_01949_gb300/csrc/scan.cu", "paper_1908_01949_gb300/csrc/tracer.cuh",
                "paper_1908_01949_gb300/csrc/cdc_dev.cuh", "paper_1908_01949_gb300/csrc/capi.cu",
                "include/cdc.h"):
        p = root / rel
        s = p.read_text()
        p.write_text(s + "\nstatic int changed_code = 3;\n")
        assert _digest(monkeypatch, root) != d0, rel
        p.write_text(s)
    assert _digest(monkeypatch, root) == d0
