"""bench.py reports the ncu traffic and instruction count of the fused kernel from the
committed profile summary only while the kernel sources hash to the value recorded there:
a changed source must drop both (host logic, no GPU)."""
import os
import shutil

import bench


def _tree(tmp_path):
    root = os.path.dirname(os.path.abspath(bench.__file__))
    os.makedirs(tmp_path / "profiles")
    shutil.copy(os.path.join(root, "profiles", "niv_query_fp16_1080p.md"), tmp_path / "profiles")
    shutil.copytree(os.path.join(root, "paper_2602_12949_gb300", "csrc"), tmp_path / "paper_2602_12949_gb300" / "csrc",
                    ignore=shutil.ignore_patterns("*.o"))
    return tmp_path


def test_record_follows_the_source_hash(tmp_path, monkeypatch):
    root = _tree(tmp_path)
    monkeypatch.setattr(bench, "ROOT", str(root))
    rec = bench._profiled_record()
    if rec is None:  # the committed summary predates the current sources: nothing to report
        return
    assert rec["traffic"] > 0 and rec["instructions"] > 0
    with open(root / "paper_2602_12949_gb300" / "csrc" / "query_tc.cu", "a") as f:
        f.write("\n// edited\n")
    assert bench._profiled_record() is None


def test_missing_or_garbled_summary_gives_none(tmp_path, monkeypatch):
    root = _tree(tmp_path)
    monkeypatch.setattr(bench, "ROOT", str(root))
    (root / "profiles" / "niv_query_fp16_1080p.md").write_text("no record here\n")
    assert bench._profiled_record() is None
    os.remove(root / "profiles" / "niv_query_fp16_1080p.md")
    assert bench._profiled_record() is None
