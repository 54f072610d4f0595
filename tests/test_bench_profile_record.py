"""bench.py reports the ncu traffic and instruction count of the fused kernel from the
committed profile summary only while the kernel's code hashes to the value recorded there:
a code change must drop both, a comment or layout change must not (host logic, no GPU)."""
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
    src = root / "paper_2602_12949_gb300" / "csrc" / "query_tc.cu"
    text = src.read_text()
    src.write_text("// a new comment line\n/* and a block\n   comment */\n" + text.replace("\n", "\n\n", 3) + "\n// end\n")
    assert bench._profiled_record() == rec
    src.write_text(text + "\nstatic const int edited_code = 1;\n")
    assert bench._profiled_record() is None


def test_code_hash_keeps_strings_and_drops_comments(tmp_path):
    a, b, c = tmp_path / "a.cu", tmp_path / "b.cu", tmp_path / "c.cu"
    a.write_text('asm("ld.x [%0]; // not a comment");  // a comment\nint x = 1;\n')
    b.write_text('asm("ld.x [%0]; // not a comment");\n\n   int x = 1; /* another */\n')
    c.write_text('asm("ld.x [%0]; // changed");\nint x = 1;\n')
    assert bench.kernel_code_hash([a]) == bench.kernel_code_hash([b])
    assert bench.kernel_code_hash([a]) != bench.kernel_code_hash([c])


def test_missing_or_garbled_summary_gives_none(tmp_path, monkeypatch):
    root = _tree(tmp_path)
    monkeypatch.setattr(bench, "ROOT", str(root))
    (root / "profiles" / "niv_query_fp16_1080p.md").write_text("no record here\n")
    assert bench._profiled_record() is None
    os.remove(root / "profiles" / "niv_query_fp16_1080p.md")
    assert bench._profiled_record() is None


def test_measured_peaks_include_the_host_link():
    """The committed peak summary gives the host link's rate on a 1080p frame's traffic, which
    bounds the end-to-end (host-buffer) figure."""
    p = bench._extra_peaks()
    assert p.get("host_frame_rw_gbs", 0) > 0
    assert p.get("fp32_ffma_tflops", 0) > 0


def test_host_link_roofline():
    moved = 2 * 1920 * 1080 * 8 + 1920 * 1080 * 8  # pos + nrm in, E out (FP16 records)
    r = bench.host_link_roofline(moved, 0.256e-3, 274.3)
    assert r["bound"] == "host link" and r["unit"] == "GB/s"
    assert abs(r["achieved"] - moved / 0.256e-3 / 1e9) < 1e-9
    assert abs(r["frac"] - r["achieved"] / 274.3) < 1e-12
    assert bench.host_link_roofline(moved, 0.256e-3, None) is None
    assert bench.host_link_roofline(moved, 0.0, 274.3) is None
