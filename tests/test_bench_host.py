"""Host-side logic of bench.py that needs no GPU: the source hash that keys the recorded
ncu traffic (compiled content only) and the parsing of that record."""
import os
import shutil
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _copy_tree(tmp):
    for d in ("paper_2504_19365_gb300/csrc", "include"):
        shutil.copytree(os.path.join(ROOT, d), os.path.join(tmp, d))


def test_source_hash_ignores_comments_but_not_code(tmp_path, monkeypatch):
    _copy_tree(tmp_path)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h0 = bench.csrc_hash()
    hdr = tmp_path / "include" / "agile.h"
    txt = hdr.read_text()
    hdr.write_text(txt + "\n/* a comment */\n// another one\n")
    assert bench.csrc_hash() == h0
    src = tmp_path / "paper_2504_19365_gb300" / "csrc" / "agile_dev.cuh"
    s = src.read_text()
    assert "constexpr int kWarps = 8;" in s
    src.write_text(s.replace("constexpr int kWarps = 8;", "constexpr int kWarps = 4;"))
    assert bench.csrc_hash() != h0


def test_recorded_traffic_is_keyed_to_the_source_hash(tmp_path, monkeypatch):
    _copy_tree(tmp_path)
    (tmp_path / "profiles").mkdir()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h = bench.csrc_hash()
    (tmp_path / "profiles" / "ncu_traffic.txt").write_text(
        "# comment\n"
        f"kernel=engine_kernel<BfsApp> source={h} dram_bytes_per_launch=123 link_bytes_per_launch=456\n"
        "kernel=engine_kernel<EmbApp<1,3>> source=0000000000000000 dram_bytes_per_launch=7\n")
    assert bench.recorded_traffic("engine_kernel<BfsApp>") == 123.0
    assert bench.recorded_traffic("engine_kernel<BfsApp>", "link_bytes_per_launch") == 456.0
    assert bench.recorded_traffic("engine_kernel<EmbApp<1,3>>") is None   # taken on other sources
    assert bench.recorded_traffic("engine_kernel<SpmvApp>") is None
