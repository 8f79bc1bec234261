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


def test_recorded_traffic_is_keyed_to_the_source_hash_and_workload(tmp_path, monkeypatch):
    _copy_tree(tmp_path)
    (tmp_path / "profiles").mkdir()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h = bench.csrc_hash()
    (tmp_path / "profiles" / "ncu_traffic.txt").write_text(
        "# comment\n"
        f"kernel=engine_kernel<BfsAppT<false>> workload=bfs_rmat20 source={h} dram_bytes_per_launch=123 "
        "link_bytes_per_launch=456\n"
        "kernel=resident_bag_kernel<1> workload=hits_1gib source=0000000000000000 dram_bytes_per_launch=7\n")
    k = "engine_kernel<BfsAppT<false>>"
    assert bench.recorded_traffic(k, workload="bfs_rmat20") == 123.0
    assert bench.recorded_traffic(k, "link_bytes_per_launch", workload="bfs_rmat20") == 456.0
    assert bench.recorded_traffic(k, workload="bfs_rmat16") is None        # another workload
    assert bench.recorded_traffic("resident_bag_kernel<1>", workload="hits_1gib") is None   # other sources
    assert bench.recorded_traffic("engine_kernel<SpmvAppT<false>>", workload="spmv_rmat20") is None
