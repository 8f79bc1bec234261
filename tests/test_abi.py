"""CPU checks of the C-ABI boundary: the library builds for sm_103a, loads, exports
every entry point declared in include/agile.h, and its host-only calls behave."""
import ctypes as C
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "agile.h")


def declared():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(agile_[a-z_]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2504_19365_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = declared()
    for must in ["agile_init", "agile_destroy", "agile_read_async", "agile_write_async", "agile_wait",
                 "agile_embedding_bag", "agile_bfs", "agile_flush", "agile_stats"]:
        assert must in names


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r"\bT (agile_[a-z_]+)\b", out))
    missing = [n for n in declared() if n not in exported]
    assert not missing, missing
    L = C.CDLL(libpath)
    for n in declared():
        assert getattr(L, n) is not None


def test_binding_names_match_header():
    import paper_2504_19365_gb300 as ag
    assert sorted(ag.EXPORTED) == declared()
    for n in declared():
        assert callable(getattr(ag, n))


def test_host_only_calls(libpath):
    import paper_2504_19365_gb300 as ag
    cfg = ag.agile_config_default()
    assert cfg.num_queues == 128 and cfg.queue_depth == 256 and cfg.ways == 8
    assert "timed out" in ag.agile_strerror(ag.AGILE_ETIMEDOUT)
    L = ag.lib()
    h = C.c_void_p()
    # argument checks happen before any device work
    bad = ag.agile_config_default(queue_depth=100)
    assert L.agile_init(C.byref(bad), C.byref(h)) == ag.AGILE_EINVAL
    bad = ag.agile_config_default(ways=0)
    assert L.agile_init(C.byref(bad), C.byref(h)) == ag.AGILE_EINVAL
    bad = ag.agile_config_default(nvme_path=b"/dev/nvme0n1")
    assert L.agile_init(C.byref(bad), C.byref(h)) == ag.AGILE_ENODEV
    assert L.agile_destroy(None) == 0
    assert L.agile_read_async(None, None, 0, None, None, 0, None) == ag.AGILE_EINVAL


def test_sqe_and_cqe_layout_constants():
    # 64-byte submission entries and 16-byte completion entries (NVMe, Sec. 2.1) as laid
    # out by the library source
    src = open(os.path.join(ROOT, "paper_2504_19365_gb300", "csrc", "agile_dev.cuh")).read()
    assert "struct alignas(64) Sqe { uint32_t dw[16]; };" in src
    assert "struct alignas(16) Cqe { uint32_t dw[4]; };" in src


def test_application_calls_reject_a_missing_context(libpath):
    # every application entry point validates its arguments on the host before it
    # touches a device
    import paper_2504_19365_gb300 as ag
    L = ag.lib()
    E = ag.AGILE_EINVAL
    assert L.agile_embedding_bag(None, 0, 10, 128, None, None, 1, None, 0, None) == E
    assert L.agile_embedding_bag_backward(None, 0, 10, 128, None, None, 1, 1, None, 0.0, None, 0, None) == E
    assert L.agile_embedding_pipeline(None, 0, 4096, 1, 10, 64, None, 1, 1, 1, 0, None, 0, None) == E
    assert L.agile_bfs(None, 0, 4096, 10, 0, None, None, 0, None) == E
    assert L.agile_bfs_noalloc(None, 0, 4096, 10, 10, 0, None, None, 0, None) == E
    assert L.agile_spmv(None, 0, 4096, 8192, 10, 10, None, None, None, 0, None) == E
    # an invalid mode is rejected the same way
    assert L.agile_spmv(None, 0, 4096, 8192, 10, 10, None, None, None, 7, None) == E
