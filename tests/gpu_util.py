"""Helpers shared by the GPU tests: a context whose store holds given byte blobs."""
from __future__ import annotations

import numpy as np

import paper_2504_19365_gb300 as ag

PAGE = 4096


def round_page(n: int) -> int:
    return (int(n) + PAGE - 1) // PAGE * PAGE


class Ctx:
    def __init__(self, store_bytes: int, **cfg):
        import torch
        self.torch = torch
        self.cfg = ag.agile_config_default(store_bytes=round_page(store_bytes), **cfg)
        self.h = ag.agile_init(self.cfg)
        self.stream = torch.cuda.current_stream().cuda_stream

    def put(self, off: int, arr: np.ndarray):
        a = np.ascontiguousarray(arr)
        ag.agile_store_write(self.h, off, a.ctypes.data, a.nbytes)

    def get(self, off: int, n: int) -> np.ndarray:
        out = np.empty(n, dtype=np.uint8)
        ag.agile_store_read(self.h, off, out.ctypes.data, n)
        return out

    def check(self):
        e = ag.agile_check(self.h)
        assert e == 0, f"device error {e}: {ag.strerror(e)}"

    def stats(self):
        return ag.agile_stats(self.h)

    def tags(self) -> np.ndarray:
        n = ag.agile_cache_lines(self.h)
        out = np.zeros(n, dtype=np.uint64)
        ag.agile_cache_tags(self.h, out.ctypes.data)
        return out

    def close(self):
        if self.h:
            ag.agile_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def tag_fields(tags: np.ndarray):
    t = tags.astype(np.uint64)
    return (t >> np.uint64(20)), (t & np.uint64(3)), ((t >> np.uint64(2)) & np.uint64(1)), \
        ((t >> np.uint64(4)) & np.uint64(0xFFFF))


def assert_cache_invariants(c: Ctx, store: np.ndarray | None = None):
    """No two valid ways of a set hold one page; nothing pinned or in flight after a
    call; every READY line equals the store page it caches."""
    tags = c.tags()
    page, state, _, pins = tag_fields(tags)
    ways = c.cfg.ways
    sets = len(tags) // ways
    assert (pins == 0).all(), "pins left after the call"
    assert not (state == 1).any(), "BUSY line after the call"
    for s in range(sets):
        sl = slice(s * ways, (s + 1) * ways)
        valid = page[sl][state[sl] != 0]
        assert len(valid) == len(set(valid.tolist())), f"duplicate tag in set {s}"
    return page, state


def build_user_kernel(name: str):
    """Compile tests/user_kernels/<name>.cu (a user kernel built against
    include/agile_device.cuh) into tests/_build/lib<name>.so, linked to libagile.so, and
    load it."""
    import ctypes
    import os
    import subprocess

    from paper_2504_19365_gb300 import build
    here = os.path.dirname(os.path.abspath(__file__))
    root = os.path.dirname(here)
    lib = build.build()
    pkg = os.path.dirname(lib)
    src = os.path.join(here, "user_kernels", name + ".cu")
    deps = [src, lib, os.path.join(root, "include", "agile_device.cuh")] + \
        [os.path.join(pkg, "csrc", f) for f in os.listdir(os.path.join(pkg, "csrc"))]
    out_dir = os.path.join(here, "_build")
    os.makedirs(out_dir, exist_ok=True)
    so = os.path.join(out_dir, f"lib{name}.so")
    if not os.path.exists(so) or os.path.getmtime(so) < max(os.path.getmtime(p) for p in deps):
        cmd = [build.nvcc(), "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17", "-shared",
               "-Xcompiler", "-fPIC", "-I", os.path.join(root, "include"), "-I", os.path.join(pkg, "csrc"),
               src, "-o", so + ".tmp", "-L", pkg, "-lagile", "-Xlinker", f"-rpath={pkg}"]
        subprocess.run(cmd, check=True, capture_output=True, text=True)
        os.replace(so + ".tmp", so)
    return ctypes.CDLL(so)


def dyadic_rows(k: int, r: np.ndarray, dim: int) -> np.ndarray:
    """Rows r of dyadic table k: T_k[r, d] = ((r*131 + d*7 + k) mod 1024) / 64 - 8, so that
    every FP32 sum of up to 2^16 of them is exact (any order gives the same bits)."""
    d = np.arange(dim, dtype=np.int64)[None, :]
    r = np.asarray(r, dtype=np.int64)[:, None]
    return (((r * 131 + d * 7 + k) % 1024).astype(np.float32) / np.float32(64.0) - np.float32(8.0))


def fill_dyadic(c: "Ctx", n_tables: int, rows: int, dim: int, stride: int, chunk_rows: int = 1 << 20):
    """Write n_tables dyadic tables (table k at byte k*stride of the store).  A table's
    rows repeat with period 1024, so one 1024-row block is tiled."""
    for k in range(n_tables):
        block = dyadic_rows(k, np.arange(1024), dim)
        big = np.tile(block, (chunk_rows // 1024 + 1, 1))
        for r0 in range(0, rows, chunk_rows):
            m = min(chunk_rows, rows - r0)
            s = r0 % 1024
            c.put(k * stride + r0 * dim * 4, big[s:s + m])
