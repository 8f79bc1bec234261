"""CPU oracle of the AGILE I/O path (arXiv 2504.19365) -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py``
may import this package.  It shares no code with the CUDA library and never imports it.
The arithmetic lives in ``agile_oracle.c`` (compiled by ``oracle/build.py``); this
module only marshals numpy arrays through ctypes.

Functions and the passage each restates:
  store_read_page / store_write_page -- 4 KiB page store (Sec. 2.3.3)
  RefCache                          -- sequential set-associative clock cache with the
                                       line states of Sec. 3.4 and the clock policy of
                                       Sec. 4.4
  embedding_bag / _backward / sgd   -- sum-pooled lookups of Sec. 4.4, fixed order
  bfs                               -- FIFO-queue BFS over CSR (Sec. 4.5)
  spmv                              -- y = A x over CSR with FP32 values (Sec. 4.5)
  fma_chain / embedding_pipeline    -- compute phase of the overlap experiment (Sec. 4.2)
  ideal_speedup                     -- Eq. 1
  set_of                            -- the cache's set-index function

Parity status: every function above is pinned by ``tests/test_oracle_*.py`` against
closed forms, brute force, library routines (torch, scipy) or hand-derived golden
traces.  The paper's own speedup figures (RTX 5000 Ada, Gen4 SSDs, BaM) are not
computed here: parity unpinned for those by construction.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import build as _build

PAGE = 4096
INVALID, BUSY, READY, MODIFIED = 0, 1, 2, 3
HIT, MISS_FILL, MISS_EVICT, MISS_WRITEBACK = 0, 1, 2, 3

_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        vp, u64, u32, i32 = C.c_void_p, C.c_uint64, C.c_uint32, C.c_int32
        L.orc_store_read_page.argtypes = [vp, u64, vp]
        L.orc_store_write_page.argtypes = [vp, u64, vp]
        L.orc_set_of.argtypes = [u64, u32]
        L.orc_set_of.restype = u32
        L.orc_cache_new.argtypes = [u32, u32, u64]
        L.orc_cache_new.restype = vp
        L.orc_cache_free.argtypes = [vp]
        L.orc_cache_set_policy.argtypes = [vp, C.c_int]
        L.orc_cache_lookup.argtypes = [vp, vp, u64, C.POINTER(u32), C.POINTER(u64)]
        L.orc_cache_lookup.restype = C.c_int
        L.orc_cache_read.argtypes = [vp, vp, u64, u32, u32, vp]
        L.orc_cache_read.restype = C.c_int
        L.orc_cache_write.argtypes = [vp, vp, u64, u32, u32, vp, C.c_int]
        L.orc_cache_write.restype = C.c_int
        L.orc_cache_flush.argtypes = [vp, vp]
        L.orc_cache_flush.restype = u64
        L.orc_cache_replay.argtypes = [vp, vp, vp, u64, vp]
        L.orc_cache_counters.argtypes = [vp, vp]
        L.orc_cache_wb_log.argtypes = [vp, vp, u64]
        L.orc_cache_wb_log.restype = u64
        L.orc_cache_tags.argtypes = [vp, vp, vp, vp]
        L.orc_cache_line.argtypes = [vp, u64, vp]
        L.orc_share_new.argtypes = [vp, u32]
        L.orc_share_new.restype = vp
        L.orc_share_free.argtypes = [vp]
        L.orc_share_acquire.argtypes = [vp, vp, vp, u64, i32]
        L.orc_share_acquire.restype = i32
        L.orc_share_write.argtypes = [vp, vp, u64, u32, vp, u32]
        L.orc_share_release.argtypes = [vp, vp, vp, u64]
        L.orc_share_release.restype = C.c_int
        L.orc_share_entry.argtypes = [vp, u64, vp]
        L.orc_share_counters.argtypes = [vp, vp]
        L.orc_embedding_bag.argtypes = [vp, u64, u32, vp, vp, u64, vp]
        L.orc_embedding_bag_backward.argtypes = [u64, u32, vp, vp, u64, vp, vp, vp]
        L.orc_sgd.argtypes = [vp, u64, u32, vp, vp, C.c_float]
        L.orc_bfs.argtypes = [u64, vp, vp, i32, vp]
        L.orc_bfs.restype = u64
        L.orc_spmv.argtypes = [u64, vp, vp, vp, vp, vp]
        L.orc_spmv.restype = u64
        L.orc_fma_chain.argtypes = [vp, u64, u32, C.c_float, C.c_float]
        L.orc_ideal_speedup.argtypes = [C.c_double]
        L.orc_ideal_speedup.restype = C.c_double
        _lib = L
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


# ----------------------------------------------------------------------------- store

def store_read_page(store: np.ndarray, page: int) -> np.ndarray:
    out = np.empty(PAGE, dtype=np.uint8)
    lib().orc_store_read_page(_p(store), page, _p(out))
    return out


def store_write_page(store: np.ndarray, page: int, data: np.ndarray) -> None:
    d = _c(data, np.uint8)
    assert d.size == PAGE
    lib().orc_store_write_page(_p(store), page, _p(d))


def set_of(page: int, sets: int) -> int:
    return int(lib().orc_set_of(page, sets))


# ----------------------------------------------------------------------------- cache

class RefCache:
    """Sequential reference cache; ``store`` is a uint8 numpy array the cache reads on
    fills and writes on write-backs (it is modified in place)."""

    CLOCK, FIFO = 0, 1

    def __init__(self, sets: int, ways: int, store: np.ndarray, wb_cap: int = 1 << 20, policy: int = 0):
        assert store.dtype == np.uint8 and store.flags.c_contiguous
        self.sets, self.ways, self.store = sets, ways, store
        self.h = lib().orc_cache_new(sets, ways, wb_cap)
        lib().orc_cache_set_policy(self.h, policy)

    def __del__(self):
        if getattr(self, "h", None):
            lib().orc_cache_free(self.h)
            self.h = None

    def lookup(self, page: int):
        w = C.c_uint32()
        v = C.c_uint64()
        code = lib().orc_cache_lookup(self.h, _p(self.store), page, C.byref(w), C.byref(v))
        return code, int(w.value), int(v.value)

    def read(self, page: int, off: int = 0, length: int = PAGE) -> tuple[int, np.ndarray]:
        out = np.empty(length, dtype=np.uint8)
        code = lib().orc_cache_read(self.h, _p(self.store), page, off, length, _p(out))
        return code, out

    def write(self, page: int, off: int, data: np.ndarray, write_through: bool = False) -> int:
        d = _c(data, np.uint8)
        return lib().orc_cache_write(self.h, _p(self.store), page, off, d.size, _p(d),
                                     1 if write_through else 0)

    def flush(self) -> int:
        return int(lib().orc_cache_flush(self.h, _p(self.store)))

    def replay(self, pages) -> np.ndarray:
        p = _c(pages, np.uint64)
        codes = np.empty(p.size, dtype=np.int32)
        lib().orc_cache_replay(self.h, _p(self.store), _p(p), p.size, _p(codes))
        return codes

    def counters(self) -> dict:
        out = np.zeros(4, dtype=np.uint64)
        lib().orc_cache_counters(self.h, _p(out))
        return dict(hits=int(out[0]), misses=int(out[1]), evictions=int(out[2]),
                    writebacks=int(out[3]))

    def writeback_log(self) -> np.ndarray:
        n = int(lib().orc_cache_wb_log(self.h, None, 0))
        out = np.zeros(max(n, 1), dtype=np.uint64)
        lib().orc_cache_wb_log(self.h, _p(out), n)
        return out[:n]

    def tags(self):
        n = self.sets * self.ways
        page = np.zeros(n, dtype=np.uint64)
        state = np.zeros(n, dtype=np.uint8)
        ref = np.zeros(n, dtype=np.uint8)
        lib().orc_cache_tags(self.h, _p(page), _p(state), _p(ref))
        return page, state, ref

    def line(self, line: int) -> np.ndarray:
        out = np.empty(PAGE, dtype=np.uint8)
        lib().orc_cache_line(self.h, line, _p(out))
        return out


# ----------------------------------------------------------------------------- share table

UB_I, UB_E, UB_S, UB_M, UB_O = 0, 1, 2, 3, 4


class ShareTable:
    """Sequential Share Table (Sec. 3.4.1) over a RefCache; ``bufs`` is a uint8 array of
    4096-byte user buffers named by index (modified in place)."""

    def __init__(self, cache: RefCache, cap: int, bufs: np.ndarray):
        assert bufs.dtype == np.uint8 and bufs.flags.c_contiguous
        self.cache, self.bufs = cache, bufs
        self.h = lib().orc_share_new(cache.h, cap)

    def __del__(self):
        if getattr(self, "h", None):
            lib().orc_share_free(self.h)
            self.h = None

    def acquire(self, page: int, mine: int) -> int:
        return int(lib().orc_share_acquire(self.h, _p(self.cache.store), _p(self.bufs), page, mine))

    def write(self, page: int, off: int, data: np.ndarray) -> None:
        d = _c(data, np.uint8)
        lib().orc_share_write(self.h, _p(self.bufs), page, off, _p(d), d.size)

    def release(self, page: int) -> bool:
        return bool(lib().orc_share_release(self.h, _p(self.cache.store), _p(self.bufs), page))

    def entry(self, page: int):
        out = np.zeros(3, dtype=np.int32)
        lib().orc_share_entry(self.h, page, _p(out))
        return int(out[0]), int(out[1]), int(out[2])

    def counters(self) -> dict:
        out = np.zeros(3, dtype=np.uint64)
        lib().orc_share_counters(self.h, _p(out))
        return dict(store_reads=int(out[0]), cache_copies=int(out[1]), propagations=int(out[2]))


# ----------------------------------------------------------------------------- embedding bag

def embedding_bag(table: np.ndarray, idx: np.ndarray, offsets: np.ndarray) -> np.ndarray:
    t = _c(table, np.float32)
    i = _c(idx, np.int64)
    o = _c(offsets, np.int64)
    rows, dim = t.shape
    nb = o.size - 1
    out = np.empty((nb, dim), dtype=np.float32)
    lib().orc_embedding_bag(_p(t), rows, dim, _p(i), _p(o), nb, _p(out))
    return out


def embedding_bag_backward(rows: int, idx, offsets, gout: np.ndarray):
    g = _c(gout, np.float32)
    i = _c(idx, np.int64)
    o = _c(offsets, np.int64)
    nb, dim = g.shape
    G = np.empty((rows, dim), dtype=np.float32)
    touched = np.empty(rows, dtype=np.uint8)
    lib().orc_embedding_bag_backward(rows, dim, _p(i), _p(o), nb, _p(g), _p(G), _p(touched))
    return G, touched


def sgd(table: np.ndarray, G: np.ndarray, touched: np.ndarray, lr: float) -> np.ndarray:
    t = np.array(table, dtype=np.float32, copy=True, order="C")
    g = _c(G, np.float32)
    tc = _c(touched, np.uint8)
    rows, dim = t.shape
    lib().orc_sgd(_p(t), rows, dim, _p(g), _p(tc), lr)
    return t


# ----------------------------------------------------------------------------- BFS

def bfs(offsets: np.ndarray, cols: np.ndarray, src: int):
    o = _c(offsets, np.int64)
    c = _c(cols, np.int32)
    n = o.size - 1
    level = np.empty(max(n, 1), dtype=np.int32)
    scanned = int(lib().orc_bfs(n, _p(o), _p(c), int(src), _p(level)))
    return level[:n], scanned


def spmv(offsets: np.ndarray, cols: np.ndarray, vals: np.ndarray, x: np.ndarray) -> np.ndarray:
    """y = A x, A in CSR (int64 offsets, int32 cols, float32 vals), FP32 in increasing
    entry order per row."""
    o = _c(offsets, np.int64)
    c = _c(cols, np.int32)
    v = _c(vals, np.float32)
    xv = _c(x, np.float32)
    n = o.size - 1
    y = np.empty(max(n, 1), dtype=np.float32)
    lib().orc_spmv(n, _p(o), _p(c), _p(v), _p(xv), _p(y))
    return y[:n]


FMA_A = 0.999755859375   # 1 - 2^-12
FMA_B = 0.0009765625     # 2^-10


def fma_chain(x: np.ndarray, iters: int, a: float = FMA_A, b: float = FMA_B) -> np.ndarray:
    """Compute phase of the overlap experiment: `iters` rounds of x = fma(x, a, b)."""
    y = np.array(x, dtype=np.float32, copy=True, order="C")
    lib().orc_fma_chain(_p(y), y.size, iters, a, b)
    return y


def embedding_pipeline(tables, idx, pooling: int, iters: int) -> np.ndarray:
    """Lookup batches over several tables followed by the compute phase.

    tables: list of (rows, dim) float32 arrays; idx: int64 [batches, tables, bags, pooling].
    Returns float32 [batches, bags, tables * dim]: the sum-pooled rows of every table,
    concatenated per bag, then `iters` multiply-add rounds per element."""
    nb_t, nt, nbags, pool = idx.shape
    assert pool == pooling and nt == len(tables)
    dim = tables[0].shape[1]
    out = np.empty((nb_t, nbags, nt * dim), dtype=np.float32)
    off = np.arange(nbags + 1, dtype=np.int64) * pooling
    for t in range(nb_t):
        for k in range(nt):
            out[t, :, k * dim:(k + 1) * dim] = embedding_bag(tables[k], idx[t, k].reshape(-1), off)
    return fma_chain(out, iters)


def ideal_speedup(ctc: float) -> float:
    return float(lib().orc_ideal_speedup(ctc))
