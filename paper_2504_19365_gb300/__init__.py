"""Thin Python binding of the C-ABI in ``include/agile.h`` (argument marshalling only).

Every function keeps the C name and takes plain integers for device pointers
(``tensor.data_ptr()``) and streams (``torch.cuda.current_stream().cuda_stream``).
All work runs in the CUDA library ``libagile.so``; there is no fallback: importing
the binding without the built library raises at the first call.

Paper: "AGILE: Lightweight and Efficient Asynchronous GPU-SSD Integration"
(arXiv 2504.19365), Sec. 3 (design) and Sec. 4 (evaluation workloads).
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libagile.so")

PAGE_SIZE = 4096
AGILE_OK = 0
AGILE_EIO = -5
AGILE_EAGAIN = -11
AGILE_ENOMEM = -12
AGILE_ENODEV = -19
AGILE_EINVAL = -22
AGILE_ETIMEDOUT = -110
AGILE_ECUDA = -1000
AGILE_SYNC = 0
AGILE_ASYNC = 1
AGILE_FAULT_EIO = 1
AGILE_FAULT_DROP_CQE = 2
AGILE_TOKEN_HIT = (1 << 64) - 1
AGILE_POLICY_CLOCK = 0
AGILE_POLICY_FIFO = 1
AGILE_NO_EXTRA_ENGINES = 0xFFFFFFFF
AGILE_NO_PREFETCH_QUEUES = 0xFFFFFFFF

EXPORTED = [
    "agile_config_default", "agile_init", "agile_destroy", "agile_store_write",
    "agile_store_read", "agile_read_async", "agile_write_async", "agile_wait",
    "agile_prefetch", "agile_flush", "agile_invalidate", "agile_embedding_bag",
    "agile_embedding_bag_backward", "agile_embedding_pipeline", "agile_bfs",
    "agile_bfs_noalloc", "agile_spmv", "agile_serve_start", "agile_serve_submit", "agile_serve_poll",
    "agile_serve_stop", "agile_serve_replay",
    "agile_cache_replay", "agile_cache_tags", "agile_cache_lines", "agile_cache_sets",
    "agile_stats", "agile_reset_stats", "agile_check", "agile_launch_shape", "agile_strerror",
    "agile_config_parallelism", "agile_page_io", "agile_trace", "agile_link_probe", "agile_set_device_model",
    "agile_bfs_hbm", "agile_spmv_hbm", "agile_device_view", "agile_run_reset",
    "agile_share_replay", "agile_lock_order_check", "agile_embedding_bag_hbm", "agile_events",
]


class agile_config(C.Structure):
    _fields_ = [
        ("store_bytes", C.c_uint64),
        ("nvme_path", C.c_char_p),
        ("cache_bytes", C.c_uint64),
        ("ways", C.c_uint32),
        ("num_queues", C.c_uint32),
        ("queue_depth", C.c_uint32),
        ("emu_latency_ns", C.c_uint32),
        ("emu_queue_gbps", C.c_double),
        ("wait_timeout_ns", C.c_uint64),
        ("device", C.c_int32),
        ("fault_flags", C.c_uint32),
        ("fault_rate", C.c_double),
        ("seed", C.c_uint64),
        ("max_ctas", C.c_uint32),
        ("prefetch_depth", C.c_uint32),
        ("app_warps", C.c_uint32),
        ("trace_records", C.c_uint32),
        ("num_devices", C.c_uint32),
        ("cache_policy", C.c_uint32),
        ("emu_device_read_gbps", C.c_double),
        ("emu_device_write_gbps", C.c_double),
        ("share_slots", C.c_uint32),
        ("emu_extra_engines", C.c_uint32),
        ("prefetch_queues", C.c_uint32),
    ]


class agile_trace_rec(C.Structure):
    _fields_ = [
        ("page", C.c_uint64),
        ("t_seen", C.c_uint64),
        ("t_start", C.c_uint64),
        ("t_done", C.c_uint64),
        ("q", C.c_uint32),
        ("cid", C.c_uint32),
        ("opcode", C.c_uint32),
        ("status", C.c_uint32),
        ("t_commit", C.c_uint64),
        ("pad", C.c_uint32 * 2),
    ]


STAT_FIELDS = [
    "hits", "misses", "busy_hits", "warp_coalesced", "share_retries", "evictions",
    "writebacks", "eagain", "sq_full", "doorbells", "commands", "cqes", "cq_doorbells",
    "io_errors", "bytes_read", "bytes_written", "prefetches", "timeouts",
]


class agile_lookup_req(C.Structure):
    _fields_ = [
        ("table_byte0", C.c_uint64),
        ("rows", C.c_uint32),
        ("dim", C.c_uint32),
        ("d_idx", C.c_void_p),
        ("d_offsets", C.c_void_p),
        ("n_bags", C.c_uint32),
        ("d_out", C.c_void_p),
    ]


class agile_stats_t(C.Structure):
    _fields_ = [(f, C.c_uint64) for f in STAT_FIELDS]


class AgileError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"{what}: {code} ({strerror(code)})")
        self.code = code


_lib = None


def lib():
    """Load ``libagile.so``; raise if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(
                f"{LIB_PATH} is missing: build the CUDA library first "
                "(python -c 'import __graft_entry__ as g; g.build()')")
        L = C.CDLL(LIB_PATH)
        vp, u64, u32, i32 = C.c_void_p, C.c_uint64, C.c_uint32, C.c_int32
        cfgp = C.POINTER(agile_config)
        sig = {
            "agile_config_default": (None, [cfgp]),
            "agile_init": (C.c_int, [cfgp, C.POINTER(vp)]),
            "agile_destroy": (C.c_int, [vp]),
            "agile_store_write": (C.c_int, [vp, u64, vp, u64]),
            "agile_store_read": (C.c_int, [vp, u64, vp, u64]),
            "agile_read_async": (C.c_int, [vp, vp, u32, vp, vp, u32, vp]),
            "agile_write_async": (C.c_int, [vp, vp, u32, vp, vp, vp]),
            "agile_wait": (C.c_int, [vp, vp, u32, vp, vp]),
            "agile_prefetch": (C.c_int, [vp, vp, u32, vp]),
            "agile_flush": (C.c_int, [vp, vp]),
            "agile_invalidate": (C.c_int, [vp, vp]),
            "agile_embedding_bag": (C.c_int, [vp, u64, u32, u32, vp, vp, u32, vp, u32, vp]),
            "agile_embedding_bag_backward": (C.c_int, [vp, u64, u32, u32, vp, vp, u32, u32, vp, C.c_float, vp,
                                                       u32, vp]),
            "agile_embedding_pipeline": (C.c_int, [vp, u64, u64, u32, u32, u32, vp, u32, u32, u32, u32, vp, u32,
                                                   vp]),
            "agile_bfs": (C.c_int, [vp, u64, u64, u32, i32, vp, vp, u32, vp]),
            "agile_bfs_noalloc": (C.c_int, [vp, u64, u64, u32, u64, i32, vp, vp, u32, vp]),
            "agile_spmv": (C.c_int, [vp, u64, u64, u64, u32, u32, vp, vp, vp, u32, vp]),
            "agile_cache_replay": (C.c_int, [vp, vp, u32, vp, vp]),
            "agile_cache_tags": (C.c_int, [vp, vp]),
            "agile_cache_lines": (u64, [vp]),
            "agile_cache_sets": (u32, [vp]),
            "agile_stats": (C.c_int, [vp, C.POINTER(agile_stats_t)]),
            "agile_reset_stats": (C.c_int, [vp]),
            "agile_check": (C.c_int, [vp]),
            "agile_launch_shape": (C.c_int, [vp, C.POINTER(u32), C.POINTER(u32)]),
            "agile_config_parallelism": (C.c_int, [vp, u32]),
            "agile_serve_start": (C.c_int, [vp, u32, u32, u64, vp, C.POINTER(vp)]),
            "agile_serve_submit": (C.c_int, [vp, C.POINTER(agile_lookup_req), C.POINTER(u64)]),
            "agile_serve_poll": (C.c_int, [vp, u64]),
            "agile_serve_stop": (C.c_int, [vp]),
            "agile_serve_replay": (C.c_int, [vp, C.POINTER(agile_lookup_req), u32, vp, vp, u32, vp]),
            "agile_strerror": (C.c_char_p, [C.c_int]),
            "agile_page_io": (C.c_int, [vp, u64, u64, vp, vp, vp]),
            "agile_device_view": (C.c_int, [vp, vp, u64]),
            "agile_events": (C.c_int, [vp, vp, u32, C.POINTER(u32)]),
            "agile_share_replay": (C.c_int, [vp, vp, u32, vp, vp, vp]),
            "agile_lock_order_check": (C.c_int, [vp, u64, vp, u32, C.POINTER(u32)]),
            "agile_run_reset": (C.c_int, [vp, vp]),
            "agile_bfs_hbm": (C.c_int, [vp, vp, vp, u32, u64, i32, vp, vp, vp]),
            "agile_embedding_bag_hbm": (C.c_int, [vp, vp, u32, u32, vp, vp, u32, vp, vp]),
            "agile_spmv_hbm": (C.c_int, [vp, vp, vp, vp, u32, u32, u64, vp, vp, vp, vp]),
            "agile_set_device_model": (C.c_int, [vp, u32, u32, C.c_double, C.c_double, C.c_double]),
            "agile_trace": (C.c_int, [vp, vp, u32, C.POINTER(u32)]),
            "agile_link_probe": (C.c_int, [vp, vp, u64, u32, u32, C.POINTER(C.c_double)]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def strerror(code: int) -> str:
    try:
        return lib().agile_strerror(int(code)).decode()
    except Exception:
        return "?"


def _ok(code: int, what: str) -> int:
    if code != 0:
        raise AgileError(code, what)
    return code


# ----------------------------------------------------------------------------- C names

def agile_config_default(**overrides) -> agile_config:
    cfg = agile_config()
    lib().agile_config_default(C.byref(cfg))
    for k, v in overrides.items():
        setattr(cfg, k, v)
    return cfg


def agile_init(cfg: agile_config) -> int:
    h = C.c_void_p()
    _ok(lib().agile_init(C.byref(cfg), C.byref(h)), "agile_init")
    return h.value


def agile_destroy(ctx: int) -> int:
    return _ok(lib().agile_destroy(ctx), "agile_destroy")


def agile_store_write(ctx: int, off: int, host_ptr: int, n: int) -> int:
    return _ok(lib().agile_store_write(ctx, off, host_ptr, n), "agile_store_write")


def agile_store_read(ctx: int, off: int, host_ptr: int, n: int) -> int:
    return _ok(lib().agile_store_read(ctx, off, host_ptr, n), "agile_store_read")


def agile_read_async(ctx, d_pages, n, d_dst, d_tok, mode, stream) -> int:
    return _ok(lib().agile_read_async(ctx, d_pages, n, d_dst, d_tok, mode, stream), "agile_read_async")


def agile_write_async(ctx, d_pages, n, d_src, d_tok, stream) -> int:
    return _ok(lib().agile_write_async(ctx, d_pages, n, d_src, d_tok, stream), "agile_write_async")


def agile_wait(ctx, d_tok, n, d_status, stream) -> int:
    return _ok(lib().agile_wait(ctx, d_tok, n, d_status, stream), "agile_wait")


def agile_prefetch(ctx, d_pages, n, stream) -> int:
    return _ok(lib().agile_prefetch(ctx, d_pages, n, stream), "agile_prefetch")


def agile_flush(ctx, stream) -> int:
    return _ok(lib().agile_flush(ctx, stream), "agile_flush")


def agile_invalidate(ctx, stream) -> int:
    return _ok(lib().agile_invalidate(ctx, stream), "agile_invalidate")


def agile_embedding_bag(ctx, table_byte0, rows, dim, d_idx, d_offsets, n_bags, d_out, mode, stream) -> int:
    return _ok(lib().agile_embedding_bag(ctx, table_byte0, rows, dim, d_idx, d_offsets, n_bags, d_out,
                                         mode, stream), "agile_embedding_bag")


def agile_embedding_bag_backward(ctx, table_byte0, rows, dim, d_idx, d_offsets, n_bags, n_indices, d_grad_out,
                                 lr, d_grad_table, mode, stream) -> int:
    return _ok(lib().agile_embedding_bag_backward(ctx, table_byte0, rows, dim, d_idx, d_offsets, n_bags, n_indices,
                                                  d_grad_out, lr, d_grad_table, mode, stream),
               "agile_embedding_bag_backward")


def agile_embedding_pipeline(ctx, table_byte0, table_stride, n_tables, rows, dim, d_idx, pooling, n_bags, n_batches,
                             compute_iters, d_out, mode, stream) -> int:
    return _ok(lib().agile_embedding_pipeline(ctx, table_byte0, table_stride, n_tables, rows, dim, d_idx, pooling,
                                              n_bags, n_batches, compute_iters, d_out, mode, stream),
               "agile_embedding_pipeline")


def agile_bfs(ctx, offsets_byte0, cols_byte0, n_vertices, src, d_level, d_edges, mode, stream) -> int:
    return _ok(lib().agile_bfs(ctx, offsets_byte0, cols_byte0, n_vertices, src, d_level, d_edges, mode,
                               stream), "agile_bfs")


def agile_spmv(ctx, offsets_byte0, cols_byte0, vals_byte0, n_rows, n_cols, d_x, d_y, d_entries, mode,
               stream) -> int:
    return _ok(lib().agile_spmv(ctx, offsets_byte0, cols_byte0, vals_byte0, n_rows, n_cols, d_x, d_y, d_entries,
                                mode, stream), "agile_spmv")


def agile_embedding_bag_hbm(ctx, d_table, rows, dim, d_idx, d_offsets, n_bags, d_out, stream) -> int:
    """Embedding bag over a table in device memory, no cache (the hit path's ceiling)."""
    return _ok(lib().agile_embedding_bag_hbm(ctx, d_table, rows, dim, d_idx, d_offsets, n_bags, d_out, stream),
               "agile_embedding_bag_hbm")


def agile_bfs_hbm(ctx, d_offsets, d_cols, n_vertices, n_cols, src, d_level, d_edges, stream) -> int:
    """BFS over a CSR in device memory without the cache (Sec. 4.5 kernel time)."""
    return _ok(lib().agile_bfs_hbm(ctx, d_offsets, d_cols, n_vertices, n_cols, src, d_level, d_edges, stream),
               "agile_bfs_hbm")


def agile_spmv_hbm(ctx, d_offsets, d_cols, d_vals, n_rows, n_cols, n_entries, d_x, d_y, d_entries, stream) -> int:
    """SpMV over a CSR in device memory without the cache (Sec. 4.5 kernel time)."""
    return _ok(lib().agile_spmv_hbm(ctx, d_offsets, d_cols, d_vals, n_rows, n_cols, n_entries, d_x, d_y, d_entries,
                                    stream), "agile_spmv_hbm")


def agile_bfs_noalloc(ctx, offsets_byte0, cols_byte0, n_vertices, n_cols, src, d_level, d_edges, mode,
                      stream) -> int:
    """BFS that allocates nothing during the call (scratch in a fixed device array)."""
    return _ok(lib().agile_bfs_noalloc(ctx, offsets_byte0, cols_byte0, n_vertices, n_cols, src, d_level,
                                       d_edges, mode, stream), "agile_bfs_noalloc")


def agile_serve_start(ctx, ring_slots, mode, session_ns, stream) -> int:
    h = C.c_void_p()
    _ok(lib().agile_serve_start(ctx, ring_slots, mode, session_ns, stream, C.byref(h)), "agile_serve_start")
    return h.value


def agile_serve_submit(srv, req: agile_lookup_req):
    """Returns the request's sequence number, or None when the ring is full."""
    q = C.c_uint64()
    r = lib().agile_serve_submit(srv, C.byref(req), C.byref(q))
    if r == AGILE_EAGAIN:
        return None
    _ok(r, "agile_serve_submit")
    return q.value


def agile_serve_poll(srv, seq) -> int:
    r = lib().agile_serve_poll(srv, seq)
    if r < 0:
        _ok(r, "agile_serve_poll")
    return r


def agile_serve_stop(srv) -> int:
    return _ok(lib().agile_serve_stop(srv), "agile_serve_stop")


def agile_serve_replay(ctx, reqs, arrival_ns_ptr, latency_ns_ptr, mode, stream) -> int:
    arr = (agile_lookup_req * len(reqs))(*reqs)
    return _ok(lib().agile_serve_replay(ctx, arr, len(reqs), arrival_ns_ptr, latency_ns_ptr, mode, stream),
               "agile_serve_replay")


def agile_cache_replay(ctx, d_pages, n, d_codes, stream) -> int:
    return _ok(lib().agile_cache_replay(ctx, d_pages, n, d_codes, stream), "agile_cache_replay")


def agile_cache_tags(ctx, host_ptr) -> int:
    return _ok(lib().agile_cache_tags(ctx, host_ptr), "agile_cache_tags")


def agile_cache_lines(ctx) -> int:
    return int(lib().agile_cache_lines(ctx))


def agile_cache_sets(ctx) -> int:
    return int(lib().agile_cache_sets(ctx))


def agile_stats(ctx) -> dict:
    s = agile_stats_t()
    _ok(lib().agile_stats(ctx, C.byref(s)), "agile_stats")
    return {f: int(getattr(s, f)) for f in STAT_FIELDS}


def agile_reset_stats(ctx) -> int:
    return _ok(lib().agile_reset_stats(ctx), "agile_reset_stats")


def agile_check(ctx) -> int:
    """Device-side error since the last check (0 if none); does not raise."""
    return int(lib().agile_check(ctx))


def agile_config_parallelism(ctx, app_warps) -> int:
    return _ok(lib().agile_config_parallelism(ctx, app_warps), "agile_config_parallelism")


def agile_launch_shape(ctx):
    a, b = C.c_uint32(), C.c_uint32()
    _ok(lib().agile_launch_shape(ctx, C.byref(a), C.byref(b)), "agile_launch_shape")
    return a.value, b.value


def agile_set_device_model(ctx, num_devices=1, emu_latency_ns=0, emu_queue_gbps=0.0, emu_device_read_gbps=0.0,
                           emu_device_write_gbps=0.0) -> int:
    return _ok(lib().agile_set_device_model(ctx, num_devices, emu_latency_ns, emu_queue_gbps, emu_device_read_gbps,
                                            emu_device_write_gbps), "agile_set_device_model")


AGILE_LOCK_ACQUIRE, AGILE_LOCK_RELEASE, AGILE_LOCK_TRY = 0, 1, 2


class agile_lock_event(C.Structure):
    _fields_ = [("thread", C.c_uint32), ("op", C.c_uint32), ("lock", C.c_uint64)]


def agile_share_replay(ctx, d_ops, n, d_bufs, d_out, stream) -> int:
    return _ok(lib().agile_share_replay(ctx, d_ops, n, d_bufs, d_out, stream), "agile_share_replay")


def agile_lock_order_check(events):
    """events: (thread, op, lock) triples.  Returns (cycles closed, first cycle's locks)."""
    arr = (agile_lock_event * max(1, len(events)))(*[agile_lock_event(t, o, k) for t, o, k in events])
    cyc = (C.c_uint64 * 64)()
    ln = C.c_uint32()
    r = lib().agile_lock_order_check(arr, len(events), cyc, 64, C.byref(ln))
    if r < 0:
        _ok(r, "agile_lock_order_check")
    return r, [int(cyc[i]) for i in range(min(64, ln.value))]


def agile_device_view(ctx, out_ptr, size) -> int:
    """Copy the context's device view (for kernels built against agile_device.cuh)."""
    return _ok(lib().agile_device_view(ctx, out_ptr, size), "agile_device_view")


def agile_run_reset(ctx, stream) -> int:
    return _ok(lib().agile_run_reset(ctx, stream), "agile_run_reset")


def agile_page_io(ctx, page0: int, n: int):
    """(reads, writes, dirtied) per store page page0 .. page0+n-1, as uint32 numpy arrays."""
    import numpy as np
    r = np.zeros(n, dtype=np.uint32)
    w = np.zeros(n, dtype=np.uint32)
    dt = np.zeros(n, dtype=np.uint32)
    _ok(lib().agile_page_io(ctx, page0, n, r.ctypes.data, w.ctypes.data, dt.ctypes.data), "agile_page_io")
    return r, w, dt


TRACE_DTYPE = [("page", "<u8"), ("t_seen", "<u8"), ("t_start", "<u8"), ("t_done", "<u8"), ("q", "<u4"),
               ("cid", "<u4"), ("opcode", "<u4"), ("status", "<u4"), ("t_commit", "<u8"), ("pad", "<u4", (2,))]


def agile_trace(ctx, cap: int):
    """(records as a numpy structured array, number logged)."""
    import numpy as np
    out = np.zeros(cap, dtype=TRACE_DTYPE)
    n = C.c_uint32()
    _ok(lib().agile_trace(ctx, out.ctypes.data, cap, C.byref(n)), "agile_trace")
    return out[:min(cap, n.value)], n.value


def agile_events(ctx, cap: int):
    """(times ns, warps, kinds, args) of the application event log, and the number logged."""
    import numpy as np
    out = np.zeros(2 * cap, dtype=np.uint64)
    n = C.c_uint32()
    _ok(lib().agile_events(ctx, out.ctypes.data, cap, C.byref(n)), "agile_events")
    k = min(cap, n.value)
    t, w = out[0:2 * k:2], out[1:2 * k:2]
    return (t, (w & np.uint64(0xFFFFFFFF)).astype(np.int64), ((w >> np.uint64(32)) & np.uint64(0xFF)).astype(np.int64),
            (w >> np.uint64(40)).astype(np.int64)), n.value


def agile_link_probe(ctx, d_dst, nbytes, ctas=0, reps=3) -> float:
    g = C.c_double()
    _ok(lib().agile_link_probe(ctx, d_dst, nbytes, ctas, reps, C.byref(g)), "agile_link_probe")
    return g.value


def agile_strerror(code: int) -> str:
    return strerror(code)


# ----------------------------------------------------------------------------- tag word
TAG_STATE_MASK = 3
INVALID, BUSY, READY, MODIFIED = 0, 1, 2, 3


def tag_page(t: int) -> int:
    return int(t) >> 20


def tag_state(t: int) -> int:
    return int(t) & 3


def tag_pins(t: int) -> int:
    return (int(t) >> 4) & 0xFFFF
