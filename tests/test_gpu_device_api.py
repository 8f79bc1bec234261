"""The device-side API (include/agile_device.cuh) used from a user kernel compiled here:
issue a read, continue with other work, test and wait on the request's token with a
bound, then use the data (Listing 1, Sec. 3.5; the transaction barrier of Sec. 3.2.1).

  - reads through the cache deliver the store's bytes, and each wait returns 0;
  - with a device latency of 2 ms every read is still in flight when its token is
    tested right after the request (the warp continued without waiting);
  - with a device latency of 30 ms and waits bounded at 1 ms, every wait returns
    AGILE_ETIMEDOUT through its token, nothing is copied, no error is recorded for the
    context, and a later launch finds the pages resident (the reads were drained).
"""
import ctypes as C
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2504_19365_gb300 as ag  # noqa: E402
from gpu_util import Ctx, build_user_kernel  # noqa: E402

DEV = "cuda:0"


@pytest.fixture(scope="module")
def user_lib():
    L = build_user_kernel("token_demo")
    L.token_demo.restype = C.c_int
    L.token_demo.argtypes = [C.c_void_p] * 6 + [C.c_uint64, C.c_uint32, C.c_void_p, C.c_uint32, C.c_void_p]
    return L


def _store(npages, seed):
    return synth.splitmix64(seed, np.arange(npages * 512, dtype=np.uint64)).view(np.uint8).copy()


def _run(L, c, pages, wait_ns, iters=200, app_warps=0):
    n = len(pages)
    d_pages = torch.from_numpy(np.asarray(pages, dtype=np.uint64).view(np.int64)).to(DEV)
    dst = torch.zeros(n * 4096, dtype=torch.uint8, device=DEV)
    status = torch.full((n,), 99, dtype=torch.int32, device=DEV)
    pending = torch.full((n,), 99, dtype=torch.int32, device=DEV)
    work = torch.zeros(n, dtype=torch.float32, device=DEV)
    rc = L.token_demo(c.h, d_pages.data_ptr(), n, dst.data_ptr(), status.data_ptr(), pending.data_ptr(), wait_ns,
                      iters, work.data_ptr(), app_warps, c.stream)
    assert rc == 0
    torch.cuda.synchronize()
    return (dst.cpu().numpy().reshape(n, 4096), status.cpu().numpy(), pending.cpu().numpy(), work.cpu().numpy())


def test_issue_continue_wait_delivers_pages(user_lib):
    npages = 900
    store = _store(npages, 71)
    pages = synth.uniform_int(72, 2500, npages)   # repeats: merged in a warp, or found in flight
    with Ctx(store.nbytes, cache_bytes=256 * 4096, ways=8, num_queues=16, queue_depth=64) as c:
        c.put(0, store)
        got, status, pending, work = _run(user_lib, c, pages, wait_ns=2_000_000_000)
        c.check()
        assert (status == 0).all()
        for i, p in enumerate(pages):
            assert np.array_equal(got[i], store[p * 4096:(p + 1) * 4096]), i
        assert set(np.unique(pending).tolist()) <= {0, 1}
        assert (work > 0).all()


def test_reads_are_in_flight_after_issue(user_lib):
    npages = 256
    store = _store(npages, 73)
    pages = np.arange(npages, dtype=np.uint64)
    with Ctx(store.nbytes, cache_bytes=512 * 4096, ways=8, num_queues=16, queue_depth=64,
             emu_latency_ns=2_000_000) as c:
        c.put(0, store)
        got, status, pending, _ = _run(user_lib, c, pages, wait_ns=2_000_000_000, app_warps=8)
        c.check()
        assert (pending == 1).all()     # tested right after the request: still in flight
        assert (status == 0).all()
        assert np.array_equal(got.reshape(-1), store)


def test_wait_times_out_through_the_token(user_lib):
    npages = 128
    store = _store(npages, 74)
    pages = np.arange(npages, dtype=np.uint64)
    with Ctx(store.nbytes, cache_bytes=512 * 4096, ways=8, num_queues=16, queue_depth=64,
             emu_latency_ns=30_000_000) as c:
        c.put(0, store)
        got, status, pending, _ = _run(user_lib, c, pages, wait_ns=1_000_000, app_warps=4)
        assert (status == ag.AGILE_ETIMEDOUT).all()
        assert (pending == 1).all()
        assert not got.any()                       # nothing copied
        assert ag.agile_check(c.h) == 0            # the timeout belongs to the caller
        assert c.stats()["commands"] == npages     # the reads were served and drained
        # the pages are now resident: a second launch finds them (hit tokens), at once
        got, status, pending, _ = _run(user_lib, c, pages, wait_ns=1_000_000, app_warps=4)
        c.check()
        assert (status == 0).all() and (pending == 0).all()
        assert np.array_equal(got.reshape(-1), store)


@pytest.fixture(scope="module")
def row_lib():
    L = build_user_kernel("row_demo")
    L.row_demo.restype = C.c_int
    L.row_demo.argtypes = [C.c_void_p] * 4 + [C.c_uint32, C.c_void_p, C.c_uint32, C.c_void_p]
    return L


def _rows(L, c, pages, offs, lens, app_warps=0):
    n = len(pages)
    d_pages = torch.from_numpy(np.asarray(pages, dtype=np.uint64).view(np.int64)).to(DEV)
    d_offs = torch.from_numpy(np.asarray(offs, dtype=np.uint32).view(np.int32)).to(DEV)
    d_lens = torch.from_numpy(np.asarray(lens, dtype=np.uint32).view(np.int32)).to(DEV)
    dst = torch.zeros(n * 4096, dtype=torch.uint8, device=DEV)
    rc = L.row_demo(c.h, d_pages.data_ptr(), d_offs.data_ptr(), d_lens.data_ptr(), n, dst.data_ptr(), app_warps,
                    c.stream)
    assert rc == 0
    torch.cuda.synchronize()
    return dst.cpu().numpy().reshape(n, 4096)


def test_get_row_reads_the_bytes_of_the_row(row_lib):
    # rows of 4-4096 bytes at 4-byte aligned offsets, through a cache of a quarter of the
    # pages (misses, hits and evictions); the rest of each slot stays untouched
    npages = 512
    store = _store(npages, 75)
    n = 3000
    pages = synth.uniform_int(76, n, npages)
    lens = 4 * (synth.uniform_int(77, n, 1024) + 1)
    offs = 4 * np.array([synth.uniform_int(78 + i, 1, (4096 - int(ln)) // 4 + 1)[0] for i, ln in enumerate(lens)])
    with Ctx(store.nbytes, cache_bytes=128 * 4096, ways=8, num_queues=16, queue_depth=64) as c:
        c.put(0, store)
        got = _rows(row_lib, c, pages, offs, lens)
        c.check()
        for i in range(n):
            p, o, ln = int(pages[i]), int(offs[i]), int(lens[i])
            assert np.array_equal(got[i, :ln], store[p * 4096 + o:p * 4096 + o + ln]), i
            assert not got[i, ln:].any(), i
        assert c.stats()["evictions"] > 0


def test_get_row_rejects_a_row_past_the_page(row_lib):
    store = _store(8, 79)
    with Ctx(store.nbytes, cache_bytes=8 * 4096, ways=8, num_queues=4, queue_depth=64) as c:
        c.put(0, store)
        got = _rows(row_lib, c, [3], [4092], [8], app_warps=1)   # 4 bytes past the page
        assert not got.any()
        assert ag.agile_check(c.h) == ag.AGILE_EINVAL
