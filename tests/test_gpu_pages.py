"""GPU parity of the page path: asyncRead / asyncWrite / wait / prefetch / flush through
the HBM cache and the emulated NVMe queues, against the oracle's page store and its
sequential reference cache (Sec. 3.2-3.4)."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2504_19365_gb300 as ag  # noqa: E402
from gpu_util import Ctx, assert_cache_invariants, tag_fields  # noqa: E402

DEV = "cuda:0"


def _store(npages, seed=1):
    return synth.splitmix64(seed, np.arange(npages * 512, dtype=np.uint64)).view(np.uint8).copy()


def _read(c, pages, mode):
    n = len(pages)
    d_pages = torch.from_numpy(np.asarray(pages, dtype=np.uint64).view(np.int64)).to(DEV)
    dst = torch.empty(n * 4096, dtype=torch.uint8, device=DEV)
    tok = torch.zeros(n, dtype=torch.int64, device=DEV)
    st = torch.full((n,), 7, dtype=torch.int32, device=DEV)
    ag.agile_read_async(c.h, d_pages.data_ptr(), n, dst.data_ptr(), tok.data_ptr(), mode, c.stream)
    ag.agile_wait(c.h, tok.data_ptr(), n, st.data_ptr(), c.stream)
    torch.cuda.synchronize()
    c.check()
    return dst.cpu().numpy().reshape(n, 4096), tok.cpu().numpy().view(np.uint64), st.cpu().numpy()


@pytest.mark.parametrize("mode", [ag.AGILE_SYNC, ag.AGILE_ASYNC])
def test_read_pages_byte_equal_store(mode):
    npages = 700
    store = _store(npages)
    pages = synth.uniform_int(5, 3000, npages)   # many repeats: hits, in-flight attaches
    with Ctx(store.nbytes, cache_bytes=64 * 4096, ways=8, num_queues=16, queue_depth=64) as c:
        c.put(0, store)
        got, tok, st = _read(c, pages, mode)
        for i, p in enumerate(pages):
            assert np.array_equal(got[i], oracle.store_read_page(store, int(p))), i
        assert (st == 0).all()
        s = c.stats()
        assert s["misses"] >= 1
        assert s["cqes"] == s["commands"] and s["io_errors"] == 0
        assert s["bytes_read"] == 4096 * s["misses"]
        assert_cache_invariants(c)


def test_cache_larger_than_working_set_misses_equal_distinct_pages():
    npages = 200
    store = _store(npages, 2)
    pages = synth.uniform_int(6, 2000, npages)
    # 4096 lines: every set has room for every page that maps to it
    with Ctx(store.nbytes, cache_bytes=4096 * 4096, ways=8, num_queues=8, queue_depth=64) as c:
        c.put(0, store)
        got, _, _ = _read(c, pages, ag.AGILE_ASYNC)
        assert all(np.array_equal(got[i], store[p * 4096:(p + 1) * 4096]) for i, p in enumerate(pages))
        s = c.stats()
        assert s["misses"] == len(np.unique(pages)) and s["evictions"] == 0


@pytest.mark.parametrize("sets,ways", [(1, 4), (8, 2), (16, 8), (5, 3)])
def test_single_thread_replay_equals_reference_cache(sets, ways):
    # With one request in flight the GPU cache must make the oracle's decisions:
    # same hit / fill / eviction sequence and the same final tags and reference bits.
    npages = 64
    store = _store(npages, 3)
    trace = np.concatenate([synth.uniform_int(7, 400, npages),
                            np.tile(np.arange(ways + 1), 5)]).astype(np.uint64)
    ref = oracle.RefCache(sets, ways, store.copy())
    want = ref.replay(trace)
    with Ctx(store.nbytes, cache_bytes=sets * ways * 4096, ways=ways, num_queues=4, queue_depth=64) as c:
        c.put(0, store)
        d_pages = torch.from_numpy(trace.view(np.int64)).to(DEV)
        codes = torch.full((len(trace),), -1, dtype=torch.int32, device=DEV)
        ag.agile_cache_replay(c.h, d_pages.data_ptr(), len(trace), codes.data_ptr(), c.stream)
        torch.cuda.synchronize()
        c.check()
        got = codes.cpu().numpy()
        assert np.array_equal(got, want), np.nonzero(got != want)[0][:10]
        page, state, refbit, pins = tag_fields(c.tags())
        opage, ostate, oref = ref.tags()
        valid = ostate != 0
        assert np.array_equal(state != 0, valid)
        assert np.array_equal(page[valid], opage[valid])
        assert np.array_equal(refbit[valid].astype(np.uint8), oref[valid])
        cnt = ref.counters()
        s = c.stats()
        assert (s["hits"], s["misses"], s["evictions"]) == (cnt["hits"], cnt["misses"], cnt["evictions"])


def test_write_then_read_then_flush_store_equals_oracle():
    npages = 300
    store = _store(npages, 4)
    truth = store.copy()
    wpages = np.unique(synth.uniform_int(8, 150, npages)).astype(np.uint64)
    data = synth.splitmix64(99, np.arange(len(wpages) * 512, dtype=np.uint64)).view(np.uint8)
    data = data.reshape(len(wpages), 4096)
    for k, p in enumerate(wpages):
        oracle.store_write_page(truth, int(p), data[k])
    with Ctx(store.nbytes, cache_bytes=32 * 4096, ways=4, num_queues=8, queue_depth=64) as c:
        c.put(0, store)
        d_pages = torch.from_numpy(wpages.view(np.int64)).to(DEV)
        src = torch.from_numpy(data.reshape(-1).copy()).to(DEV)
        tok = torch.zeros(len(wpages), dtype=torch.int64, device=DEV)
        st = torch.full((len(wpages),), 7, dtype=torch.int32, device=DEV)
        ag.agile_write_async(c.h, d_pages.data_ptr(), len(wpages), src.data_ptr(), tok.data_ptr(), c.stream)
        ag.agile_wait(c.h, tok.data_ptr(), len(wpages), st.data_ptr(), c.stream)
        torch.cuda.synchronize()
        c.check()
        assert (st.cpu().numpy() == 0).all()
        # reads see the new data whether the line is still cached or re-read from the store
        rp = synth.uniform_int(9, 1000, npages)
        got, _, _ = _read(c, rp, ag.AGILE_ASYNC)
        for i, p in enumerate(rp):
            assert np.array_equal(got[i], truth[p * 4096:(p + 1) * 4096]), (i, p)
        ag.agile_flush(c.h, c.stream)
        torch.cuda.synchronize()
        c.check()
        assert np.array_equal(c.get(0, store.nbytes), truth)
        s = c.stats()
        assert s["bytes_written"] == 4096 * s["writebacks"]
        # every page written once by the device: one write per page write (or per
        # dirty epoch of a page whose write found no queue slot), none for other pages
        _, writes, dirtied = ag.agile_page_io(c.h, 0, npages)
        assert np.array_equal(writes, dirtied)
        mask = np.zeros(npages, dtype=bool)
        mask[wpages.astype(np.int64)] = True
        assert (writes[mask] == 1).all() and (writes[~mask] == 0).all()
        assert_cache_invariants(c)


@pytest.mark.parametrize("policy", [ag.AGILE_POLICY_CLOCK, ag.AGILE_POLICY_FIFO])
@pytest.mark.parametrize("ndev", [1, 3])
def test_replay_with_policy_and_devices_equals_reference_cache(policy, ndev):
    # the same single-request replay for each replacement policy, with the pages spread
    # over one or three backing devices (where a page lives changes no decision)
    sets, ways, npages = 4, 4, 64
    store = _store(npages, 13)
    trace = np.concatenate([synth.uniform_int(17, 500, npages), np.tile(np.arange(ways + 1), 4),
                            np.array([1, 2, 3, 4, 2, 5, 2] * 3)]).astype(np.uint64)
    ref = oracle.RefCache(sets, ways, store.copy(), policy=policy)
    want = ref.replay(trace)
    with Ctx(store.nbytes, cache_bytes=sets * ways * 4096, ways=ways, num_queues=6, queue_depth=64,
             cache_policy=policy, num_devices=ndev) as c:
        c.put(0, store)
        d_pages = torch.from_numpy(trace.view(np.int64)).to(DEV)
        codes = torch.full((len(trace),), -1, dtype=torch.int32, device=DEV)
        ag.agile_cache_replay(c.h, d_pages.data_ptr(), len(trace), codes.data_ptr(), c.stream)
        torch.cuda.synchronize()
        c.check()
        got = codes.cpu().numpy()
        assert np.array_equal(got, want), np.nonzero(got != want)[0][:10]
        page, state, _, _ = tag_fields(c.tags())
        opage, ostate, _ = ref.tags()
        valid = ostate != 0
        assert np.array_equal(state != 0, valid)
        assert np.array_equal(page[valid], opage[valid])


@pytest.mark.parametrize("mode", [ag.AGILE_SYNC, ag.AGILE_ASYNC])
def test_tiny_ring_and_tiny_cache_finish(mode):
    # Sec. 2.3.1 / 2.3.2 deadlock scenarios: one queue of depth 64 (at most 63 commands
    # outstanding) and a 1-set x 2-way cache, with every app warp of the grid asking for
    # many pages.  Completions are consumed by the service warps, and no thread waits
    # while it holds a line or a slot, so the call must finish with correct bytes.
    npages = 64
    store = _store(npages, 5)
    pages = synth.uniform_int(10, 5000, npages)
    with Ctx(store.nbytes, cache_bytes=2 * 4096, ways=2, num_queues=1, queue_depth=64,
             wait_timeout_ns=20_000_000_000, max_ctas=8) as c:
        c.put(0, store)
        got, _, st = _read(c, pages, mode)
        for i, p in enumerate(pages):
            assert np.array_equal(got[i], store[p * 4096:(p + 1) * 4096])
        assert (st == 0).all()
        s = c.stats()
        assert s["cqes"] == s["commands"]
        # the CQ head doorbell is written once per full 32-entry window (Alg. 1)
        assert s["cq_doorbells"] == s["cqes"] // 32


def test_prefetch_then_read_hits():
    npages = 128
    store = _store(npages, 6)
    pages = np.arange(0, 64, dtype=np.uint64)
    with Ctx(store.nbytes, cache_bytes=1024 * 4096, ways=8, num_queues=8, queue_depth=64) as c:
        c.put(0, store)
        d_pages = torch.from_numpy(pages.view(np.int64)).to(DEV)
        ag.agile_prefetch(c.h, d_pages.data_ptr(), len(pages), c.stream)
        torch.cuda.synchronize()
        c.check()
        ag.agile_reset_stats(c.h)
        got, tok, _ = _read(c, pages, ag.AGILE_SYNC)
        s = c.stats()
        assert s["misses"] == 0 and s["hits"] >= len(pages)
        assert (tok == ag.AGILE_TOKEN_HIT).all()
        for i, p in enumerate(pages):
            assert np.array_equal(got[i], store[p * 4096:(p + 1) * 4096])


def test_injected_io_errors_are_retried_and_counted():
    npages = 256
    store = _store(npages, 7)
    pages = synth.uniform_int(11, 2000, npages)
    with Ctx(store.nbytes, cache_bytes=64 * 4096, ways=8, num_queues=8, queue_depth=64,
             fault_flags=ag.AGILE_FAULT_EIO, fault_rate=0.05, seed=3) as c:
        c.put(0, store)
        got, _, _ = _read(c, pages, ag.AGILE_ASYNC)
        for i, p in enumerate(pages):
            assert np.array_equal(got[i], store[p * 4096:(p + 1) * 4096])
        s = c.stats()
        assert s["io_errors"] > 0


def test_dropped_completion_times_out_without_hanging():
    # The emulated device never posts some completions: the bounded waits expire, the
    # call returns, the error is reported on the host and the GPU stays usable.
    npages = 64
    store = _store(npages, 8)
    pages = np.arange(npages, dtype=np.uint64)
    with Ctx(store.nbytes, cache_bytes=128 * 4096, ways=8, num_queues=4, queue_depth=64,
             fault_flags=ag.AGILE_FAULT_DROP_CQE, fault_rate=0.5, seed=5,
             wait_timeout_ns=200_000_000) as c:
        c.put(0, store)
        d_pages = torch.from_numpy(pages.view(np.int64)).to(DEV)
        dst = torch.empty(npages * 4096, dtype=torch.uint8, device=DEV)
        ag.agile_read_async(c.h, d_pages.data_ptr(), npages, dst.data_ptr(), 0, ag.AGILE_ASYNC, c.stream)
        torch.cuda.synchronize()
        assert ag.agile_check(c.h) == ag.AGILE_ETIMEDOUT
        assert c.stats()["timeouts"] >= 1
    # the device is still healthy
    x = torch.arange(10, device=DEV)
    assert int(x.sum().item()) == 45
