"""GPU checks of the emulated NVMe device's model, read from its command trace and its
per-page counters.

Sec. 2.1 describes the device side of a queue pair (commands fetched from the
submission ring after a doorbell, completions posted with a phase bit); Sec. 4.3 gives
the device figures the model stands in for (about 3.7 GB/s of 4 KiB random reads and
2.2 GB/s of writes per SSD, requests interleaved over the SSDs).  Here:
  - no command is taken before the configured latency has passed since the device saw
    its doorbell;
  - a queue capped at R GB/s never serves faster than R, and serves at R, within 10 %,
    while it has commands waiting;
  - n devices capped at R each serve about n R together, and a page's command always
    goes to a queue of the page's device (page p on device p mod n);
  - write-backs that leave for another device than the read that replaces them keep
    the store exact and write each dirty epoch exactly once.
"""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2504_19365_gb300 as ag  # noqa: E402
from gpu_util import Ctx, assert_cache_invariants  # noqa: E402

DEV = "cuda:0"


def _store(npages, seed):
    return synth.splitmix64(seed, np.arange(npages * 512, dtype=np.uint64)).view(np.uint8).copy()


def _read(c, pages, mode=ag.AGILE_ASYNC):
    n = len(pages)
    d_pages = torch.from_numpy(np.asarray(pages, dtype=np.uint64).view(np.int64)).to(DEV)
    dst = torch.empty(n * 4096, dtype=torch.uint8, device=DEV)
    ag.agile_read_async(c.h, d_pages.data_ptr(), n, dst.data_ptr(), 0, mode, c.stream)
    torch.cuda.synchronize()
    c.check()
    return dst.cpu().numpy().reshape(n, 4096)


def test_latency_is_respected():
    lat = 300_000   # 300 us
    npages = 512
    store = _store(npages, 51)
    pages = synth.uniform_int(52, 1200, npages)
    with Ctx(store.nbytes, cache_bytes=1024 * 4096, ways=8, num_queues=8, queue_depth=64,
             emu_latency_ns=lat, trace_records=4096) as c:
        c.put(0, store)
        got = _read(c, pages)
        assert all(np.array_equal(got[i], store[p * 4096:(p + 1) * 4096]) for i, p in enumerate(pages))
        tr, n = ag.agile_trace(c.h, 4096)
        assert n == c.stats()["commands"] == len(np.unique(pages)) == tr.size
        assert (tr["t_seen"] > 0).all()
        waited = tr["t_start"].astype(np.int64) - tr["t_seen"].astype(np.int64)
        assert waited.min() >= lat, waited.min()
        assert (tr["t_done"] >= tr["t_start"]).all()


def test_queue_throughput_cap():
    cap = 0.5   # GB/s per queue: 8.2 us a page
    q = 4
    npages = 1600
    store = _store(npages, 53)
    pages = np.arange(npages, dtype=np.uint64)
    with Ctx(store.nbytes, cache_bytes=2048 * 4096, ways=8, num_queues=q, queue_depth=256,
             emu_queue_gbps=cap, trace_records=4096, prefetch_queues=ag.AGILE_NO_PREFETCH_QUEUES) as c:
        c.put(0, store)
        _read(c, pages)
        tr, n = ag.agile_trace(c.h, 4096)
        assert n == npages
        per_page = 4096 / cap   # ns
        for k in range(q):
            sel = tr[tr["q"] == k]
            order = np.argsort(sel["t_start"], kind="stable")
            t = sel["t_start"][order].astype(np.float64)
            seen = sel["t_seen"][order].astype(np.float64)
            assert t.size > 100
            # never faster than the cap over the whole run (one slack window of 16 us)
            assert (t.size - 1) * per_page <= t[-1] - t[0] + 16_000, k
            # while the queue has work waiting (a command seen before the one ahead of it
            # started), it is served at the cap: the mean spacing of those starts is one
            # page time
            back = seen[1:] <= t[:-1]
            assert back.sum() > 50, k
            gap = (t[1:] - t[:-1])[back].mean()
            assert 0.9 * per_page <= gap <= 1.1 * per_page, (k, gap, per_page)


@pytest.mark.parametrize("ndev", [1, 2, 3])
def test_devices_interleave_and_add_up(ndev):
    cap = 2.0   # GB/s of reads per device
    npages = 6000
    store = _store(npages, 54)
    pages = synth.splitmix64(55, np.arange(npages, dtype=np.uint64)) % np.uint64(npages)
    pages = np.unique(pages)
    with Ctx(store.nbytes, cache_bytes=8192 * 4096, ways=8, num_queues=12 * ndev, queue_depth=256,
             num_devices=ndev, emu_device_read_gbps=cap, trace_records=8192) as c:
        c.put(0, store)
        got = _read(c, pages)
        assert all(np.array_equal(got[i], store[p * 4096:(p + 1) * 4096]) for i, p in enumerate(pages))
        tr, n = ag.agile_trace(c.h, 8192)
        assert n == pages.size
        # each command went to a queue of its page's device
        assert ((tr["q"] % ndev) == (tr["page"] % np.uint64(ndev))).all()
        span = float(tr["t_done"].max() - tr["t_start"].min())
        total = pages.size * 4096 / span
        assert 0.85 * ndev * cap <= total <= 1.1 * ndev * cap, total
        for k in range(ndev):
            sel = (tr["page"] % np.uint64(ndev)) == k
            t = np.sort(tr["t_start"][sel]).astype(np.float64)
            assert (t.size - 1) * 4096 / (t[-1] - t[0]) <= 1.1 * cap


def test_device_write_cap():
    cap = 1.0   # GB/s of writes per device
    npages = 1500
    store = _store(npages, 56)
    wp = np.arange(npages, dtype=np.uint64)
    data = synth.splitmix64(57, np.arange(npages * 512, dtype=np.uint64)).view(np.uint8)
    with Ctx(store.nbytes, cache_bytes=2048 * 4096, ways=8, num_queues=16, queue_depth=256, num_devices=2,
             emu_device_write_gbps=cap, trace_records=4096) as c:
        c.put(0, store)
        d_pages = torch.from_numpy(wp.view(np.int64)).to(DEV)
        src = torch.from_numpy(data.copy()).to(DEV)
        ag.agile_write_async(c.h, d_pages.data_ptr(), npages, src.data_ptr(), 0, c.stream)
        torch.cuda.synchronize()
        c.check()
        tr, _ = ag.agile_trace(c.h, 4096)   # the writes of the call itself
        w = tr[tr["opcode"] == 1]
        assert w.size > npages // 2
        for k in range(2):
            t = np.sort(w["t_start"][(w["page"] % np.uint64(2)) == k]).astype(np.float64)
            rate = (t.size - 1) * 4096 / (t[-1] - t[0])
            assert 0.85 * cap <= rate <= 1.1 * cap, (k, rate)
        # a write that found no free slot stays in its MODIFIED line until a flush
        ag.agile_flush(c.h, c.stream)
        torch.cuda.synchronize()
        c.check()
        assert np.array_equal(c.get(0, store.nbytes), data)
        _, writes, dirtied = ag.agile_page_io(c.h, 0, npages)
        assert (writes == 1).all() and (dirtied == 1).all()


@pytest.mark.parametrize("mode", [ag.AGILE_SYNC, ag.AGILE_ASYNC])
def test_writebacks_across_devices_exact_and_once(mode):
    # SGD rows through a cache of 1/8 of the table with the pages on two devices: a
    # MODIFIED victim and the page that replaces it are on different devices about half
    # of the time (the write-back then leaves on the victim's device)
    rows, dim = 8192, 128
    T = synth.table_normal(58, rows, dim)
    idx = synth.Zipf(rows, 1.05, permute=True, seed=59).rows(60, 1000 * 20)
    off = synth.bags_fixed(1000, 20)
    gout = synth.table_normal(61, 1000, dim)
    lr = 2.0 ** -6
    G, touched = oracle.embedding_bag_backward(rows, idx, off, gout)
    want = oracle.sgd(T, G, touched, lr)
    with Ctx(T.nbytes, cache_bytes=T.nbytes // 8, ways=8, num_queues=32, queue_depth=128, num_devices=2) as c:
        c.put(0, T)
        d_idx = torch.from_numpy(idx).to(DEV)
        d_off = torch.from_numpy(off).to(DEV)
        d_g = torch.from_numpy(gout).to(DEV)
        ag.agile_embedding_bag_backward(c.h, 0, rows, dim, d_idx.data_ptr(), d_off.data_ptr(), 1000, idx.size,
                                        d_g.data_ptr(), lr, 0, mode, c.stream)
        ag.agile_flush(c.h, c.stream)
        torch.cuda.synchronize()
        c.check()
        got = c.get(0, T.nbytes).view(np.float32).reshape(rows, dim)
        assert np.array_equal(got.view(np.uint32), want.view(np.uint32))
        _, writes, dirtied = ag.agile_page_io(c.h, 0, T.nbytes // 4096)
        assert np.array_equal(writes, dirtied) and writes.sum() > 0
        assert c.stats()["evictions"] > 0
        assert_cache_invariants(c)


def test_model_switch_between_calls():
    # one context: no model, then an SSD-like model (latency 200 us, 2 devices capped at
    # 3 GB/s), then no model again; every read is right and the latency holds in between
    npages = 1200
    store = _store(npages, 62)
    with Ctx(store.nbytes, cache_bytes=2048 * 4096, ways=8, num_queues=16, queue_depth=64,
             trace_records=4096) as c:
        c.put(0, store)
        parts = np.array_split(np.arange(npages, dtype=np.uint64), 3)
        got = _read(c, parts[0])
        assert np.array_equal(got.reshape(-1), store[:parts[0].size * 4096])
        ag.agile_set_device_model(c.h, num_devices=2, emu_latency_ns=200_000, emu_device_read_gbps=3.0)
        ag.agile_reset_stats(c.h)
        got = _read(c, parts[1])
        assert np.array_equal(got.reshape(-1), store[parts[1][0] * 4096:(parts[1][-1] + 1) * 4096])
        tr, n = ag.agile_trace(c.h, 4096)
        assert n == parts[1].size
        assert ((tr["t_start"].astype(np.int64) - tr["t_seen"].astype(np.int64)) >= 200_000).all()
        assert ((tr["q"] % 2) == (tr["page"] % np.uint64(2))).all()
        ag.agile_set_device_model(c.h)
        got = _read(c, parts[2])
        assert np.array_equal(got.reshape(-1), store[parts[2][0] * 4096:])


def test_demand_queues_are_served_before_prefetch_queues():
    # the lookup + compute pipeline in async mode requests rows ahead (prefetch queues)
    # and waits for the rows it sums (demand queues); with the device saturated (one
    # device capped at 1 GB/s), demand commands wait less for the device than prefetches
    nt, rows, dim, nbags, pool = 2, 200_000, 64, 512, 16
    stride = 200_000 * dim * 4
    tabs = [np.array(synth.table_normal(70 + k, rows, dim)) for k in range(nt)]
    idx = synth.indices_uniform(72, nt * nbags * pool, rows).reshape(1, nt, nbags, pool)
    # 32 queues of depth 64: room for more than the 32 warps' own groups of 32 rows, so
    # the asynchronous call keeps its lookahead
    with Ctx(stride * nt, cache_bytes=4096 * 4096, ways=8, num_queues=32, queue_depth=64,
             emu_device_read_gbps=1.0, trace_records=65536) as c:
        for k in range(nt):
            c.put(k * stride, tabs[k])
        d_idx = torch.from_numpy(idx).to(DEV)
        out = torch.empty((1, nbags, nt * dim), dtype=torch.float32, device=DEV)
        ag.agile_config_parallelism(c.h, 32)
        ag.agile_embedding_pipeline(c.h, 0, stride, nt, rows, dim, d_idx.data_ptr(), pool, nbags, 1, 8,
                                    out.data_ptr(), ag.AGILE_ASYNC, c.stream)
        torch.cuda.synchronize()
        c.check()
        assert np.array_equal(out.cpu().numpy().view(np.uint32),
                              oracle.embedding_pipeline(tabs, idx, pool, 8).view(np.uint32))
        tr, n = ag.agile_trace(c.h, 65536)
        assert n == tr.size
        wait = tr["t_start"].astype(np.int64) - tr["t_seen"].astype(np.int64)
        pf = tr["q"] >= 16                     # queues 16..31 carry the prefetches
        assert pf.sum() > 100 and (~pf).sum() > 100
        assert wait[~pf].mean() < wait[pf].mean(), (wait[~pf].mean(), wait[pf].mean())
