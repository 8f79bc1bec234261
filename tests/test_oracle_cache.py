"""Pins for the oracle's page store and sequential reference cache (Sec. 3.4, Sec. 4.4).

Each pin comes from outside the oracle: hand-derived golden traces, closed forms
(cache at least as large as the working set, direct-mapped caches, cyclic thrash under
clock), and the transparency of a cache (after a flush the store must equal the result
of applying every write in order to a plain dictionary of pages).
"""
import os

import numpy as np
import pytest

import oracle
import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _store(pages, seed=11):
    return synth.splitmix64(seed, np.arange(pages * 512, dtype=np.uint64)).view(np.uint8).copy()


def _rows(name):
    out = []
    with open(os.path.join(GOLD, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                out.append(line.split())
    return out


def test_store_roundtrip():
    st = _store(8)
    ref = st.copy()
    assert np.array_equal(oracle.store_read_page(st, 3), ref[3 * 4096:4 * 4096])
    new = np.arange(4096, dtype=np.uint32).astype(np.uint8)
    oracle.store_write_page(st, 5, new)
    ref[5 * 4096:6 * 4096] = new
    assert np.array_equal(st, ref)


def test_golden_clock_trace():
    st = _store(32)
    c = oracle.RefCache(1, 3, st)
    for page, code, way, victim in _rows("clock_trace_1set_3way.txt"):
        got = c.lookup(int(page))
        assert got[0] == int(code) and got[1] == int(way), (page, got)
        if int(victim) >= 0:
            assert got[2] == int(victim)
    assert c.counters() == dict(hits=4, misses=8, evictions=5, writebacks=0)
    pages, state, ref = c.tags()
    assert list(pages) == [11, 12, 10] and list(ref) == [1, 1, 1]
    assert all(s == oracle.READY for s in state)


def test_golden_writeback_trace():
    st = _store(8)
    orig = st.copy()
    c = oracle.RefCache(1, 2, st)
    payload = {}
    for op, page, code, way in _rows("clock_writeback_1set_2way.txt"):
        page = int(page)
        if op == "W":
            data = np.full(4096, page * 3 + 1, dtype=np.uint8)
            payload[page] = data
            got = c.write(page, 0, data)
            assert got == int(code)
        elif op == "R":
            got, out = c.read(page)
            assert got == int(code)
            want = payload.get(page, orig[page * 4096:(page + 1) * 4096])
            assert np.array_equal(out, want)
        else:
            assert c.flush() == 0
    assert list(c.writeback_log()) == [1, 3]
    assert c.counters() == dict(hits=1, misses=5, evictions=3, writebacks=2)
    # the store now holds the written pages, the rest is untouched
    for p in range(8):
        want = payload.get(p, orig[p * 4096:(p + 1) * 4096])
        assert np.array_equal(st[p * 4096:(p + 1) * 4096], want)


@pytest.mark.parametrize("sets,ways", [(1, 8), (4, 4), (16, 8), (7, 3)])
def test_large_cache_misses_equal_distinct_pages(sets, ways):
    # every set has room for every page that maps to it -> misses = distinct pages
    rng_pages = synth.uniform_int(5, 400, 64)
    st = _store(64)
    c = oracle.RefCache(sets, ways, st)
    per_set = {}
    for p in np.unique(rng_pages):
        per_set.setdefault(oracle.set_of(int(p), sets), set()).add(int(p))
    fits = all(len(v) <= ways for v in per_set.values())
    codes = c.replay(rng_pages)
    cnt = c.counters()
    if fits:
        assert cnt["misses"] == len(np.unique(rng_pages))
        assert cnt["evictions"] == 0
    assert cnt["hits"] + cnt["misses"] == len(rng_pages)
    assert (codes == oracle.HIT).sum() == cnt["hits"]


def test_direct_mapped_closed_form():
    # one way per set: a request hits iff the previous request to the same set was
    # for the same page
    pages = synth.uniform_int(9, 3000, 40)
    sets = 8
    c = oracle.RefCache(sets, 1, _store(40))
    codes = c.replay(pages)
    last = {}
    for i, p in enumerate(pages):
        s = oracle.set_of(int(p), sets)
        expect_hit = last.get(s) == int(p)
        assert (codes[i] == oracle.HIT) == expect_hit
        last[s] = int(p)


@pytest.mark.parametrize("ways", [2, 3, 8])
def test_clock_cyclic_thrash(ways):
    # W+1 pages cycled through one W-way set: clock degenerates to FIFO and every
    # request misses
    pages = np.tile(np.arange(ways + 1, dtype=np.uint64), 6)
    c = oracle.RefCache(1, ways, _store(ways + 1))
    codes = c.replay(pages)
    assert (codes != oracle.HIT).all()


def test_set_index_range_and_spread():
    for sets in (1, 3, 128, 425, 131072):
        s = np.array([oracle.set_of(p, sets) for p in range(0, 200000, 97)])
        assert s.min() >= 0 and s.max() < sets
    s = np.array([oracle.set_of(p, 128) for p in range(8192)])
    counts = np.bincount(s, minlength=128)
    assert counts.min() > 0.5 * 64 and counts.max() < 1.5 * 64


@pytest.mark.parametrize("write_through", [False, True])
def test_cache_transparency_random_rw(write_through):
    # A cache is invisible: reads return what a plain dictionary of pages would hold,
    # and after a flush the store equals it byte for byte.
    npages = 48
    st = _store(npages, seed=3)
    truth = {p: st[p * 4096:(p + 1) * 4096].copy() for p in range(npages)}
    c = oracle.RefCache(4, 2, st)
    ops = synth.uniform_int(21, 1500, 4)
    pages = synth.uniform_int(22, 1500, npages)
    offs = synth.uniform_int(23, 1500, 4096 - 64)
    dirty_epochs = 0
    for i in range(1500):
        p, off = int(pages[i]), int(offs[i])
        if ops[i] == 0:
            data = synth.splitmix64(1000 + i, np.arange(8, dtype=np.uint64)).view(np.uint8)
            c.write(p, off, data, write_through)
            truth[p][off:off + 64] = data
        else:
            _, out = c.read(p, off, 64)
            assert np.array_equal(out, truth[p][off:off + 64])
    c.flush()
    for p in range(npages):
        assert np.array_equal(st[p * 4096:(p + 1) * 4096], truth[p])
    cnt = c.counters()
    if write_through:
        assert cnt["writebacks"] == 0
    else:
        # each write-back ends one dirty epoch: never more write-backs than writes
        assert 0 < cnt["writebacks"] <= int((ops == 0).sum())
    page, state, _ = c.tags()
    valid = page[state != oracle.INVALID]
    for s in range(4):
        ways = [page[s * 2 + w] for w in range(2) if state[s * 2 + w] != oracle.INVALID]
        assert len(ways) == len(set(ways)), "duplicate tag in a set"
    assert valid.size <= 8


def test_writeback_exactly_once_per_dirty_epoch():
    # Dirty a page, evict it (write-back 1), dirty it again, flush (write-back 2);
    # untouched pages are never written back.
    st = _store(16)
    c = oracle.RefCache(1, 2, st)
    c.write(5, 0, np.ones(16, np.uint8))
    c.read(6)
    c.read(7)       # evicts 5 (dirty) after clearing both bits
    c.read(8)
    c.write(5, 0, np.full(16, 2, np.uint8))
    assert c.flush() == 1
    assert list(c.writeback_log()) == [5, 5]
    assert c.flush() == 0


# ---------------------------------------------------------------- FIFO policy
# First-in first-out replacement (the policy is the user's choice, Sec. 3.4).  Pins:
# Belady's anomaly (Belady, Nelson and Shedler, CACM 1969), the textbook example in
# which FIFO takes more misses with more frames, and brute force against a per-set
# queue of pages written here.

def test_fifo_belady_anomaly():
    trace = np.array([1, 2, 3, 4, 1, 2, 5, 1, 2, 3, 4, 5], dtype=np.uint64)
    misses = {}
    for ways in (3, 4):
        c = oracle.RefCache(1, ways, _store(8), policy=oracle.RefCache.FIFO)
        codes = c.replay(trace)
        misses[ways] = int((codes != oracle.HIT).sum())
    assert misses == {3: 9, 4: 10}


@pytest.mark.parametrize("sets,ways", [(1, 2), (1, 4), (4, 3), (8, 8)])
def test_fifo_brute_force_queue(sets, ways):
    import collections
    npages = 40
    pages = synth.uniform_int(31, 3000, npages)
    c = oracle.RefCache(sets, ways, _store(npages), policy=oracle.RefCache.FIFO)
    codes = c.replay(pages)
    q = collections.defaultdict(collections.deque)   # per set: pages, oldest first
    for i, p in enumerate(pages.tolist()):
        dq = q[oracle.set_of(p, sets)]
        if p in dq:
            assert codes[i] == oracle.HIT, i
        else:
            assert codes[i] == (oracle.MISS_FILL if len(dq) < ways else oracle.MISS_EVICT), i
            if len(dq) == ways:
                dq.popleft()
            dq.append(p)


def test_fifo_differs_from_clock_on_reuse():
    # 1, 2, 3 fill three ways; 4 replaces 1 (clock: after clearing every reference bit);
    # 2 is used again; 5 must replace a page.  FIFO takes 2 (the oldest fill) although
    # it was just used; clock gives 2 a second chance and takes 3
    trace = np.array([1, 2, 3, 4, 2, 5, 2], dtype=np.uint64)
    fifo = oracle.RefCache(1, 3, _store(8), policy=oracle.RefCache.FIFO).replay(trace)
    clock = oracle.RefCache(1, 3, _store(8)).replay(trace)
    assert fifo[-1] != oracle.HIT
    assert clock[-1] == oracle.HIT
