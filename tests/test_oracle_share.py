"""Pins of the oracle's Share Table (Sec. 3.4.1), from outside the oracle: a hand-derived
trace (tests/golden/share_trace_1set_2way.txt), and a brute-force transparency check
against a plain dictionary of page contents: every acquire returns the bytes the page
holds at that moment (the latest write to a shared buffer, else what the cache or the
store holds), and after the last release and a flush the store equals the dictionary."""
import os

import numpy as np

import oracle
import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")
STATES = {"I": oracle.UB_I, "E": oracle.UB_E, "S": oracle.UB_S, "M": oracle.UB_M, "O": oracle.UB_O}


def _store(npages, seed=1):
    return synth.splitmix64(seed, np.arange(npages * 512, dtype=np.uint64)).view(np.uint8).copy()


def test_golden_share_trace():
    store = _store(16)
    orig = store.copy()
    bufs = np.zeros((4, 4096), dtype=np.uint8)
    cache = oracle.RefCache(1, 2, store)
    st = oracle.ShareTable(cache, 8, bufs)
    aa = np.full(16, 0xAA, dtype=np.uint8)
    rows = [ln.split() for ln in open(os.path.join(GOLD, "share_trace_1set_2way.txt"))
            if ln.strip() and not ln.startswith("#")]
    for op, page, buf, ret, state, count in rows:
        page = int(page)
        if op == "a":
            assert st.acquire(page, int(buf)) == int(ret)
        elif op == "w":
            st.write(page, 0, aa)
        else:
            st.release(page)
        s, n, _ = st.entry(page)
        assert (s, n) == (STATES[state], int(count)), (op, page)
    assert st.counters() == dict(store_reads=2, cache_copies=1, propagations=1)
    # buffers: b0 = p5 with AA in front, b2 = p7, b3 = b0 (read back from the cache line)
    want5 = orig[5 * 4096:6 * 4096].copy()
    want5[:16] = 0xAA
    assert np.array_equal(bufs[0], want5) and np.array_equal(bufs[3], want5)
    assert np.array_equal(bufs[2], orig[7 * 4096:8 * 4096])
    assert not bufs[1].any()                      # shared by pointer: b1 never written
    assert np.array_equal(store, orig)            # nothing reached the store yet
    assert cache.flush() == 1 and list(cache.writeback_log()) == [5]
    assert np.array_equal(store[5 * 4096:6 * 4096], want5)


def test_one_user_modified_goes_to_cache_on_release():
    store = _store(8, 2)
    bufs = np.zeros((2, 4096), dtype=np.uint8)
    cache = oracle.RefCache(2, 2, store)
    st = oracle.ShareTable(cache, 4, bufs)
    assert st.acquire(3, 1) == 1 and st.entry(3)[:2] == (oracle.UB_E, 1)
    st.write(3, 100, np.arange(8, dtype=np.uint8))
    assert st.entry(3)[:2] == (oracle.UB_M, 1)
    assert st.release(3) is True and st.entry(3)[:2] == (oracle.UB_I, 0)
    assert cache.flush() == 1
    assert np.array_equal(store[3 * 4096 + 100:3 * 4096 + 108], np.arange(8, dtype=np.uint8))


def test_transparency_brute_force():
    npages, nbufs = 12, 64
    store = _store(npages, 3)
    truth = {p: store[p * 4096:(p + 1) * 4096].copy() for p in range(npages)}
    bufs = np.zeros((nbufs, 4096), dtype=np.uint8)
    cache = oracle.RefCache(2, 2, store)
    st = oracle.ShareTable(cache, nbufs, bufs)
    held = {}            # page -> references held by the test's "threads"
    free = list(range(nbufs))
    inuse = {}           # page -> buffer index while an entry exists
    ops = synth.uniform_int(81, 3000, 3)
    pages = synth.uniform_int(82, 3000, npages)
    offs = synth.uniform_int(83, 3000, 4096 - 32)
    for i in range(3000):
        p, op = int(pages[i]), int(ops[i])
        if op == 0 or p not in held:                      # acquire
            mine = inuse.get(p, free[-1])
            got = st.acquire(p, mine)
            if p not in inuse:
                assert got == mine
                free.pop()
                inuse[p] = got
            assert got == inuse[p]
            assert np.array_equal(bufs[got], truth[p]), i
            held[p] = held.get(p, 0) + 1
        elif op == 1:                                     # write through a held reference
            data = synth.splitmix64(1000 + i, np.arange(4, dtype=np.uint64)).view(np.uint8)
            st.write(p, int(offs[i]), data)
            truth[p][int(offs[i]):int(offs[i]) + 32] = data
        else:                                             # release
            st.release(p)
            held[p] -= 1
            if held[p] == 0:
                del held[p]
                free.append(inuse.pop(p))
    for p in list(held):
        for _ in range(held[p]):
            st.release(p)
    cache.flush()
    for p in range(npages):
        assert np.array_equal(store[p * 4096:(p + 1) * 4096], truth[p]), p
