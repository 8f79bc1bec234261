"""GPU parity of the Share Table (Sec. 3.4.1) against the oracle's sequential Share Table.

  - served by one GPU thread, a sequence of acquire / write / release makes the
    oracle's decisions: the same buffer returned, the same entry states and counts, the
    same buffer bytes, and after a flush the same store (the hand-derived golden trace
    and seeded random sequences over a 2-way cache);
  - concurrently, from a user kernel: requests for one page held at the same time share
    one buffer (one store read per page, none of the other buffers written), a write by
    the buffer's owner is seen by every sharer through the shared pointer, and the last
    release carries it into the cache, from where a flush writes it to the store once.
"""
import ctypes as C
import os

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2504_19365_gb300 as ag  # noqa: E402
from gpu_util import Ctx, build_user_kernel, tag_fields  # noqa: E402

DEV = "cuda:0"
GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _store(npages, seed):
    return synth.splitmix64(seed, np.arange(npages * 512, dtype=np.uint64)).view(np.uint8).copy()


def _replay_both(store, sets, ways, nbufs, ops):
    """Run ops = [(op, page, a, b)] on the GPU (one thread) and on the oracle."""
    ref_store = store.copy()
    cache = oracle.RefCache(sets, ways, ref_store)
    bufs = np.zeros((nbufs, 4096), dtype=np.uint8)
    st = oracle.ShareTable(cache, 64, bufs)
    want = []
    for op, page, a, b in ops:
        if op == 0:
            ret = st.acquire(page, a)
        elif op == 1:
            st.write(page, a, np.full(16, b, dtype=np.uint8))
            ret = -1
        else:
            ret = int(st.release(page))
        s_, n_, _ = st.entry(page)
        want.append((ret, s_, n_))
    with Ctx(store.nbytes, cache_bytes=sets * ways * 4096, ways=ways, num_queues=4, queue_depth=64,
             share_slots=64) as c:
        c.put(0, store)
        d_ops = torch.tensor(np.array(ops, dtype=np.int32).reshape(-1), device=DEV)
        d_bufs = torch.zeros(nbufs * 4096, dtype=torch.uint8, device=DEV)
        d_out = torch.full((len(ops) * 3,), -9, dtype=torch.int32, device=DEV)
        ag.agile_share_replay(c.h, d_ops.data_ptr(), len(ops), d_bufs.data_ptr(), d_out.data_ptr(), c.stream)
        torch.cuda.synchronize()
        c.check()
        got = [tuple(r) for r in d_out.cpu().numpy().reshape(-1, 3).tolist()]
        assert got == want, next((i, g, w) for i, (g, w) in enumerate(zip(got, want)) if g != w)
        assert np.array_equal(d_bufs.cpu().numpy().reshape(nbufs, 4096), bufs)
        # the cache decided as the oracle's: same pages, states and reference bits
        page, state, refbit, pins = tag_fields(c.tags())
        opage, ostate, oref = cache.tags()
        valid = ostate != 0
        assert np.array_equal(state != 0, valid) and (pins == 0).all()
        assert np.array_equal(page[valid], opage[valid]) and np.array_equal(state[valid], ostate[valid])
        assert np.array_equal(refbit[valid].astype(np.uint8), oref[valid])
        ag.agile_flush(c.h, c.stream)
        torch.cuda.synchronize()
        cache.flush()
        assert np.array_equal(c.get(0, store.nbytes), ref_store)


def test_golden_trace_on_the_gpu():
    codes = {"a": 0, "w": 1, "r": 2}
    ops = []
    for ln in open(os.path.join(GOLD, "share_trace_1set_2way.txt")):
        if not ln.strip() or ln.startswith("#"):
            continue
        op, page, buf = ln.split()[:3]
        if op == "a":
            ops.append((0, int(page), int(buf), 0))
        elif op == "w":
            ops.append((1, int(page), 0, 0xAA))
        else:
            ops.append((2, int(page), 0, 0))
    _replay_both(_store(16, 91), 1, 2, 4, ops)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_random_sequences_match_the_oracle(seed):
    npages, nbufs = 10, 48
    ops, held, inuse, free = [], {}, {}, list(range(nbufs))
    kinds = synth.uniform_int(100 + seed, 400, 3)
    pages = synth.uniform_int(200 + seed, 400, npages)
    offs = synth.uniform_int(300 + seed, 400, 255) * 16
    for i in range(400):
        p, k = int(pages[i]), int(kinds[i])
        if k == 0 or p not in held:
            mine = inuse.get(p, free[-1] if free else 0)
            if p not in inuse:
                free.pop()
                inuse[p] = mine
            ops.append((0, p, mine, 0))
            held[p] = held.get(p, 0) + 1
        elif k == 1:
            ops.append((1, p, int(offs[i]), (i * 37) & 0xFF))
        else:
            ops.append((2, p, 0, 0))
            held[p] -= 1
            if held[p] == 0:
                del held[p]
                free.append(inuse.pop(p))
    for p, cnt in held.items():
        ops += [(2, p, 0, 0)] * cnt
    _replay_both(_store(npages, 92 + seed), 2, 2, nbufs, ops)


@pytest.fixture(scope="module")
def share_lib():
    L = build_user_kernel("share_demo")
    L.share_demo.restype = C.c_int
    L.share_demo.argtypes = [C.c_void_p, C.c_void_p, C.c_uint32] + [C.c_void_p] * 6
    return L


@pytest.mark.parametrize("cached", [False, True])
def test_concurrent_sharing_from_a_user_kernel(share_lib, cached):
    npages, n = 64, 2000
    store = _store(npages, 95)
    pages = synth.uniform_int(96, n, npages).astype(np.uint64)
    with Ctx(store.nbytes, cache_bytes=128 * 4096, ways=8, num_queues=16, queue_depth=64, share_slots=256) as c:
        c.put(0, store)
        if cached:   # every page resident: the buffers are filled from the cache
            d_p = torch.from_numpy(np.arange(npages, dtype=np.int64)).to(DEV)
            ag.agile_prefetch(c.h, d_p.data_ptr(), npages, c.stream)
            torch.cuda.synchronize()
        ag.agile_reset_stats(c.h)
        bufs = torch.zeros(n * 4096, dtype=torch.uint8, device=DEV)
        used = torch.full((n,), -7, dtype=torch.int32, device=DEV)
        first8 = torch.zeros(n, dtype=torch.int64, device=DEV)
        seen = torch.zeros(n, dtype=torch.int32, device=DEV)
        prop = torch.full((n,), -7, dtype=torch.int32, device=DEV)
        d_pages = torch.from_numpy(pages.view(np.int64)).to(DEV)
        rc = share_lib.share_demo(c.h, d_pages.data_ptr(), n, bufs.data_ptr(), used.data_ptr(), first8.data_ptr(),
                                  seen.data_ptr(), prop.data_ptr(), c.stream)
        assert rc == 0
        torch.cuda.synchronize()
        c.check()
        used, first8, seen, prop = (t.cpu().numpy() for t in (used, first8, seen, prop))
        # one buffer per page while its requests overlap (the slot of whichever request
        # registered it first)
        assert (used >= 0).all()
        assert len({(int(p), int(u)) for p, u in zip(pages, used)}) == len(np.unique(pages))
        for i, p in enumerate(pages):
            assert first8[i] == store[int(p) * 4096:int(p) * 4096 + 8].view(np.int64)[0], i
        assert seen.all()                                    # the owner's mark, through the shared pointer
        # exactly one release per page propagated its buffer into the cache
        assert int(prop.sum()) == len(np.unique(pages))
        reads, _, _ = ag.agile_page_io(c.h, 0, npages)
        if cached:
            assert reads.sum() == 0
        else:
            assert (reads[np.unique(pages).astype(np.int64)] == 1).all()   # one fetch per page, shared
        ag.agile_flush(c.h, c.stream)
        torch.cuda.synchronize()
        c.check()
        want = store.copy()
        for p in np.unique(pages):
            want[int(p) * 4096 + 32:int(p) * 4096 + 48] = (int(p) & 0xFF) ^ 0x5A
        assert np.array_equal(c.get(0, store.nbytes), want)
        _, writes, dirtied = ag.agile_page_io(c.h, 0, npages)
        assert np.array_equal(writes, dirtied)
        assert (writes[np.unique(pages).astype(np.int64)] == 1).all()
