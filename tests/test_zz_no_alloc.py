"""The BFS entry point that allocates nothing (agile_bfs_noalloc).

Some callers cannot allocate device memory while they run a BFS: code running under
stream capture, where cudaMalloc is not allowed, and latency-critical loops, where the
device synchronisation an allocation implies would stall other streams.
agile_bfs_noalloc serves them with its scratch in fixed device arrays.  Here it must
give the same levels and edge counts as agile_bfs on two calls in a row, leave the
device's free memory unchanged, and refuse a graph larger than its arrays can serve.
This file is collected last so that a failure here comes after every other test has
run.
"""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2504_19365_gb300 as ag  # noqa: E402
from gpu_util import Ctx, round_page  # noqa: E402

DEV = "cuda:0"


def _graph():
    n, off, cols = synth.rmat_csr(5, 16, 16)   # hubs above 1,024 entries: the queue is used
    col0 = round_page(off.nbytes)
    return n, off, cols, col0, col0 + round_page(cols.nbytes)


@pytest.mark.parametrize("mode", [ag.AGILE_SYNC, ag.AGILE_ASYNC])
def test_noalloc_bfs_matches_bfs_on_two_calls_in_a_row(mode):
    n, off, cols, col0, total = _graph()
    assert np.diff(off).max() >= 1024
    lines = max(8, (cols.nbytes // 8 + 4095) // 4096)
    with Ctx(total, cache_bytes=(lines + 7) // 8 * 8 * 4096, ways=8) as c:
        c.put(0, off)
        c.put(col0, cols)
        srcs = [int(x) for x in synth.bfs_sources(5, off, 2)]
        want = []
        for src in srcs:
            lv = torch.full((n,), 7, dtype=torch.int32, device=DEV)
            ed = torch.zeros(1, dtype=torch.int64, device=DEV)
            ag.agile_bfs(c.h, 0, col0, n, src, lv.data_ptr(), ed.data_ptr(), mode, c.stream)
            want.append((lv, ed))
        got = []
        for src in srcs:   # two calls of the new entry point in a row
            lv = torch.full((n,), 9, dtype=torch.int32, device=DEV)
            ed = torch.zeros(1, dtype=torch.int64, device=DEV)
            ag.agile_bfs_noalloc(c.h, 0, col0, n, int(cols.size), src, lv.data_ptr(), ed.data_ptr(), mode,
                                 c.stream)
            got.append((lv, ed))
        torch.cuda.synchronize()
        c.check()
        for (lv_a, ed_a), (lv_b, ed_b) in zip(want, got):
            # levels and edge counts are integers: equal bit for bit
            assert torch.equal(lv_a, lv_b)
            assert int(ed_a.item()) == int(ed_b.item()) > 0


def test_noalloc_bfs_allocates_no_device_memory():
    # On a context that never ran agile_bfs (so it holds no BFS scratch of its own), two
    # calls leave the device's free memory exactly as it was.  The store has 1 GiB of
    # room beyond the columns, so agile_bfs on the same context sizes its queue of long
    # lists for it (16 MiB, far above the driver's 2 MiB allocation granule): the same
    # measurement sees that allocation.
    n, off, cols, col0, total = _graph()
    total += 1 << 30
    lines = max(8, (cols.nbytes // 8 + 4095) // 4096)
    cache = (lines + 7) // 8 * 8 * 4096
    src = int(synth.bfs_sources(5, off, 1)[0])
    lv = torch.empty(n, dtype=torch.int32, device=DEV)
    ed = torch.zeros(1, dtype=torch.int64, device=DEV)
    with Ctx(total, cache_bytes=cache, ways=8) as warm:   # loads the kernels once
        warm.put(0, off)
        warm.put(col0, cols)
        ag.agile_bfs_noalloc(warm.h, 0, col0, n, int(cols.size), src, lv.data_ptr(), ed.data_ptr(),
                             ag.AGILE_SYNC, warm.stream)
        torch.cuda.synchronize()
        warm.check()
    want = lv.clone()
    with Ctx(total, cache_bytes=cache, ways=8) as c:
        c.put(0, off)
        c.put(col0, cols)
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        for mode in (ag.AGILE_SYNC, ag.AGILE_ASYNC):
            lv.fill_(5)
            ag.agile_bfs_noalloc(c.h, 0, col0, n, int(cols.size), src, lv.data_ptr(), ed.data_ptr(), mode,
                                 c.stream)
            torch.cuda.synchronize()
            c.check()
            assert torch.equal(lv, want)
        assert torch.cuda.mem_get_info()[0] == free0
        ag.agile_bfs(c.h, 0, col0, n, src, lv.data_ptr(), ed.data_ptr(), ag.AGILE_SYNC, c.stream)
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] < free0   # the allocating entry point is seen


def test_noalloc_bfs_rejects_graph_beyond_its_scratch():
    n, off, cols, col0, total = _graph()
    with Ctx(total + (128 << 20), cache_bytes=64 * 4096, ways=8, num_queues=8, queue_depth=64) as c:
        lv = torch.empty(n, dtype=torch.int32, device=DEV)
        too_many = 131072 * 256   # needs 131,073 queue slots, one more than the array has
        with pytest.raises(ag.AgileError) as e:
            ag.agile_bfs_noalloc(c.h, 0, col0, n, too_many, 0, lv.data_ptr(), 0, ag.AGILE_SYNC, c.stream)
        assert e.value.code == ag.AGILE_EINVAL


def test_noalloc_bfs_rejects_more_vertices_than_its_bitmap():
    # 2^25 + 1 vertices need one bitmap word more than the fixed array has; the call is
    # rejected on the host before anything is launched
    nv = (1 << 25) + 1
    store = ((nv + 1) * 8 + 4095) // 4096 * 4096 + 4096
    with Ctx(store, cache_bytes=64 * 4096, ways=8, num_queues=8, queue_depth=64) as c:
        lv = torch.empty(1, dtype=torch.int32, device=DEV)
        with pytest.raises(ag.AgileError) as e:
            ag.agile_bfs_noalloc(c.h, 0, store - 4096, nv, 1, 0, lv.data_ptr(), 0, ag.AGILE_SYNC, c.stream)
        assert e.value.code == ag.AGILE_EINVAL
