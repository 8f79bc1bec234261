"""The BFS entry point that allocates nothing (agile_bfs_noalloc).

Some callers cannot allocate device memory while they run a BFS: code being recorded
into a CUDA graph or running under stream capture, where cudaMalloc is not allowed, and
latency-critical loops, where the device synchronisation an allocation implies would
stall other streams.  agile_bfs_noalloc serves them with its scratch in a fixed device
array.  Here it must give the same levels and edge counts as agile_bfs on two calls in
a row, and refuse a graph larger than that array can serve.  This file is collected
last so that a failure here comes after every other test has run.
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


def test_noalloc_bfs_rejects_graph_beyond_its_scratch():
    n, off, cols, col0, total = _graph()
    with Ctx(total + (128 << 20), cache_bytes=64 * 4096, ways=8, num_queues=8, queue_depth=64) as c:
        lv = torch.empty(n, dtype=torch.int32, device=DEV)
        too_many = 32768 * 1024   # needs 32,769 queue slots, one more than the array has
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
