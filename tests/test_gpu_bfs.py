"""GPU parity of BFS through the HBM cache (Sec. 4.5) against the oracle's FIFO BFS:
levels bit-exact, edges scanned exact."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2504_19365_gb300 as ag  # noqa: E402
from gpu_util import Ctx, assert_cache_invariants, round_page  # noqa: E402

DEV = "cuda:0"


def _layout(offsets, cols):
    col0 = round_page(offsets.nbytes)
    return col0, col0 + round_page(cols.nbytes)


def _bfs(c, col0, n, src, mode):
    level = torch.full((n,), 12345, dtype=torch.int32, device=DEV)
    edges = torch.zeros(1, dtype=torch.int64, device=DEV)
    ag.agile_bfs(c.h, 0, col0, n, int(src), level.data_ptr(), edges.data_ptr(), mode, c.stream)
    torch.cuda.synchronize()
    c.check()
    return level.cpu().numpy(), int(edges.item())


def _cache_for(cols, ways=8):
    lines = max(ways, (cols.nbytes // 8 + 4095) // 4096)
    return (lines + ways - 1) // ways * ways * 4096


@pytest.mark.parametrize("mode", [ag.AGILE_SYNC, ag.AGILE_ASYNC])
@pytest.mark.parametrize("graph", ["path", "star", "tree", "isolated"])
def test_special_graphs(mode, graph):
    if graph == "path":
        off, cols = synth.graph_path(3000)
    elif graph == "star":
        off, cols = synth.graph_star(5000)
    elif graph == "tree":
        off, cols = synth.graph_binary_tree(4095)
    else:
        off, cols = synth.csr_from_edges(2000, np.arange(1000), np.arange(1, 1001))
    n = len(off) - 1
    col0, total = _layout(off, cols)
    with Ctx(total, cache_bytes=16 * 4096, ways=4, num_queues=8, queue_depth=64) as c:
        c.put(0, off)
        c.put(col0, cols)
        for src in [0, n // 2, n - 1]:
            want, scanned = oracle.bfs(off, cols, src)
            got, edges = _bfs(c, col0, n, src, mode)
            assert np.array_equal(got, want)
            assert edges == scanned
        assert_cache_invariants(c)


@pytest.mark.parametrize("mode", [ag.AGILE_SYNC, ag.AGILE_ASYNC])
def test_rmat_small_cache_one_eighth(mode):
    n, off, cols = synth.rmat_csr(3, 14, 16)
    col0, total = _layout(off, cols)
    with Ctx(total, cache_bytes=_cache_for(cols), ways=8) as c:
        c.put(0, off)
        c.put(col0, cols)
        for src in synth.bfs_sources(3, off, 3):
            want, scanned = oracle.bfs(off, cols, src)
            got, edges = _bfs(c, col0, n, src, mode)
            assert np.array_equal(got, want)
            assert edges == scanned
        s = c.stats()
        assert s["cqes"] == s["commands"]
        assert_cache_invariants(c)


def test_rmat_scale20_config_parity():
    # RMAT scale 20, edge factor 16, (a, b, c) = (.57, .19, .19), symmetrised CSR,
    # HBM cache = 1/8 of the column array, 8 seeded sources, sync and async
    n, off, cols = synth.rmat_csr(3, 20, 16)
    col0, total = _layout(off, cols)
    with Ctx(total, cache_bytes=_cache_for(cols), ways=8) as c:
        c.put(0, off)
        c.put(col0, cols)
        for k, src in enumerate(synth.bfs_sources(3, off, 8)):
            want, scanned = oracle.bfs(off, cols, src)
            for mode in (ag.AGILE_ASYNC, ag.AGILE_SYNC) if k < 2 else (ag.AGILE_ASYNC,):
                got, edges = _bfs(c, col0, n, src, mode)
                assert np.array_equal(got, want)
                assert edges == scanned
        assert_cache_invariants(c)


@pytest.mark.parametrize("mode", [ag.AGILE_SYNC, ag.AGILE_ASYNC])
def test_tiny_ring_and_tiny_cache(mode):
    # one queue of depth 64 and an 8-line cache: every warp must let its pin go before
    # it waits, or the search could not finish
    n, off, cols = synth.rmat_csr(31, 10, 8)
    col0 = round_page(off.nbytes)
    total = col0 + round_page(cols.nbytes)
    src = int(synth.bfs_sources(31, off, 1)[0])
    want, scanned = oracle.bfs(off, cols, src)
    with Ctx(total, cache_bytes=8 * 4096, ways=2, num_queues=1, queue_depth=64) as c:
        c.put(0, off)
        c.put(col0, cols)
        lv = torch.empty(n, dtype=torch.int32, device=DEV)
        ed = torch.zeros(1, dtype=torch.int64, device=DEV)
        ag.agile_bfs(c.h, 0, col0, n, src, lv.data_ptr(), ed.data_ptr(), mode, c.stream)
        torch.cuda.synchronize()
        c.check()
        assert np.array_equal(lv.cpu().numpy(), want) and int(ed.item()) == scanned
        assert_cache_invariants(c)


@pytest.mark.parametrize("mode", [ag.AGILE_SYNC, ag.AGILE_ASYNC])
def test_uniform_random_graph_scale20(mode):
    # the "-U" graphs of Sec. 4.5: every edge's endpoints uniform, scale 20, edge factor
    # 16, cache 1/8 of the columns; 2 seeded sources
    n, off, cols = synth.uniform_csr(8, 20, 16)
    col0, total = _layout(off, cols)
    with Ctx(total, cache_bytes=_cache_for(cols), ways=8) as c:
        c.put(0, off)
        c.put(col0, cols)
        for src in synth.bfs_sources(8, off, 2):
            lv, edges = _bfs(c, col0, n, src, mode)
            want, scanned = oracle.bfs(off, cols, int(src))
            assert np.array_equal(lv, want)
            assert edges == scanned


@pytest.mark.parametrize("graph", ["rmat", "uniform", "path"])
def test_hbm_kernel_equals_oracle(graph):
    # the breakdown's kernel-time baseline: the same kernel over the CSR in HBM
    if graph == "rmat":
        n, off, cols = synth.rmat_csr(3, 16, 16)
    elif graph == "uniform":
        n, off, cols = synth.uniform_csr(9, 16, 16)
    else:
        off, cols = synth.graph_path(5000)
        n = off.size - 1
    col0, total = _layout(off, cols)
    with Ctx(total, cache_bytes=_cache_for(cols), ways=8) as c:
        d_off = torch.from_numpy(off).to(DEV)
        d_cols = torch.from_numpy(cols).to(DEV)
        for src in synth.bfs_sources(10, off, 2):
            level = torch.full((n,), 77, dtype=torch.int32, device=DEV)
            edges = torch.zeros(1, dtype=torch.int64, device=DEV)
            ag.agile_bfs_hbm(c.h, d_off.data_ptr(), d_cols.data_ptr(), n, int(cols.size), int(src),
                             level.data_ptr(), edges.data_ptr(), c.stream)
            torch.cuda.synchronize()
            c.check()
            want, scanned = oracle.bfs(off, cols, int(src))
            assert np.array_equal(level.cpu().numpy(), want)
            assert int(edges.item()) == scanned
        assert c.stats()["commands"] == 0   # no page went through the queues
