"""GPU parity of the differentiable embedding bag: backward scatter-add and the fused SGD
step written back through the cache and the queues, against the oracle's gradient, its
SGD table and finite differences."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2504_19365_gb300 as ag  # noqa: E402
from paper_2504_19365_gb300.autograd import cached_embedding_bag  # noqa: E402
from gpu_util import Ctx, assert_cache_invariants  # noqa: E402

DEV = "cuda:0"


def _bags(seed, n_bags, rows, lo=0, hi=24, zipf=False):
    sizes = synth.uniform_int(seed, n_bags, hi - lo + 1) + lo
    off = np.zeros(n_bags + 1, dtype=np.int64)
    np.cumsum(sizes, out=off[1:])
    if zipf:
        idx = synth.Zipf(rows, 1.1, permute=True, seed=seed).rows(seed + 1, int(off[-1]))
    else:
        idx = synth.indices_uniform(seed + 1, int(off[-1]), rows)
    return idx, off


def _backward(c, rows, dim, idx, off, gout, lr, want_grad, mode):
    d_idx = torch.from_numpy(idx).to(DEV)
    d_off = torch.from_numpy(off).to(DEV)
    d_g = torch.from_numpy(np.ascontiguousarray(gout, dtype=np.float32)).to(DEV)
    G = torch.full((rows, dim), float("nan"), dtype=torch.float32, device=DEV) if want_grad else None
    ag.agile_embedding_bag_backward(c.h, 0, rows, dim, d_idx.data_ptr(), d_off.data_ptr(), len(off) - 1, len(idx),
                                    d_g.data_ptr(), lr, G.data_ptr() if want_grad else 0, mode, c.stream)
    torch.cuda.synchronize()
    c.check()
    return G.cpu().numpy() if want_grad else None


@pytest.mark.parametrize("mode", [ag.AGILE_SYNC, ag.AGILE_ASYNC])
@pytest.mark.parametrize("zipf", [False, True])
def test_gradient_bit_exact_vs_oracle(mode, zipf):
    rows, dim = 3000, 64
    T = synth.table_normal(1, rows, dim)
    idx, off = _bags(2, 400, rows, zipf=zipf)
    gout = synth.table_normal(3, 400, dim)
    Gw, _ = oracle.embedding_bag_backward(rows, idx, off, gout)
    with Ctx(T.nbytes, cache_bytes=64 * 4096, ways=8, num_queues=16, queue_depth=64) as c:
        c.put(0, T)
        G = _backward(c, rows, dim, idx, off, gout, 0.0, True, mode)
        assert np.array_equal(G.view(np.uint32), Gw.view(np.uint32))
        # lr = 0: the table is untouched
        ag.agile_flush(c.h, c.stream)
        torch.cuda.synchronize()
        assert np.array_equal(c.get(0, T.nbytes).view(np.float32).reshape(rows, dim), T)


@pytest.mark.parametrize("mode", [ag.AGILE_SYNC, ag.AGILE_ASYNC])
def test_sgd_written_back_through_small_cache(mode):
    # the cache holds 1/8 of the table: MODIFIED lines are evicted (written back from a
    # staging copy) during the call, the rest at flush; the store must equal the oracle
    rows, dim = 8192, 128
    T = synth.table_normal(4, rows, dim)
    idx, off = _bags(5, 1000, rows, 1, 20, zipf=True)
    gout = synth.table_normal(6, 1000, dim)
    lr = 2.0 ** -6
    G, touched = oracle.embedding_bag_backward(rows, idx, off, gout)
    want = oracle.sgd(T, G, touched, lr)
    with Ctx(T.nbytes, cache_bytes=T.nbytes // 8, ways=8, num_queues=32, queue_depth=128) as c:
        c.put(0, T)
        _backward(c, rows, dim, idx, off, gout, lr, False, mode)
        s1 = c.stats()
        ag.agile_flush(c.h, c.stream)
        torch.cuda.synchronize()
        c.check()
        got = c.get(0, T.nbytes).view(np.float32).reshape(rows, dim)
        assert np.array_equal(got.view(np.uint32), want.view(np.uint32))
        s = c.stats()
        assert s1["writebacks"] > 0, "evictions of MODIFIED lines during the call"
        assert s["bytes_written"] == 4096 * s["writebacks"]
        # the device's per-page write log: every dirty epoch of a page (a clean line of
        # it turned MODIFIED) ended in exactly one write-back, and no other page was
        # written; some pages went through several epochs (evicted, then dirtied again)
        npages = T.nbytes // 4096
        _, writes, dirtied = ag.agile_page_io(c.h, 0, npages)
        hit = np.zeros(npages, dtype=bool)
        hit[np.unique((np.nonzero(touched)[0] * dim * 4) // 4096)] = True
        assert np.array_equal(writes, dirtied)
        assert (dirtied[hit] >= 1).all() and (dirtied[~hit] == 0).all()
        assert int(writes.sum()) == s["writebacks"]
        assert_cache_invariants(c)
        # a following forward sees the updated rows
        d_idx = torch.from_numpy(idx).to(DEV)
        d_off = torch.from_numpy(off).to(DEV)
        out = torch.empty((1000, dim), dtype=torch.float32, device=DEV)
        ag.agile_embedding_bag(c.h, 0, rows, dim, d_idx.data_ptr(), d_off.data_ptr(), 1000, out.data_ptr(), mode,
                               c.stream)
        torch.cuda.synchronize()
        assert np.array_equal(out.cpu().numpy(), oracle.embedding_bag(want, idx, off))


def test_gradient_matches_finite_differences():
    # loss = sum(out * gout) is linear in the table; with dyadic values and h = 1/4 the
    # central difference of GPU forwards is exact
    rows, dim = 16, 4
    T = synth.table_dyadic(rows, dim)
    idx, off = _bags(7, 6, rows, 1, 5)
    gout = (synth.table_dyadic(6, dim) - 8.0).astype(np.float32)
    h = 0.25
    d_idx = torch.from_numpy(idx).to(DEV)
    d_off = torch.from_numpy(off).to(DEV)
    with Ctx(T.nbytes, cache_bytes=8 * 4096, ways=8, num_queues=4, queue_depth=64) as c:
        def loss(table):
            c.put(0, table)
            out = torch.empty((6, dim), dtype=torch.float32, device=DEV)
            ag.agile_embedding_bag(c.h, 0, rows, dim, d_idx.data_ptr(), d_off.data_ptr(), 6, out.data_ptr(),
                                   ag.AGILE_SYNC, c.stream)
            torch.cuda.synchronize()
            return float((out.cpu().numpy().astype(np.float64) * gout).sum())
        fd = np.zeros((rows, dim))
        for r in range(rows):
            for d in range(dim):
                tp, tm = T.copy(), T.copy()
                tp[r, d] += h
                tm[r, d] -= h
                fd[r, d] = (loss(tp) - loss(tm)) / (2 * h)
        c.put(0, T)
        G = _backward(c, rows, dim, idx, off, gout, 0.0, True, ag.AGILE_SYNC)
        assert np.allclose(G, fd, rtol=1e-5, atol=1e-6)


def test_autograd_function_forward_backward_sgd():
    rows, dim = 4096, 64
    T = synth.table_normal(8, rows, dim)
    idx, off = _bags(9, 300, rows, 1, 16)
    gout = synth.table_normal(10, 300, dim)
    lr = 2.0 ** -5
    G, touched = oracle.embedding_bag_backward(rows, idx, off, gout)
    want_T = oracle.sgd(T, G, touched, lr)
    with Ctx(T.nbytes, cache_bytes=32 * 4096, ways=8, num_queues=16, queue_depth=64) as c:
        c.put(0, T)
        d_idx = torch.from_numpy(idx).to(DEV)
        d_off = torch.from_numpy(off).to(DEV)
        out = cached_embedding_bag(c.h, 0, rows, dim, d_idx, d_off, lr)
        assert np.array_equal(out.detach().cpu().numpy(), oracle.embedding_bag(T, idx, off))
        (out * torch.from_numpy(gout).to(DEV)).sum().backward()
        ag.agile_flush(c.h, c.stream)
        torch.cuda.synchronize()
        c.check()
        got = c.get(0, T.nbytes).view(np.float32).reshape(rows, dim)
        assert np.array_equal(got.view(np.uint32), want_T.view(np.uint32))
