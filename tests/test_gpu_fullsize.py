"""GPU parity at the stated sizes of the DLRM-shaped workloads, on seeded samples the
oracle computes one by one.

  - Lookup + compute pipeline over 8 FP32 tables of 10,000,000 x 64 (20.48 GB on the
    store) with a 4 GiB cache, Zipf(1.05) rows, 2048 bags x pooling 32 per table, one
    batch, then the FP32 multiply-add phase: 1,024 sampled bags (all 8 tables each)
    against the oracle, sync and async, at the full grid and at 32 warps.
  - Serving against the same tables and cache: 120 requests of 1-4096 bags (log-uniform)
    x pooling 1-64, all of their bags against the oracle, with requests arriving at once
    and arriving spread out.
  - Training step over 4 tables of 4,194,304 x 128 (8 GiB) with a 2 GiB cache, Zipf(1.1)
    rows, batch 4096 x pooling 20: forward, backward with the SGD step (lr 2^-6), flush;
    1,024 sampled bags of each forward and 2,000 touched plus 500 untouched rows of each
    table on the store after the flush against the oracle, and every dirty epoch of a
    page written back exactly once.
Tables are dyadic, so every FP32 sum is exact and every comparison is bit for bit.
"""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2504_19365_gb300 as ag  # noqa: E402
from gpu_util import Ctx, dyadic_rows, fill_dyadic, round_page  # noqa: E402

DEV = "cuda:0"
NT3, ROWS3, DIM3 = 8, 10_000_000, 64
STRIDE3 = round_page(ROWS3 * DIM3 * 4)


@pytest.fixture(scope="module")
def dlrm():
    c = Ctx(STRIDE3 * NT3, cache_bytes=4 << 30, ways=8, wait_timeout_ns=60_000_000_000)
    try:
        fill_dyadic(c, NT3, ROWS3, DIM3, STRIDE3)
        yield c
    finally:
        c.close()


def _local(tables_rows, k, dim):
    """Rows needed from table k as a compact table, and the map row -> local index."""
    uniq = np.unique(tables_rows)
    return dyadic_rows(k, uniq, dim), uniq


@pytest.mark.parametrize("app_warps", [0, 32])
def test_pipeline_config3_sampled(dlrm, app_warps):
    nbags, pool, iters = 2048, 32, 40
    idx = synth.Zipf(ROWS3, 1.05, permute=True, seed=4).rows(5, NT3 * nbags * pool).reshape(1, NT3, nbags, pool)
    sample = np.sort(synth.uniform_int(31, 1024, nbags))
    sample = np.unique(sample)
    tabs, lidx = [], np.empty((1, NT3, sample.size, pool), dtype=np.int64)
    for k in range(NT3):
        t, uniq = _local(idx[0, k, sample].reshape(-1), k, DIM3)
        tabs.append(t)
        lidx[0, k] = np.searchsorted(uniq, idx[0, k, sample])
    want = oracle.embedding_pipeline(tabs, lidx, pool, iters)[0]
    c = dlrm
    d_idx = torch.from_numpy(idx).to(DEV)
    ag.agile_config_parallelism(c.h, app_warps)
    try:
        for mode in (ag.AGILE_SYNC, ag.AGILE_ASYNC):
            ag.agile_invalidate(c.h, c.stream)
            out = torch.full((1, nbags, NT3 * DIM3), float("nan"), dtype=torch.float32, device=DEV)
            ag.agile_embedding_pipeline(c.h, 0, STRIDE3, NT3, ROWS3, DIM3, d_idx.data_ptr(), pool, nbags, 1, iters,
                                        out.data_ptr(), mode, c.stream)
            torch.cuda.synchronize()
            c.check()
            got = out.cpu().numpy()[0, sample]
            assert np.array_equal(got.view(np.uint32), want.view(np.uint32)), mode
    finally:
        ag.agile_config_parallelism(c.h, 0)


@pytest.mark.parametrize("mode", [ag.AGILE_SYNC, ag.AGILE_ASYNC])
def test_serving_config5_sampled(dlrm, mode):
    n_req = 120
    sizes = np.minimum(4096, np.maximum(1, np.round(2.0 ** (synth.uniform01(7, n_req) * 12)))).astype(int)
    pools = synth.uniform_int(8, n_req, 64) + 1
    which = synth.uniform_int(9, n_req, NT3)
    zipf = synth.Zipf(ROWS3, 1.05, permute=True, seed=4)
    reqs, keep, wants = [], [], []
    for i in range(n_req):
        nb, pool, k = int(sizes[i]), int(pools[i]), int(which[i])
        idx = zipf.rows(1000 + i, nb * pool)
        off = synth.bags_fixed(nb, pool)
        t, uniq = _local(idx, k, DIM3)
        wants.append(oracle.embedding_bag(t, np.searchsorted(uniq, idx), off))
        d_idx, d_off = torch.from_numpy(idx).to(DEV), torch.from_numpy(off).to(DEV)
        out = torch.full((nb, DIM3), float("nan"), dtype=torch.float32, device=DEV)
        keep.append((d_idx, d_off, out))
        reqs.append(ag.agile_lookup_req(k * STRIDE3, ROWS3, DIM3, d_idx.data_ptr(), d_off.data_ptr(), nb,
                                        out.data_ptr()))
    c = dlrm
    for arrival in (np.zeros(n_req, dtype=np.uint64), (np.arange(n_req) * 20_000).astype(np.uint64)):
        for _, _, out in keep:
            out.fill_(float("nan"))
        lat = np.zeros(n_req, dtype=np.uint64)
        ag.agile_serve_replay(c.h, reqs, arrival.ctypes.data, lat.ctypes.data, mode, c.stream)
        torch.cuda.synchronize()
        c.check()
        for i, (_, _, out) in enumerate(keep):
            assert np.array_equal(out.cpu().numpy().view(np.uint32), wants[i].view(np.uint32)), i
        assert (lat > 0).all()


def test_training_config4_sampled():
    nt, rows, dim, nb, pool = 4, 1 << 22, 128, 4096, 20
    stride = round_page(rows * dim * 4)
    lr = 2.0 ** -6
    zipf = synth.Zipf(rows, 1.1, permute=True, seed=6)
    off = synth.bags_fixed(nb, pool)
    gout = synth.table_normal(12, nb, dim)
    sample = np.unique(synth.uniform_int(33, 1024, nb))
    with Ctx(stride * nt, cache_bytes=2 << 30, ways=8, wait_timeout_ns=60_000_000_000) as c:
        fill_dyadic(c, nt, rows, dim, stride)
        d_off, d_g = torch.from_numpy(off).to(DEV), torch.from_numpy(gout).to(DEV)
        out = torch.empty((nb, dim), dtype=torch.float32, device=DEV)
        idxs = [zipf.rows(100 + k, nb * pool) for k in range(nt)]
        for mode, k in ((ag.AGILE_SYNC, 0), (ag.AGILE_ASYNC, 1), (ag.AGILE_SYNC, 2), (ag.AGILE_ASYNC, 3)):
            d_idx = torch.from_numpy(idxs[k]).to(DEV)
            ag.agile_embedding_bag(c.h, k * stride, rows, dim, d_idx.data_ptr(), d_off.data_ptr(), nb, out.data_ptr(),
                                   mode, c.stream)
            torch.cuda.synchronize()
            c.check()
            # forward: sampled bags against the oracle (the table before its SGD step)
            rows_s = idxs[k].reshape(nb, pool)[sample].reshape(-1)
            t, uniq = _local(rows_s, k, dim)
            want = oracle.embedding_bag(t, np.searchsorted(uniq, rows_s), synth.bags_fixed(sample.size, pool))
            assert np.array_equal(out.cpu().numpy()[sample].view(np.uint32), want.view(np.uint32)), k
            ag.agile_embedding_bag_backward(c.h, k * stride, rows, dim, d_idx.data_ptr(), d_off.data_ptr(), nb,
                                            nb * pool, d_g.data_ptr(), lr, 0, mode, c.stream)
        ag.agile_flush(c.h, c.stream)
        torch.cuda.synchronize()
        c.check()
        for k in range(nt):
            # the oracle's gradient and SGD step over the touched rows, relabelled 0..u-1
            uniq, local = np.unique(idxs[k], return_inverse=True)
            G, touched = oracle.embedding_bag_backward(uniq.size, local.astype(np.int64), off, gout)
            new = oracle.sgd(dyadic_rows(k, uniq, dim), G, touched, lr)
            pick = np.unique(synth.uniform_int(40 + k, 2000, uniq.size))
            for j in pick:
                r = int(uniq[j])
                got = c.get(k * stride + r * dim * 4, dim * 4).view(np.float32)
                assert np.array_equal(got.view(np.uint32), new[j].view(np.uint32)), (k, r)
            untouched = np.setdiff1d(synth.uniform_int(50 + k, 600, rows), uniq)[:500]
            for r in untouched:
                got = c.get(k * stride + int(r) * dim * 4, dim * 4).view(np.float32)
                assert np.array_equal(got, dyadic_rows(k, np.array([r]), dim)[0]), (k, r)
        npages = stride * nt // 4096
        _, writes, dirtied = ag.agile_page_io(c.h, 0, npages)
        assert np.array_equal(writes, dirtied) and writes.sum() > 0
