"""GPU parity of the cache-backed embedding bag (Sec. 4.4) against the oracle.

Pooled sums are compared bit for bit: both sides add the rows of a bag in increasing
index order in FP32 with round-to-nearest and no fused multiply-add."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2504_19365_gb300 as ag  # noqa: E402
from gpu_util import Ctx, assert_cache_invariants  # noqa: E402

DEV = "cuda:0"


def _bag(c, table_byte0, rows, dim, idx, off, mode):
    d_idx = torch.from_numpy(np.ascontiguousarray(idx, dtype=np.int64)).to(DEV)
    d_off = torch.from_numpy(np.ascontiguousarray(off, dtype=np.int64)).to(DEV)
    nb = len(off) - 1
    out = torch.full((nb, dim), float("nan"), dtype=torch.float32, device=DEV)
    ag.agile_embedding_bag(c.h, table_byte0, rows, dim, d_idx.data_ptr(), d_off.data_ptr(), nb,
                           out.data_ptr(), mode, c.stream)
    torch.cuda.synchronize()
    c.check()
    return out.cpu().numpy()


@pytest.mark.parametrize("mode", [ag.AGILE_SYNC, ag.AGILE_ASYNC])
@pytest.mark.parametrize("dim", [128, 64, 16, 1024])
def test_bag_bit_exact_vs_oracle(mode, dim):
    rows = 3000
    T = synth.table_normal(1, rows, dim)
    sizes = synth.uniform_int(2, 300, 41)   # 0..40 indices: empty bags and >32 (two groups)
    off = np.zeros(301, dtype=np.int64)
    np.cumsum(sizes, out=off[1:])
    idx = synth.indices_uniform(3, int(off[-1]), rows)
    want = oracle.embedding_bag(T, idx, off)
    with Ctx(T.nbytes, cache_bytes=64 * 4096, ways=8, num_queues=16, queue_depth=64) as c:
        c.put(0, T)
        got = _bag(c, 0, rows, dim, idx, off, mode)
        assert np.array_equal(got.view(np.uint32), want.view(np.uint32))
        assert_cache_invariants(c)


def test_config1_small_full_size_sync_async_equal_and_exact():
    # 65,536 x 128 FP32 table (32 MiB, 8192 pages), 4 MiB 8-way cache, 16 batches of
    # 256 bags x 16 uniform indices, sum pooling
    rows, dim = 65536, 128
    T = synth.table_normal(1, rows, dim)
    nb, pool, batches = 256, 16, 16
    off = synth.bags_fixed(nb, pool)
    with Ctx(T.nbytes, cache_bytes=4 << 20, ways=8) as c:
        c.put(0, T)
        for bt in range(batches):
            idx = synth.indices_uniform(2, nb * pool, rows, offset=bt * nb * pool)
            want = oracle.embedding_bag(T, idx, off)
            a = _bag(c, 0, rows, dim, idx, off, ag.AGILE_ASYNC)
            s = _bag(c, 0, rows, dim, idx, off, ag.AGILE_SYNC)
            assert np.array_equal(a.view(np.uint32), want.view(np.uint32))
            assert np.array_equal(s.view(np.uint32), want.view(np.uint32))
        st = c.stats()
        assert st["cqes"] == st["commands"] and st["io_errors"] == 0
        assert_cache_invariants(c)


def test_dyadic_table_and_pooling_one():
    rows, dim = 4096, 64
    T = synth.table_dyadic(rows, dim)
    idx = synth.indices_uniform(4, 500, rows)
    off = np.arange(501, dtype=np.int64)   # pooling 1: each bag copies one row
    with Ctx(T.nbytes, cache_bytes=32 * 4096, ways=4, num_queues=8, queue_depth=64) as c:
        c.put(0, T)
        got = _bag(c, 0, rows, dim, idx, off, ag.AGILE_ASYNC)
        assert np.array_equal(got, T[idx])


def test_table_at_offset_and_out_of_range_index_reported():
    rows, dim = 512, 32
    T = synth.table_normal(5, rows, dim)
    base = 3 * 4096
    with Ctx(base + T.nbytes, cache_bytes=16 * 4096, ways=4, num_queues=4, queue_depth=64) as c:
        c.put(base, T)
        idx = np.array([0, 511, 7], dtype=np.int64)
        off = np.array([0, 2, 3], dtype=np.int64)
        got = _bag(c, base, rows, dim, idx, off, ag.AGILE_SYNC)
        assert np.array_equal(got, oracle.embedding_bag(T, idx, off))
        # an index outside the table is refused on the GPU and reported on the host
        bad = np.array([0, rows], dtype=np.int64)
        d_idx = torch.from_numpy(bad).to(DEV)
        d_off = torch.from_numpy(np.array([0, 2], dtype=np.int64)).to(DEV)
        out = torch.empty((1, dim), dtype=torch.float32, device=DEV)
        ag.agile_embedding_bag(c.h, base, rows, dim, d_idx.data_ptr(), d_off.data_ptr(), 1, out.data_ptr(),
                               ag.AGILE_SYNC, c.stream)
        torch.cuda.synchronize()
        assert ag.agile_check(c.h) == ag.AGILE_EINVAL


@pytest.mark.parametrize("app_warps", [0, 1024])
def test_large_cache_cold_then_warm_hits(app_warps):
    # A cache with room for more warps than two CTAs per SM hold (the three-CTA kernel is
    # taken by default, the two-CTA one with 1,024 app warps); bags of 0..40 rows take
    # the all-resident path (<= 32 rows, every page pinned at once) and the general one.
    rows, dim = 131072, 128
    T = synth.table_normal(11, rows, dim)
    sizes = synth.uniform_int(12, 8192, 41)
    off = np.zeros(8193, dtype=np.int64)
    np.cumsum(sizes, out=off[1:])
    idx = synth.indices_uniform(13, int(off[-1]), rows)
    want = oracle.embedding_bag(T, idx, off)
    with Ctx(T.nbytes, cache_bytes=96 << 20, ways=8) as c:
        c.put(0, T)
        if app_warps:
            ag.agile_config_parallelism(c.h, app_warps)
        for mode in (ag.AGILE_SYNC, ag.AGILE_ASYNC):
            ag.agile_invalidate(c.h, c.stream)
            cold = _bag(c, 0, rows, dim, idx, off, mode)
            ag.agile_reset_stats(c.h)
            warm = _bag(c, 0, rows, dim, idx, off, mode)
            st = c.stats()
            assert np.array_equal(cold.view(np.uint32), want.view(np.uint32))
            assert np.array_equal(warm.view(np.uint32), want.view(np.uint32))
            assert st["misses"] == 0 and st["hits"] > 0
            # every looked-up row was served by a probe of its own or of a warp-mate
            assert st["hits"] + st["warp_coalesced"] >= int(off[-1])
        assert_cache_invariants(c)


@pytest.mark.parametrize("dim", [16, 128, 512])
def test_hbm_gather_ceiling_equals_oracle(dim):
    # the hit path's plain-gather ceiling (table in HBM, no cache) computes the same bits
    rows, nb = 5000, 700
    T = synth.table_normal(21, rows, dim)
    lens = synth.uniform_int(22, nb, 40)           # 0-39 indices a bag, empty bags included
    off = np.zeros(nb + 1, dtype=np.int64)
    off[1:] = np.cumsum(lens)
    idx = synth.indices_uniform(23, int(off[-1]), rows)
    with Ctx(4096 * 16, cache_bytes=8 * 4096, ways=8, num_queues=4, queue_depth=64) as c:
        d_t = torch.from_numpy(T).to(DEV)
        d_idx, d_off = torch.from_numpy(idx).to(DEV), torch.from_numpy(off).to(DEV)
        out = torch.full((nb, dim), float("nan"), dtype=torch.float32, device=DEV)
        ag.agile_embedding_bag_hbm(c.h, d_t.data_ptr(), rows, dim, d_idx.data_ptr(), d_off.data_ptr(), nb,
                                   out.data_ptr(), c.stream)
        torch.cuda.synchronize()
        c.check()
        want = oracle.embedding_bag(T, idx, off)
        assert np.array_equal(out.cpu().numpy().view(np.uint32), want.view(np.uint32))
