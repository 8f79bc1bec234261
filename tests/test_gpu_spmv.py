"""GPU parity of SpMV through the cache (Sec. 4.5 runs SpMV over the CSR graphs of its
BFS) against the oracle.

Every row is summed in increasing entry order on both sides, each product rounded
before it is added: rows of fewer than 1024 entries by a chain over the lanes of one
warp, longer rows as slices of 1024 entries that hand their running sum on to the next
slice.  Every row is therefore compared bit for bit, whatever its length, the values'
distribution or the cache size; repeated calls give the same bits."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2504_19365_gb300 as ag  # noqa: E402
from gpu_util import Ctx, assert_cache_invariants, round_page  # noqa: E402

DEV = "cuda:0"
HUB = 1024


def _layout(off, cols, vals):
    col0 = round_page(off.nbytes)
    val0 = col0 + round_page(cols.nbytes)
    return col0, val0, val0 + round_page(vals.nbytes)


def _spmv(c, off, cols, vals, x, mode, col0, val0, n_cols=None):
    n = off.size - 1
    d_x = torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).to(DEV)
    d_y = torch.full((n,), float("nan"), dtype=torch.float32, device=DEV)
    ent = torch.zeros(1, dtype=torch.int64, device=DEV)
    ag.agile_spmv(c.h, 0, col0, val0, n, x.size if n_cols is None else n_cols, d_x.data_ptr(), d_y.data_ptr(),
                  ent.data_ptr(), mode, c.stream)
    torch.cuda.synchronize()
    return d_y.cpu().numpy(), int(ent.item())


def _check(off, cols, vals, x, y):
    want = oracle.spmv(off, cols, vals, x)
    bad = np.nonzero(y.view(np.uint32) != want.view(np.uint32))[0]
    deg = np.diff(off)
    assert bad.size == 0, f"{bad.size} rows differ, e.g. row {bad[:5]} of degree {deg[bad[:5]]}"


def _store(c, off, cols, vals):
    col0, val0, _ = _layout(off, cols, vals)
    c.put(0, off)
    c.put(col0, cols)
    c.put(val0, vals)
    return col0, val0


@pytest.mark.parametrize("mode", [ag.AGILE_SYNC, ag.AGILE_ASYNC])
def test_identity_empty_rows_and_one_long_row(mode):
    n = 3000
    rows = []
    for i in range(n):
        if i == 1234:
            rows.append(list(range(0, 2 * 2500, 2)))   # 2500 entries: the slice path
        elif i % 5 == 0:
            rows.append([])
        else:
            rows.append([i])
    off = np.zeros(n + 1, dtype=np.int64)
    off[1:] = np.cumsum([len(r) for r in rows])
    cols = np.array([c for r in rows for c in r], dtype=np.int32)
    vals = np.ones(cols.size, dtype=np.float32)
    vals[off[1234]:off[1235]] = ((synth.uniform_int(3, 2500, 64) - 32) / 8.0).astype(np.float32)
    x = ((synth.uniform_int(4, 2 * 2500, 256) - 128) / 16.0).astype(np.float32)[:max(n, 5000)]
    _, _, total = _layout(off, cols, vals)
    with Ctx(total, cache_bytes=16 * 4096, ways=8, num_queues=8, queue_depth=64) as c:
        col0, val0 = _store(c, off, cols, vals)
        y, ent = _spmv(c, off, cols, vals, x, mode, col0, val0)
        c.check()
        want = oracle.spmv(off, cols, vals, x)
        # dyadic values: every row exact, the long one included
        assert np.array_equal(y.view(np.uint32), want.view(np.uint32))
        assert ent == cols.size
        assert_cache_invariants(c)


@pytest.mark.parametrize("mode", [ag.AGILE_SYNC, ag.AGILE_ASYNC])
@pytest.mark.parametrize("cache_pages", [64, 4096])
def test_rmat_normal_values(mode, cache_pages):
    n, off, cols = synth.rmat_csr(21, 14, 16)
    vals = synth.normal(22, cols.size).astype(np.float32)
    x = synth.normal(23, n).astype(np.float32)
    _, _, total = _layout(off, cols, vals)
    with Ctx(total, cache_bytes=cache_pages * 4096, ways=8) as c:
        col0, val0 = _store(c, off, cols, vals)
        y, ent = _spmv(c, off, cols, vals, x, mode, col0, val0)
        c.check()
        _check(off, cols, vals, x, y)
        assert ent == cols.size
        assert_cache_invariants(c)


@pytest.mark.parametrize("mode", [ag.AGILE_SYNC, ag.AGILE_ASYNC])
def test_very_long_rows_in_entry_order(mode):
    # rows of 40,000 and 9,000 entries (40 and 9 slices handing their running sums on)
    # with N(0,1) values, beside short rows; two calls give the same bits
    lens = [40000, 3, 0, 9000, 1023, 1024, 1025, 2047, 2048, 5]
    n_cols = 50000
    off = np.zeros(len(lens) + 1, dtype=np.int64)
    off[1:] = np.cumsum(lens)
    cols = synth.uniform_int(41, int(off[-1]), n_cols).astype(np.int32)
    vals = synth.normal(42, cols.size).astype(np.float32)
    x = synth.normal(43, n_cols).astype(np.float32)
    _, _, total = _layout(off, cols, vals)
    with Ctx(total, cache_bytes=32 * 4096, ways=8, num_queues=16, queue_depth=64) as c:
        col0, val0 = _store(c, off, cols, vals)
        y1, ent = _spmv(c, off, cols, vals, x, mode, col0, val0)
        y2, _ = _spmv(c, off, cols, vals, x, mode, col0, val0)
        c.check()
        _check(off, cols, vals, x, y1)
        assert np.array_equal(y1.view(np.uint32), y2.view(np.uint32))
        assert ent == cols.size
        assert_cache_invariants(c)


def test_rmat_dyadic_values_bit_exact_sync_equals_async():
    n, off, cols = synth.rmat_csr(24, 13, 16)
    vals = ((synth.uniform_int(25, cols.size, 32) - 16) / 4.0).astype(np.float32)
    x = ((synth.uniform_int(26, n, 32) - 16) / 4.0).astype(np.float32)
    _, _, total = _layout(off, cols, vals)
    with Ctx(total, cache_bytes=256 * 4096, ways=8) as c:
        col0, val0 = _store(c, off, cols, vals)
        want = oracle.spmv(off, cols, vals, x)
        for mode in (ag.AGILE_SYNC, ag.AGILE_ASYNC):
            y, _ = _spmv(c, off, cols, vals, x, mode, col0, val0)
            c.check()
            assert np.array_equal(y.view(np.uint32), want.view(np.uint32))


def test_column_out_of_range_is_reported():
    off = np.array([0, 2, 3], dtype=np.int64)
    cols = np.array([0, 7, 1], dtype=np.int32)   # 7 >= n_cols = 2
    vals = np.ones(3, dtype=np.float32)
    x = np.array([1.0, 2.0], dtype=np.float32)
    _, _, total = _layout(off, cols, vals)
    with Ctx(total, cache_bytes=16 * 4096, ways=8, num_queues=4, queue_depth=64) as c:
        col0, val0 = _store(c, off, cols, vals)
        y, _ = _spmv(c, off, cols, vals, x, ag.AGILE_SYNC, col0, val0, n_cols=2)
        assert ag.agile_check(c.h) == ag.AGILE_EINVAL
        assert y[0] == 1.0 and y[1] == 2.0   # the bad entry contributes 0


def test_full_rmat20_against_oracle():
    # the benchmark's matrix: RMAT scale 20 graph with N(0,1) values, cache 1/8 of the
    # column and value arrays
    n, off, cols = synth.rmat_csr(3, 20, 16)
    vals = synth.normal(6, cols.size).astype(np.float32)
    x = synth.normal(7, n).astype(np.float32)
    _, _, total = _layout(off, cols, vals)
    cache = round_page((cols.nbytes + vals.nbytes) // 8) // (8 * 4096) * (8 * 4096)
    with Ctx(total, cache_bytes=cache, ways=8) as c:
        col0, val0 = _store(c, off, cols, vals)
        for mode in (ag.AGILE_ASYNC, ag.AGILE_SYNC):
            y, ent = _spmv(c, off, cols, vals, x, mode, col0, val0)
            c.check()
            _check(off, cols, vals, x, y)
            assert ent == cols.size


@pytest.mark.parametrize("mode", [ag.AGILE_SYNC, ag.AGILE_ASYNC])
def test_tiny_ring_and_tiny_cache(mode):
    # one queue of depth 64 and an 8-line cache while warps pin pages of three arrays:
    # a warp that has to wait lets all of its pins go first
    n, off, cols = synth.rmat_csr(32, 10, 8)
    vals = ((synth.uniform_int(33, cols.size, 32) - 16) / 4.0).astype(np.float32)
    x = ((synth.uniform_int(34, n, 32) - 16) / 4.0).astype(np.float32)
    _, _, total = _layout(off, cols, vals)
    with Ctx(total, cache_bytes=8 * 4096, ways=2, num_queues=1, queue_depth=64) as c:
        col0, val0 = _store(c, off, cols, vals)
        y, ent = _spmv(c, off, cols, vals, x, mode, col0, val0)
        c.check()
        assert np.array_equal(y.view(np.uint32), oracle.spmv(off, cols, vals, x).view(np.uint32))
        assert ent == cols.size


@pytest.mark.parametrize("graph", ["rmat", "uniform"])
def test_hbm_kernel_and_uniform_graph(graph):
    # the breakdown's kernel-time baseline over the CSR in HBM, and the cached SpMV, on
    # RMAT and uniform random ("-U", Sec. 4.5) scale-16 graphs with N(0,1) values
    if graph == "rmat":
        n, off, cols = synth.rmat_csr(44, 16, 16)
    else:
        n, off, cols = synth.uniform_csr(45, 16, 16)
    vals = synth.normal(46, cols.size).astype(np.float32)
    x = synth.normal(47, n).astype(np.float32)
    _, _, total = _layout(off, cols, vals)
    with Ctx(total, cache_bytes=round_page((cols.nbytes + vals.nbytes) // 8) // 32768 * 32768, ways=8) as c:
        d_off = torch.from_numpy(off).to(DEV)
        d_cols = torch.from_numpy(cols).to(DEV)
        d_vals = torch.from_numpy(vals).to(DEV)
        d_x = torch.from_numpy(x).to(DEV)
        d_y = torch.full((n,), float("nan"), dtype=torch.float32, device=DEV)
        ent = torch.zeros(1, dtype=torch.int64, device=DEV)
        ag.agile_spmv_hbm(c.h, d_off.data_ptr(), d_cols.data_ptr(), d_vals.data_ptr(), n, n, int(cols.size),
                          d_x.data_ptr(), d_y.data_ptr(), ent.data_ptr(), c.stream)
        torch.cuda.synchronize()
        c.check()
        _check(off, cols, vals, x, d_y.cpu().numpy())
        assert int(ent.item()) == cols.size and c.stats()["commands"] == 0
        col0, val0 = _store(c, off, cols, vals)
        for mode in (ag.AGILE_SYNC, ag.AGILE_ASYNC):
            y, e2 = _spmv(c, off, cols, vals, x, mode, col0, val0)
            c.check()
            _check(off, cols, vals, x, y)
            assert e2 == cols.size
