"""GPU tests of the serving loop: lookup requests of uneven sizes submitted while others
run are served in one resident session, and every request's result is bit-identical
alone and in the mix (and equal to the oracle)."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2504_19365_gb300 as ag  # noqa: E402
from gpu_util import Ctx, assert_cache_invariants, round_page  # noqa: E402

DEV = "cuda:0"


def _requests(seed, n, tables, stride, rows, dim):
    reqs, keep, want = [], [], []
    sizes = np.minimum(4096, np.maximum(1, np.round(2.0 ** (synth.uniform01(seed, n) * 9)))).astype(int)
    pools = synth.uniform_int(seed + 1, n, 64) + 1
    which = synth.uniform_int(seed + 2, n, len(tables))
    for i in range(n):
        nb, pool, k = int(sizes[i]), int(pools[i]), int(which[i])
        zipf = synth.Zipf(rows, 1.05, permute=True, seed=k)
        idx = zipf.rows(seed * 1000 + i, nb * pool)
        off = synth.bags_fixed(nb, pool)
        want.append(oracle.embedding_bag(tables[k], idx, off))
        d_idx = torch.from_numpy(idx).to(DEV)
        d_off = torch.from_numpy(off).to(DEV)
        out = torch.full((nb, dim), float("nan"), dtype=torch.float32, device=DEV)
        keep.append((d_idx, d_off, out))
        reqs.append(ag.agile_lookup_req(k * stride, rows, dim, d_idx.data_ptr(), d_off.data_ptr(), nb, out.data_ptr()))
    return reqs, keep, want


def _setup(c, n_tables, rows, dim):
    stride = round_page(rows * dim * 4)
    tables = [synth.table_normal(60 + k, rows, dim) for k in range(n_tables)]
    for k in range(n_tables):
        c.put(k * stride, tables[k])
    return tables, stride


@pytest.mark.parametrize("mode", [ag.AGILE_SYNC, ag.AGILE_ASYNC])
def test_mixed_requests_equal_alone_and_oracle(mode):
    n_tables, rows, dim = 3, 20000, 64
    with Ctx(n_tables * round_page(rows * dim * 4), cache_bytes=512 * 4096, ways=8, num_queues=32,
             queue_depth=128) as c:
        tables, stride = _setup(c, n_tables, rows, dim)
        reqs, keep, want = _requests(3, 40, tables, stride, rows, dim)
        srv = ag.agile_serve_start(c.h, 64, mode, 0, c.stream)
        seqs = []
        for r in reqs:
            q = ag.agile_serve_submit(srv, r)
            assert q is not None
            seqs.append(q)
        ag.agile_serve_stop(srv)
        torch.cuda.synchronize()
        c.check()
        for i, (d_idx, d_off, out) in enumerate(keep):
            got = out.cpu().numpy()
            assert np.array_equal(got.view(np.uint32), want[i].view(np.uint32)), i
            # the same request alone, through agile_embedding_bag
            alone = torch.empty_like(out)
            ag.agile_embedding_bag(c.h, reqs[i].table_byte0, rows, dim, d_idx.data_ptr(), d_off.data_ptr(),
                                   reqs[i].n_bags, alone.data_ptr(), mode, c.stream)
            torch.cuda.synchronize()
            assert torch.equal(alone, out)
        assert_cache_invariants(c)


def test_small_ring_defers_and_finishes():
    n_tables, rows, dim = 2, 8000, 128
    with Ctx(n_tables * round_page(rows * dim * 4), cache_bytes=128 * 4096, ways=8, num_queues=16,
             queue_depth=64) as c:
        tables, stride = _setup(c, n_tables, rows, dim)
        reqs, keep, want = _requests(5, 30, tables, stride, rows, dim)
        srv = ag.agile_serve_start(c.h, 4, ag.AGILE_ASYNC, 0, c.stream)
        pending = list(range(len(reqs)))
        seqs = {}
        deferred = 0
        import time
        t_end = time.time() + 60
        while pending and time.time() < t_end:
            i = pending[0]
            q = ag.agile_serve_submit(srv, reqs[i])
            if q is None:
                deferred += 1
                continue
            seqs[i] = q
            pending.pop(0)
        assert not pending
        assert all(ag.agile_serve_poll(srv, q) in (0, 1) for q in seqs.values())
        ag.agile_serve_stop(srv)
        torch.cuda.synchronize()
        c.check()
        assert deferred > 0, "a 4-entry ring must have refused some submissions"
        for i, (_, _, out) in enumerate(keep):
            assert np.array_equal(out.cpu().numpy().view(np.uint32), want[i].view(np.uint32))


def test_replay_trace_latencies():
    n_tables, rows, dim = 2, 10000, 64
    with Ctx(n_tables * round_page(rows * dim * 4), cache_bytes=256 * 4096, ways=8) as c:
        tables, stride = _setup(c, n_tables, rows, dim)
        reqs, keep, want = _requests(7, 50, tables, stride, rows, dim)
        gaps = -np.log1p(-synth.uniform01(8, len(reqs))) * 200_000   # Poisson, mean 200 us
        arrival = np.cumsum(gaps).astype(np.uint64)
        lat = np.zeros(len(reqs), dtype=np.uint64)
        ag.agile_serve_replay(c.h, reqs, arrival.ctypes.data, lat.ctypes.data, ag.AGILE_ASYNC, c.stream)
        torch.cuda.synchronize()
        c.check()
        assert (lat > 0).all()
        for i, (_, _, out) in enumerate(keep):
            assert np.array_equal(out.cpu().numpy().view(np.uint32), want[i].view(np.uint32))
