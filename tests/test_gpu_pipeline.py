"""GPU parity of the lookup + compute pipeline of the overlap experiment (Sec. 4.2 CTC,
Sec. 4.4 prefetch of the next batch) against the oracle, bit for bit."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2504_19365_gb300 as ag  # noqa: E402
from gpu_util import Ctx, assert_cache_invariants, round_page  # noqa: E402

DEV = "cuda:0"


@pytest.mark.parametrize("mode", [ag.AGILE_SYNC, ag.AGILE_ASYNC])
@pytest.mark.parametrize("dim,iters", [(64, 7), (128, 0), (256, 3)])
def test_pipeline_bit_exact(mode, dim, iters):
    n_tables, rows, n_bags, pooling, batches = 3, 5000, 64, 8, 3
    tables = [synth.table_normal(40 + k, rows, dim) for k in range(n_tables)]
    stride = round_page(rows * dim * 4)
    zipf = synth.Zipf(rows, 1.05, permute=True, seed=3)
    idx = zipf.rows(41, batches * n_tables * n_bags * pooling).reshape(batches, n_tables, n_bags, pooling)
    want = oracle.embedding_pipeline(tables, idx, pooling, iters)
    with Ctx(stride * n_tables, cache_bytes=96 * 4096, ways=8, num_queues=16, queue_depth=64) as c:
        for k in range(n_tables):
            c.put(k * stride, tables[k])
        d_idx = torch.from_numpy(np.ascontiguousarray(idx)).to(DEV)
        out = torch.full((batches, n_bags, n_tables * dim), float("nan"), dtype=torch.float32, device=DEV)
        ag.agile_embedding_pipeline(c.h, 0, stride, n_tables, rows, dim, d_idx.data_ptr(), pooling, n_bags, batches,
                                    iters, out.data_ptr(), mode, c.stream)
        torch.cuda.synchronize()
        c.check()
        assert np.array_equal(out.cpu().numpy().view(np.uint32), want.view(np.uint32))
        assert_cache_invariants(c)
