"""Closed-form pins of the embedding-bag workload at its stated size (65,536 x 128 FP32
table = 8,192 pages of 8 rows, batches of 256 bags x 16 uniform indices, a 4 MiB cache
of 1,024 lines in 128 sets of 8 ways), checked on the index generator and the oracle's
sequential cache:

  - the distinct pages of a batch: 4,096 uniform draws over 8,192 pages leave a page
    untouched with probability (1 - 1/8192)^4096 (about e^-0.5), so a batch touches
    8192 (1 - (1 - 1/8192)^4096) = 3,223.6 pages on average (occupancy problem; the
    standard deviation of one batch's count is about 21);
  - the steady hit rate of the cache: under uniform references each set s receives the
    share n_s / 8192 of them and keeps 8 of its n_s pages, whatever the replacement
    policy, so the hit rate is sum_s (n_s / 8192)(8 / n_s) = 128 x 8 / 8192 = 1/8.
"""
import numpy as np
import pytest

import oracle
import synth

ROWS, DIM, NB, POOL, BATCHES = 65_536, 128, 256, 16, 16
PAGES = ROWS * DIM * 4 // 4096
ROWS_PER_PAGE = 4096 // (DIM * 4)


def _batches():
    # the index stream of the workload (the bench's config-1 leg draws it the same way)
    return [synth.indices_uniform(2, NB * POOL, ROWS, offset=b * NB * POOL) for b in range(BATCHES)]


def test_distinct_pages_per_batch_match_the_occupancy_formula():
    n = NB * POOL
    want = PAGES * (1.0 - (1.0 - 1.0 / PAGES) ** n)
    sd = np.sqrt(PAGES * ((1 - 1 / PAGES) ** n - (1 + n / PAGES) * (1 - 1 / PAGES) ** (2 * n)))
    counts = np.array([np.unique(b // ROWS_PER_PAGE).size for b in _batches()])
    assert abs(want - 3223.6) < 0.5
    assert 15 < sd < 30
    assert (np.abs(counts - want) < 6 * sd).all(), counts
    assert abs(counts.mean() - want) < 5 * sd / np.sqrt(BATCHES), counts.mean()


@pytest.mark.parametrize("policy", [oracle.RefCache.CLOCK, oracle.RefCache.FIFO])
def test_steady_hit_rate_is_cache_over_table(policy):
    store = np.zeros(PAGES * 4096, dtype=np.uint8)
    ref = oracle.RefCache(128, 8, store, policy=policy)
    pages = [b // ROWS_PER_PAGE for b in _batches()]
    ref.replay(pages[0].astype(np.uint64))   # warm-up batch: the cache fills
    c0 = ref.counters()
    ref.replay(np.concatenate(pages[1:]).astype(np.uint64))
    c1 = ref.counters()
    hits, misses = c1["hits"] - c0["hits"], c1["misses"] - c0["misses"]
    rate = hits / (hits + misses)
    assert hits + misses == (BATCHES - 1) * NB * POOL
    assert abs(rate - 1 / 8) < 0.01, rate
