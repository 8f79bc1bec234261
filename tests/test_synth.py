"""Checks of the seeded input generators (not the method): reproducibility, ranges and
the shape of the distributions the workloads ask for."""
import numpy as np

import synth


def test_splitmix64_reference_values():
    # SplitMix64 seeded with 0: the first outputs of the generator as published with
    # the algorithm (Vigna's splitmix64.c: state += golden gamma, then the mix).
    got = synth.splitmix64(0, np.arange(3, dtype=np.uint64))
    assert [int(x) for x in got] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_uniform_ranges_and_mean():
    u = synth.uniform01(1, 100000)
    assert u.min() >= 0 and u.max() < 1 and abs(u.mean() - 0.5) < 0.01
    k = synth.uniform_int(2, 100000, 7)
    assert k.min() == 0 and k.max() == 6
    assert np.all(np.abs(np.bincount(k) / 1e5 - 1 / 7) < 0.01)


def test_zipf_frequencies():
    z = synth.Zipf(1000, 1.05, permute=False)
    r = z.ranks(3, 200000)
    f = np.bincount(r, minlength=1000) / 200000
    p = np.arange(1, 1001) ** -1.05
    p /= p.sum()
    assert abs(f[0] - p[0]) < 0.01 and abs(f[9] - p[9]) < 0.005
    zp = synth.Zipf(1000, 1.05, permute=True, seed=4)
    rows = zp.rows(3, 1000)
    assert np.array_equal(np.sort(np.unique((np.arange(1000) * zp.a + zp.c) % 1000)), np.arange(1000))
    assert rows.min() >= 0 and rows.max() < 1000


def test_rmat_quadrant_skew():
    s, d = synth.rmat_edges(5, 12, 4)
    # with a = .57 the top-left quadrant holds about a fraction a of all edges at the
    # first level
    half = 1 << 11
    top_left = np.mean((s < half) & (d < half))
    assert abs(top_left - 0.57) < 0.01


def test_generators_deterministic():
    a = synth.rmat_csr(9, 9, 4)
    b = synth.rmat_csr(9, 9, 4)
    assert np.array_equal(a[1], b[1]) and np.array_equal(a[2], b[2])


def test_uniform_csr_is_a_simple_undirected_graph():
    n, off, cols = synth.uniform_csr(3, 10, 8)
    assert n == 1024 and off[0] == 0 and off[-1] == cols.size
    src = np.repeat(np.arange(n), np.diff(off))
    assert (src != cols).all()                                   # no self loops
    pairs = set(zip(src.tolist(), cols.tolist()))
    assert all((b, a) in pairs for a, b in pairs)               # symmetric
    for v in range(n):
        lst = cols[off[v]:off[v + 1]]
        assert (np.diff(lst) > 0).all()                          # sorted, no duplicates
    # about 2 * 8 * 1024 entries (a few duplicates and loops dropped); same seed, same graph
    assert 0.95 * 2 * 8 * 1024 < cols.size <= 2 * 8 * 1024
    n2, off2, cols2 = synth.uniform_csr(3, 10, 8)
    assert np.array_equal(off, off2) and np.array_equal(cols, cols2)
