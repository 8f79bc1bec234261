"""Pins for the oracle BFS (Sec. 4.5 graph workloads over CSR) and the graph inputs.

Independent references: closed-form levels of paths, stars and binary trees, an
isolated vertex, and scipy's unweighted shortest paths on random graphs.
"""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.csgraph as csg

import oracle
import synth


def test_path_levels_equal_index():
    off, cols = synth.graph_path(50)
    lv, scanned = oracle.bfs(off, cols, 0)
    assert np.array_equal(lv, np.arange(50))
    assert scanned == 2 * 49


def test_star_levels():
    off, cols = synth.graph_star(30)
    lv, scanned = oracle.bfs(off, cols, 0)
    assert lv[0] == 0 and np.all(lv[1:] == 1)
    lv, _ = oracle.bfs(off, cols, 7)
    assert lv[7] == 0 and lv[0] == 1 and np.all(np.delete(lv, [0, 7]) == 2)
    assert scanned == 2 * 29


def test_binary_tree_levels():
    n = 127
    off, cols = synth.graph_binary_tree(n)
    lv, _ = oracle.bfs(off, cols, 0)
    assert np.array_equal(lv, np.floor(np.log2(np.arange(n) + 1)).astype(np.int32))


def test_isolated_vertex_unreached():
    # vertex 9 has no edges
    off, cols = synth.csr_from_edges(10, np.arange(8), np.arange(1, 9))
    lv, scanned = oracle.bfs(off, cols, 0)
    assert lv[9] == -1 and np.array_equal(lv[:9], np.arange(9))
    lv, scanned = oracle.bfs(off, cols, 9)
    assert lv[9] == 0 and np.all(lv[:9] == -1) and scanned == 0


@pytest.mark.parametrize("seed,n,m", [(1, 200, 300), (2, 1000, 3000), (3, 500, 450)])
def test_random_graph_vs_scipy(seed, n, m):
    off, cols = synth.graph_uniform(seed, n, m)
    A = sp.csr_matrix((np.ones(cols.size), cols, off), shape=(n, n))
    for src in synth.bfs_sources(seed, off, 3):
        lv, scanned = oracle.bfs(off, cols, int(src))
        dist = csg.shortest_path(A, unweighted=True, indices=int(src))
        want = np.where(np.isinf(dist), -1, dist).astype(np.int32)
        assert np.array_equal(lv, want)
        deg = np.diff(off)
        assert scanned == int(deg[want >= 0].sum())


def test_rmat_small_csr_valid_and_bfs_vs_scipy():
    n, off, cols = synth.rmat_csr(4, 10, 8)
    assert off[0] == 0 and off[-1] == cols.size and np.all(np.diff(off) >= 0)
    A = sp.csr_matrix((np.ones(cols.size), cols, off), shape=(n, n))
    assert (A != A.T).nnz == 0, "symmetrised"
    assert A.diagonal().sum() == 0, "no self loops"
    for v in range(n):
        nb = cols[off[v]:off[v + 1]]
        assert np.all(np.diff(nb) > 0), "sorted, no duplicates"
    src = int(synth.bfs_sources(4, off, 1)[0])
    lv, _ = oracle.bfs(off, cols, src)
    dist = csg.shortest_path(A, unweighted=True, indices=src)
    assert np.array_equal(lv, np.where(np.isinf(dist), -1, dist).astype(np.int32))
