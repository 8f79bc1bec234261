"""Pins for the oracle's SpMV over CSR (Sec. 4.5 runs SpMV on the graphs of its BFS).

Independent references: scipy.sparse in float64 within the float32 error bound, exact
dyadic values (any order gives the same bits), the identity matrix, empty rows, a row
whose left-to-right rounding is observable, and brute force from dense on a tiny
matrix."""
import numpy as np
import pytest

import oracle
import synth

sp = pytest.importorskip("scipy.sparse")


def _values(seed, n):
    return synth.normal(seed, n).astype(np.float32)


def test_vs_scipy_float64_within_bound():
    n, off, cols = synth.rmat_csr(11, 10, 8)
    vals = _values(12, cols.size)
    x = _values(13, n)
    y = oracle.spmv(off, cols, vals, x)
    A = sp.csr_matrix((vals.astype(np.float64), cols, off), shape=(n, n))
    ref = A @ x.astype(np.float64)
    absA = sp.csr_matrix((np.abs(vals.astype(np.float64)), cols, off), shape=(n, n))
    mag = absA @ np.abs(x.astype(np.float64))
    deg = np.diff(off)
    # n terms, each product rounded once, n-1 roundings of the sum: |err| <= n u sum|a x|
    bound = (deg + 1) * 2.0 ** -24 * mag + 1e-30
    assert np.all(np.abs(y - ref) <= bound)


def test_dyadic_values_exact():
    n, off, cols = synth.rmat_csr(14, 9, 8)
    vals = ((synth.uniform_int(15, cols.size, 64) - 32) / 16.0).astype(np.float32)
    x = ((synth.uniform_int(16, n, 64) - 32) / 16.0).astype(np.float32)
    y = oracle.spmv(off, cols, vals, x)
    A = sp.csr_matrix((vals.astype(np.float64), cols, off), shape=(n, n))
    assert np.array_equal(y.astype(np.float64), A @ x.astype(np.float64))


def test_identity_and_empty_rows():
    n = 50
    # rows i with i % 7 == 0 are empty; the others hold their diagonal entry
    off = np.zeros(n + 1, dtype=np.int64)
    cols, vals = [], []
    for i in range(n):
        if i % 7:
            cols.append(i)
            vals.append(1.0)
        off[i + 1] = len(cols)
    x = _values(17, n)
    y = oracle.spmv(off, np.array(cols, dtype=np.int32), np.array(vals, dtype=np.float32), x)
    for i in range(n):
        if i % 7:
            assert y[i] == x[i]
        else:
            assert y[i] == 0.0 and not np.signbit(y[i])


def test_left_to_right_order_observable():
    off = np.array([0, 3], dtype=np.int64)
    cols = np.array([0, 1, 2], dtype=np.int32)
    vals = np.array([1e8, 1.0, -1e8], dtype=np.float32)
    x = np.ones(3, dtype=np.float32)
    y = oracle.spmv(off, cols, vals, x)
    want = np.float32(np.float32(np.float32(0) + np.float32(1e8)) + np.float32(1.0)) + np.float32(-1e8)
    assert y[0] == want == np.float32(0.0)


def test_brute_force_dense_tiny():
    rng_vals = _values(18, 40)
    n = 8
    dense = np.zeros((n, n), dtype=np.float32)
    k = 0
    off = np.zeros(n + 1, dtype=np.int64)
    cols = []
    vals = []
    for i in range(n):
        for j in range(n):
            if (i * 3 + j * 5) % 4 == 0:
                dense[i, j] = rng_vals[k % 40]
                cols.append(j)
                vals.append(dense[i, j])
                k += 1
        off[i + 1] = len(cols)
    x = _values(19, n)
    y = oracle.spmv(off, np.array(cols, dtype=np.int32), np.array(vals, dtype=np.float32), x)
    for i in range(n):
        acc = np.float32(0.0)
        for j in range(n):
            if dense[i, j] != 0:
                acc = np.float32(acc + np.float32(dense[i, j] * x[j]))
        assert y[i] == acc


def test_product_rounded_before_the_add():
    # (1 + 2^-12)^2 = 1 + 2^-11 + 2^-24 rounds to 1 + 2^-11 in float32 (a tie, to even);
    # added to -(1 + 2^-11) that gives 0, where a fused multiply-add would give 2^-24
    a = np.float32(1 + 2.0 ** -12)
    off = np.array([0, 2], dtype=np.int64)
    cols = np.array([0, 1], dtype=np.int32)
    vals = np.array([-(1 + 2.0 ** -11), a], dtype=np.float32)
    x = np.array([1.0, a], dtype=np.float32)
    y = oracle.spmv(off, cols, vals, x)
    assert y[0] == 0.0
