"""Pins for the oracle's sum-pooled embedding bag, its backward and the SGD step
(Sec. 4.4 DLRM embedding lookups).

Independent references: exact dyadic sums (any order gives the same bits), torch's
``embedding_bag`` and autograd in float64 (a library routine), fp64 central finite
differences, a single-index bag that must copy the row, and empty bags.
"""
import numpy as np
import pytest
import torch

import oracle
import synth


def _bags(seed, n_bags, rows, lo=0, hi=9):
    sizes = synth.uniform_int(seed, n_bags, hi - lo + 1) + lo
    off = np.zeros(n_bags + 1, dtype=np.int64)
    np.cumsum(sizes, out=off[1:])
    idx = synth.uniform_int(seed + 1, int(off[-1]), rows)
    return idx, off


def test_dyadic_exact_vs_float64_sum():
    T = synth.table_dyadic(300, 40)
    idx, off = _bags(1, 64, 300)
    out = oracle.embedding_bag(T, idx, off)
    T64 = T.astype(np.float64)
    for b in range(64):
        want = T64[idx[off[b]:off[b + 1]]].sum(axis=0)
        assert np.array_equal(out[b].astype(np.float64), want)


def test_normal_table_vs_torch_embedding_bag():
    T = synth.table_normal(2, 500, 32)
    idx, off = _bags(3, 100, 500)
    out = oracle.embedding_bag(T, idx, off)
    ref = torch.nn.functional.embedding_bag(
        torch.from_numpy(idx), torch.from_numpy(T.astype(np.float64)),
        torch.from_numpy(off[:-1]), mode="sum").numpy()
    # float32 accumulation vs float64: |err| <= n * eps32 * sum|x|
    absT = np.abs(T.astype(np.float64))
    for b in range(100):
        n = off[b + 1] - off[b]
        bound = n * 2.0 ** -24 * absT[idx[off[b]:off[b + 1]]].sum(axis=0) + 1e-30
        assert np.all(np.abs(out[b] - ref[b]) <= bound)


def test_fixed_order_is_left_to_right_float32():
    # the accumulation order is observable with non-associative values
    T = np.array([[1e8], [1.0], [-1e8]], dtype=np.float32)
    idx = np.array([0, 1, 2], dtype=np.int64)
    off = np.array([0, 3], dtype=np.int64)
    out = oracle.embedding_bag(T, idx, off)
    want = np.float32(np.float32(np.float32(0) + np.float32(1e8)) + np.float32(1.0)) + np.float32(-1e8)
    assert out[0, 0] == want == np.float32(0.0)


def test_pooling_one_copies_rows_and_empty_bags_are_zero():
    T = synth.table_normal(4, 64, 16)
    idx = np.array([5, 7, 63], dtype=np.int64)
    off = np.array([0, 1, 1, 2, 3], dtype=np.int64)   # bag 1 is empty
    out = oracle.embedding_bag(T, idx, off)
    assert np.array_equal(out[0], T[5]) and np.array_equal(out[2], T[7])
    assert np.array_equal(out[3], T[63])
    assert np.all(out[1] == 0) and not np.signbit(out[1]).any()


def test_backward_vs_torch_autograd():
    rows, dim = 200, 24
    T = synth.table_normal(5, rows, dim).astype(np.float64)
    idx, off = _bags(6, 50, rows)
    gout = synth.table_dyadic(50, dim)
    G, touched = oracle.embedding_bag_backward(rows, idx, off, gout)
    Tt = torch.tensor(T, requires_grad=True)
    o = torch.nn.functional.embedding_bag(torch.from_numpy(idx), Tt, torch.from_numpy(off[:-1]),
                                          mode="sum")
    (o * torch.from_numpy(gout.astype(np.float64))).sum().backward()
    # dyadic gout: all partial sums exact in float32
    assert np.array_equal(G.astype(np.float64), Tt.grad.numpy())
    assert np.array_equal(touched.astype(bool), np.isin(np.arange(rows), idx))


def test_backward_finite_differences():
    # loss = sum(out * gout) is linear in T, so the fp64 central difference equals the
    # gradient up to rounding
    rows, dim = 12, 3
    T = synth.table_normal(7, rows, dim).astype(np.float64)
    idx, off = _bags(8, 6, rows, 1, 5)
    gout = synth.normal(9, 6 * dim).reshape(6, dim).astype(np.float32)
    G, _ = oracle.embedding_bag_backward(rows, idx, off, gout)

    def loss(t):
        s = 0.0
        for b in range(6):
            s += float((t[idx[off[b]:off[b + 1]]].sum(axis=0) * gout[b].astype(np.float64)).sum())
        return s

    h = 1e-3
    fd = np.zeros_like(T)
    for r in range(rows):
        for d in range(dim):
            tp, tm = T.copy(), T.copy()
            tp[r, d] += h
            tm[r, d] -= h
            fd[r, d] = (loss(tp) - loss(tm)) / (2 * h)
    assert np.allclose(G, fd, rtol=1e-5, atol=1e-5)


def test_sgd_vs_torch_optimizer_dyadic():
    rows, dim = 64, 8
    T = synth.table_dyadic(rows, dim)
    idx, off = _bags(10, 20, rows)
    gout = synth.table_dyadic(20, dim)
    lr = 2.0 ** -6
    G, touched = oracle.embedding_bag_backward(rows, idx, off, gout)
    newT = oracle.sgd(T, G, touched, lr)
    p = torch.nn.Parameter(torch.tensor(T.astype(np.float64)))
    opt = torch.optim.SGD([p], lr=lr)
    p.grad = torch.tensor(G.astype(np.float64))
    opt.step()
    assert np.array_equal(newT.astype(np.float64), p.detach().numpy())
    # untouched rows are unchanged bit for bit
    assert np.array_equal(newT[touched == 0], T[touched == 0])


def test_ideal_speedup_eq1():
    assert oracle.ideal_speedup(0.0) == 1.0
    assert oracle.ideal_speedup(0.5) == 1.5
    assert oracle.ideal_speedup(1.0) == 2.0
    assert oracle.ideal_speedup(2.0) == 1.5
    assert oracle.ideal_speedup(4.0) == 1.25
    # continuous at CTC = 1 and maximal there
    xs = np.linspace(0, 3, 301)
    ys = [oracle.ideal_speedup(x) for x in xs]
    assert max(ys) == 2.0 and abs(xs[int(np.argmax(ys))] - 1.0) < 1e-12


def test_fma_chain_is_correctly_rounded_fma():
    # x*a + b is exact in float64 for |x| in [2^-5, 2^10] (x: 24 bits, a: 13 bits, b = 2^-10),
    # so rounding it once to float32 is the fused multiply-add by definition
    u = synth.uniform01(12, 4000)
    x = ((u * 2 - 1) * 2.0 ** (u * 15 - 5)).astype(np.float32)
    x = x[np.abs(x) >= 2.0 ** -5]
    want = (x.astype(np.float64) * oracle.FMA_A + oracle.FMA_B).astype(np.float32)
    assert np.array_equal(oracle.fma_chain(x, 1), want)
    y = x.copy()
    for _ in range(6):
        y = (y.astype(np.float64) * oracle.FMA_A + oracle.FMA_B).astype(np.float32)
    assert np.array_equal(oracle.fma_chain(x, 6), y)
    assert np.array_equal(oracle.fma_chain(x, 0), x)


def test_embedding_pipeline_composes_bag_and_chain():
    tables = [synth.table_normal(20 + k, 300, 16) for k in range(3)]
    idx = synth.indices_uniform(30, 2 * 3 * 10 * 4, 300).reshape(2, 3, 10, 4)
    got = oracle.embedding_pipeline(tables, idx, 4, 3)
    off = np.arange(11, dtype=np.int64) * 4
    for t in range(2):
        for k in range(3):
            want = oracle.fma_chain(oracle.embedding_bag(tables[k], idx[t, k].reshape(-1), off), 3)
            assert np.array_equal(got[t, :, k * 16:(k + 1) * 16], want)
