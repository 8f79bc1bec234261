"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the benchmark.

This module holds no arithmetic of the I/O method itself: it only draws numbers and
builds input data structures (embedding tables, bag index lists, CSR graphs).  Every
draw comes from SplitMix64 (Steele, Lea, Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014), evaluated as a counter-based generator

    z_i = mix(seed + (i + 1) * 0x9E3779B97F4A7C15)

so that the same (seed, counter) pair gives the same value on every machine and in
every numpy version.

Workload shapes follow the paper's evaluation (Sec. 4.4 DLRM embedding lookups with a
Criteo-like skew, Sec. 4.5 BFS over Kronecker graphs in CSR form); public datasets are
not available, so these seeded generators stand in for them.
"""
from __future__ import annotations

import math

import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
PAGE = 4096


def splitmix64(seed: int, counters: np.ndarray) -> np.ndarray:
    """SplitMix64 outputs for the given counters (uint64 array) under ``seed``."""
    with np.errstate(over="ignore"):
        c = np.asarray(counters, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + (c + np.uint64(1)) * GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def uniform01(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """n doubles in [0, 1) with 53 random bits each."""
    u = splitmix64(seed, np.arange(offset, offset + n, dtype=np.uint64))
    return (u >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def uniform_int(seed: int, n: int, hi: int, offset: int = 0) -> np.ndarray:
    """n integers uniform on [0, hi), as int64 (floor(u * hi) with a 53-bit u)."""
    if hi <= 0:
        raise ValueError("hi must be positive")
    u = uniform01(seed, n, offset)
    r = np.floor(u * hi).astype(np.int64)
    return np.minimum(r, hi - 1)


def normal(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """n standard normal doubles by the Box-Muller transform of paired uniforms."""
    m = (n + 1) // 2
    u1 = uniform01(seed, m, 2 * offset)
    u2 = uniform01(seed, m, 2 * offset + m)
    r = np.sqrt(-2.0 * np.log1p(-u1))
    th = 2.0 * math.pi * u2
    z = np.concatenate([r * np.cos(th), r * np.sin(th)])
    return z[:n]


# ----------------------------------------------------------------------------- tables

def table_normal(seed: int, rows: int, dim: int) -> np.ndarray:
    """FP32 embedding table, entries N(0, 1) rounded to float32."""
    return normal(seed, rows * dim).astype(np.float32).reshape(rows, dim)


def table_dyadic(rows: int, dim: int) -> np.ndarray:
    """FP32 table whose entries are multiples of 1/64 below 16.

    Sums of up to 2^18 such values are exact in FP32, so any summation order gives
    the same bits; used to pin pooled sums independently of order.
    """
    r = np.arange(rows, dtype=np.int64)[:, None]
    d = np.arange(dim, dtype=np.int64)[None, :]
    return (((r * 131 + d * 7) % 1024).astype(np.float32) / np.float32(64.0))


# ----------------------------------------------------------------------------- bags

def bags_fixed(n_bags: int, pooling: int) -> np.ndarray:
    """Offsets (int64, length n_bags + 1) for bags of equal size."""
    return np.arange(n_bags + 1, dtype=np.int64) * pooling


def indices_uniform(seed: int, n: int, rows: int, offset: int = 0) -> np.ndarray:
    return uniform_int(seed, n, rows, offset)


class Zipf:
    """Zipf(alpha) ranks on {0, .., n-1} with P(k) proportional to (k + 1)^-alpha.

    Sampled by inversion of the cumulative distribution (a table of n partial sums and
    a binary search), then mapped to rows by the affine bijection
    row = (a * rank + c) mod n with gcd(a, n) = 1 so that hot rows are spread over the
    table instead of packed into its first pages.
    """

    def __init__(self, n: int, alpha: float, permute: bool = True, seed: int = 0):
        self.n = int(n)
        self.alpha = float(alpha)
        w = np.arange(1, self.n + 1, dtype=np.float64) ** (-self.alpha)
        cdf = np.cumsum(w)
        self.cdf = cdf / cdf[-1]
        self.permute = permute
        a = 0x9E3779B1 % self.n if self.n > 1 else 1
        a = max(a, 1)
        while math.gcd(a, self.n) != 1:
            a += 1
        self.a = a
        self.c = (seed * 7919) % self.n if self.n > 0 else 0

    def ranks(self, seed: int, count: int, offset: int = 0) -> np.ndarray:
        u = uniform01(seed, count, offset)
        r = np.searchsorted(self.cdf, u, side="right").astype(np.int64)
        return np.minimum(r, self.n - 1)

    def rows(self, seed: int, count: int, offset: int = 0) -> np.ndarray:
        r = self.ranks(seed, count, offset)
        if not self.permute:
            return r
        return (r * self.a + self.c) % self.n


# ----------------------------------------------------------------------------- graphs

def csr_from_edges(n: int, src: np.ndarray, dst: np.ndarray, symmetrize: bool = True):
    """CSR (int64 offsets [n+1], int32 cols) with self-loops dropped, duplicates removed
    and each neighbour list sorted ascending."""
    src = np.asarray(src, dtype=np.int64)
    dst = np.asarray(dst, dtype=np.int64)
    if symmetrize:
        src, dst = np.concatenate([src, dst]), np.concatenate([dst, src])
    keep = src != dst
    key = np.sort(src[keep] * np.int64(n) + dst[keep])
    if key.size:
        key = key[np.concatenate([[True], key[1:] != key[:-1]])]
    s = key // n
    d = (key % n).astype(np.int32)
    deg = np.bincount(s, minlength=n).astype(np.int64)
    offsets = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(deg, out=offsets[1:])
    return offsets, d


def rmat_edges(seed: int, scale: int, edge_factor: int, a=0.57, b=0.19, c=0.19):
    """R-MAT edge list (Chakrabarti, Zhan, Faloutsos, SDM 2004): for each edge and each of
    ``scale`` bit levels one uniform draw picks a quadrant with probabilities
    (a, b, c, 1 - a - b - c); no vertex relabelling.  Each draw is a 16-bit field of a
    SplitMix64 output (four levels per output), compared with the thresholds scaled
    to 2^16."""
    m = edge_factor << scale
    src = np.zeros(m, dtype=np.int64)
    dst = np.zeros(m, dtype=np.int64)
    ta = np.uint64(round(a * 65536))
    tab = np.uint64(round((a + b) * 65536))
    tabc = np.uint64(round((a + b + c) * 65536))
    edges = np.arange(m, dtype=np.uint64)
    for blk in range((scale + 3) // 4):
        u = splitmix64(seed, edges + np.uint64(blk * m))
        for k in range(4):
            lvl = blk * 4 + k
            if lvl >= scale:
                break
            x = (u >> np.uint64(16 * k)) & np.uint64(0xFFFF)
            sh = np.int64(scale - 1 - lvl)
            right = ((x >= ta) & (x < tab)) | (x >= tabc)   # quadrants b and d set the dst bit
            down = x >= tab                                  # quadrants c and d set the src bit
            src |= down.astype(np.int64) << sh
            dst |= right.astype(np.int64) << sh
    return src, dst


def rmat_csr(seed: int, scale: int, edge_factor: int, a=0.57, b=0.19, c=0.19):
    n = 1 << scale
    s, d = rmat_edges(seed, scale, edge_factor, a, b, c)
    offsets, cols = csr_from_edges(n, s, d, symmetrize=True)
    return n, offsets, cols


def bfs_sources(seed: int, offsets: np.ndarray, count: int) -> np.ndarray:
    """``count`` distinct seeded vertices of positive degree."""
    deg = np.diff(offsets)
    cand = np.nonzero(deg > 0)[0]
    out = []
    k = 0
    while len(out) < count and k < 64 * count + 64:
        v = int(cand[int(uniform_int(seed, 1, len(cand), offset=k)[0])])
        k += 1
        if v not in out:
            out.append(v)
    return np.array(out, dtype=np.int32)


def graph_path(n: int):
    s = np.arange(n - 1)
    return csr_from_edges(n, s, s + 1)


def graph_star(n: int):
    s = np.zeros(n - 1, dtype=np.int64)
    return csr_from_edges(n, s, np.arange(1, n))


def graph_binary_tree(n: int):
    ch = np.arange(1, n)
    return csr_from_edges(n, (ch - 1) // 2, ch)


def graph_uniform(seed: int, n: int, m: int):
    s = uniform_int(seed, m, n)
    d = uniform_int(seed, m, n, offset=m)
    return csr_from_edges(n, s, d)


def uniform_csr(seed: int, scale: int, edge_factor: int):
    """Uniform random graph (Erdos-Renyi style, as GAP's uniform generator: every edge's
    two endpoints drawn uniformly from the 2^scale vertices), edge_factor * 2^scale
    edges, then symmetrised, self-loops dropped, duplicates removed, lists sorted."""
    n = 1 << scale
    offsets, cols = graph_uniform(seed, n, edge_factor << scale)
    return n, offsets, cols


def pages_for(nbytes: int) -> int:
    return (int(nbytes) + PAGE - 1) // PAGE
