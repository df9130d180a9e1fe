"""Seeded synthetic inputs for the APSP library, its tests and its benchmark.

This module only draws random graphs, sizes and arrival times.  It contains none of the
shortest-path arithmetic, so both the CUDA path and the CPU oracle can take their inputs
from it without sharing any of the method.

Cost-matrix convention (the paper's H, Sec. 3.1 and Sec. 3.4): a dense row-major n x n matrix
whose entry [i, j] is the cost of the edge i -> j, the diagonal is 0, and a missing edge holds
the "no edge" sentinel: INF_I32 = 0x3FFFFFFF for int32 matrices and +inf for float32 ones.

Graph families:
  * er_graph: directed Erdos-Renyi, every ordered pair i != j is an edge independently with
    probability p, weights drawn from a named distribution.  Generation runs in fixed blocks
    of rows, each from its own PCG64 stream keyed by (seed, block), so the matrix does not
    depend on how many threads draw it and any row block can be regenerated on its own.
  * paper_graph: the paper's generator f(V, rho, alpha) of Sec. 3.4: a uniform probability
    matrix P scaled by rho, a Bernoulli draw per entry, integer costs in [0, alpha], zero
    diagonal.  rho * P is clipped to [0, 1] (the paper's rho ~ U[0, 100] would otherwise give
    "probabilities" above 1).  paper_sweep draws the paper's 1000 such graphs (Sec. 4).
"""
from __future__ import annotations

import math
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np

INF_I32 = 0x3FFFFFFF
ROWS_PER_BLOCK = 256


def _block_rng(seed: int, block: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64([int(seed), int(block), 0x41505350]))


def _fill_block(out, r0, r1, n, p, dtype, dist, lo, hi, seed, block, inf):
    rng = _block_rng(seed, block)
    rows = r1 - r0
    u = rng.random((rows, n))
    edge = u < p
    if dtype == np.int32:
        w = rng.integers(lo, hi, size=(rows, n), endpoint=True, dtype=np.int64)
        blk = np.where(edge, w, inf).astype(np.int32)
    else:
        if dist == "lognormal":
            w = rng.lognormal(mean=lo, sigma=hi, size=(rows, n))
        elif dist == "uniform01":  # uniform in (0, 1]
            w = 1.0 - rng.random((rows, n))
        elif dist == "uniform":
            w = rng.uniform(lo, hi, size=(rows, n))
        else:
            raise ValueError(f"unknown weight distribution {dist!r}")
        blk = np.where(edge, w, np.inf).astype(np.float32)
    idx = np.arange(r0, r1)
    blk[idx - r0, idx] = 0
    out[r0:r1] = blk


def er_graph(n: int, p: float, dtype="int32", dist: str = "uniform", lo=1, hi=100,
             seed: int = 0, inf: int = INF_I32, threads: int | None = None) -> np.ndarray:
    """Directed Erdos-Renyi cost matrix (n x n, row-major, diagonal 0).

    int32: weights uniform integers in [lo, hi], missing edges = inf.
    float32: dist "lognormal" (lo = mu, hi = sigma), "uniform01" (uniform in (0, 1]) or
    "uniform" (uniform in [lo, hi)); missing edges = +inf.
    """
    dt = np.dtype(dtype)
    if dt not in (np.dtype(np.int32), np.dtype(np.float32)):
        raise ValueError("dtype must be int32 or float32")
    out = np.empty((n, n), dtype=dt)
    if n == 0:
        return out
    nblk = (n + ROWS_PER_BLOCK - 1) // ROWS_PER_BLOCK
    jobs = [(b * ROWS_PER_BLOCK, min(n, (b + 1) * ROWS_PER_BLOCK), b) for b in range(nblk)]
    threads = threads or min(16, os.cpu_count() or 1)
    args = (n, p, dt.type, dist, lo, hi, seed)
    if threads <= 1 or nblk == 1:
        for r0, r1, b in jobs:
            _fill_block(out, r0, r1, *args, b, inf)
    else:
        with ThreadPoolExecutor(threads) as ex:
            list(ex.map(lambda j: _fill_block(out, j[0], j[1], *args, j[2], inf), jobs))
    return out


def paper_graph(V: int, rho: float, alpha: int = 100, seed: int = 0, inf: int = INF_I32) -> np.ndarray:
    """The generator f(V, rho, alpha) of Sec. 3.4 as an int32 cost matrix (missing = inf)."""
    rng = np.random.Generator(np.random.PCG64([int(seed), 0x50415052]))
    P = rng.random((V, V))
    A = rng.random((V, V)) < np.clip(rho * P, 0.0, 1.0)
    H = np.where(A, rng.integers(0, alpha, size=(V, V), endpoint=True), inf).astype(np.int32)
    np.fill_diagonal(H, 0)
    return H


def signed_graph(n: int, p: float, dtype="int32", lo=1, hi=100, pot: float = 60, seed: int = 0,
                 inf: int = INF_I32):
    """A directed graph with negative edges and no negative cycle, by potentials: start from
    er_graph(n, p) with non-negative weights w and draw a potential pi[v] uniform in [0, pot]
    (integers for int32); the edge u -> v gets w(u, v) + pi[u] - pi[v].  Every cycle keeps its
    (non-negative) weight, and every distance becomes d(u, v) + pi[u] - pi[v].
    Returns (cost matrix, pi)."""
    if np.dtype(dtype) == np.int32:
        h = er_graph(n, p, "int32", lo=lo, hi=hi, seed=seed, inf=inf).astype(np.int64)
        rng = np.random.Generator(np.random.PCG64([int(seed), 0x504F5445]))
        pi = rng.integers(0, int(pot), size=n, endpoint=True).astype(np.int64)
        out = np.where(h < inf, h + pi[:, None] - pi[None, :], inf)
        np.fill_diagonal(out, 0)
        return out.astype(np.int32), pi
    h = er_graph(n, p, "float32", dist="uniform", lo=lo, hi=hi, seed=seed).astype(np.float64)
    rng = np.random.Generator(np.random.PCG64([int(seed), 0x504F5445]))
    pi = rng.uniform(0.0, float(pot), size=n)
    out = h + pi[:, None] - pi[None, :]
    np.fill_diagonal(out, 0.0)
    return out.astype(np.float32), pi


def paper_sweep(count: int = 1000, v_lo: int = 4, v_hi: int = 1000, rho_hi: float = 100.0, alpha: int = 100,
                seed: int = 0, threads: int | None = None):
    """The paper's experiment inputs (Sec. 3.4 and Sec. 4): ``count`` graphs f(V, rho, alpha) with V
    uniform on the integers [v_lo, v_hi], rho uniform in [0, rho_hi] and alpha = 100, sorted by
    ascending number of edges as the paper sorts them.  Graph g of the draw is
    paper_graph(V[g], rho[g], alpha, seed=2000 + g).  Returns (ns, rhos, edges, mats) in that order."""
    rng = np.random.Generator(np.random.PCG64([int(seed), 0x53574550]))
    Vs = rng.integers(v_lo, v_hi, size=count, endpoint=True)
    rhos = rng.uniform(0.0, rho_hi, size=count)
    with ThreadPoolExecutor(threads or min(16, os.cpu_count() or 1)) as ex:
        mats = list(ex.map(lambda g: paper_graph(int(Vs[g]), float(rhos[g]), alpha, seed=2000 + g), range(count)))
    edges = np.array([int(np.count_nonzero(m < INF_I32)) - m.shape[0] for m in mats], np.int64)
    order = np.argsort(edges, kind="stable")
    return (Vs[order].astype(np.int64), rhos[order], edges[order], [mats[g] for g in order])


def batch_specs(count: int = 2048, n_lo: int = 32, n_hi: int = 1024, p_lo: float = 0.02,
                p_hi: float = 0.8, seed: int = 0):
    """Sizes and densities of a batch: n log-uniform in [n_lo, n_hi], p uniform in [p_lo, p_hi].

    Graph g of the batch is then er_graph(n[g], p[g], seed=1000 + g).
    """
    rng = np.random.Generator(np.random.PCG64([int(seed), 0x42415443]))
    ns = np.rint(np.exp(rng.uniform(math.log(n_lo), math.log(n_hi), size=count))).astype(np.int64)
    ps = rng.uniform(p_lo, p_hi, size=count)
    return ns, ps


def batch_graphs(ns, ps, dtype="int32", lo=1, hi=100, inf: int = INF_I32, dist: str = "uniform",
                 threads: int | None = None):
    """Graph g = er_graph(ns[g], ps[g], dtype, dist, lo, hi, seed=1000 + g) (float32: dist
    "lognormal" with lo = mu, hi = sigma, as in er_graph), drawn on a pool of threads."""
    def one(g):
        return er_graph(int(ns[g]), float(ps[g]), dtype=dtype, dist=dist, lo=lo, hi=hi, seed=1000 + g, inf=inf,
                        threads=1)
    with ThreadPoolExecutor(threads or min(16, os.cpu_count() or 1)) as ex:
        return list(ex.map(one, range(len(ns))))


def request_library(count: int = 128, n_lo: int = 64, n_hi: int = 8192, p_lo: float = 0.01, p_hi: float = 0.5,
                    seed: int = 0, threads: int | None = None):
    """Graphs for a request stream: entry i has n log-uniform in [n_lo, n_hi], p uniform in
    [p_lo, p_hi]; even entries int32 weights in [1, 100], odd entries float32 lognormal(0, 1).
    Request k of a stream carries entry k mod count (count even keeps the dtype alternation)."""
    rng = np.random.Generator(np.random.PCG64([int(seed), 0x4C494252]))
    ns = np.rint(np.exp(rng.uniform(math.log(n_lo), math.log(n_hi), size=count))).astype(np.int64)
    ps = rng.uniform(p_lo, p_hi, size=count)

    def make(i):
        if i % 2 == 0:
            return er_graph(int(ns[i]), float(ps[i]), "int32", lo=1, hi=100, seed=5000 + i, threads=1)
        return er_graph(int(ns[i]), float(ps[i]), "float32", dist="lognormal", lo=0.0, hi=1.0, seed=5000 + i,
                        threads=1)

    with ThreadPoolExecutor(threads or min(16, os.cpu_count() or 1)) as ex:
        mats = list(ex.map(make, range(count)))
    return ns, ps, mats


class RequestPool:
    """Pre-drawn variates from which request matrices are cut quickly (a serving stream needs
    several GB/s of fresh cost matrices, more than drawing each one from scratch delivers):
    ``u`` holds uniform 32-bit integers, ``logn`` float32 lognormal(0, 1) weights.  Request k
    takes windows of both at offsets drawn from its own seeded stream (see request_matrix)."""

    def __init__(self, seed: int = 0, size_u: int = 1 << 28, size_w: int = 1 << 26, threads: int | None = None):
        blocks = 64
        self.u = np.empty(size_u, np.uint32)
        self.logn = np.empty(size_w, np.float32)

        def fill(b):
            rng = np.random.Generator(np.random.PCG64([int(seed), 0x504F4F4C, int(b)]))
            lo, hi = size_u * b // blocks, size_u * (b + 1) // blocks
            self.u[lo:hi] = rng.integers(0, 1 << 32, size=hi - lo, dtype=np.uint32)
            lo, hi = size_w * b // blocks, size_w * (b + 1) // blocks
            self.logn[lo:hi] = rng.lognormal(0.0, 1.0, size=hi - lo).astype(np.float32)

        with ThreadPoolExecutor(threads or min(16, os.cpu_count() or 1)) as ex:
            list(ex.map(fill, range(blocks)))


def request_matrix(pool: RequestPool, k: int, n: int, p: float, dtype: str, out: np.ndarray | None = None,
                   seed: int = 0, inf: int = INF_I32) -> np.ndarray:
    """The cost matrix of request k: a directed Erdos-Renyi graph on n vertices with edge
    probability p.  Entry (i, j), i != j, is an edge when the pool variate u at the request's
    offset o + i n + j is below p 2^32; an int32 weight is 1 + (u mod 100) (uniform in [1, 100]
    up to a bias below 100 / (p 2^32)), a float32 weight the lognormal(0, 1) variate at the
    request's second offset.  Missing edges hold the sentinel (+inf for float32); the diagonal
    is 0.  ``out`` (n x n, any row stride) receives it in place when given."""
    nn = n * n
    rng = np.random.Generator(np.random.PCG64([int(seed), 0x52455155, int(k)]))
    o = int(rng.integers(0, pool.u.size - nn + 1))
    ow = int(rng.integers(0, pool.logn.size - min(nn, pool.logn.size) + 1))
    thr = np.uint32(min(int(p * 4294967296.0), 4294967295))
    dt = np.dtype(dtype)
    if out is None:
        out = np.empty((n, n), dt)
    rows = max(1, (1 << 22) // max(n, 1))  # about 4M entries per step
    for r0 in range(0, n, rows):
        r1 = min(n, r0 + rows)
        u = pool.u[o + r0 * n: o + r1 * n].reshape(r1 - r0, n)
        edge = u < thr
        if dt == np.int32:
            w = (u % np.uint32(100)).astype(np.int32) + 1
            out[r0:r1] = np.where(edge, w, np.int32(inf))
        else:
            a = (ow + r0 * n) % pool.logn.size
            b = a + (r1 - r0) * n
            wv = pool.logn[a:b] if b <= pool.logn.size else np.concatenate([pool.logn[a:], pool.logn[:b - pool.logn.size]])
            out[r0:r1] = np.where(edge, wv.reshape(r1 - r0, n), np.float32(np.inf))
        idx = np.arange(r0, r1)
        out[idx, idx] = 0
    return out


def poisson_requests(rate: float = 200.0, duration: float = 60.0, n_lo: int = 64, n_hi: int = 8192,
                     p_lo: float = 0.01, p_hi: float = 0.5, seed: int = 0):
    """Arrival times (s), sizes, densities and dtypes of a Poisson request stream.

    Even request ids carry int32 weights uniform in [1, 100]; odd ones float32 lognormal(0, 1).
    """
    rng = np.random.Generator(np.random.PCG64([int(seed), 0x53455256]))
    gaps = rng.exponential(1.0 / rate, size=int(rate * duration * 1.5) + 16)
    t = np.cumsum(gaps)
    t = t[t < duration]
    m = len(t)
    ns = np.rint(np.exp(rng.uniform(math.log(n_lo), math.log(n_hi), size=m))).astype(np.int64)
    ps = rng.uniform(p_lo, p_hi, size=m)
    dtypes = np.where(np.arange(m) % 2 == 0, "int32", "float32")
    return t, ns, ps, dtypes
