"""Pins for the CPU oracle: each check compares it with something other than itself.

  * brute force: enumeration of every simple path on graphs of <= 7 vertices (the definition
    of a shortest distance, Sec. 2), written here independently of the oracle;
  * library routines: scipy's Dijkstra/Johnson and networkx's Floyd-Warshall;
  * closed forms: path, cycle, complete and empty graphs, n = 0 and n = 1;
  * a hand-worked example (tests/golden/hand_6node.json);
  * the (min,+) product against the paper's own 3-D broadcast formulation (Sec. 3.1:
    L = H[:, :, None] + H'[None, :, :], then a min over the middle axis), its identity
    element and K = 1;
  * invariants and idempotence;
  * planted mistakes: variants of the oracle compiled with a deliberate error must each
    fail at least one of these pins.
"""
import itertools
import json
import os

import numpy as np
import pytest

import oracle
import workloads

INF = oracle.INF_I32
HERE = os.path.dirname(os.path.abspath(__file__))


def _rand_graph(rng, n, p, dtype, zero_diag=True):
    if dtype == np.int32:
        w = rng.integers(0, 20, size=(n, n))
        h = np.where(rng.random((n, n)) < p, w, INF).astype(np.int32)
    else:
        w = rng.lognormal(0.0, 1.0, size=(n, n))
        h = np.where(rng.random((n, n)) < p, w, np.inf).astype(np.float32)
    if zero_diag:
        np.fill_diagonal(h, 0)
    return h


def _brute_force(h):
    """min over every simple path i -> j of the summed edge costs (exact; n <= 7)."""
    n = h.shape[0]
    isint = h.dtype.kind in "iu"
    edge = (h < INF) if isint else np.isfinite(h)
    unreach = INF if isint else np.inf
    out = np.full((n, n), unreach, dtype=np.int64 if isint else np.float64)
    for i in range(n):
        out[i, i] = 0
        others = [v for v in range(n) if v != i]
        for L in range(1, n):
            for mids in itertools.permutations(others, L - 1):
                for j in others:
                    if j in mids:
                        continue
                    path = (i,) + mids + (j,)
                    if all(edge[a, b] for a, b in zip(path, path[1:])):
                        cost = sum((int(h[a, b]) if isint else float(h[a, b])) for a, b in zip(path, path[1:]))
                        if cost < out[i, j]:
                            out[i, j] = cost
    if isint:
        out = np.minimum(out, INF)
    return out


@pytest.mark.parametrize("dtype", [np.int32, np.float32])
def test_fw_matches_simple_path_enumeration(dtype):
    rng = np.random.default_rng(1)
    for trial in range(120):
        n = int(rng.integers(1, 8))
        h = _rand_graph(rng, n, float(rng.uniform(0.1, 0.9)), dtype)
        got = oracle.fw(h)
        want = _brute_force(h)
        if dtype == np.int32:
            assert np.array_equal(got.astype(np.int64), want), (trial, h, got, want)
        else:
            assert np.allclose(got, want, rtol=1e-12, atol=0), (trial, h, got, want)


def test_golden_hand_example():
    g = json.load(open(os.path.join(HERE, "golden", "hand_6node.json")))
    n, inf = g["n"], g["inf"]
    h = np.full((n, n), inf, np.int32)
    np.fill_diagonal(h, 0)
    for u, v, c in g["edges"]:
        h[u, v] = c
    assert np.array_equal(oracle.fw(h, inf=inf), np.array(g["expected"], np.int32))


@pytest.mark.parametrize("dtype,n,p", [(np.int32, 120, 0.05), (np.int32, 300, 0.3),
                                       (np.float32, 150, 0.1), (np.float32, 257, 0.02)])
def test_fw_matches_scipy(dtype, n, p):
    sp = pytest.importorskip("scipy.sparse.csgraph")
    if dtype == np.int32:
        h = workloads.er_graph(n, p, "int32", lo=1, hi=100, seed=n)
        dense = np.where(h < INF, h.astype(np.float64), np.inf)
    else:
        h = workloads.er_graph(n, p, "float32", dist="lognormal", lo=0.0, hi=1.0, seed=n)
        dense = h.astype(np.float64)
    g = sp.csgraph_from_dense(dense, null_value=np.inf)
    ref = sp.shortest_path(g, method="D", directed=True)
    got = oracle.fw(h)
    if dtype == np.int32:
        ref = np.where(np.isinf(ref), INF, ref).astype(np.int64)
        assert np.array_equal(got.astype(np.int64), ref)
    else:
        assert np.array_equal(np.isinf(got), np.isinf(ref))
        f = np.isfinite(ref)
        assert np.allclose(got[f], ref[f], rtol=1e-12, atol=0)


def test_fw_matches_networkx():
    nx = pytest.importorskip("networkx")
    h = workloads.er_graph(40, 0.1, "int32", lo=1, hi=50, seed=7)
    G = nx.DiGraph()
    G.add_nodes_from(range(40))
    for i, j in zip(*np.nonzero(oracle.edge_mask(h))):
        G.add_edge(int(i), int(j), weight=int(h[i, j]))
    ref = nx.floyd_warshall_numpy(G, nodelist=list(range(40)), weight="weight")
    ref = np.where(np.isinf(ref), INF, ref).astype(np.int64)
    assert np.array_equal(oracle.fw(h).astype(np.int64), ref)


@pytest.mark.parametrize("dtype", [np.int32, np.float32])
def test_dijkstra_rows_match_fw(dtype):
    if dtype == np.int32:
        h = workloads.er_graph(200, 0.03, "int32", lo=1, hi=1000, seed=3)
    else:
        h = workloads.er_graph(200, 0.03, "float32", dist="uniform01", seed=3)
    full = oracle.fw(h)
    src = [0, 5, 17, 199]
    rows = oracle.dijkstra_rows(h, src, threads=2)
    if dtype == np.int32:
        assert np.array_equal(rows, full[src])
    else:
        assert np.array_equal(np.isinf(rows), np.isinf(full[src]))
        f = np.isfinite(rows)
        assert np.allclose(rows[f], full[src][f], rtol=1e-12)


def test_closed_forms():
    n = 9
    w = np.arange(1, n, dtype=np.int64) * 3
    # directed path 0 -> 1 -> ... -> n-1: d[i, j] = sum of w[i..j-1] for i < j, unreachable otherwise
    h = np.full((n, n), INF, np.int32)
    np.fill_diagonal(h, 0)
    for i in range(n - 1):
        h[i, i + 1] = w[i]
    d = oracle.fw(h).astype(np.int64)
    pref = np.concatenate([[0], np.cumsum(w)])
    for i in range(n):
        for j in range(n):
            assert d[i, j] == (pref[j] - pref[i] if i <= j else INF)
    # directed cycle: going round from i to j costs the arc length
    h[n - 1, 0] = 5
    total = int(pref[-1]) + 5
    d = oracle.fw(h).astype(np.int64)
    for i in range(n):
        for j in range(n):
            fwd = pref[j] - pref[i] if i <= j else total - (pref[i] - pref[j])
            assert d[i, j] == fwd
    # complete graph with unit weights: every distinct pair at distance 1
    h = np.ones((n, n), np.int32)
    np.fill_diagonal(h, 0)
    assert np.array_equal(oracle.fw(h), h)
    # empty graph: nothing changes; diagonal is forced to zero
    h = np.full((n, n), INF, np.int32)
    np.fill_diagonal(h, 7)
    want = np.full((n, n), INF, np.int32)
    np.fill_diagonal(want, 0)
    assert np.array_equal(oracle.fw(h), want)
    # n = 1 and n = 0
    assert oracle.fw(np.array([[4]], np.int32))[0, 0] == 0
    assert oracle.fw(np.zeros((0, 0), np.int32)).shape == (0, 0)
    # float: +inf off the path, exact prefix sums of dyadic weights
    hf = np.full((4, 4), np.inf, np.float32)
    np.fill_diagonal(hf, 0)
    hf[0, 1], hf[1, 2], hf[2, 3] = 0.5, 0.25, 0.125
    df = oracle.fw(hf)
    assert df[0, 3] == 0.875 and np.isinf(df[3, 0])


def _broadcast_minplus(x, y, inf=None):
    """Sec. 3.1: the 3-D tensor L[i, k, j] = x[i, k] + y[k, j], then min over k."""
    if inf is not None:
        X = np.where(x >= inf, np.inf, x.astype(np.float64))
        Y = np.where(y >= inf, np.inf, y.astype(np.float64))
        Z = (X[:, :, None] + Y[None, :, :]).min(axis=1) if x.shape[1] else np.full((x.shape[0], y.shape[1]), np.inf)
        return np.where(np.isinf(Z), inf, Z).astype(np.int64)
    return (x.astype(np.float64)[:, :, None] + y.astype(np.float64)[None, :, :]).min(axis=1)


@pytest.mark.parametrize("M,N,K", [(1, 1, 1), (7, 5, 3), (33, 17, 31), (40, 64, 1), (12, 9, 65)])
def test_minplus_matches_broadcast_tensor(M, N, K):
    rng = np.random.default_rng(M * 100 + N * 10 + K)
    x = np.where(rng.random((M, K)) < 0.7, rng.integers(0, 1000, (M, K)), INF).astype(np.int32)
    y = np.where(rng.random((K, N)) < 0.7, rng.integers(0, 1000, (K, N)), INF).astype(np.int32)
    assert np.array_equal(oracle.minplus(x, y).astype(np.int64), _broadcast_minplus(x, y, INF))
    z = rng.integers(0, 3000, (M, N)).astype(np.int32)
    want = np.minimum(z.astype(np.int64), _broadcast_minplus(x, y, INF))
    assert np.array_equal(oracle.minplus(x, y, z).astype(np.int64), want)
    xf, yf = rng.lognormal(size=(M, K)).astype(np.float32), rng.lognormal(size=(K, N)).astype(np.float32)
    assert np.array_equal(oracle.minplus(xf, yf), _broadcast_minplus(xf, yf))


def _rows_pin_passes(lib):
    """Selected rows of the product (unsorted, repeated, with a fold into z) against the paper's
    3-D broadcast formulation of the same rows; True if every case agrees."""
    rng = np.random.default_rng(77)
    for M, N, K in [(9, 7, 5), (31, 40, 17), (16, 3, 64), (5, 5, 1)]:
        rows = rng.integers(0, M, size=6)
        x = np.where(rng.random((M, K)) < 0.6, rng.integers(0, 1000, (M, K)), INF).astype(np.int32)
        y = np.where(rng.random((K, N)) < 0.6, rng.integers(0, 1000, (K, N)), INF).astype(np.int32)
        want = _broadcast_minplus(x[rows], y, INF)
        if not np.array_equal(oracle.minplus_rows(x, y, rows, lib=lib).astype(np.int64), want):
            return False
        z = rng.integers(0, 1500, (len(rows), N)).astype(np.int32)
        if not np.array_equal(oracle.minplus_rows(x, y, rows, z=z, lib=lib).astype(np.int64),
                              np.minimum(z.astype(np.int64), want)):
            return False
        xf = np.where(rng.random((M, K)) < 0.6, rng.lognormal(size=(M, K)), np.inf).astype(np.float32)
        yf = np.where(rng.random((K, N)) < 0.6, rng.lognormal(size=(K, N)), np.inf).astype(np.float32)
        if not np.array_equal(oracle.minplus_rows(xf, yf, rows, threads=3, lib=lib), _broadcast_minplus(xf[rows], yf)):
            return False
    return True


def test_minplus_rows_match_broadcast_tensor():
    assert _rows_pin_passes(oracle.load())


def test_minplus_rows_pin_catches_a_wrong_row():
    """Plant 8 reads the r-th row of X instead of row rows[r]: the pin must fail."""
    assert not _rows_pin_passes(oracle.load(plant=8))


def test_minplus_rows_equal_full_product():
    h = workloads.er_graph(300, 0.05, "int32", lo=1, hi=100, seed=4)
    rows = np.array([0, 299, 17, 150])
    assert np.array_equal(oracle.minplus_rows(h, h, rows, threads=4), oracle.minplus(h, h)[rows])
    hf = workloads.er_graph(200, 0.1, "float32", dist="uniform01", seed=4)
    assert np.array_equal(oracle.minplus_rows(hf, hf, rows[rows < 200]), oracle.minplus(hf, hf)[rows[rows < 200]])


def test_minplus_identity_and_outer_sum():
    rng = np.random.default_rng(5)
    n = 23
    eye = np.full((n, n), INF, np.int32)
    np.fill_diagonal(eye, 0)
    b = rng.integers(0, 500, (n, 11)).astype(np.int32)
    assert np.array_equal(oracle.minplus(eye, b), b)
    a = rng.integers(0, 500, (13, n)).astype(np.int32)
    assert np.array_equal(oracle.minplus(a, eye), a)
    x = rng.integers(0, 500, (6, 1)).astype(np.int32)
    y = rng.integers(0, 500, (1, 8)).astype(np.int32)
    assert np.array_equal(oracle.minplus(x, y), x + y)


@pytest.mark.parametrize("dtype", [np.int32, np.float32])
def test_invariants_and_idempotence(dtype):
    if dtype == np.int32:
        h = workloads.er_graph(160, 0.04, "int32", lo=1, hi=100, seed=11)
    else:
        h = workloads.er_graph(160, 0.04, "float32", dist="lognormal", lo=0.0, hi=1.0, seed=11)
    d = oracle.fw(h)
    assert oracle.check_invariants(d, h, rtol=0 if dtype == np.int32 else 1e-12) == []
    sq = oracle.minplus(d, d)
    if dtype == np.int32:
        assert np.array_equal(sq, d)
    else:
        assert np.array_equal(np.isinf(sq), np.isinf(d))
        f = np.isfinite(d)
        assert np.allclose(sq[f], d[f], rtol=1e-12)
    # a wrong matrix must be flagged: raise one reachable entry above a path through k
    bad = d.copy()
    i, j = np.argwhere((d > 0) & (d < (INF if dtype == np.int32 else np.inf)))[0]
    bad[i, j] = bad[i, j] + 1
    assert oracle.check_invariants(bad, h, rtol=0 if dtype == np.int32 else 1e-12) != []


def _pins_pass(lib):
    """Run a compact set of the pins above against an oracle library; True if all pass."""
    rng = np.random.default_rng(2)
    for _ in range(40):
        n = int(rng.integers(2, 7))
        h = _rand_graph(rng, n, 0.5, np.int32, zero_diag=False)  # a self-loop still costs 0
        if not np.array_equal(oracle.fw(h, lib=lib).astype(np.int64), _brute_force(h)):
            return False
    for M in (5, 8):
        x = rng.integers(0, 100, (M, M)).astype(np.int32)
        y = rng.integers(0, 100, (M, M)).astype(np.int32)
        if not np.array_equal(oracle.minplus(x, y, lib=lib).astype(np.int64), _broadcast_minplus(x, y, INF)):
            return False
    return True


def test_pins_pass_on_the_oracle():
    assert _pins_pass(oracle.load())


@pytest.mark.parametrize("plant", [1, 2, 3, 4])
def test_pins_catch_planted_mistakes(plant):
    """Each compiled-in mistake (no zero diagonal, k innermost, swapped index, transposed
    product operand) must make the pins fail."""
    assert not _pins_pass(oracle.load(plant=plant))


def test_squaring_reaches_eq1_closure():
    """Sec. 3.2's repeated squaring ends at the same closure as Eq. 1."""
    rng = np.random.default_rng(21)
    for trial in range(30):
        n = int(rng.integers(1, 40))
        h = _rand_graph(rng, n, float(rng.uniform(0.05, 0.6)), np.int32)
        d, _ = oracle.squaring(h)
        assert np.array_equal(d, oracle.fw(h)), trial
    hf = workloads.er_graph(70, 0.05, "float32", dist="lognormal", lo=0.0, hi=1.0, seed=21)
    df, _ = oracle.squaring(hf)
    want = oracle.fw(hf)
    assert np.array_equal(np.isinf(df), np.isinf(want))
    f = np.isfinite(want)
    assert np.allclose(df[f], want[f], rtol=1e-12)


@pytest.mark.parametrize("n", [2, 3, 5, 9, 17, 40])
def test_squaring_on_a_path_closed_form(n):
    """On the directed path 0 -> 1 -> ... -> n-1, t products reach exactly the pairs j - i <= 2^t
    (a shortest walk of at most 2^t edges), so ceil(log2(n - 1)) products change something and
    the next one does not."""
    h = np.full((n, n), INF, np.int32)
    np.fill_diagonal(h, 0)
    for v in range(n - 1):
        h[v, v + 1] = 1
    need = int(np.ceil(np.log2(n - 1))) if n > 2 else 0
    assert oracle.squaring(h)[1] == need
    for t in range(need + 1):
        d, _ = oracle.squaring(h, max_iters=t)
        i, j = np.indices((n, n))
        want = np.where((j >= i) & (j - i <= 2 ** t), j - i, INF)
        assert np.array_equal(d, want), t
