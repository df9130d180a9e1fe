"""Pins for the oracle's predecessor functions (pred[i, j] of Sec. 2), each against something
other than the oracle itself:

  * brute force: on graphs of <= 7 vertices every simple path is enumerated; the last hops of
    the shortest ones form the set of valid predecessors (with positive weights every shortest
    path can be taken simple), and ``last_hop`` must return the smallest of them;
  * the hand-worked example of tests/golden/hand_6node.json;
  * closed forms: a directed path and a directed cycle;
  * the paper's own Floyd-Warshall with predecessor indices (``fw_pred``) must give valid
    predecessors and the same distances as Eq. 1;
  * ``check_predecessors`` must reject deliberately broken matrices;
  * planted mistakes (a transposed cost, j allowed as its own last hop) must fail the pins.
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


def _positive_graph(rng, n, p, dtype):
    if dtype == np.int32:
        h = np.where(rng.random((n, n)) < p, rng.integers(1, 6, (n, n)), INF).astype(np.int32)
    else:
        h = np.where(rng.random((n, n)) < p, rng.lognormal(0.0, 1.0, (n, n)), np.inf).astype(np.float32)
    np.fill_diagonal(h, 0)
    return h


def _valid_last_hops(h):
    """{(i, j): set of k that end some shortest simple i -> j path} and the distances, by
    enumerating every simple path (exact: Python ints or fp64)."""
    n = h.shape[0]
    isint = h.dtype.kind in "iu"
    edge = (h < INF) if isint else np.isfinite(h)
    best, hops = {}, {}
    for i in range(n):
        others = [v for v in range(n) if v != i]
        for L in range(1, n):
            for mids in itertools.permutations(others, L - 1):
                for j in others:
                    if j in mids:
                        continue
                    path = (i,) + mids + (j,)
                    if not all(edge[a, b] for a, b in zip(path, path[1:])):
                        continue
                    cost = sum((int(h[a, b]) if isint else float(h[a, b])) for a, b in zip(path, path[1:]))
                    key = (i, j)
                    if key not in best or cost < best[key]:
                        best[key], hops[key] = cost, {path[-2]}
                    elif cost == best[key]:
                        hops[key].add(path[-2])
    return best, hops


def _last_hop_pins_pass(lib, trials=60, seed=3):
    rng = np.random.default_rng(seed)
    for _ in range(trials):
        n = int(rng.integers(2, 7))
        h = _positive_graph(rng, n, float(rng.uniform(0.2, 0.9)), np.int32)
        d = oracle.fw(h)
        got = oracle.last_hop(d, h, lib=lib)
        best, hops = _valid_last_hops(h)
        for i in range(n):
            for j in range(n):
                want = min(hops[(i, j)]) if (i, j) in hops else -1
                if got[i, j] != want:
                    return False
    return True


def test_last_hop_matches_simple_path_enumeration_int():
    assert _last_hop_pins_pass(oracle.load())


def test_last_hop_matches_simple_path_enumeration_float():
    rng = np.random.default_rng(4)
    for _ in range(60):
        n = int(rng.integers(2, 7))
        h = _positive_graph(rng, n, float(rng.uniform(0.2, 0.9)), np.float32)
        d = oracle.fw(h).astype(np.float32)
        got = oracle.last_hop(d, h)
        best, hops = _valid_last_hops(h)
        for i in range(n):
            for j in range(n):
                if (i, j) in hops:
                    assert got[i, j] in hops[(i, j)], (h, i, j, got[i, j], hops[(i, j)])
                else:
                    assert got[i, j] == -1


def test_fw_pred_is_valid_and_keeps_eq1_distances():
    rng = np.random.default_rng(5)
    for _ in range(40):
        n = int(rng.integers(2, 7))
        h = _positive_graph(rng, n, float(rng.uniform(0.2, 0.9)), np.int32)
        d, pred = oracle.fw_pred(h)
        assert np.array_equal(d, oracle.fw(h))
        best, hops = _valid_last_hops(h)
        for (i, j), ks in hops.items():
            assert pred[i, j] in ks
    h = workloads.er_graph(120, 0.05, "int32", lo=1, hi=100, seed=6)
    d, pred = oracle.fw_pred(h)
    assert oracle.check_predecessors(pred, d, h) == []
    hf = workloads.er_graph(90, 0.08, "float32", dist="lognormal", lo=0.0, hi=1.0, seed=6)
    df, predf = oracle.fw_pred(hf)
    assert oracle.check_predecessors(predf, df, hf, rtol=1e-12) == []


def test_golden_hand_example_predecessors():
    g = json.load(open(os.path.join(HERE, "golden", "hand_6node.json")))
    n, inf = g["n"], g["inf"]
    h = np.full((n, n), inf, np.int32)
    np.fill_diagonal(h, 0)
    for u, v, c in g["edges"]:
        h[u, v] = c
    want = np.array(g["expected_pred"], np.int32)
    d = np.array(g["expected"], np.int32)
    assert np.array_equal(oracle.last_hop(d, h, inf=inf), want)
    assert np.array_equal(oracle.fw_pred(h, inf=inf)[1], want)
    assert oracle.check_predecessors(want, d, h, inf=inf) == []


def test_closed_forms():
    n = 9
    path_g = np.full((n, n), INF, np.int32)
    np.fill_diagonal(path_g, 0)
    for v in range(n - 1):
        path_g[v, v + 1] = v + 1
    d = oracle.fw(path_g)
    pred = oracle.last_hop(d, path_g)
    want = np.full((n, n), -1, np.int32)
    for i in range(n):
        for j in range(i + 1, n):
            want[i, j] = j - 1
    assert np.array_equal(pred, want)
    cyc = np.full((n, n), INF, np.int32)
    np.fill_diagonal(cyc, 0)
    for v in range(n):
        cyc[v, (v + 1) % n] = 3
    d = oracle.fw(cyc)
    pred = oracle.last_hop(d, cyc)
    want = np.array([[-1 if i == j else (j - 1) % n for j in range(n)] for i in range(n)], np.int32)
    assert np.array_equal(pred, want)


def test_check_predecessors_rejects_broken_matrices():
    h = workloads.er_graph(60, 0.1, "int32", lo=1, hi=50, seed=7)
    d = oracle.fw(h)
    pred = oracle.last_hop(d, h)
    assert oracle.check_predecessors(pred, d, h) == []
    i, j = np.argwhere((pred >= 0))[5]
    for wrong in ({"v": -1}, {"v": int(j)}, {"v": int((pred[i, j] + 1) % 60)}):
        bad = pred.copy()
        bad[i, j] = wrong["v"]
        if wrong["v"] >= 0 and wrong["v"] != j and h[wrong["v"], j] < INF and d[i, wrong["v"]] + h[wrong["v"], j] == d[i, j]:
            continue  # happens to be another valid last hop
        assert oracle.check_predecessors(bad, d, h) != [], wrong
    bad = pred.copy()
    bad[0, 0] = 1
    assert oracle.check_predecessors(bad, d, h) != []
    # a two-cycle of predecessors: tight-looking locally only if costs allow; walks must catch it
    bad = pred.copy()
    a, b = np.argwhere((pred >= 0) & (pred != np.arange(60)[:, None]))[0]
    bad[a, pred[a, b]] = b
    assert oracle.check_predecessors(bad, d, h) != []


@pytest.mark.parametrize("plant", [5, 6])
def test_pred_pins_catch_planted_mistakes(plant):
    """A transposed cost (w[j][k]) and a last hop allowed to be j itself must each fail."""
    assert not _last_hop_pins_pass(oracle.load(plant=plant), trials=30)


def test_last_hop_rows_subset_equals_full():
    h = workloads.er_graph(150, 0.05, "int32", lo=1, hi=100, seed=8)
    d = oracle.fw(h)
    rows = [0, 7, 149]
    assert np.array_equal(oracle.last_hop(d, h, rows=rows), oracle.last_hop(d, h)[rows])
    hf = workloads.er_graph(150, 0.05, "float32", dist="lognormal", lo=0.0, hi=1.0, seed=8)
    df = oracle.fw(hf).astype(np.float32)
    assert np.array_equal(oracle.last_hop(df[rows], hf, rows=rows), oracle.last_hop(df, hf)[rows])
