"""Pins for the oracle on graphs with negative edges (Sec. 3.1 assumes only that no cycle is
negative), each against something other than the oracle itself:

  * brute force: every simple path on graphs of <= 7 vertices (with no negative cycle a
    shortest path can always be taken simple);
  * a closed form: reweighting by potentials, w'(u, v) = w(u, v) + pi[u] - pi[v], keeps every
    cycle's weight and turns every distance into d(u, v) + pi[u] - pi[v];
  * Bellman-Ford from every source, the textbook algorithm for negative weights, against Eq. 1;
  * negative cycles: Eq. 1 leaves a negative diagonal entry and Bellman-Ford flags the sources
    that reach the cycle;
  * a planted mistake (one relaxation round too few) must fail the Bellman-Ford pin.
"""
import numpy as np
import pytest

import oracle
import workloads
from test_oracle_pins import _brute_force

INF = oracle.INF_I32


def _small_signed(rng, n, p):
    w = np.where(rng.random((n, n)) < p, rng.integers(1, 9, (n, n)), INF).astype(np.int64)
    pi = rng.integers(0, 12, n)
    h = np.where(w < INF, w + pi[:, None] - pi[None, :], INF)
    np.fill_diagonal(h, 0)
    return h.astype(np.int32)


def test_signed_fw_matches_simple_path_enumeration():
    rng = np.random.default_rng(31)
    seen_negative = 0
    for trial in range(150):
        n = int(rng.integers(2, 8))
        h = _small_signed(rng, n, float(rng.uniform(0.2, 0.9)))
        seen_negative += int((h < 0).any())
        assert np.array_equal(oracle.fw(h, threads=1).astype(np.int64), _brute_force(h)), (trial, h)
    assert seen_negative > 100


@pytest.mark.parametrize("dtype", ["int32", "float32"])
def test_potentials_closed_form(dtype):
    n = 90
    h, pi = workloads.signed_graph(n, 0.06, dtype, lo=1, hi=50, pot=40, seed=3)
    assert (h < 0).any()
    base = workloads.er_graph(n, 0.06, "int32", lo=1, hi=50, seed=3) if dtype == "int32" else \
        workloads.er_graph(n, 0.06, "float32", dist="uniform", lo=1, hi=50, seed=3)
    d0 = oracle.fw(base).astype(np.float64)
    d = oracle.fw(h, threads=1).astype(np.float64)
    reach = d0 < (INF if dtype == "int32" else np.inf)
    want = d0 + pi[:, None] - pi[None, :]
    if dtype == "int32":
        assert np.array_equal(d[reach], want[reach])
        assert np.all(d[~reach] == INF)
    else:
        assert np.allclose(d[reach], want[reach], rtol=1e-6, atol=1e-4)
        assert np.all(np.isinf(d[~reach]))


@pytest.mark.parametrize("dtype", ["int32", "float32"])
def test_bellman_ford_matches_eq1(dtype):
    n = 70
    h, _ = workloads.signed_graph(n, 0.08, dtype, lo=1, hi=30, pot=25, seed=4)
    d = oracle.fw(h, threads=1)
    bf, neg = oracle.bellman_ford_rows(h, np.arange(n))
    assert not neg.any()
    if dtype == "int32":
        assert np.array_equal(bf, d)
    else:
        f = np.isfinite(d)
        assert np.array_equal(np.isfinite(bf), f) and np.allclose(bf[f], d[f], rtol=1e-12)


def test_negative_cycle_is_seen_by_both():
    n = 40
    h, _ = workloads.signed_graph(n, 0.1, "int32", lo=1, hi=20, pot=10, seed=5)
    h[7, 8], h[8, 9], h[9, 7] = 3, -10, 2  # a cycle of weight -5
    d = oracle.fw(h, threads=1)
    assert np.diagonal(d).min() < 0
    assert np.diagonal(d)[[7, 8, 9]].max() < 0
    _, neg = oracle.bellman_ford_rows(h, [7, 8, 9])
    assert neg.all()
    reach = oracle.reachability(h)
    _, neg_all = oracle.bellman_ford_rows(h, np.arange(n))
    assert np.array_equal(neg_all, reach[:, 7])  # exactly the sources that reach the cycle


def _bf_pin_passes(lib):
    """A directed path n-1 -> n-2 -> ... -> 0 relaxed in increasing vertex order advances one
    edge per round, so from vertex n-1 it needs every one of the n - 1 rounds."""
    n = 12
    h = np.full((n, n), INF, np.int32)
    np.fill_diagonal(h, 0)
    for v in range(n - 1):
        h[v + 1, v] = -1 if v % 3 == 0 else 2
    bf, _ = oracle.bellman_ford_rows(h, [n - 1], lib=lib)
    return np.array_equal(bf[0], oracle.fw(h, threads=1)[n - 1])


def test_bellman_ford_pin_passes_and_catches_a_missing_round():
    assert _bf_pin_passes(oracle.load())
    assert not _bf_pin_passes(oracle.load(plant=7))
