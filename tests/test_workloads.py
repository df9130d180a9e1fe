"""The seeded input generators: deterministic, thread-count independent, right shape."""
import numpy as np

import workloads


def test_er_graph_is_deterministic_and_thread_independent():
    a = workloads.er_graph(600, 0.1, "int32", seed=4, threads=1)
    b = workloads.er_graph(600, 0.1, "int32", seed=4, threads=4)
    assert np.array_equal(a, b)
    assert not np.array_equal(a, workloads.er_graph(600, 0.1, "int32", seed=5))
    assert np.all(np.diagonal(a) == 0)
    off = ~np.eye(600, dtype=bool)
    edges = (a < workloads.INF_I32) & off
    assert abs(edges.sum() / off.sum() - 0.1) < 0.01
    w = a[edges]
    assert w.min() >= 1 and w.max() <= 100


def test_er_graph_float_distributions():
    f = workloads.er_graph(300, 0.5, "float32", dist="uniform01", seed=1)
    w = f[np.isfinite(f) & ~np.eye(300, dtype=bool)]
    assert f.dtype == np.float32 and w.min() > 0 and w.max() <= 1
    g = workloads.er_graph(300, 0.5, "float32", dist="lognormal", lo=0.0, hi=1.0, seed=1)
    lw = np.log(g[np.isfinite(g) & ~np.eye(300, dtype=bool)].astype(np.float64))
    assert abs(lw.mean()) < 0.05 and abs(lw.std() - 1) < 0.05


def test_batch_and_requests():
    ns, ps = workloads.batch_specs(2048, seed=0)
    assert ns.min() >= 32 and ns.max() <= 1024 and len(ns) == 2048
    assert ps.min() >= 0.02 and ps.max() <= 0.8
    t, n, p, dt = workloads.poisson_requests(200, 60, seed=0)
    assert 10000 < len(t) < 14000 and np.all(np.diff(t) > 0)
    assert set(dt) == {"int32", "float32"}


def test_paper_generator():
    h = workloads.paper_graph(50, rho=30.0, alpha=100, seed=2)
    assert np.all(np.diagonal(h) == 0)
    w = h[h < workloads.INF_I32]
    assert w.min() >= 0 and w.max() <= 100


def test_paper_sweep_shape_and_order():
    ns, rhos, edges, mats = workloads.paper_sweep(count=60, seed=3)
    assert len(mats) == 60 and all(m.shape == (n, n) for n, m in zip(ns, mats))
    assert ns.min() >= 4 and ns.max() <= 1000 and rhos.min() >= 0 and rhos.max() <= 100
    assert np.all(np.diff(edges) >= 0)  # ascending number of edges, as the paper orders them
    for n, e, m in zip(ns, edges, mats):
        assert np.all(np.diagonal(m) == 0)
        fin = m[m < workloads.INF_I32]
        assert fin.min() >= 0 and fin.max() <= 100
        assert e == np.count_nonzero(m < workloads.INF_I32) - n
    ns2, _, _, mats2 = workloads.paper_sweep(count=60, seed=3)
    assert np.array_equal(ns, ns2) and all(np.array_equal(a, b) for a, b in zip(mats, mats2))
