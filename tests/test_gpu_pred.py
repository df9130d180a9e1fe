"""Predecessors (pred[i, j] of Sec. 2) on the GPU against the CPU oracle, through the C ABI.

The library defines pred[i][j] as the smallest k != j minimising d[i][k] + w[k][j] (-1 on the
diagonal and for unreachable pairs), so the index is unique and compared exactly:
  * int32: the oracle sums in int64; the encoded (min,+) product on the tropical-GEMM engine
    and the direct argmin kernel must both match it entry for entry;
  * float32: the decision is taken in float32 on both sides (one round-to-nearest add per
    sum, ties to the smallest k), so the indices must match exactly too.
The closed matrix d fed to the kernel is the oracle's.  End-to-end runs (GPU closure, then GPU
predecessors) are checked by the properties every valid predecessor matrix has: tight last
edges, and walks back to the source whose costs re-sum to the distance.
"""
import os

import numpy as np
import pytest
import torch

import oracle
import workloads

pytestmark = pytest.mark.gpu

INF = workloads.INF_I32
THREADS = os.cpu_count() or 4


@pytest.fixture(scope="module")
def apsp():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import paper_2310_03983_gb300 as m
    assert m.apsp_device_status() == 0
    return m


def _graph(n, p, dtype, seed, hi=100):
    if dtype == np.int32:
        return workloads.er_graph(n, p, "int32", lo=1, hi=hi, seed=seed)
    return workloads.er_graph(n, p, "float32", dist="lognormal", lo=0.0, hi=1.0, seed=seed)


def _oracle_d(h):
    d = oracle.fw(h, threads=THREADS)
    return d if h.dtype == np.int32 else d.astype(np.float32)


def _pred_gpu(apsp, d, h, strided=False):
    n = h.shape[0]
    dd = torch.from_numpy(np.ascontiguousarray(d)).cuda()
    ww = torch.from_numpy(np.ascontiguousarray(h)).cuda()
    if strided:  # leading dimension n + 1: not a TMA operand, so the direct kernel runs
        buf = torch.empty((n, n + 1), dtype=torch.int32, device="cuda")
        pred = buf[:, :n]
        apsp.apsp_predecessors(dd, ww, pred)
    else:
        pred = apsp.apsp_predecessors(dd, ww)
    return pred.cpu().numpy()


@pytest.mark.parametrize("n", [1, 2, 5, 127, 128, 129, 300, 520])
@pytest.mark.parametrize("dtype", [np.int32, np.float32])
def test_predecessors_match_oracle(apsp, n, dtype):
    h = _graph(n, 0.05 if n > 100 else 0.4, dtype, seed=100 + n)
    d = _oracle_d(h)
    got = _pred_gpu(apsp, d, h)
    want = oracle.last_hop(d, h, threads=THREADS)
    bad = np.argwhere(got != want)
    assert bad.size == 0, f"{len(bad)} mismatches, first {bad[:5].tolist()}"
    assert apsp.apsp_device_status() == 0


@pytest.mark.parametrize("n", [129, 300])
def test_direct_kernel_matches_oracle(apsp, n):
    """pred with a leading dimension that TMA cannot take -> the direct argmin kernel."""
    h = _graph(n, 0.3, np.int32, seed=7 + n)
    d = _oracle_d(h)
    got = _pred_gpu(apsp, d, h, strided=True)
    assert np.array_equal(got, oracle.last_hop(d, h, threads=THREADS))


def test_encoding_overflow_falls_back(apsp):
    """Weights near 2^22 at n = 300 break the index encoding ((d + w) << 9 >= 2^30): the
    device must skip the encoded product and run the direct kernel, with the same answer."""
    n = 300
    rng = np.random.default_rng(9)
    h = np.where(rng.random((n, n)) < 0.05, rng.integers(1, 1 << 22, (n, n)), INF).astype(np.int32)
    np.fill_diagonal(h, 0)
    d = _oracle_d(h)
    assert int(d[d < INF].max()) + int(h[h < INF].max()) > (1 << 21)
    got = _pred_gpu(apsp, d, h)
    assert np.array_equal(got, oracle.last_hop(d, h, threads=THREADS))
    assert apsp.apsp_device_status() == 0


def test_dense_ties_and_int32_dpx_path(apsp):
    """Dense graph with few distinct weights (many ties: smallest k must win) and encoded sums
    above 2^24 (so the engine's int32 instruction path runs rather than the fp32 one)."""
    n = 384
    rng = np.random.default_rng(10)
    h = np.where(rng.random((n, n)) < 0.9, rng.integers(1, 3, (n, n)), INF).astype(np.int32)
    np.fill_diagonal(h, 0)
    d = _oracle_d(h)
    got = _pred_gpu(apsp, d, h)
    assert np.array_equal(got, oracle.last_hop(d, h, threads=THREADS))
    h2 = np.where(rng.random((n, n)) < 0.2, rng.integers(1000, 40000, (n, n)), INF).astype(np.int32)
    np.fill_diagonal(h2, 0)
    d2 = _oracle_d(h2)
    assert (int(d2[d2 < INF].max()) + int(h2[h2 < INF].max())) << 9 >= (1 << 24)
    assert np.array_equal(_pred_gpu(apsp, d2, h2), oracle.last_hop(d2, h2, threads=THREADS))


def test_float32_ties(apsp):
    """Integer-valued float32 weights: sums are exact and ties common, so the kernel's rule
    (the first k in order whose sum equals the running minimum) is tested against the
    oracle's strict-less scan."""
    n = 333
    rng = np.random.default_rng(16)
    h = np.where(rng.random((n, n)) < 0.5, rng.integers(1, 3, (n, n)), np.inf).astype(np.float32)
    np.fill_diagonal(h, 0)
    d = _oracle_d(h)
    assert np.array_equal(_pred_gpu(apsp, d, h), oracle.last_hop(d, h, threads=THREADS))


def test_unreachable_and_sentinel(apsp):
    """Two components, entries above the sentinel in w, a custom sentinel."""
    n = 200
    h = _graph(n, 0.1, np.int32, seed=11)
    h[:100, 100:] = INF + 5  # above the sentinel: no edge
    h[100:, :100] = INF
    d = _oracle_d(np.minimum(h, INF))
    got = _pred_gpu(apsp, d, h)
    want = oracle.last_hop(d, np.minimum(h, INF), threads=THREADS)
    assert np.array_equal(got, want)
    assert np.all(got[:100, 100:] == -1) and np.all(got[100:, :100] == -1)
    inf2 = 1 << 20
    h3 = np.where(h >= INF, inf2, h).astype(np.int32)
    d3 = np.where(d >= INF, inf2, d).astype(np.int32)
    dd, ww = torch.from_numpy(d3).cuda(), torch.from_numpy(h3).cuda()
    got3 = apsp.apsp_predecessors(dd, ww, inf=inf2).cpu().numpy()
    assert np.array_equal(got3, oracle.last_hop(d3, h3, inf=inf2, threads=THREADS))


def test_negative_weight_sets_domain(apsp):
    h = _graph(64, 0.2, np.int32, seed=12)
    d = _oracle_d(h)
    h[3, 5] = -4
    _pred_gpu(apsp, d, h)
    assert apsp.apsp_device_status() == 2


@pytest.mark.parametrize("algo", ["fw", "rkleene"])
@pytest.mark.parametrize("dtype", [np.int32, np.float32])
def test_end_to_end_paths(apsp, algo, dtype):
    """solve(..., predecessors=True): GPU closure then GPU predecessors; every walk is a real
    path whose costs re-sum to the distance; int32 matches the oracle's definition exactly."""
    n = 700
    h = _graph(n, 0.02, dtype, seed=13)
    d, pred = apsp.solve(h, algo=algo, param=256 if algo == "rkleene" else 0, predecessors=True)
    d, pred = d.numpy(), pred.numpy()
    rows = list(range(0, n, 7))
    viol = oracle.check_predecessors(pred, d, h, rtol=0 if dtype == np.int32 else 1e-5, rows=rows)
    assert viol == [], viol[:3]
    if dtype == np.int32:
        want_d = _oracle_d(h)
        assert np.array_equal(d, want_d)
        assert np.array_equal(pred[rows], oracle.last_hop(want_d, h, rows=rows, threads=THREADS))
    j = int(np.nonzero(pred[0] >= 0)[0][-1])
    p = apsp.path(pred, 0, j)
    assert p[0] == 0 and p[-1] == j and len(set(p)) == len(p)
    cost = sum(float(h[a, b]) for a, b in zip(p, p[1:]))
    assert abs(cost - float(d[0, j])) <= 1e-5 * max(1.0, float(d[0, j]))


def test_large_sampled_rows(apsp):
    """n = 4096 int32 (the encoded product on the exact fp32 path), checked on 24 source rows
    against the oracle's definition and by walks on every pair of those rows."""
    n = 4096
    h = _graph(n, 0.01, np.int32, seed=14)
    dd = torch.from_numpy(h).cuda()
    w = dd.clone()
    apsp.apsp_fw(dd)
    pred = apsp.apsp_predecessors(dd, w).cpu().numpy()
    d = dd.cpu().numpy()
    rows = np.random.default_rng(15).choice(n, 24, replace=False)
    want_rows = oracle.dijkstra_rows(h, rows, threads=THREADS)
    assert np.array_equal(d[rows], want_rows)
    assert np.array_equal(pred[rows], oracle.last_hop(want_rows, h, rows=rows, threads=THREADS))
    assert oracle.check_predecessors(pred, d, h, rows=rows) == []
