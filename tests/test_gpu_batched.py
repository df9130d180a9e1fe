"""a7: the batched persistent kernel against the oracle, graph by graph."""
import os

import numpy as np
import pytest
import torch

import oracle
import workloads
from test_gpu_parity import assert_dist_equal

pytestmark = pytest.mark.gpu
THREADS = os.cpu_count() or 4
INF = workloads.INF_I32


@pytest.fixture(scope="module")
def apsp():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import paper_2310_03983_gb300 as m
    assert m.apsp_device_status() == 0
    return m


SIZES = [1, 2, 3, 5, 17, 31, 32, 33, 64, 100, 127, 128, 129, 130, 200, 255, 256, 257, 300, 383, 400, 513]


@pytest.mark.parametrize("dtype", ["int32", "float32"])
def test_batched_matches_oracle(apsp, dtype):
    rng = np.random.default_rng(11)
    mats = []
    for g, n in enumerate(SIZES * 2):
        p = float(rng.uniform(0.02, 0.6))
        if dtype == "int32":
            mats.append(workloads.er_graph(n, p, "int32", lo=1, hi=100, seed=500 + g))
        else:
            mats.append(workloads.er_graph(n, p, "float32", dist="lognormal", lo=0.0, hi=1.0, seed=500 + g))
    b = apsp.Batch(mats)
    apsp.apsp_batched(b)
    out = b.pool.cpu()
    for g, m in enumerate(mats):
        assert_dist_equal(b.graph(g, out).numpy(), oracle.fw(m, threads=THREADS), f"graph {g} n={m.shape[0]}")
    assert apsp.apsp_device_status() == 0


def test_batched_large_weights_use_int_path(apsp):
    """Weights up to 10^6 on 300 vertices: (n - 1) * w > 2^24, the int32 sequence runs."""
    mats = [workloads.er_graph(n, 0.05, "int32", lo=1, hi=10**6, seed=n) for n in (150, 300, 260)]
    b = apsp.Batch(mats)
    apsp.apsp_batched(b)
    out = b.pool.cpu()
    for g, m in enumerate(mats):
        assert_dist_equal(b.graph(g, out).numpy(), oracle.fw(m, threads=THREADS), f"graph {g}")


def test_batched_equals_single_graph_calls(apsp):
    rng = np.random.default_rng(3)
    ns, ps = workloads.batch_specs(64, n_lo=32, n_hi=600, seed=5)
    mats = workloads.batch_graphs(ns, ps)
    b = apsp.Batch(mats)
    apsp.apsp_batched(b)
    out = b.pool.cpu()
    for g, m in enumerate(mats):
        d = torch.from_numpy(m).cuda()
        apsp.apsp_fw(d)
        assert np.array_equal(b.graph(g, out).numpy(), d.cpu().numpy()), f"graph {g}"


def test_batched_bad_entries_are_skipped(apsp):
    mats = [workloads.er_graph(40, 0.2, "int32", seed=1), workloads.er_graph(50, 0.2, "int32", seed=2)]
    b = apsp.Batch(mats)
    b.d_lds[1] = 49  # not a multiple of 4: skipped and reported
    apsp.apsp_batched(b)
    assert apsp.apsp_device_status() == 1
    assert_dist_equal(b.graph(0).cpu().numpy(), oracle.fw(mats[0]), "graph 0")


def test_batched_balanced_batch_runs_one_cta_per_graph(apsp):
    """600 graphs of 150 vertices: no graph dominates, so the launch uses one CTA per graph
    with no clusters; the same pool closed with the cluster shape must agree bit for bit."""
    mats = [workloads.er_graph(150, 0.05, "int32", lo=1, hi=100, seed=70 + g) for g in range(600)]
    b = apsp.Batch(mats)
    pristine = b.pool.clone()
    apsp.apsp_batched(b)                          # host sizes given: plain launch
    plain = b.pool.clone()
    b.pool.copy_(pristine)
    apsp.apsp_batched_raw(b.pool, b.d_offsets, b.d_ns, b.d_lds, b.d_order, len(b), b.ws)  # no hint: clusters
    assert torch.equal(plain, b.pool)
    for g in (0, 299, 599):
        assert_dist_equal(b.graph(g, plain).cpu().numpy(), oracle.fw(mats[g]), f"graph {g}")
    assert apsp.apsp_device_status() == 0


def test_paper_sweep_through_batched(apsp):
    """The paper's 1000 generator graphs (Sec. 3.4, Sec. 4: V uniform in [4, 1000], rho uniform
    in [0, 100], costs in [0, 100] including zero) closed in one apsp_batched call.  Every graph
    of at most 320 vertices is compared with the oracle in full, plus the ten largest graphs on
    32 sampled source rows each (Dijkstra), all bit-exact."""
    ns, _, _, mats = workloads.paper_sweep(1000, seed=0)
    batch = apsp.Batch(mats)
    apsp.apsp_batched(batch)
    out = batch.pool.cpu()
    assert apsp.apsp_device_status() == 0
    small = [g for g in range(len(mats)) if ns[g] <= 320]
    assert len(small) > 250
    for g in small:
        assert_dist_equal(batch.graph(g, out).numpy(), oracle.fw(mats[g], threads=THREADS), f"graph {g} (n={ns[g]})")
    rng = np.random.default_rng(5)
    for g in np.argsort(ns)[-10:]:
        rows = rng.choice(int(ns[g]), 32, replace=False)
        got = batch.graph(int(g), out).numpy()[rows]
        assert_dist_equal(got, oracle.dijkstra_rows(mats[g], rows, threads=THREADS), f"graph {g}")


def test_batched_long_paths(apsp):
    """Directed paths (diameter n - 1, distances up to 8 * 10^5) mixed with ordinary graphs:
    every phase-1 and phase-3 relaxation matters; all bit-exact."""
    def path(n, w):
        h = np.full((n, n), INF, np.int32)
        np.fill_diagonal(h, 0)
        idx = np.arange(n - 1)
        h[idx, idx + 1] = w
        return h
    mats = [path(300, 100), path(400, 40), path(200, 4000), path(160, 1), path(129, 128)]
    mats += [workloads.er_graph(n, 0.05, "int32", lo=1, hi=100, seed=600 + n) for n in (130, 257, 511)]
    b = apsp.Batch(mats)
    apsp.apsp_batched(b)
    out = b.pool.cpu()
    assert apsp.apsp_device_status() == 0
    for g, m in enumerate(mats):
        assert_dist_equal(b.graph(g, out).numpy(), oracle.fw(m, threads=THREADS), f"graph {g} n={m.shape[0]}")
