"""a7, staged path: the larger graphs of a batch (257..2048 vertices) closed in lockstep on the
tropical-GEMM engine (int32: 16-bit phase 3 certified per graph, an int32 pass for the rest;
float32: one fp32 pass), against the persistent kernel alone and the oracle."""
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
CAP = 0x3FFF


@pytest.fixture(scope="module")
def apsp():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import paper_2310_03983_gb300 as m
    assert m.apsp_device_status() == 0
    return m


def _path(n, w):
    h = np.full((n, n), INF, np.int32)
    np.fill_diagonal(h, 0)
    idx = np.arange(n - 1)
    h[idx, idx + 1] = w
    return h


def _run(apsp, b):
    torch.cuda.synchronize()
    apsp.apsp_launch_count(reset=True)
    apsp.apsp_batched(b)
    launches = apsp.apsp_launch_count()
    torch.cuda.synchronize()
    return b.pool.cpu(), launches


def test_staged_equals_persistent_kernel(apsp):
    ns, ps = workloads.batch_specs(300, n_lo=32, n_hi=1100, seed=7)
    mats = workloads.batch_graphs(ns, ps)
    staged = apsp.Batch(mats)
    plain = apsp.Batch(mats, staged=False)
    assert staged.ws.numel() > plain.ws.numel()
    out_s, launches_s = _run(apsp, staged)
    out_p, launches_p = _run(apsp, plain)
    assert launches_p == 1 and launches_s > 10  # the staged sequence ran
    assert torch.equal(out_s, out_p)
    assert apsp.apsp_device_status() == 0
    for g in np.argsort(ns)[-6:]:
        g = int(g)
        assert_dist_equal(staged.graph(g, out_s).numpy(), oracle.fw(mats[g], threads=THREADS), f"graph {g}")


def _check_batch_against_oracle(b, mats, out, full_max=512, rows_per_large=16):
    """Every graph of at most full_max vertices in full against the oracle's Eq. 1 closure;
    rows_per_large seeded Dijkstra rows of every larger graph."""
    from concurrent.futures import ThreadPoolExecutor

    def check(g):
        m = mats[g]
        n = m.shape[0]
        got = b.graph(g, out).numpy()
        if n <= full_max:
            assert_dist_equal(got, oracle.fw(m), f"graph {g} n={n}")
        else:
            src = np.sort(np.random.default_rng(g).choice(n, rows_per_large, replace=False))
            assert_dist_equal(got[src], oracle.dijkstra_rows(m, src), f"graph {g} n={n} rows")
        return n <= full_max

    with ThreadPoolExecutor(THREADS) as ex:
        full = list(ex.map(check, range(len(mats))))
    return sum(full)


def test_config4_batch_against_oracle(apsp):
    """The benchmark's 2048-graph batch itself (n log-uniform in [32, 1024], p uniform in
    [0.02, 0.8], int32 weights in [1, 100], graph g seeded 1000 + g), closed by one apsp_batched
    call on the staged path, as the benchmark closes it."""
    from concurrent.futures import ThreadPoolExecutor
    ns, ps = workloads.batch_specs(2048, seed=0)
    with ThreadPoolExecutor(THREADS) as ex:
        mats = list(ex.map(lambda g: workloads.er_graph(int(ns[g]), float(ps[g]), "int32", lo=1, hi=100,
                                                        seed=1000 + g, threads=1), range(len(ns))))
    b = apsp.Batch(mats)
    out, launches = _run(apsp, b)
    assert launches > 10  # the staged sequence ran
    assert apsp.apsp_device_status() == 0
    full = _check_batch_against_oracle(b, mats, out)
    assert full > 1500 and len(mats) - full > 300


def test_staged_float32_equals_persistent_kernel(apsp):
    """Float32 batches stage too (one fp32 lockstep pass, no certificate): the same distances
    as the persistent kernel alone and as the oracle (1e-5 relative of fp64)."""
    ns, ps = workloads.batch_specs(300, n_lo=32, n_hi=1100, seed=9)
    mats = workloads.batch_graphs(ns, ps, dtype="float32", dist="lognormal", lo=0.0, hi=1.0)
    staged = apsp.Batch(mats)
    plain = apsp.Batch(mats, staged=False)
    assert staged.ws.numel() > plain.ws.numel()
    out_s, launches_s = _run(apsp, staged)
    out_p, launches_p = _run(apsp, plain)
    assert launches_p == 1 and launches_s > 10
    assert apsp.apsp_device_status() == 0
    for g in range(len(mats)):
        assert_dist_equal(staged.graph(g, out_s).numpy(), staged.graph(g, out_p).numpy().astype(np.float64),
                          f"graph {g} staged vs persistent")
    full = _check_batch_against_oracle(staged, mats, out_s)
    assert full > 100


def test_config4_float32_batch_against_oracle(apsp):
    """The 2048-graph batch shape with float32 lognormal(0, 1) weights, staged."""
    ns, ps = workloads.batch_specs(2048, seed=0)
    mats = workloads.batch_graphs(ns, ps, dtype="float32", dist="lognormal", lo=0.0, hi=1.0)
    b = apsp.Batch(mats)
    out, launches = _run(apsp, b)
    assert launches > 10
    assert apsp.apsp_device_status() == 0
    full = _check_batch_against_oracle(b, mats, out)
    assert full > 1500


def test_certificate_both_sides_of_the_cap(apsp):
    """Paths whose longest distance plus the largest weight lands just below CAP (certified)
    and just above it (the int32 pass finishes them), next to ordinary graphs."""
    w_ok = (CAP - 1) // 400          # (399 + 1) * w < CAP
    w_fail = CAP // 299 + 1          # 299 * w >= CAP: certificate fails
    mats = [_path(400, w_ok), _path(300, w_fail), _path(600, 1), _path(1024, 16)]
    mats += [workloads.er_graph(n, 0.05, "int32", lo=1, hi=100, seed=800 + n) for n in (260, 700, 1000)]
    b = apsp.Batch(mats)
    out, _ = _run(apsp, b)
    assert apsp.apsp_device_status() == 0
    for g, m in enumerate(mats):
        assert_dist_equal(b.graph(g, out).numpy(), oracle.fw(m, threads=THREADS), f"graph {g} n={m.shape[0]}")


def test_heavy_and_zero_weights(apsp):
    """Weights above CAP / 4 skip the 16-bit pass (int32 pass only), weights up to 10^6 take the
    int32 instruction sequence, zero weights are allowed."""
    mats = [workloads.er_graph(300, 0.05, "int32", lo=1, hi=10**6, seed=1),
            workloads.er_graph(500, 0.02, "int32", lo=4000, hi=9000, seed=2),
            workloads.er_graph(400, 0.1, "int32", lo=0, hi=3, seed=3),
            workloads.er_graph(270, 0.3, "int32", lo=1, hi=100, seed=4)]
    b = apsp.Batch(mats)
    out, _ = _run(apsp, b)
    assert apsp.apsp_device_status() == 0
    for g, m in enumerate(mats):
        assert_dist_equal(b.graph(g, out).numpy(), oracle.fw(m, threads=THREADS), f"graph {g}")


def test_bad_staged_graphs_are_left_alone(apsp):
    """A staged graph with an unaligned leading dimension, and one whose device size disagrees
    with the host sizes the plan was made from: both untouched and reported (APSP_ERR_ARG);
    every other graph closed."""
    mats = [workloads.er_graph(n, 0.05, "int32", lo=1, hi=100, seed=900 + n) for n in (300, 520, 640, 90, 384)]
    b = apsp.Batch(mats)
    before = b.pool.clone()
    b.d_lds[1] = 519                  # 520-vertex graph: ld not a multiple of 4
    b.d_ns[2] = 200                   # 640 on the host, 200 on the device: another block count
    out, _ = _run(apsp, b)
    assert apsp.apsp_device_status() == 1
    for g in (1, 2):
        assert torch.equal(b.graph(g, out), b.graph(g, before.cpu())), f"graph {g} was modified"
    for g in (0, 3, 4):
        assert_dist_equal(b.graph(g, out).numpy(), oracle.fw(mats[g], threads=THREADS), f"graph {g}")


def test_negative_entry_is_reported(apsp):
    mats = [workloads.er_graph(n, 0.05, "int32", lo=1, hi=100, seed=950 + n) for n in (300, 400)]
    mats[1][5, 7] = -3
    b = apsp.Batch(mats)
    out, _ = _run(apsp, b)
    assert apsp.apsp_device_status() == 2
    assert_dist_equal(b.graph(0, out).numpy(), oracle.fw(mats[0], threads=THREADS), "graph 0")


def test_small_sentinel_takes_the_persistent_kernel(apsp):
    """A sentinel at or below the 16-bit cap cannot use the staged path: one launch, same
    distances as the oracle with that sentinel."""
    inf = 5000
    mats = [workloads.er_graph(n, 0.05, "int32", lo=1, hi=40, seed=990 + n, inf=inf) for n in (300, 260)]
    b = apsp.Batch(mats)
    torch.cuda.synchronize()
    apsp.apsp_launch_count(reset=True)
    apsp.apsp_batched(b, inf=inf)
    assert apsp.apsp_launch_count() == 1
    out = b.pool.cpu()
    assert apsp.apsp_device_status() == 0
    for g, m in enumerate(mats):
        want = oracle.fw(m, inf=inf, threads=THREADS)
        assert np.array_equal(b.graph(g, out).numpy(), want), f"graph {g}"


def test_staged_sequence_replays_in_a_cuda_graph(apsp):
    ns, ps = workloads.batch_specs(120, n_lo=100, n_hi=900, seed=11)
    mats = workloads.batch_graphs(ns, ps)
    b = apsp.Batch(mats)
    pristine = b.pool.clone()
    apsp.apsp_batched(b)
    torch.cuda.synchronize()
    want = b.pool.clone()
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        b.pool.copy_(pristine)
        apsp.apsp_batched(b)
    for _ in range(3):
        b.pool.zero_()
        g.replay()
        torch.cuda.synchronize()
        assert torch.equal(b.pool, want)
    assert apsp.apsp_device_status() == 0
