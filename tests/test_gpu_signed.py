"""Negative weights (Sec. 3.1 assumes only that no cycle is negative): apsp_fw_signed on the
GPU against the CPU oracle through the C ABI.  int32 is bit-exact.  float32 distances of a
signed graph are differences of path sums that can nearly cancel, so their error is bounded
relative to the magnitudes involved: |gpu - oracle| <= 1e-5 (|oracle| + 2 max|pi|) for graphs
built from non-negative weights w and potentials pi (every distance is d_w + pi_u - pi_v)."""
import os

import numpy as np
import pytest
import torch

import oracle
import workloads
from test_gpu_parity import assert_dist_equal

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


@pytest.mark.parametrize("n", [1, 2, 50, 127, 129, 300, 520, 1100])
def test_signed_int32_matches_oracle(apsp, n):
    h, _ = workloads.signed_graph(n, 0.05 if n > 100 else 0.3, "int32", lo=1, hi=100, pot=80, seed=400 + n)
    assert n < 3 or (h < 0).any()
    d = torch.from_numpy(h).cuda()
    apsp.apsp_fw_signed(d)
    assert apsp.apsp_device_status() == 0
    assert_dist_equal(d.cpu().numpy(), oracle.fw(h, threads=THREADS), f"signed n={n}")


@pytest.mark.parametrize("n", [60, 257, 700])
def test_signed_float32_matches_oracle(apsp, n):
    pot = 30.0
    h, _ = workloads.signed_graph(n, 0.05, "float32", lo=1, hi=20, pot=pot, seed=500 + n)
    d = torch.from_numpy(h).cuda()
    apsp.apsp_fw_signed(d)
    assert apsp.apsp_device_status() == 0
    got, want = d.cpu().numpy().astype(np.float64), oracle.fw(h, threads=THREADS)
    assert np.array_equal(np.isinf(got), np.isinf(want))
    f = np.isfinite(want)
    assert np.all(np.abs(got[f] - want[f]) <= 1e-5 * (np.abs(want[f]) + 2 * pot))


def test_potentials_on_the_gpu(apsp):
    """Closed form, GPU against GPU: the signed closure equals the unsigned closure of the base
    graph shifted by the potentials, entry for entry."""
    n = 1500
    h, pi = workloads.signed_graph(n, 0.01, "int32", lo=1, hi=100, pot=200, seed=7)
    base = workloads.er_graph(n, 0.01, "int32", lo=1, hi=100, seed=7)
    d = torch.from_numpy(h).cuda()
    apsp.apsp_fw_signed(d)
    b = torch.from_numpy(base).cuda()
    apsp.apsp_fw(b)
    ds, bs = d.cpu().numpy().astype(np.int64), b.cpu().numpy().astype(np.int64)
    reach = bs < INF
    assert np.array_equal(ds[reach], (bs + pi[:, None] - pi[None, :])[reach])
    assert np.all(ds[~reach] == INF)


def test_large_signed_rows(apsp):
    """n = 4100 (33 diagonal blocks, a ragged last one): 32 source rows by Bellman-Ford."""
    n = 4100
    h, _ = workloads.signed_graph(n, 0.002, "int32", lo=1, hi=100, pot=100, seed=8)
    d = torch.from_numpy(h).cuda()
    apsp.apsp_fw_signed(d)
    assert apsp.apsp_device_status() == 0
    rows = np.random.default_rng(9).choice(n, 32, replace=False)
    got = d.cpu().numpy()[rows]
    want = oracle.fw(h, threads=THREADS)[rows]
    assert_dist_equal(got, want, "rows")


@pytest.mark.parametrize("where", [(7, 8, 9), (300, 1000, 1300)])
def test_negative_cycle_is_reported(apsp, where):
    n = 1400
    h, _ = workloads.signed_graph(n, 0.01, "int32", lo=1, hi=50, pot=20, seed=10)
    a, b, c = where
    h[a, b], h[b, c], h[c, a] = 5, -20, 4  # a cycle of weight -11
    d = torch.from_numpy(h).cuda()
    apsp.apsp_fw_signed(d)
    assert apsp.apsp_device_status() == 7
    assert apsp.apsp_device_status() == 0  # read clears


def test_float32_negative_cycle_and_range(apsp):
    h, _ = workloads.signed_graph(300, 0.05, "float32", lo=1, hi=10, pot=5, seed=11)
    h[3, 4], h[4, 3] = -2.0, 1.0
    d = torch.from_numpy(h).cuda()
    apsp.apsp_fw_signed(d)
    assert apsp.apsp_device_status() == 7
    # int32 entries too large for the signed range: a data error, the matrix is not closed
    g = workloads.er_graph(300, 0.05, "int32", lo=1, hi=10**6, seed=12)
    g[1, 2] = -5
    e = torch.from_numpy(g).cuda()
    apsp.apsp_fw_signed(e)
    assert apsp.apsp_device_status() == 2


def test_small_sentinel_is_rejected(apsp):
    d = torch.zeros((64, 64), dtype=torch.int32, device="cuda")
    with pytest.raises(apsp.ApspError):
        apsp.apsp_fw_signed(d, inf=1000)
