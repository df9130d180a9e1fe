"""The n = 32768 configuration, in the launch configuration bench.py times.

Directed ER n = 32768, p = 0.05, int32 weights in [1, 100] (the bench's input, seed 0), the fp32
variant with weights uniform in (0, 1], and int32 weights in [1, 10^6] (too heavy for the 16-bit
pass and for the a-priori exact fp32 bound).  The oracle cannot close the whole matrix, so it
checks 64 seeded source rows by array Dijkstra (int32 bit-exact, fp32 within 1e-5 relative of
fp64), and 64 seeded rows of the standalone tropical GEMM (A = B = the input matrix, Eq. 2) by
its row-wise product.  A whole-matrix property holds at any size: a closed matrix is idempotent
under (min,+) squaring, D (x) D == D, checked on the GPU with the tropical GEMM as an extra.
"""
import os

import numpy as np
import pytest
import torch

import oracle
import workloads
from test_gpu_parity import assert_dist_equal

pytestmark = pytest.mark.gpu
THREADS = os.cpu_count() or 4
N = 32768


@pytest.fixture(scope="module")
def apsp():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import paper_2310_03983_gb300 as m
    return m


@pytest.mark.parametrize("algo", ["fw", "rkleene"])
def test_n32768_int32_rows_match_dijkstra(apsp, algo):
    h = workloads.er_graph(N, 0.05, "int32", lo=1, hi=100, seed=0)
    d = torch.from_numpy(h).cuda()
    (apsp.apsp_fw if algo == "fw" else apsp.apsp_rkleene)(d)
    src = np.sort(np.random.default_rng(0).choice(N, 64, replace=False))
    got = d[torch.from_numpy(src).cuda()].cpu().numpy()
    assert_dist_equal(got, oracle.dijkstra_rows(h, src, threads=THREADS), f"{algo} rows")
    if algo == "fw":
        sq = torch.empty_like(d)
        apsp.tropical_gemm(sq, d, d)
        assert torch.equal(sq, d), "closed matrix is not idempotent under (min,+) squaring"
    assert apsp.apsp_device_status() == 0


def test_n32768_fp32_rows_match_dijkstra(apsp):
    h = workloads.er_graph(N, 0.05, "float32", dist="uniform01", seed=0)
    d = torch.from_numpy(h).cuda()
    apsp.apsp_fw(d)
    src = np.sort(np.random.default_rng(1).choice(N, 64, replace=False))
    got = d[torch.from_numpy(src).cuda()].cpu().numpy()
    assert_dist_equal(got, oracle.dijkstra_rows(h, src, threads=THREADS), "fp32 rows")
    assert apsp.apsp_device_status() == 0


def test_n32768_fp32_rkleene_rows_match_dijkstra(apsp):
    h = workloads.er_graph(N, 0.05, "float32", dist="uniform01", seed=0)
    d = torch.from_numpy(h).cuda()
    ws = torch.empty(apsp.apsp_rkleene_workspace_bytes(N, N, torch.float32, 1024), dtype=torch.uint8, device="cuda")
    apsp.apsp_rkleene(d, cutoff=1024, ws=ws)
    src = np.sort(np.random.default_rng(2).choice(N, 64, replace=False))
    got = d[torch.from_numpy(src).cuda()].cpu().numpy()
    assert_dist_equal(got, oracle.dijkstra_rows(h, src, threads=THREADS), "fp32 R-Kleene rows")
    assert apsp.apsp_device_status() == 0


@pytest.mark.parametrize("dtype", ["int32", "float32"])
def test_n32768_tropical_gemm_rows_match_oracle(apsp, dtype):
    """The standalone product of the bench's tgemm_n32768 workload (C = A (x) A on the input
    matrix, with the workspace the bench passes), 64 seeded rows against the oracle's Eq. 2."""
    if dtype == "int32":
        h = workloads.er_graph(N, 0.05, "int32", lo=1, hi=100, seed=0)
    else:
        h = workloads.er_graph(N, 0.05, "float32", dist="uniform01", seed=0)
    a = torch.from_numpy(h).cuda()
    c = torch.empty_like(a)
    ws = torch.empty(apsp.tropical_gemm_workspace_bytes(N, N, N, a.dtype), dtype=torch.uint8, device="cuda")
    apsp.tropical_gemm(c, a, a, ws=ws)
    rows = np.sort(np.random.default_rng(3).choice(N, 64, replace=False))
    got = c[torch.from_numpy(rows).cuda()].cpu().numpy()
    assert_dist_equal(got, oracle.minplus_rows(h, h, rows, threads=THREADS), f"{dtype} product rows")
    assert apsp.apsp_device_status() == 0


def test_n32768_heavy_int32_rows_match_dijkstra(apsp):
    """int32 weights in [1, 10^6]: (n - 1) w_max far above 2^24 and w_max far above the 16-bit
    cap, so no a-priori bound admits the faster instruction sequences; the result must still be
    bit-exact."""
    h = workloads.er_graph(N, 0.05, "int32", lo=1, hi=10**6, seed=0)
    d = torch.from_numpy(h).cuda()
    apsp.apsp_fw(d)
    src = np.sort(np.random.default_rng(4).choice(N, 64, replace=False))
    got = d[torch.from_numpy(src).cuda()].cpu().numpy()
    assert_dist_equal(got, oracle.dijkstra_rows(h, src, threads=THREADS), "heavy int32 rows")
    assert apsp.apsp_device_status() == 0
