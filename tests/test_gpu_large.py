"""The n = 32768 configuration, in the launch configuration bench.py times.

Directed ER n = 32768, p = 0.05, int32 weights in [1, 100] (the bench's input, seed 0), and the
fp32 variant with weights uniform in (0, 1].  The oracle cannot close the whole matrix, so it
checks 64 seeded source rows by array Dijkstra (int32 bit-exact, fp32 within 1e-5 relative of
fp64).  A whole-matrix property holds at any size: a closed matrix is idempotent under (min,+)
squaring, D (x) D == D, checked on the GPU with the tropical GEMM.
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
