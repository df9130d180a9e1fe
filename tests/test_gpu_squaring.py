"""Repeated (min,+) squaring (the paper's "Floyd-Warshall on GPU", Sec. 3.2) on the GPU against
the CPU oracle, through the C ABI: int32 bit-exact, float32 within 1e-5 relative (only the
order of summation differs from the oracle's Eq. 1 closure)."""
import numpy as np
import pytest
import torch

import oracle
import workloads
from test_gpu_parity import THREADS, assert_dist_equal

pytestmark = pytest.mark.gpu

INF = workloads.INF_I32


@pytest.fixture(scope="module")
def apsp():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import paper_2310_03983_gb300 as m
    assert m.apsp_device_status() == 0
    return m


def _path(n, w=1):
    h = np.full((n, n), INF, np.int32)
    np.fill_diagonal(h, 0)
    for v in range(n - 1):
        h[v, v + 1] = w
    return h


@pytest.mark.parametrize("n", [1, 2, 3, 100, 129, 300, 513])
@pytest.mark.parametrize("dtype", ["int32", "float32"])
def test_squaring_matches_oracle(apsp, n, dtype):
    if dtype == "int32":
        h = workloads.er_graph(n, 0.03, "int32", lo=1, hi=100, seed=300 + n)
    else:
        h = workloads.er_graph(n, 0.03, "float32", dist="lognormal", lo=0.0, hi=1.0, seed=300 + n)
    d = torch.from_numpy(h).cuda()
    apsp.apsp_squaring(d)
    assert_dist_equal(d.cpu().numpy(), oracle.fw(h, threads=THREADS), f"squaring n={n} {dtype}")
    assert apsp.apsp_device_status() == 0


def test_long_path_needs_every_product(apsp):
    """A directed path of 300 vertices has diameter 299: all ceil(log2 299) = 9 products change
    something, and the result equals the closure."""
    h = _path(300, 3)
    d = torch.from_numpy(h).cuda()
    apsp.apsp_squaring(d)
    assert_dist_equal(d.cpu().numpy(), oracle.fw(h), "path")


@pytest.mark.parametrize("t", [1, 3, 5])
def test_capped_products_match_oracle(apsp, t):
    """max_iters = t leaves the shortest paths of at most 2^t edges (oracle: t products of Eq. 2)."""
    h = workloads.er_graph(257, 0.006, "int32", lo=1, hi=100, seed=31)
    d = torch.from_numpy(h).cuda()
    apsp.apsp_squaring(d, max_iters=t)
    want, _ = oracle.squaring(h, max_iters=t)
    assert_dist_equal(d.cpu().numpy(), want, f"t={t}")


def test_unaligned_ld_and_int32_dpx_path(apsp):
    """ld = n + 1 (not a multiple of 4: the aligned-copy path) and weights whose (n - 1) * w_max
    exceeds 2^24 (the engine's int32 instruction path)."""
    n = 211
    h = workloads.er_graph(n, 0.05, "int32", lo=1, hi=200000, seed=32)
    base = torch.full((n, n + 1), 7, dtype=torch.int32, device="cuda")
    d = base[:, :n]
    d.copy_(torch.from_numpy(h))
    apsp.apsp_squaring(d)
    assert_dist_equal(d.cpu().numpy(), oracle.fw(h), "unaligned")
    assert torch.all(base[:, n] == 7)


def test_solve_and_equal_to_fw(apsp):
    h = workloads.er_graph(1500, 0.01, "int32", lo=1, hi=100, seed=33)
    a = apsp.solve(h, algo="squaring").numpy()
    b = apsp.solve(h, algo="fw").numpy()
    assert np.array_equal(a, b)
