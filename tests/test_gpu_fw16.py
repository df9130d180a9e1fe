"""Blocked Floyd-Warshall with phase 3 on packed 16-bit pairs (int32 closures of at least 4096
vertices whose largest weight is at most 0x3FFF / 4), against the CPU oracle, bit-exact.

The 16-bit pass computes the closure truncated at 0x3FFF; a device-side certificate (largest
stored value below the cap plus the largest weight stays below the cap) proves it exact, and
otherwise the int32 pass runs again over the stored matrix.  Covered here: graphs that pass the
certificate, graphs whose long paths fail it (the int32 pass must finish the job), weights too
large for the 16-bit pass, and a workspace without room for the packed panels."""
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


def _close(apsp, h, ws_bytes=None):
    d = torch.from_numpy(h).cuda()
    ws = None
    if ws_bytes is not None:
        ws = torch.empty(ws_bytes, dtype=torch.uint8, device="cuda")
    apsp.apsp_fw(d, ws=ws)
    assert apsp.apsp_device_status() == 0
    return d.cpu().numpy()


@pytest.mark.parametrize("n,p,hi", [(4096, 0.01, 100), (4100, 0.3, 1000), (4133, 0.002, 4095)])
def test_fw16_matches_oracle(apsp, n, p, hi):
    h = workloads.er_graph(n, p, "int32", lo=1, hi=hi, seed=n + hi)
    assert_dist_equal(_close(apsp, h), oracle.fw(h, threads=THREADS), f"n={n} p={p} hi={hi}")


def _path_graph(n, w, extra=0, seed=0):
    h = np.full((n, n), INF, np.int32)
    np.fill_diagonal(h, 0)
    idx = np.arange(n - 1)
    h[idx, idx + 1] = w
    if extra:  # a few random shortcuts
        rng = np.random.default_rng(seed)
        a, b = rng.integers(0, n, extra), rng.integers(0, n, extra)
        h[a, b] = np.where(a != b, rng.integers(1, w + 1, extra), 0)
    return h


def test_long_paths_below_the_cap_certify(apsp):
    """A directed path of 4096 vertices with weight 3: distances up to 12285, still below the
    cap, so the certificate holds; every entry must be exact."""
    n = 4096
    h = _path_graph(n, 3)
    i, j = np.indices((n, n))
    want = np.where(j >= i, 3 * (j - i), INF)
    assert np.array_equal(_close(apsp, h), want)


@pytest.mark.parametrize("w,extra", [(100, 0), (1000, 300)])
def test_long_paths_above_the_cap_rerun_in_int32(apsp, w, extra):
    """Paths far longer than the cap: the truncated pass cannot be certified and the int32
    pass must produce the exact closure."""
    n = 4200
    h = _path_graph(n, w, extra, seed=w)
    assert_dist_equal(_close(apsp, h), oracle.fw(h, threads=THREADS), f"w={w}")


def test_heavy_weights_skip_the_16bit_pass(apsp):
    n = 4096
    h = workloads.er_graph(n, 0.02, "int32", lo=1, hi=50000, seed=5)
    assert_dist_equal(_close(apsp, h), oracle.fw(h, threads=THREADS), "heavy")


def test_base_workspace_uses_the_plain_phase3(apsp):
    """A workspace without room for the packed panels is accepted; the result is identical."""
    n = 4352
    h = workloads.er_graph(n, 0.01, "int32", lo=1, hi=100, seed=6)
    full = apsp.apsp_fw_workspace_bytes(n, n)
    assert full > 256
    a = _close(apsp, h)
    b = _close(apsp, h, ws_bytes=256)
    c = _close(apsp, h, ws_bytes=full)
    assert np.array_equal(a, b) and np.array_equal(a, c)
    rows = np.random.default_rng(7).choice(n, 16, replace=False)
    assert_dist_equal(a[rows], oracle.dijkstra_rows(h, rows, threads=THREADS), "rows")


@pytest.mark.parametrize("n,hi", [(2600, 100), (2300, 3000)])
def test_rkleene_packed_products_match_oracle(apsp, n, hi):
    """R-Kleene with products of >= 10^9 pairs on packed 16-bit pairs (operand maxima summing
    below 0x3FFF, checked per product on the device); with hi = 3000 some products exceed the
    cap and take the plain path.  Bit-exact, and identical with a workspace without the packed
    room."""
    h = workloads.er_graph(n, 0.01, "int32", lo=1, hi=hi, seed=n)
    d = torch.from_numpy(h).cuda()
    apsp.apsp_rkleene(d, cutoff=256)
    got = d.cpu().numpy()
    assert apsp.apsp_device_status() == 0
    assert_dist_equal(got, oracle.fw(h, threads=THREADS), f"rkleene n={n} hi={hi}")
    base = apsp.apsp_rkleene_workspace_bytes(n, n, torch.float32, 256)  # same size minus the packed room
    d2 = torch.from_numpy(h).cuda()
    apsp.apsp_rkleene(d2, cutoff=256, ws=torch.empty(base, dtype=torch.uint8, device="cuda"))
    assert np.array_equal(d2.cpu().numpy(), got)


@pytest.mark.parametrize("inf", [1 << 20, 5000])
def test_custom_sentinel(apsp, inf):
    """A sentinel above the 16-bit cap keeps the packed phase 3 (unreachable pairs must come
    back as exactly that sentinel); one below it takes the plain phase 3.  Bit-exact both ways."""
    n = 4096
    h = workloads.er_graph(n, 0.003, "int32", lo=1, hi=40, seed=inf % 97)
    h[:, :64] = INF          # columns nobody reaches except themselves
    np.fill_diagonal(h, 0)
    hc = np.where(h >= INF, inf, h).astype(np.int32)
    d = torch.from_numpy(hc).cuda()
    apsp.apsp_fw(d, inf=inf)
    assert apsp.apsp_device_status() == 0
    want = oracle.fw(hc, inf=inf, threads=THREADS)
    assert_dist_equal(d.cpu().numpy(), want, f"inf={inf}")


def test_wide_blocks_rows(apsp):
    """n = 16400: the 16-bit pass on 256-vertex blocks (a ragged last block of 16 vertices),
    checked on 24 source rows by Dijkstra, bit-exact."""
    n = 16400
    h = workloads.er_graph(n, 0.004, "int32", lo=1, hi=100, seed=77)
    d = torch.from_numpy(h).cuda()
    apsp.apsp_fw(d)
    assert apsp.apsp_device_status() == 0
    rows = np.random.default_rng(78).choice(n, 24, replace=False)
    got = d.cpu().numpy()[rows]
    assert_dist_equal(got, oracle.dijkstra_rows(h, rows, threads=THREADS), "rows")


def test_wide_blocks_long_path_reruns(apsp):
    """A directed path of 16384 vertices with unit weights: distances reach the cap, the
    certificate fails and the int32 pass must produce the closed form exactly."""
    n = 16384
    h = _path_graph(n, 1)
    d = torch.from_numpy(h).cuda()
    apsp.apsp_fw(d)
    assert apsp.apsp_device_status() == 0
    got = d.cpu().numpy()
    for i in (0, 1, 255, 256, 8191, 16383):
        row = got[i]
        j = np.arange(n)
        assert np.array_equal(row, np.where(j >= i, j - i, INF)), i
