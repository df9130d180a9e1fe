"""int32 closures too heavy for the 16-bit pass and for the exact fp32 bound: phase 3 runs in
fp32 on the int32 bit patterns truncated at 2^24 and is certified on the device, or, when a
distance crosses 2^24, the exact int32 pass finishes the closure.  And R-Kleene leaves, whose
blocks hold path lengths rather than edge weights: the certificates' step must be the leaf's
own largest entry.

Every case compares with the CPU oracle (bit-exact), and the FW cases also with the plain loop
that runs when the workspace has no room for the pass (a workspace of the bound words only).
"""
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


def _fw(apsp, h, full=True):
    n = h.shape[0]
    d = torch.from_numpy(h).cuda()
    # the required part only: the bound words and, for n % 4 != 0, the aligned copy of d
    base = 256 + ((n * ((n + 3) // 4 * 4) * 4 + 255) // 256 * 256 if n % 4 else 0)
    size = apsp.apsp_fw_workspace_bytes(n, n, d.dtype) if full else base
    apsp.apsp_fw(d, ws=torch.empty(size, dtype=torch.uint8, device="cuda"))
    assert apsp.apsp_device_status() == 0
    return d.cpu().numpy()


@pytest.mark.parametrize("n,hi", [(4096, 10**6), (4133, 3 * 10**6),   # truncated at 2^24, certified
                                  (4100, 2 * 10**8)])                 # beyond 2^22: exact int32
def test_heavy_weights_match_oracle(apsp, n, hi):
    h = workloads.er_graph(n, 0.05, "int32", lo=1, hi=hi, seed=n)
    got = _fw(apsp, h)
    assert_dist_equal(got, oracle.fw(h, threads=THREADS), f"n={n} hi={hi}")
    assert np.array_equal(got, _fw(apsp, h, full=False))


def _path(n, w):
    h = np.full((n, n), INF, np.int32)
    np.fill_diagonal(h, 0)
    idx = np.arange(n - 1)
    h[idx, idx + 1] = w
    return h


@pytest.mark.parametrize("n,w", [(4200, 5000), (4500, 60000)])
def test_long_paths_fail_the_certificate(apsp, n, w):
    """Directed paths whose distances cross 2^24 (the 2^24 certificate fails: the exact int32
    pass must finish), with a few shortcuts."""
    h = _path(n, w)
    rng = np.random.default_rng(n)
    a, b = rng.integers(0, n, 40), rng.integers(0, n, 40)
    h[a, b] = np.where(a != b, rng.integers(1, w + 1, 40), 0)
    assert (n - 1) * w >= 1 << 24
    assert_dist_equal(_fw(apsp, h), oracle.fw(h, threads=THREADS), f"path n={n} w={w}")


def test_just_below_the_cap_certifies(apsp):
    """A path whose longest distance plus the largest weight stays below 2^24 while
    (n - 1) w_max is far above it (one heavy edge back from the last vertex): the certificate
    holds and the truncated pass alone gives the closure."""
    n, w, heavy = 4096, 3000, 10**6
    h = _path(n, w)
    h[n - 1, n - 2] = heavy
    want = oracle.fw(h, threads=THREADS)
    assert want[want < INF].max() + heavy < 1 << 24 <= (n - 1) * heavy
    assert_dist_equal(_fw(apsp, h), want, "just below 2^24")


def _alternating_path(n, w):
    """u_0 -> f_0 -> u_1 -> f_1 -> ... with u_k = n/2 + k and f_k = k, every edge of weight w:
    after R-Kleene's update through the first half, the second half's leaf holds steps of 2w."""
    h = np.full((n, n), INF, np.int32)
    np.fill_diagonal(h, 0)
    half = n // 2
    seq = np.empty(n, np.int64)
    seq[0::2] = half + np.arange(half)
    seq[1::2] = np.arange(half)
    h[seq[:-1], seq[1:]] = w
    return h, seq


@pytest.mark.parametrize("w", [100, 16417])
def test_rkleene_leaf_certificate_uses_leaf_steps(apsp, w):
    """n = 8192, cutoff 4096: the second leaf's entries are multiples of 2w.  w = 100: it closes
    on packed 16-bit pairs, and no multiple of 200 lies in [0x3FFF - 100, 0x3FFF), so a
    certificate stepping by the largest weight would pass while distances beyond the cap exist.
    w = 16417: the same with phase 3 truncated at 2^24 (510 * 2w lies below 2^24 - w, and
    511 * 2w is above 2^24)."""
    n, cutoff = 8192, 4096
    h, seq = _alternating_path(n, w)
    d = torch.from_numpy(h).cuda()
    ws = torch.empty(apsp.apsp_rkleene_workspace_bytes(n, n, torch.int32, cutoff), dtype=torch.uint8, device="cuda")
    apsp.apsp_rkleene(d, cutoff=cutoff, ws=ws)
    assert apsp.apsp_device_status() == 0
    got = d.cpu().numpy()
    pos = np.empty(n, np.int64)
    pos[seq] = np.arange(n)
    pi, pj = np.meshgrid(pos, pos, indexing="ij")
    want = np.where(pj >= pi, (pj - pi) * w, INF)
    want = np.where(want >= INF, INF, want)
    assert np.array_equal(got.astype(np.int64), want)
    src = np.array([int(seq[0]), int(seq[1]), int(seq[n // 3]), int(seq[-2])])
    assert_dist_equal(got[src], oracle.dijkstra_rows(h, src, threads=THREADS), "rows")
