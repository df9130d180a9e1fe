"""Parity of the CUDA path (through the C ABI) with the CPU oracle, element by element.

int32 results must be bit-exact.  float32 results must be within 1e-5 relative of the fp64
oracle, with +inf (unreachable) and 0 matching exactly.  The 1e-5 bound follows from the
arithmetic: each finite distance is a sum of L non-negative fp32 weights, computed with one
round-to-nearest add per hop, so its relative error is at most (L - 1) * 2^-24 ~ 6e-8 * L;
1e-5 therefore covers paths of up to ~160 hops, far beyond the shortest paths of these graphs.
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


def assert_dist_equal(got, want, what=""):
    got = np.asarray(got)
    want = np.asarray(want)
    assert got.shape == want.shape, what
    if got.dtype == np.int32 or want.dtype.kind in "iu":
        bad = np.argwhere(got.astype(np.int64) != want.astype(np.int64))
        assert bad.size == 0, f"{what}: {len(bad)} mismatches, first {bad[:5].tolist()}"
        return
    g = got.astype(np.float64)
    w = want.astype(np.float64)
    assert np.array_equal(np.isinf(g), np.isinf(w)), f"{what}: reachability differs"
    f = np.isfinite(w)
    assert np.array_equal(g[f] == 0, w[f] == 0), f"{what}: zeros differ"
    rel = np.abs(g[f] - w[f]) / np.maximum(np.abs(w[f]), 1e-30)
    assert rel.size == 0 or rel.max() <= 1e-5, f"{what}: max rel err {rel.max():.3g}"


def _rand(rng, shape, dtype, p_inf=0.3):
    if dtype == np.int32:
        v = rng.integers(0, 1000, size=shape)
        return np.where(rng.random(shape) < p_inf, INF, v).astype(np.int32)
    v = rng.lognormal(size=shape)
    return np.where(rng.random(shape) < p_inf, np.inf, v).astype(np.float32)


# ------------------------------------------------------------------ a1: normalise
def test_normalise(apsp):
    h = np.array([[5, 3, INF + 7], [2**31 - 1, 9, 0], [1, 2, 3]], np.int32)
    d = torch.from_numpy(h).cuda()
    apsp.apsp_normalise(d)
    assert d.cpu().numpy().tolist() == [[0, 3, INF], [INF, 0, 0], [1, 2, 0]]
    assert apsp.apsp_device_status() == 0
    bad = torch.tensor([[0, -1], [2, 0]], dtype=torch.int32, device="cuda")
    apsp.apsp_normalise(bad)
    assert apsp.apsp_device_status() == 2
    assert apsp.apsp_device_status() == 0  # read clears the sticky word
    f = torch.tensor([[3.0, 1e30], [float("nan"), 1.0]], device="cuda")
    apsp.apsp_normalise(f, inf=1e29)
    assert apsp.apsp_device_status() == 2
    g = torch.tensor([[3.0, 1e30], [2.5, 1.0]], device="cuda")
    apsp.apsp_normalise(g, inf=1e29)
    assert g.cpu().numpy().tolist() == [[0.0, float("inf")], [2.5, 0.0]]
    assert apsp.apsp_device_status() == 0


def test_normalise_custom_sentinel_and_ld(apsp):
    base = torch.full((5, 7), 50, dtype=torch.int32, device="cuda")
    d = base[:, :5]  # leading dimension 7
    d[1, 2] = 80
    apsp.apsp_normalise(d, inf=60)
    got = d.cpu().numpy()
    assert got[1, 2] == 60 and got[0, 1] == 50 and np.all(np.diagonal(got) == 0)
    assert np.all(base[:, 5:].cpu().numpy() == 50)  # padding columns untouched


# ------------------------------------------------------------------ a2: tropical GEMM
SHAPES = [(1, 1, 1), (7, 5, 3), (31, 33, 32), (128, 128, 128), (129, 127, 33), (130, 257, 129),
          (300, 200, 100), (256, 384, 512), (5, 600, 7), (1000, 64, 31)]


@pytest.mark.parametrize("dtype", [np.int32, np.float32])
@pytest.mark.parametrize("M,N,K", SHAPES)
def test_tropical_gemm_parity(apsp, dtype, M, N, K):
    rng = np.random.default_rng(M * 7919 + N * 31 + K)
    a, b, c = _rand(rng, (M, K), dtype), _rand(rng, (K, N), dtype), _rand(rng, (M, N), dtype, 0.5)
    A, B = torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda()
    C = torch.empty((M, N), dtype=A.dtype, device="cuda")
    apsp.tropical_gemm(C, A, B)
    assert_dist_equal(C.cpu().numpy(), oracle.minplus(a, b), f"overwrite {M}x{N}x{K}")
    C2 = torch.from_numpy(c).cuda()
    apsp.tropical_gemm(C2, A, B, accumulate=True)
    assert_dist_equal(C2.cpu().numpy(), oracle.minplus(a, b, c), f"accumulate {M}x{N}x{K}")
    assert apsp.apsp_device_status() == 0


@pytest.mark.parametrize("dtype", [np.int32, np.float32])
def test_tropical_gemm_strided_and_unaligned(apsp, dtype):
    rng = np.random.default_rng(3)
    M, N, K = 70, 45, 37
    a, b = _rand(rng, (M, K), dtype), _rand(rng, (K, N), dtype)
    # aligned views with padded leading dimensions (TMA engine)
    Abig = torch.from_numpy(_rand(rng, (M, 64), dtype)).cuda()
    Abig[:, :K] = torch.from_numpy(a).cuda()
    Bbig = torch.from_numpy(_rand(rng, (K, 52), dtype)).cuda()
    Bbig[:, :N] = torch.from_numpy(b).cuda()
    Cbig = torch.zeros((M, 48), dtype=Abig.dtype, device="cuda")
    apsp.tropical_gemm(Cbig[:, :N], Abig[:, :K], Bbig[:, :N])
    want = oracle.minplus(a, b)
    assert_dist_equal(Cbig[:, :N].cpu().numpy(), want, "padded ld")
    assert np.all(Cbig[:, N:].cpu().numpy() == 0)
    # odd leading dimensions and offsets (plain-load kernel)
    Aodd = torch.from_numpy(_rand(rng, (M, K + 3), dtype)).cuda()
    Aodd[:, 1:K + 1] = torch.from_numpy(a).cuda()
    C = torch.empty((M, N), dtype=Abig.dtype, device="cuda")
    apsp.tropical_gemm(C, Aodd[:, 1:K + 1], torch.from_numpy(b).cuda())
    assert_dist_equal(C.cpu().numpy(), want, "unaligned")


@pytest.mark.parametrize("hi", [1000, 8191, 8192, 2**23 - 1, 2**23, 2**24, 10**8])
def test_tropical_gemm_int_paths(apsp, hi):
    """Entries up to `hi`: largest entries summing below 0x3FFF take the packed 16-bit path
    (8191 + 8191 = 0x3FFE), below 2^24 the exact fp32 path, above it the int32 path; all must
    give the oracle's values, including sums right at each boundary."""
    rng = np.random.default_rng(hi % 1000)
    M, N, K = 200, 160, 140
    a = np.where(rng.random((M, K)) < 0.8, rng.integers(hi // 2, hi, (M, K), endpoint=True), INF).astype(np.int32)
    b = np.where(rng.random((K, N)) < 0.8, rng.integers(hi // 2, hi, (K, N), endpoint=True), INF).astype(np.int32)
    C = torch.empty((M, N), dtype=torch.int32, device="cuda")
    apsp.tropical_gemm(C, torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda())
    assert_dist_equal(C.cpu().numpy(), oracle.minplus(a, b), f"hi={hi}")


@pytest.mark.parametrize("M,N,K", [(129, 130, 1), (200, 160, 141), (64, 512, 256)])
def test_tropical_gemm_16bit_path_equals_others(apsp, M, N, K):
    """The same product with the full workspace (packed 16-bit path), with only the 256 bytes
    of bound words (exact fp32 path), and in accumulate mode over a C with entries above the
    16-bit cap: identical, and equal to the oracle."""
    rng = np.random.default_rng(M + N + K)
    a = np.where(rng.random((M, K)) < 0.7, rng.integers(0, 5000, (M, K)), INF).astype(np.int32)
    b = np.where(rng.random((K, N)) < 0.7, rng.integers(0, 5000, (K, N)), INF).astype(np.int32)
    c = np.where(rng.random((M, N)) < 0.7, rng.integers(0, 40000, (M, N)), INF).astype(np.int32)
    A, B = torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda()
    full = torch.empty(apsp.tropical_gemm_workspace_bytes(M, N, K), dtype=torch.uint8, device="cuda")
    small = torch.empty(256, dtype=torch.uint8, device="cuda")
    outs = []
    for ws in (full, small):
        C = torch.from_numpy(c).cuda()
        apsp.tropical_gemm(C, A, B, accumulate=True, ws=ws)
        outs.append(C.cpu().numpy())
        C = torch.empty((M, N), dtype=torch.int32, device="cuda")
        apsp.tropical_gemm(C, A, B, ws=ws)
        outs.append(C.cpu().numpy())
    assert_dist_equal(outs[0], oracle.minplus(a, b, c), "16-bit accumulate")
    assert_dist_equal(outs[1], oracle.minplus(a, b), "16-bit overwrite")
    assert np.array_equal(outs[0], outs[2]) and np.array_equal(outs[1], outs[3])


def test_tropical_gemm_16bit_small_sentinel(apsp):
    """A sentinel below the 16-bit cap: finite sums that reach it must come back as the
    sentinel, exactly as on the int32 path."""
    rng = np.random.default_rng(17)
    inf = 1000
    M, N, K = 150, 140, 90
    a = np.where(rng.random((M, K)) < 0.7, rng.integers(0, 900, (M, K)), inf).astype(np.int32)
    b = np.where(rng.random((K, N)) < 0.7, rng.integers(0, 900, (K, N)), inf).astype(np.int32)
    C = torch.empty((M, N), dtype=torch.int32, device="cuda")
    apsp.tropical_gemm(C, torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda(), inf=inf)
    assert_dist_equal(C.cpu().numpy(), oracle.minplus(a, b, inf=inf), "inf=1000")


def test_tropical_gemm_identity_and_k0(apsp):
    n = 200
    eye = np.full((n, n), INF, np.int32)
    np.fill_diagonal(eye, 0)
    b = np.random.default_rng(1).integers(0, 100, (n, 150)).astype(np.int32)
    C = torch.empty((n, 150), dtype=torch.int32, device="cuda")
    apsp.tropical_gemm(C, torch.from_numpy(eye).cuda(), torch.from_numpy(b).cuda())
    assert np.array_equal(C.cpu().numpy(), b)
    A0 = torch.empty((n, 0), dtype=torch.int32, device="cuda")
    B0 = torch.empty((0, 150), dtype=torch.int32, device="cuda")
    apsp.tropical_gemm(C, A0, B0)
    assert np.all(C.cpu().numpy() == INF)


def test_tropical_gemm_rejects_overlap(apsp):
    X = torch.zeros((64, 64), dtype=torch.int32, device="cuda")
    with pytest.raises(apsp.ApspError):
        apsp.tropical_gemm(X, X, X)


# ------------------------------------------------------------------ a3-a6: closures
def _graph(n, p, dtype, seed):
    if dtype == np.int32:
        return workloads.er_graph(n, p, "int32", lo=1, hi=100, seed=seed)
    return workloads.er_graph(n, p, "float32", dist="lognormal", lo=0.0, hi=1.0, seed=seed)


ALGOS = [("fw", 0), ("rkleene", 128), ("rkleene", 256), ("cta", 0)]


def _close(apsp, d, algo, param):
    if algo == "fw":
        apsp.apsp_fw(d)
    elif algo == "cta":
        apsp.apsp_close_cta(d)
    else:
        apsp.apsp_rkleene(d, cutoff=param)


@pytest.mark.parametrize("dtype", [np.int32, np.float32])
@pytest.mark.parametrize("n", [1, 2, 3, 17, 64, 127, 128, 129, 200, 255, 256, 257, 300, 383, 520])
def test_closure_parity_small(apsp, dtype, n):
    h = _graph(n, min(1.0, 4.0 / n), dtype, seed=n)
    want = oracle.fw(h, threads=THREADS)
    for algo, param in ALGOS:
        d = torch.from_numpy(h).cuda()
        _close(apsp, d, algo, param)
        assert_dist_equal(d.cpu().numpy(), want, f"{algo}/{param} n={n}")
    assert apsp.apsp_device_status() == 0


def test_config_n512_bit_exact(apsp):
    """Directed ER n=512, p=0.1, int32 weights in [1, 100], seed 0: FW bit-exact."""
    h = workloads.er_graph(512, 0.1, "int32", lo=1, hi=100, seed=0)
    want = oracle.fw(h, threads=THREADS)
    d = torch.from_numpy(h).cuda()
    apsp.apsp_fw(d)
    assert_dist_equal(d.cpu().numpy(), want, "fw n=512")
    assert oracle.check_invariants(d.cpu().numpy(), h, sample_k=64) == []


@pytest.mark.parametrize("n", [700, 1001])
def test_closure_odd_leading_dimension(apsp, n):
    h = _graph(n, 0.01, np.int32, seed=5)
    want = oracle.fw(h, threads=THREADS)
    for fn in (apsp.apsp_fw, apsp.apsp_rkleene):
        big = torch.zeros((n, n + 3), dtype=torch.int32, device="cuda")
        d = big[:, :n]
        d.copy_(torch.from_numpy(h))
        fn(d)
        assert_dist_equal(d.cpu().numpy(), want, f"{fn.__name__} ld={n + 3}")
        assert np.all(big[:, n:].cpu().numpy() == 0)


def test_special_graphs(apsp):
    n = 300
    empty = np.full((n, n), INF, np.int32)
    d = torch.from_numpy(empty).cuda()
    apsp.apsp_fw(d)
    want = empty.copy()
    np.fill_diagonal(want, 0)
    assert np.array_equal(d.cpu().numpy(), want)
    # directed path: distances are prefix sums
    path = empty.copy()
    w = np.arange(1, n, dtype=np.int64) % 7 + 1
    for i in range(n - 1):
        path[i, i + 1] = w[i]
    pref = np.concatenate([[0], np.cumsum(w)])
    expect = np.where(np.arange(n)[:, None] <= np.arange(n)[None, :], pref[None, :] - pref[:, None], INF)
    for fn in (apsp.apsp_fw, apsp.apsp_rkleene):
        d = torch.from_numpy(path).cuda()
        fn(d)
        assert np.array_equal(d.cpu().numpy().astype(np.int64), expect)
    # complete graph, unit weights
    comp = np.ones((n, n), np.int32)
    d = torch.from_numpy(comp).cuda()
    apsp.apsp_rkleene(d, cutoff=128)
    np.fill_diagonal(comp, 0)
    assert np.array_equal(d.cpu().numpy(), comp)


def test_saturation_near_inf(apsp):
    """Weights just below the sentinel: sums exceed it, results must clamp to exactly INF."""
    n = 260
    h = np.full((n, n), INF, np.int32)
    np.fill_diagonal(h, 0)
    for i in range(n - 1):
        h[i, i + 1] = INF - 1 if i % 2 == 0 else 1
    want = oracle.fw(h)
    for fn in (apsp.apsp_fw, apsp.apsp_rkleene):
        d = torch.from_numpy(h).cuda()
        fn(d)
        assert_dist_equal(d.cpu().numpy(), want, fn.__name__)


@pytest.mark.parametrize("hi", [100, 65000, 66000, 10**6])
def test_closure_int_paths(apsp, hi):
    """n = 258 with weights up to `hi`: (n - 1) * hi crosses 2^24 between 65000 and 66000, so
    both the exact fp32 path and the int32 path are exercised on long shortest paths."""
    n = 258
    rng = np.random.default_rng(hi)
    h = np.full((n, n), INF, np.int32)
    np.fill_diagonal(h, 0)
    perm = rng.permutation(n)
    for a, b in zip(perm[:-1], perm[1:]):  # a Hamiltonian path of heavy edges: long distances
        h[a, b] = rng.integers(hi - 50, hi, endpoint=True)
    extra = rng.random((n, n)) < 0.01
    h[extra] = rng.integers(hi // 2, hi, size=int(extra.sum()), endpoint=True)
    np.fill_diagonal(h, 0)
    want = oracle.fw(h)
    for fn, kw in ((apsp.apsp_fw, {}), (apsp.apsp_rkleene, {"cutoff": 128})):
        d = torch.from_numpy(h).cuda()
        fn(d, **kw)
        assert_dist_equal(d.cpu().numpy(), want, f"{fn.__name__} hi={hi}")


def test_empty_matrix(apsp):
    d = torch.empty((0, 0), dtype=torch.int32, device="cuda")
    apsp.apsp_fw(d)
    apsp.apsp_rkleene(d)


def test_domain_error_reported(apsp):
    h = _graph(130, 0.05, np.int32, seed=1)
    h[3, 7] = -5
    d = torch.from_numpy(h).cuda()
    apsp.apsp_fw(d)
    assert apsp.apsp_device_status() == 2


# ------------------------------------------------------------------ n = 4096 configuration
@pytest.mark.parametrize("p,dtype", [(0.01, np.int32), (0.5, np.int32), (0.5, np.float32)])
def test_config_n4096(apsp, p, dtype):
    """n=4096 directed ER; int32 weights in [1, 1000] (p=0.01, 0.5), fp32 lognormal(0,1):
    blocked FW and R-Kleene (cutoff 256) against the full oracle."""
    if dtype == np.int32:
        h = workloads.er_graph(4096, p, "int32", lo=1, hi=1000, seed=1)
    else:
        h = workloads.er_graph(4096, p, "float32", dist="lognormal", lo=0.0, hi=1.0, seed=2)
    want = oracle.fw(h, threads=THREADS)
    for fn, kw in ((apsp.apsp_fw, {}), (apsp.apsp_rkleene, {"cutoff": 256})):
        d = torch.from_numpy(h).cuda()
        fn(d, **kw)
        assert_dist_equal(d.cpu().numpy(), want, f"{fn.__name__} p={p}")
    assert apsp.apsp_device_status() == 0
