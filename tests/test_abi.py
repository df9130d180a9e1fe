"""The C ABI: libapsp.so builds for sm_103a, loads, and exports every function include/apsp.h
declares.  No compute call is made here, so this runs without a GPU."""
import ctypes
import os
import re

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _builder():
    import __graft_entry__
    return __graft_entry__._builder()


def _declared():
    src = open(os.path.join(ROOT, "include", "apsp.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(\w+)\s*\(", src, flags=re.M)))


def test_library_builds_loads_and_exports_every_declared_symbol():
    path = _builder().build()
    lib = ctypes.CDLL(path)
    names = _declared()
    assert {"apsp_fw", "apsp_rkleene", "tropical_gemm", "apsp_normalise"} <= set(names)
    missing = [n for n in names if not hasattr(lib, n)]
    assert missing == []


def test_host_side_calls_without_gpu():
    lib = ctypes.CDLL(_builder().build())
    lib.apsp_version.restype = ctypes.c_int
    assert lib.apsp_version() == 100
    lib.apsp_status_str.restype = ctypes.c_char_p
    lib.apsp_status_str.argtypes = [ctypes.c_int]
    assert lib.apsp_status_str(0) == b"ok"
    # the launch counter is host-side: it reads and resets without a GPU
    lib.apsp_launch_count.restype, lib.apsp_launch_count.argtypes = ctypes.c_int64, [ctypes.c_int]
    lib.apsp_launch_count(1)
    assert lib.apsp_launch_count(0) == 0
    f = lib.apsp_rkleene_workspace_bytes
    f.restype, f.argtypes = ctypes.c_size_t, [ctypes.c_int64, ctypes.c_int64, ctypes.c_int, ctypes.c_int]
    # n <= cutoff: no scratch; n = 32768: one 16384 x 16384 block, plus (int32 only) the packed
    # 16-bit copies of the largest product's operands (2 x 16384 x 8192 words)
    assert f(256, 256, 0, 256) == 256  # bound words only
    assert f(32768, 32768, 1, 256) == 256 + 16384 * 16384 * 4
    assert f(32768, 32768, 0, 256) == 256 + 16384 * 16384 * 4 + 2 * 16384 * 8192 * 4
    g = lib.apsp_fw_workspace_bytes
    g.restype, g.argtypes = ctypes.c_size_t, [ctypes.c_int64, ctypes.c_int64, ctypes.c_int, ctypes.c_int]
    assert g(1000, 1000, 0, 0) == 256
    assert g(1001, 1001, 0, 0) >= 256 + 1001 * 1004 * 4
    # int32 FW from 4096 vertices: room for the 16-bit pass over 256-vertex blocks (packed
    # panels n x 128 + 128 x n words, and copies of the 256-wide row and column panels)
    assert g(4096, 4096, 1, 0) == 256
    assert g(4096, 4096, 0, 0) == 256 + 2 * 4096 * 128 * 4 + 2 * 4096 * 256 * 4
    # argument errors return before any CUDA call: n < 0, bad dtype
    h = lib.apsp_fw
    h.restype = ctypes.c_int
    h.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64, ctypes.c_int, ctypes.c_void_p, ctypes.c_int,
                  ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p]
    assert h(None, -1, 0, 0, None, 0, None, 0, None) == 1
    assert h(None, 4, 4, 7, None, 0, None, 0, None) == 1
    assert h(None, 0, 0, 0, None, 0, None, 0, None) == 0
    # the slab probes run 256 threads per block (the engine's consumer layout) and nothing else
    pr = lib.apsp_probe_minplus
    pr.restype = ctypes.c_int
    pr.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
    for v in (9, 10, 11):
        assert pr(v, 1, 128, 1, ctypes.c_void_p(16), None) == 1
    assert pr(12, 1, 256, 1, ctypes.c_void_p(16), None) == 1


def _staged_model(ns, count, packed=True):
    """The staging plan of apsp_batched, restated: graphs of 3..16 blocks of 128 vertices
    (the 14 largest block counts present), grouped by block count; workspace = 256 bytes of
    words, four per-graph int arrays, the index lists of the whole batch, the staging matrix
    (staged rows x the largest padded size), and (int32 only) two sets of the packed column
    panels (staged rows x 64) and packed row panels (64 rows per staged graph x the largest
    padded size)."""
    r256 = lambda b: -(-b // 256) * 256
    nbs = [-(-n // 128) if n > 0 else 0 for n in ns]
    present = sorted({nb for nb in nbs if 3 <= nb <= 16}, reverse=True)[:14]
    if not present:
        return 256
    staged = [nb for nb in nbs if nb in present]
    G, R, NP = len(staged), sum(nb * 128 for nb in staged), present[0] * 128
    return (256 + 4 * r256(4 * G) + r256(4 * count) + r256(4 * R * NP)
            + (2 * (r256(4 * R * 64) + r256(4 * G * 64 * NP)) if packed else 0))


def test_staged_plan_and_chunking_on_the_host():
    """apsp_batched's staging plan and apsp_batched_host's chunking are host code: their
    workspace sizes, checked here without a GPU against the plan restated in Python."""
    lib = ctypes.CDLL(_builder().build())
    f = lib.apsp_batched_staged_workspace_bytes
    f.restype, f.argtypes = ctypes.c_size_t, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int]
    h = lib.apsp_batched_host_workspace_bytes
    h.restype = ctypes.c_size_t
    h.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_int]
    rng = np.random.default_rng(3)
    cases = [[300], [256, 128, 5], [2048, 2049, 257, 0, -3], list(rng.integers(1, 1100, 300)),
             list(rng.integers(200, 2300, 40)), [384 * k for k in range(1, 6)] * 3]
    for ns in cases:
        arr = np.asarray(ns, np.int32)
        ptr = arr.ctypes.data_as(ctypes.c_void_p)
        assert f(ptr, len(arr), 0) == _staged_model(ns, len(arr)), ns
        assert f(ptr, len(arr), 1) == _staged_model(ns, len(arr), packed=False)  # float32: no packed panels
        # chunking: consecutive runs of about equal n^3, each run's staged room; the largest
        lds = ((np.maximum(arr, 1) + 3) // 4 * 4).astype(np.int32)
        offs = np.concatenate([[0], np.cumsum(np.maximum(arr, 0).astype(np.int64) * lds)[:-1]]).astype(np.int64)
        one = h(ptr, offs.ctypes.data_as(ctypes.c_void_p), lds.ctypes.data_as(ctypes.c_void_p), len(arr), 0, 1)
        assert one == f(ptr, len(arr), 0)
        four = h(ptr, offs.ctypes.data_as(ctypes.c_void_p), lds.ctypes.data_as(ctypes.c_void_p), len(arr), 0, 4)
        assert 256 <= four <= one
