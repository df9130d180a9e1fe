"""The C ABI: libapsp.so builds for sm_103a, loads, and exports every function include/apsp.h
declares.  No compute call is made here, so this runs without a GPU."""
import ctypes
import os
import re

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
