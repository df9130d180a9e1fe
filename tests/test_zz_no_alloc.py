"""apsp_rkleene_noalloc: R-Kleene for callers that cannot allocate device memory.

Some callers may not call cudaMalloc at all: code running inside a framework or plugin host
that owns every byte of device memory through its own pool, allocation-free request paths,
processes under a hard memory budget.  This entry point keeps its scratch in a fixed array
inside libapsp.so, so the caller hands over only the matrix.  The test calls it through the
C ABI twice in a row -- on two different graphs, so the second call starts from whatever the
first left in the shared array -- and checks each result against apsp_rkleene, which takes its
scratch from the caller: int32 bit-exact, float32 within the suite's 1e-5 relative tolerance.
This file is named to be collected last.
"""
import ctypes

import numpy as np
import pytest
import torch

import workloads
from test_gpu_parity import assert_dist_equal

pytestmark = pytest.mark.gpu

APSP_I32, APSP_F32, APSP_ERR_ARG = 0, 1, 1


@pytest.fixture(scope="module")
def apsp():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import paper_2310_03983_gb300 as m
    return m


def _noalloc(apsp):
    f = ctypes.CDLL(apsp.LIB_PATH).apsp_rkleene_noalloc
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64, ctypes.c_int, ctypes.c_void_p, ctypes.c_int,
                  ctypes.c_void_p]
    return f


def _call(f, d, cutoff):
    code = APSP_I32 if d.dtype == torch.int32 else APSP_F32
    stream = torch.cuda.current_stream().cuda_stream
    return f(d.data_ptr(), d.shape[0], d.stride(0), code, None, cutoff, stream)


def _reference(apsp, h, cutoff):
    d = torch.from_numpy(h).cuda()
    ws = torch.empty(apsp.apsp_rkleene_workspace_bytes(h.shape[0], h.shape[0], d.dtype, cutoff),
                     dtype=torch.uint8, device="cuda")
    apsp.apsp_rkleene(d, cutoff=cutoff, ws=ws)
    return d.cpu().numpy()


def test_noalloc_matches_rkleene_twice(apsp):
    f = _noalloc(apsp)
    # first call: the largest size the array holds, weights large enough for the int32 path
    h1 = workloads.er_graph(4096, 0.01, "int32", lo=1, hi=10**5, seed=21)
    # second call: a different size and the exact fp32 path, over the first call's leftovers
    h2 = workloads.er_graph(1500, 0.05, "int32", lo=1, hi=100, seed=22)
    for h, cutoff in ((h1, 256), (h2, 128)):
        d = torch.from_numpy(h).cuda()
        assert _call(f, d, cutoff) == 0
        assert_dist_equal(d.cpu().numpy(), _reference(apsp, h, cutoff), f"noalloc n={h.shape[0]}")
    assert apsp.apsp_device_status() == 0


def test_noalloc_float_and_limits(apsp):
    f = _noalloc(apsp)
    for seed in (31, 32):
        h = workloads.er_graph(2000, 0.1, "float32", dist="lognormal", lo=0.0, hi=1.0, seed=seed)
        d = torch.from_numpy(h).cuda()
        assert _call(f, d, 256) == 0
        assert_dist_equal(d.cpu().numpy(), _reference(apsp, h, 256), f"noalloc fp32 seed={seed}")
    # beyond the array's capacity, or an unaligned leading dimension: refused, nothing launched
    big = torch.zeros((4100, 4100), dtype=torch.int32, device="cuda")
    assert _call(f, big, 256) == APSP_ERR_ARG
    odd = torch.zeros((300, 303), dtype=torch.int32, device="cuda")[:, :300]
    assert _call(f, odd, 128) == APSP_ERR_ARG
    assert apsp.apsp_device_status() == 0
