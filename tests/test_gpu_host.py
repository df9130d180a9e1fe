"""Entry points on host buffers: apsp_solve_host (one matrix: copy in, close, copy back) and
apsp_batched_host (a batch pipelined in chunks over copy streams), against the device calls
and the oracle."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import workloads
from test_gpu_parity import assert_dist_equal

pytestmark = pytest.mark.gpu
APSP_I32, APSP_F32, APSP_ERR_ARG = 0, 1, 1


@pytest.fixture(scope="module")
def apsp():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import paper_2310_03983_gb300 as m
    assert m.apsp_device_status() == 0
    return m


@pytest.mark.parametrize("algo,param", [("fw", 0), ("rkleene", 256), ("squaring", 0)])
def test_solve_host_matches_device_calls(apsp, algo, param):
    h = workloads.er_graph(700, 0.03, "int32", lo=1, hi=100, seed=41)
    got = apsp.solve(h, algo=algo, param=param).numpy()
    d = torch.from_numpy(h).cuda()
    {"fw": lambda: apsp.apsp_fw(d), "rkleene": lambda: apsp.apsp_rkleene(d, cutoff=param),
     "squaring": lambda: apsp.apsp_squaring(d)}[algo]()
    assert np.array_equal(got, d.cpu().numpy())
    assert_dist_equal(got, oracle.fw(h), algo)
    assert apsp.apsp_device_status() == 0


def test_solve_host_padded_rows_pinned_and_in_place(apsp):
    """A host matrix with a leading dimension past n, pinned, closed in place (h_in == h_out)
    in a caller-given device buffer; float32 as well."""
    lib = apsp.lib()
    for dtype in ("int32", "float32"):
        n, ld = 301, 307
        h = (workloads.er_graph(n, 0.05, "int32", lo=1, hi=50, seed=42) if dtype == "int32" else
             workloads.er_graph(n, 0.05, "float32", dist="lognormal", lo=0.0, hi=1.0, seed=42))
        host = torch.zeros((n, ld), dtype=getattr(torch, dtype)).pin_memory()
        host[:, :n] = torch.from_numpy(h)
        dbuf = torch.empty((n, 304), dtype=host.dtype, device="cuda")
        code = APSP_I32 if dtype == "int32" else APSP_F32
        r = lib.apsp_solve_host(host.data_ptr(), host.data_ptr(), n, ld, code, 0, 0, None, dbuf.data_ptr(), 304,
                                None, 0, torch.cuda.current_stream().cuda_stream)
        assert r == 0
        assert_dist_equal(host[:, :n].numpy(), oracle.fw(h), dtype)
        assert torch.all(host[:, n:] == 0)  # the padding of the host rows is left alone
    # a host leading dimension below n is refused before any copy
    assert lib.apsp_solve_host(host.data_ptr(), host.data_ptr(), n, n - 1, code, 0, 0, None, None, 0, None, 0,
                               None) == APSP_ERR_ARG


@pytest.mark.parametrize("chunks", [1, 3, 4, 9])
def test_batched_host_matches_device_call(apsp, chunks):
    ns, ps = workloads.batch_specs(200, n_lo=20, n_hi=900, seed=13)
    mats = workloads.batch_graphs(ns, ps)
    b = apsp.Batch(mats)
    apsp.apsp_batched(b)
    want = b.pool.cpu()
    b.pool.zero_()  # the host call must copy everything in itself
    out = apsp.apsp_batched_host(b, chunks=chunks)
    assert torch.equal(out, want)
    assert torch.equal(apsp.Batch(mats).host, b.host)  # the input stays as it was
    assert apsp.apsp_device_status() == 0
    for g in np.argsort(ns)[-3:]:
        g = int(g)
        assert_dist_equal(b.graph(g, out).numpy(), oracle.fw(mats[g]), f"graph {g}")


def test_batched_host_in_place_and_out_of_order_layout(apsp):
    """h_in == h_out works; a pool that stores the even-indexed graphs first and the odd ones
    after them (runs of consecutive graphs then cover interleaved pool ranges) runs as one
    chunk with the same results."""
    ns, ps = workloads.batch_specs(60, n_lo=20, n_hi=600, seed=14)
    mats = workloads.batch_graphs(ns, ps)
    b = apsp.Batch(mats)
    apsp.apsp_batched(b)
    want = b.pool.cpu()
    buf = b.host.clone().pin_memory()
    out = apsp.apsp_batched_host(b, buf, buf, chunks=4)
    assert out.data_ptr() == buf.data_ptr() and torch.equal(buf, want)
    order = list(range(0, len(mats), 2)) + list(range(1, len(mats), 2))
    rev = apsp.Batch([mats[g] for g in order])
    perm = apsp.Batch(mats)
    perm.offsets = np.empty_like(rev.offsets)
    perm.offsets[order] = rev.offsets
    perm.d_offsets = torch.from_numpy(perm.offsets).cuda()
    host = torch.zeros_like(rev.host).pin_memory()
    for g, m in enumerate(mats):
        o, n, ld = int(perm.offsets[g]), int(perm.ns[g]), int(perm.lds[g])
        host[o:o + n * ld].view(n, ld)[:, :n] = torch.from_numpy(m)
    perm.pool = host.cuda()
    out = apsp.apsp_batched_host(perm, host, None, chunks=4)
    for g in range(len(mats)):
        o, n, ld = int(perm.offsets[g]), int(perm.ns[g]), int(perm.lds[g])
        got = out[o:o + n * ld].view(n, ld)[:, :n].numpy()
        assert np.array_equal(got, b.graph(g, want).numpy()), f"graph {g}"
    assert apsp.apsp_device_status() == 0


@pytest.mark.parametrize("shape", [(7, 5), (8192, 8192)])
def test_host_alloc_buffers(apsp, shape):
    """apsp_host_alloc / host_empty: page-locked (registered) host memory, small buffers from
    cudaHostAlloc and large ones on huge pages; exact round trips through the device, solve()
    on them, and the free of a pointer the library did not allocate refused."""
    t = apsp.host_empty(shape, torch.int32)
    assert t.is_pinned() and t.shape == shape
    rng = np.random.default_rng(shape[0])
    t.numpy()[:] = rng.integers(0, 1 << 30, shape, dtype=np.int32)
    d = t.to("cuda", non_blocking=True)
    back = apsp.host_empty(shape, torch.int32)
    back.copy_(d, non_blocking=True)
    torch.cuda.synchronize()
    assert np.array_equal(back.numpy(), t.numpy())
    if shape[0] == shape[1] and shape[0] >= 1024:
        h = workloads.er_graph(shape[0], 0.01, "int32", lo=1, hi=100, seed=3)
        t.numpy()[:] = h
        out = apsp.solve(t, out=back)
        d2 = torch.from_numpy(h).cuda()
        apsp.apsp_fw(d2)
        assert np.array_equal(out.numpy(), d2.cpu().numpy())
    x = np.zeros(16, np.int32)
    assert apsp.lib().apsp_host_free(x.ctypes.data) == APSP_ERR_ARG
    assert apsp.lib().apsp_host_free(None) == 0
