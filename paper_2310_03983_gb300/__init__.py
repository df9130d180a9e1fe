"""Python binding of libapsp.so: all-pairs shortest paths over the (min,+) semiring on GB300.

Thin ctypes wrappers with the same names as the C ABI (include/apsp.h).  They only marshal
arguments: torch CUDA tensors become device pointers, leading dimensions and the current
stream; every step of the computation runs in the library's CUDA kernels.  There is no CPU
fallback: if libapsp.so is missing this module raises on import.

    d = torch.from_numpy(h).cuda()          # n x n int32 or float32 cost matrix
    apsp_fw(d)                               # closed in place: shortest distances
    apsp_rkleene(d, cutoff=256)              # same result by R-Kleene (Sec. 3.3)
    tropical_gemm(C, A, B)                   # C = A (x) B, Eq. 2
"""
from __future__ import annotations

import ctypes
import os
import weakref

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libapsp.so")

APSP_I32, APSP_F32 = 0, 1
APSP_INF_I32 = 0x3FFFFFFF
STATUS = {0: "ok", 1: "invalid argument", 2: "negative weight, NaN or out-of-range entry", 3: "out of memory",
          4: "CUDA error", 5: "device wait timed out", 6: "unsupported", 7: "negative cycle"}


class ApspError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"{what}: {STATUS.get(code, code)} (status {code})")
        self.code = code


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libapsp.so not built at {LIB_PATH}; run __graft_entry__.build() "
                          "(python -m paper_2310_03983_gb300.build)")
    lib = ctypes.CDLL(LIB_PATH)
    vp, i64, i32, sz = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_size_t
    sigs = {
        "apsp_version": ([], i32),
        "apsp_workspace_pool_trim": ([], i32),
        "apsp_status_str": ([i32], ctypes.c_char_p),
        "apsp_device_status": ([vp, ctypes.POINTER(i32)], i32),
        "apsp_normalise": ([vp, i64, i64, i32, vp, vp], i32),
        "tropical_gemm_workspace_bytes": ([i64, i64, i64, i32], sz),
        "tropical_gemm": ([vp, vp, vp, i64, i64, i64, i64, i64, i64, i32, vp, i32, vp, sz, vp], i32),
        "apsp_fw_workspace_bytes": ([i64, i64, i32, i32], sz),
        "apsp_fw": ([vp, i64, i64, i32, vp, i32, vp, sz, vp], i32),
        "apsp_rkleene_workspace_bytes": ([i64, i64, i32, i32], sz),
        "apsp_rkleene": ([vp, i64, i64, i32, vp, i32, vp, sz, vp], i32),
        "apsp_probe_minplus": ([i32, i32, i32, i32, vp, vp], i32),
        "apsp_fw_signed_workspace_bytes": ([i64, i64, i32], sz),
        "apsp_fw_signed": ([vp, i64, i64, i32, vp, vp, sz, vp], i32),
        "apsp_squaring_workspace_bytes": ([i64, i64, i32], sz),
        "apsp_squaring": ([vp, i64, i64, i32, vp, i32, vp, sz, vp], i32),
        "apsp_predecessors_workspace_bytes": ([i64, i32], sz),
        "apsp_predecessors": ([vp, i64, vp, i64, vp, i64, i64, i32, vp, vp, sz, vp], i32),
        "apsp_batched_workspace_bytes": ([i64], sz),
        "apsp_batched_staged_workspace_bytes": ([vp, i64, i32], sz),
        "apsp_solve_host": ([vp, vp, i64, i64, i32, i32, i32, vp, vp, i64, vp, sz, vp], i32),
        "apsp_batched_host_workspace_bytes": ([vp, vp, vp, i64, i32, i32], sz),
        "apsp_batched_host": ([vp, vp, vp, vp, vp, vp, vp, vp, vp, i64, i32, vp, i32, vp, sz, vp], i32),
        "apsp_batched": ([vp, vp, vp, vp, vp, vp, i64, i32, vp, vp, sz, vp], i32),
        "apsp_mlp_param_count": ([i32], i64),
        "apsp_mlp_backward_workspace_bytes": ([i32, i32], sz),
        "apsp_mlp_forward": ([vp, i32, vp, i32, vp, vp, vp], i32),
        "apsp_mlp_loss": ([vp, vp, i32, vp, vp, vp], i32),
        "apsp_mlp_backward": ([vp, i32, vp, vp, vp, i32, vp, vp, sz, vp], i32),
        "apsp_mlp_adam": ([vp, vp, vp, vp, i64, ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_float, i32,
                           vp], i32),
        "apsp_host_alloc": ([sz], vp),
        "apsp_host_free": ([vp], i32),
        "apsp_trace_enable": ([i32], i32),
        "apsp_launch_count": ([i32], i64),
        "apsp_trace_read": ([i32, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(i64),
                             ctypes.POINTER(ctypes.c_double)], i32),
    }
    for name, (args, res) in sigs.items():
        f = getattr(lib, name)
        f.argtypes, f.restype = args, res
    return lib


_lib = _load()
EXPORTS = ("apsp_version", "apsp_workspace_pool_trim", "apsp_status_str", "apsp_device_status", "apsp_normalise",
           "tropical_gemm_workspace_bytes", "tropical_gemm",
           "apsp_fw_workspace_bytes", "apsp_fw", "apsp_rkleene_workspace_bytes", "apsp_rkleene",
           "apsp_fw_signed_workspace_bytes", "apsp_fw_signed", "apsp_squaring_workspace_bytes", "apsp_squaring", "apsp_predecessors_workspace_bytes", "apsp_predecessors",
           "apsp_probe_minplus", "apsp_trace_enable", "apsp_trace_read", "apsp_launch_count",
           "apsp_batched_workspace_bytes", "apsp_batched_staged_workspace_bytes", "apsp_solve_host",
           "apsp_batched_host_workspace_bytes", "apsp_batched_host", "apsp_host_alloc", "apsp_host_free",
           "apsp_batched", "apsp_mlp_param_count", "apsp_mlp_backward_workspace_bytes", "apsp_mlp_forward",
           "apsp_mlp_loss", "apsp_mlp_backward", "apsp_mlp_adam")


def lib():
    return _lib


def _check(code: int, what: str):
    if code != 0:
        raise ApspError(code, what)


def _dtype_code(t: torch.Tensor) -> int:
    if t.dtype == torch.int32:
        return APSP_I32
    if t.dtype == torch.float32:
        return APSP_F32
    raise TypeError(f"dtype must be int32 or float32, got {t.dtype}")


def _mat(t: torch.Tensor, name: str):
    if not t.is_cuda or t.dim() != 2 or (t.numel() > 0 and t.stride(1) != 1):
        raise ValueError(f"{name} must be a 2-D CUDA tensor with unit column stride")
    return t.data_ptr(), t.stride(0) if t.shape[0] > 1 else max(t.shape[1], 1)


def _stream(stream) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream if hasattr(s, "cuda_stream") else int(s)


def _inf_arg(inf, code):
    if inf is None:
        return None, None
    box = ctypes.c_int32(int(inf)) if code == APSP_I32 else ctypes.c_float(float(inf))
    return ctypes.cast(ctypes.pointer(box), ctypes.c_void_p), box


def apsp_version() -> int:
    return _lib.apsp_version()


def apsp_workspace_pool_trim():
    """Release the memory the library's workspace pool keeps for the current device."""
    _check(_lib.apsp_workspace_pool_trim(), "apsp_workspace_pool_trim")


def apsp_device_status(stream=None) -> int:
    """Synchronise the stream, read and clear the device's sticky data-status word."""
    out = ctypes.c_int32(0)
    _check(_lib.apsp_device_status(_stream(stream), ctypes.byref(out)), "apsp_device_status")
    return out.value


def apsp_normalise(d: torch.Tensor, inf=None, stream=None):
    p, ld = _mat(d, "d")
    code = _dtype_code(d)
    ip, _keep = _inf_arg(inf, code)
    _check(_lib.apsp_normalise(p, d.shape[0], ld, code, ip, _stream(stream)), "apsp_normalise")
    return d


def tropical_gemm_workspace_bytes(M: int, N: int, K: int, dtype=torch.int32) -> int:
    return _lib.tropical_gemm_workspace_bytes(M, N, K, APSP_I32 if dtype == torch.int32 else APSP_F32)


def tropical_gemm(C: torch.Tensor, A: torch.Tensor, B: torch.Tensor, accumulate: bool = False, inf=None,
                  ws: torch.Tensor | None = None, stream=None):
    """C = A (x) B, or C = min(C, A (x) B) when accumulate (Eq. 2)."""
    M, K = A.shape
    K2, N = B.shape
    if K != K2 or tuple(C.shape) != (M, N):
        raise ValueError("shape mismatch")
    code = _dtype_code(C)
    if A.dtype != C.dtype or B.dtype != C.dtype:
        raise TypeError("A, B and C must share a dtype")
    pc, ldc = _mat(C, "C")
    pa, lda = _mat(A, "A")
    pb, ldb = _mat(B, "B")
    ip, _keep = _inf_arg(inf, code)
    wp, wb = (None, 0) if ws is None else (ws.data_ptr(), ws.numel() * ws.element_size())
    _check(_lib.tropical_gemm(pc, pa, pb, M, N, K, lda, ldb, ldc, code, ip, int(bool(accumulate)), wp, wb,
                              _stream(stream)), "tropical_gemm")
    return C


def _closure(fn, wsfn, d, inf, param, ws, stream, what):
    n = d.shape[0]
    if d.shape[1] != n:
        raise ValueError("d must be square")
    p, ld = _mat(d, "d")
    code = _dtype_code(d)
    ip, _keep = _inf_arg(inf, code)
    if ws is None:
        wp, wb = None, 0
    else:
        wp, wb = ws.data_ptr(), ws.numel() * ws.element_size()
    _check(fn(p, n, ld, code, ip, int(param), wp, wb, _stream(stream)), what)
    return d


def apsp_fw_workspace_bytes(n: int, ld: int, dtype=torch.int32, tile: int = 0) -> int:
    return _lib.apsp_fw_workspace_bytes(n, ld, APSP_I32 if dtype == torch.int32 else APSP_F32, tile)


def apsp_rkleene_workspace_bytes(n: int, ld: int, dtype=torch.int32, cutoff: int = 0) -> int:
    return _lib.apsp_rkleene_workspace_bytes(n, ld, APSP_I32 if dtype == torch.int32 else APSP_F32, cutoff)


def apsp_fw(d: torch.Tensor, inf=None, tile: int = 0, ws: torch.Tensor | None = None, stream=None):
    """Close d in place by blocked Floyd-Warshall (Eq. 1 over 128 x 128 tiles)."""
    return _closure(_lib.apsp_fw, _lib.apsp_fw_workspace_bytes, d, inf, tile, ws, stream, "apsp_fw")


def apsp_rkleene(d: torch.Tensor, inf=None, cutoff: int = 0, ws: torch.Tensor | None = None, stream=None):
    """Close d in place by R-Kleene (Sec. 3.3) with blocked-FW leaves of <= cutoff vertices."""
    return _closure(_lib.apsp_rkleene, _lib.apsp_rkleene_workspace_bytes, d, inf, cutoff, ws, stream,
                    "apsp_rkleene")


def apsp_fw_signed(d: torch.Tensor, inf=None, ws: torch.Tensor | None = None, stream=None):
    """Close d in place by blocked Floyd-Warshall when finite entries may be negative (no
    negative cycle, Sec. 3.1); a negative cycle is reported by apsp_device_status() as 7."""
    n = d.shape[0]
    if d.shape[1] != n:
        raise ValueError("d must be square")
    p, ld = _mat(d, "d")
    code = _dtype_code(d)
    ip, _keep = _inf_arg(inf, code)
    wp, wb = (None, 0) if ws is None else (ws.data_ptr(), ws.numel() * ws.element_size())
    _check(_lib.apsp_fw_signed(p, n, ld, code, ip, wp, wb, _stream(stream)), "apsp_fw_signed")
    return d


def apsp_squaring_workspace_bytes(n: int, ld: int, dtype=torch.int32) -> int:
    return _lib.apsp_squaring_workspace_bytes(n, ld, APSP_I32 if dtype == torch.int32 else APSP_F32)


def apsp_squaring(d: torch.Tensor, inf=None, max_iters: int = 0, ws: torch.Tensor | None = None, stream=None):
    """Close d in place by repeated (min,+) squaring until nothing changes (Sec. 3.2);
    max_iters > 0 caps the number of products."""
    return _closure(_lib.apsp_squaring, None, d, inf, max_iters, ws, stream, "apsp_squaring")


def apsp_predecessors_workspace_bytes(n: int, dtype=torch.int32) -> int:
    return _lib.apsp_predecessors_workspace_bytes(n, APSP_I32 if dtype == torch.int32 else APSP_F32)


def apsp_predecessors(d: torch.Tensor, w: torch.Tensor, pred: torch.Tensor | None = None, inf=None,
                      ws: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """pred[i][j] = the vertex before j on a shortest i -> j path (-1 on the diagonal and for
    unreachable pairs), from the closed matrix d and the cost matrix w it was closed from."""
    n = d.shape[0]
    if tuple(d.shape) != (n, n) or tuple(w.shape) != (n, n):
        raise ValueError("d and w must be n x n")
    if w.dtype != d.dtype:
        raise TypeError("d and w must share a dtype")
    code = _dtype_code(d)
    if pred is None:
        pred = torch.empty((n, n), dtype=torch.int32, device=d.device)
    if pred.dtype != torch.int32 or tuple(pred.shape) != (n, n):
        raise ValueError("pred must be an n x n int32 tensor")
    pd, ldd = _mat(d, "d")
    pw, ldw = _mat(w, "w")
    pp, ldp = _mat(pred, "pred")
    ip, _keep = _inf_arg(inf, code)
    wp, wb = (None, 0) if ws is None else (ws.data_ptr(), ws.numel() * ws.element_size())
    _check(_lib.apsp_predecessors(pd, ldd, pw, ldw, pp, ldp, n, code, ip, wp, wb, _stream(stream)),
           "apsp_predecessors")
    return pred


def path(pred, i: int, j: int) -> list[int] | None:
    """Vertices of the shortest i -> j path spelled out by a predecessor matrix (host array or
    CPU tensor), or None when j is unreachable from i.  Raises if the walk does not reach i
    within n steps (possible only with zero-cost cycles)."""
    pred = np.asarray(pred)
    n = pred.shape[0]
    if i == j:
        return [i]
    if pred[i, j] < 0:
        return None
    out = [j]
    v = j
    for _ in range(n):
        v = int(pred[i, v])
        if v < 0:
            raise ValueError(f"broken predecessor chain {i} -> {j}")
        out.append(v)
        if v == i:
            return out[::-1]
    raise ValueError(f"predecessor walk {i} -> {j} did not reach {i} in {n} steps")


def apsp_probe_minplus(variant: int, blocks: int, threads: int, iters: int, sink: torch.Tensor, stream=None):
    _check(_lib.apsp_probe_minplus(variant, blocks, threads, iters, sink.data_ptr(), _stream(stream)),
           "apsp_probe_minplus")


def apsp_trace_enable(on: bool = True):
    _check(_lib.apsp_trace_enable(int(bool(on))), "apsp_trace_enable")


def apsp_trace_read(mode: int = -1):
    """(total_ms, launches, pairs) of traced engine launches of `mode` since the last read."""
    ms, n, pairs = ctypes.c_double(), ctypes.c_int64(), ctypes.c_double()
    _check(_lib.apsp_trace_read(mode, ctypes.byref(ms), ctypes.byref(n), ctypes.byref(pairs)), "apsp_trace_read")
    return ms.value, n.value, pairs.value


def apsp_launch_count(reset: bool = False) -> int:
    """Kernel launches the library has enqueued in this process; reset=True also zeroes it."""
    return int(_lib.apsp_launch_count(int(bool(reset))))


class Batch:
    """A batch of graphs packed into one device pool, in the layout apsp_batched expects:
    graph g at element offset offsets[g], leading dimension round_up(n_g, 4)."""

    def __init__(self, mats, device=None, pin=True, staged=True):
        dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        mats = [np.asarray(m) for m in mats]
        if not mats:
            raise ValueError("empty batch")
        dt = mats[0].dtype
        if any(m.dtype != dt for m in mats) or dt not in (np.int32, np.float32):
            raise TypeError("all graphs must share one dtype, int32 or float32")
        self.ns = np.array([m.shape[0] for m in mats], np.int32)
        self.lds = ((self.ns + 3) // 4 * 4).astype(np.int32)
        sizes = self.ns.astype(np.int64) * self.lds
        self.offsets = np.concatenate([[0], np.cumsum(sizes)[:-1]]).astype(np.int64)
        total = int(sizes.sum())
        host = np.zeros(max(total, 4), dtype=dt)
        for m, o, n, ld in zip(mats, self.offsets, self.ns, self.lds):
            host[o:o + n * ld].reshape(n, ld)[:, :n] = m
        if pin:  # page-locked (huge pages when large) for full-rate copies
            self.host = host_empty(host.shape, torch.int32 if dt == np.int32 else torch.float32)
            self.host.numpy()[:] = host
        else:
            self.host = torch.from_numpy(host)
        self.dtype = self.host.dtype
        self.pool = self.host.to(dev, non_blocking=True)
        self.d_offsets = torch.from_numpy(self.offsets).to(dev)
        self.d_ns = torch.from_numpy(self.ns).to(dev)
        self.d_lds = torch.from_numpy(self.lds).to(dev)
        self.order = np.argsort(-self.ns, kind="stable").astype(np.int32)  # largest first
        self.d_order = torch.from_numpy(self.order).to(dev)
        # staged: room for closing the larger int32 graphs in lockstep on the GEMM engine
        wsb = (apsp_batched_staged_workspace_bytes(self.ns, self.dtype) if staged
               else _lib.apsp_batched_workspace_bytes(len(mats)))
        self.ws = torch.empty(wsb, dtype=torch.uint8, device=dev)

    def __len__(self):
        return len(self.ns)

    def graph(self, g, src=None):
        """Graph g of a pool (the device pool by default) as an n x n view."""
        src = self.pool if src is None else src
        o, n, ld = int(self.offsets[g]), int(self.ns[g]), int(self.lds[g])
        return src[o:o + n * ld].view(n, ld)[:, :n]


class _OneGraph:
    """Device descriptor arrays of a batch holding one graph (offset 0), cached by shape."""
    _cache: dict = {}

    @classmethod
    def get(cls, n: int, ld: int, dev):
        key = (n, ld, str(dev))
        if key not in cls._cache:
            cls._cache[key] = (torch.zeros(1, dtype=torch.int64, device=dev),
                               torch.tensor([n], dtype=torch.int32, device=dev),
                               torch.tensor([ld], dtype=torch.int32, device=dev),
                               torch.empty(_lib.apsp_batched_workspace_bytes(1), dtype=torch.uint8, device=dev))
        return cls._cache[key]


def apsp_batched_staged_workspace_bytes(ns_host, dtype=torch.int32) -> int:
    """Workspace bytes with which apsp_batched runs the larger int32 graphs in lockstep."""
    ns = np.ascontiguousarray(ns_host, dtype=np.int32)
    code = APSP_I32 if dtype == torch.int32 else APSP_F32
    return int(_lib.apsp_batched_staged_workspace_bytes(ns.ctypes.data_as(ctypes.c_void_p), len(ns), code))


def apsp_close_cta(d: torch.Tensor, inf=None, stream=None):
    """Close one graph with a single CTA (apsp_batched on a batch of one): one launch, no
    inter-CTA phases -- the cheapest plan for small graphs."""
    n = d.shape[0]
    p, ld = _mat(d, "d")
    if d.shape[1] != n:
        raise ValueError("d must be square")
    if n <= 1:
        ld = 4  # a single row: the leading dimension is never used to address memory
    elif ld % 4 != 0:
        return apsp_fw(d, inf=inf, stream=stream)  # the single-CTA kernel needs 16-byte rows
    off, ns, lds, ws = _OneGraph.get(n, ld, d.device)
    code = _dtype_code(d)
    ip, _keep = _inf_arg(inf, code)
    nh = (ctypes.c_int32 * 1)(n)
    _check(_lib.apsp_batched(p, off.data_ptr(), ns.data_ptr(), lds.data_ptr(), None, nh, 1, code, ip, ws.data_ptr(),
                             ws.numel(), _stream(stream)), "apsp_batched")
    return d


def apsp_batched_raw(pool, d_offsets, d_ns, d_lds, d_order, count: int, ws, inf=None, stream=None, ns_host=None):
    """apsp_batched on caller-built device descriptor arrays (int64 offsets, int32 ns, lds and
    order) over `pool` (a 1-D int32 or float32 CUDA tensor); ns_host: optional numpy copy of ns."""
    code = _dtype_code(pool)
    ip, _keep = _inf_arg(inf, code)
    nh = None if ns_host is None else np.ascontiguousarray(ns_host, dtype=np.int32)
    _check(_lib.apsp_batched(pool.data_ptr(), d_offsets.data_ptr(), d_ns.data_ptr(), d_lds.data_ptr(),
                             None if d_order is None else d_order.data_ptr(),
                             None if nh is None else nh.ctypes.data_as(ctypes.c_void_p), count, code, ip,
                             ws.data_ptr(), ws.numel() * ws.element_size(), _stream(stream)), "apsp_batched")


def apsp_batched(batch: Batch, inf=None, stream=None, pool=None):
    """Close every graph of `batch` (its device pool, or `pool`) in one persistent launch."""
    code = _dtype_code(batch.pool)
    ip, _keep = _inf_arg(inf, code)
    p = batch.pool if pool is None else pool
    _check(_lib.apsp_batched(p.data_ptr(), batch.d_offsets.data_ptr(), batch.d_ns.data_ptr(),
                             batch.d_lds.data_ptr(), batch.d_order.data_ptr(),
                             batch.ns.ctypes.data_as(ctypes.c_void_p), len(batch), code, ip,
                             batch.ws.data_ptr(), batch.ws.numel(), _stream(stream)), "apsp_batched")
    return batch


def apsp_batched_host(batch: Batch, host_in=None, host_out=None, chunks: int = 4, inf=None, stream=None):
    """Close a batch given in HOST memory, laid out like batch.host (the default input): the
    batch is copied to the device pool chunk by chunk, each chunk closed while the next is
    copied in and the previous copied out (apsp_batched_host).  Returns the host result
    (host_out, or a new pinned tensor); the call returns once it is written."""
    src = batch.host if host_in is None else host_in
    if src.is_cuda or src.numel() < batch.pool.numel() or not src.is_contiguous():
        raise ValueError("host_in must be a contiguous CPU tensor laid out like batch.host")
    out = host_empty(tuple(src.shape), src.dtype) if host_out is None else host_out
    if out.is_cuda or out.numel() < batch.pool.numel() or not out.is_contiguous():
        raise ValueError("host_out must be a contiguous CPU tensor laid out like batch.host")
    code = _dtype_code(batch.pool)
    ip, _keep = _inf_arg(inf, code)
    vpp = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    _check(_lib.apsp_batched_host(src.data_ptr(), out.data_ptr(), batch.pool.data_ptr(), vpp(batch.offsets),
                                  vpp(batch.ns), vpp(batch.lds), batch.d_offsets.data_ptr(), batch.d_ns.data_ptr(),
                                  batch.d_lds.data_ptr(), len(batch), code, ip, chunks, batch.ws.data_ptr(),
                                  batch.ws.numel(), _stream(stream)), "apsp_batched_host")
    return out


def _fptr(t):
    if t is None:
        return None
    if not t.is_cuda or t.dtype != torch.float32 or not t.is_contiguous():
        raise ValueError("expected a contiguous float32 CUDA tensor")
    return t.data_ptr()


def apsp_mlp_param_count(in_dim: int) -> int:
    return int(_lib.apsp_mlp_param_count(in_dim))


def apsp_mlp_forward(params, x, out, acts=None, stream=None):
    batch, in_dim = x.shape
    _check(_lib.apsp_mlp_forward(_fptr(params), in_dim, _fptr(x), batch, _fptr(out), _fptr(acts), _stream(stream)),
           "apsp_mlp_forward")
    return out


def apsp_mlp_loss(out, y, dout, loss=None, stream=None):
    _check(_lib.apsp_mlp_loss(_fptr(out), _fptr(y), out.numel(), _fptr(dout), _fptr(loss), _stream(stream)),
           "apsp_mlp_loss")
    return dout


def apsp_mlp_backward(params, x, acts, dout, grads, ws=None, stream=None):
    batch, in_dim = x.shape
    need = _lib.apsp_mlp_backward_workspace_bytes(in_dim, batch)
    if ws is None or ws.numel() * ws.element_size() < need:
        raise ValueError(f"backward needs a workspace of {need} bytes")
    _check(_lib.apsp_mlp_backward(_fptr(params), in_dim, _fptr(x), _fptr(acts), _fptr(dout), batch, _fptr(grads),
                                  ws.data_ptr(), ws.numel() * ws.element_size(), _stream(stream)),
           "apsp_mlp_backward")
    return grads


def apsp_mlp_adam(params, grads, m, v, lr, step, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
    _check(_lib.apsp_mlp_adam(_fptr(params), _fptr(grads), _fptr(m), _fptr(v), params.numel(), lr, beta1, beta2, eps,
                              step, _stream(stream)), "apsp_mlp_adam")


ALGOS = {"fw": apsp_fw, "rkleene": apsp_rkleene, "squaring": apsp_squaring}


_NP_OF = {torch.int32: np.int32, torch.float32: np.float32, torch.int64: np.int64, torch.uint8: np.uint8}


def host_empty(shape, dtype=torch.int32) -> torch.Tensor:
    """A page-locked host tensor from apsp_host_alloc (huge pages for large buffers, which keep
    host-device copies at full rate after large closures); freed when the last tensor or array
    viewing it is garbage-collected."""
    npdt = np.dtype(_NP_OF[dtype])
    shape = tuple(int(x) for x in (shape if isinstance(shape, (tuple, list)) else (shape,)))
    count = int(np.prod(shape)) if shape else 1
    nbytes = max(1, count * npdt.itemsize)
    p = _lib.apsp_host_alloc(nbytes)
    if not p:
        raise MemoryError(f"apsp_host_alloc({nbytes}) failed")
    arr = np.frombuffer((ctypes.c_byte * nbytes).from_address(p), dtype=npdt, count=count).reshape(shape)
    weakref.finalize(arr, _lib.apsp_host_free, p)
    return torch.from_numpy(arr)


def solve(h, algo: str = "fw", inf=None, param: int = 0, device=None, out=None, predecessors: bool = False):
    """End-to-end solve of a HOST cost matrix (numpy array or CPU tensor): copy it to the
    device, close it there, copy the distances back.  Returns a CPU tensor (``out`` if given,
    pinned memory recommended); with predecessors=True, a pair (distances, pred) where pred is
    the int32 predecessor matrix of apsp_predecessors (walk it with ``path``)."""
    algos = {"fw": 0, "rkleene": 1, "squaring": 2}
    if algo not in algos:
        raise ValueError(f"unknown algorithm {algo!r}")
    t = torch.as_tensor(h)
    if t.is_cuda or t.dim() != 2 or t.shape[0] != t.shape[1]:
        raise ValueError("h must be a square host matrix")
    dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
    if predecessors:  # the weights stay on the device for the predecessor pass
        d = t.to(dev, non_blocking=True)
        w = d.clone()
        {"fw": lambda: apsp_fw(d, inf=inf, tile=param), "rkleene": lambda: apsp_rkleene(d, inf=inf, cutoff=param),
         "squaring": lambda: apsp_squaring(d, inf=inf, max_iters=param)}[algo]()
        pred = apsp_predecessors(d, w, inf=inf).cpu()
        out = d.cpu() if out is None else out.copy_(d)
        return out, pred
    t = t.contiguous()
    n = t.shape[0]
    code = _dtype_code(t)
    if out is None:
        out = host_empty(tuple(t.shape), t.dtype)
    elif out.is_cuda or out.dtype != t.dtype or tuple(out.shape) != (n, n) or not out.is_contiguous():
        raise ValueError("out must be a contiguous host tensor of h's shape and dtype")
    ip, _keep = _inf_arg(inf, code)
    with torch.cuda.device(dev):
        _check(_lib.apsp_solve_host(t.data_ptr(), out.data_ptr(), n, max(n, 1), code, algos[algo], param, ip, None,
                                    0, None, 0, _stream(None)), "apsp_solve_host")
    return out
