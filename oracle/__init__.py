"""CPU oracle for APSP over the (min,+) semiring.  TEST INFRASTRUCTURE ONLY.

Only the test suite, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg
(``bench.py --impl reference`` and the ``cpu_baseline`` field) may import this package.  The
product library never does, and this package never imports the product library: the two share
nothing but the seeded inputs of ``workloads.py``.

What is here, each citing the passage it follows:
  * ``fw``            -- Eq. 1 (Sec. 2) as the textbook k-i-j triple loop, in C (apsp_oracle.c),
                         int64 for int32 inputs and fp64 for float32 inputs; ``fw_steps`` runs
                         the same loop over a range of intermediate vertices.
  * ``minplus``       -- Eq. 2 (Sec. 3), the (min,+) product, as a triple loop in C.
  * ``minplus_rows``  -- selected rows of the same product, on int32 / float32 operands widened
                         value by value (checks rows of products too large for ``minplus``).
  * ``squaring``      -- the paper's "Floyd-Warshall on GPU" (Sec. 3.2): H <- H (x) H with
                         ``minplus`` until nothing changes (or a given number of products).
  * ``dijkstra_rows`` -- single-source distances from chosen sources by array Dijkstra: an
                         independent algorithm for the same definition, used to check large
                         matrices row by row.
  * ``fw_pred``       -- Eq. 1 with the predecessor indices of Sec. 2 (pred[i, j] becomes
                         pred[k, j] whenever the path through k is shorter).
  * ``last_hop``      -- the predecessor matrix by definition from a closed d and the costs w:
                         the smallest k != j minimising d[i, k] + w[k, j] (the argmin of
                         Sec. 3.1 over the last edge); float32 sums in float32.
  * ``check_predecessors`` -- what any valid predecessor matrix satisfies: -1 exactly on the
                         diagonal and unreachable pairs, a real last edge that is tight
                         (d[i, p] + w[p, j] = d[i, j]), and walks back to the source whose
                         edge costs re-sum to d[i, j] (the path recovery of Sec. 2).
  * ``bellman_ford_rows`` -- single-source distances by Bellman-Ford, valid with negative
                         weights, with negative-cycle detection: the independent check for
                         signed graphs (Sec. 3.1 only excludes negative cycles).
  * ``reachability``  -- the transitive closure by breadth-first search (which pairs are
                         connected at all; needs no arithmetic).
  * ``check_invariants`` -- properties every closed distance matrix has: zero diagonal,
                         d <= w, the triangle inequality d[i,j] <= d[i,k] + d[k,j], idempotence
                         under (min,+) squaring, and the reachability pattern.

Unreachable pairs: int32 matrices use the sentinel ``inf`` (default 0x3FFFFFFF) and every
result >= inf is reported as exactly inf; float32 matrices use +inf.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import tempfile

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "apsp_oracle.c")
_LIB = os.path.join(_HERE, "_oracle.so")
INF_I32 = 0x3FFFFFFF

_lib = None


def build(out: str = _LIB, plant: int = 0, force: bool = False) -> str:
    """Compile apsp_oracle.c into a shared library (OpenMP when the compiler has it)."""
    if not force and plant == 0 and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(_SRC):
        return out
    base = ["gcc", "-O2", "-std=c99", "-shared", "-fPIC", _SRC, "-o", out + ".tmp", "-lm"]
    if plant:
        base.insert(1, f"-DORACLE_PLANT={int(plant)}")
    r = subprocess.run(base[:1] + ["-fopenmp"] + base[1:], capture_output=True, text=True)
    if r.returncode != 0:
        r = subprocess.run(base, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("oracle build failed:\n" + r.stderr)
    os.replace(out + ".tmp", out)
    return out


def _bind(lib):
    i64p = np.ctypeslib.ndpointer(np.int64, flags="C_CONTIGUOUS")
    f64p = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")
    I64, INT = ctypes.c_int64, ctypes.c_int
    lib.oracle_fw_i64.argtypes = [i64p, I64, I64, INT]
    lib.oracle_fw_i64_steps.argtypes = [i64p, I64, I64, I64, I64, INT]
    lib.oracle_fw_f64_steps.argtypes = [f64p, I64, I64, I64, INT]
    lib.oracle_fw_f64.argtypes = [f64p, I64, INT]
    lib.oracle_minplus_i64.argtypes = [i64p, i64p, i64p, I64, I64, I64, I64, INT]
    lib.oracle_minplus_f64.argtypes = [f64p, f64p, f64p, I64, I64, I64, INT]
    lib.oracle_dijkstra_rows_i64.argtypes = [i64p, I64, I64, i64p, I64, i64p, INT]
    lib.oracle_dijkstra_rows_f64.argtypes = [f64p, I64, i64p, I64, f64p, INT]
    f32p = np.ctypeslib.ndpointer(np.float32, flags="C_CONTIGUOUS")
    i32p = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
    lib.oracle_bellman_ford_rows_i64.argtypes = [i64p, I64, I64, i64p, I64, i64p, i32p, INT]
    lib.oracle_bellman_ford_rows_f64.argtypes = [f64p, I64, i64p, I64, f64p, i32p, INT]
    lib.oracle_bellman_ford_rows_i64.restype = None
    lib.oracle_bellman_ford_rows_f64.restype = None
    lib.oracle_fw_pred_i64.argtypes = [i64p, i64p, I64, I64]
    lib.oracle_fw_pred_f64.argtypes = [f64p, i64p, I64]
    lib.oracle_last_hop_i64.argtypes = [i64p, i64p, i64p, I64, i64p, I64, I64, INT]
    lib.oracle_last_hop_f32.argtypes = [f32p, f32p, i64p, I64, i64p, I64, INT]
    for f in ("oracle_fw_pred_i64", "oracle_fw_pred_f64", "oracle_last_hop_i64", "oracle_last_hop_f32"):
        getattr(lib, f).restype = None
    lib.oracle_minplus_rows_i32.argtypes = [i64p, i32p, i32p, I64, I64, i64p, I64, I64, INT, INT]
    lib.oracle_minplus_rows_f32.argtypes = [f64p, f32p, f32p, I64, I64, i64p, I64, INT, INT]
    lib.oracle_minplus_rows_i32.restype = None
    lib.oracle_minplus_rows_f32.restype = None
    lib.oracle_openmp_enabled.restype = INT
    for f in ("oracle_fw_i64", "oracle_fw_f64", "oracle_fw_i64_steps", "oracle_fw_f64_steps", "oracle_minplus_i64", "oracle_minplus_f64",
              "oracle_dijkstra_rows_i64", "oracle_dijkstra_rows_f64"):
        getattr(lib, f).restype = None
    return lib


def load(plant: int = 0):
    """The oracle library; ``plant`` > 0 builds a deliberately broken variant (tests only)."""
    global _lib
    if plant:
        d = tempfile.mkdtemp(prefix="oracle_plant_")
        return _bind(ctypes.CDLL(build(os.path.join(d, f"_oracle_plant{plant}.so"), plant=plant)))
    if _lib is None:
        _lib = _bind(ctypes.CDLL(build()))
    return _lib


def openmp_enabled() -> bool:
    return bool(load().oracle_openmp_enabled())


def _threads(threads):
    return int(threads) if threads else 1


def fw(h: np.ndarray, inf: int = INF_I32, threads: int | None = None, lib=None) -> np.ndarray:
    """All-pairs shortest distances of cost matrix h by Eq. 1 (Sec. 2).

    int32 h -> int32 result (computed in int64, >= inf reported as inf);
    float32/float64 h -> float64 result (computed in fp64, +inf = unreachable).
    """
    lib = lib or load()
    h = np.asarray(h)
    n = h.shape[0]
    assert h.shape == (n, n)
    if h.dtype.kind in "iu":
        d = np.ascontiguousarray(h, dtype=np.int64).copy()
        lib.oracle_fw_i64(d, n, int(inf), _threads(threads))
        return d.astype(np.int32) if h.dtype == np.int32 else d
    d = np.ascontiguousarray(h, dtype=np.float64).copy()
    lib.oracle_fw_f64(d, n, _threads(threads))
    return d


def fw_steps(d: np.ndarray, k0: int, k1: int, inf: int = INF_I32, threads: int | None = None, lib=None):
    """Run the Eq. 1 loop for intermediate vertices k in [k0, k1) in place on a prepared
    matrix (int64 with threshold inf, or float64 with +inf; zero diagonal)."""
    lib = lib or load()
    n = d.shape[0]
    assert d.flags.c_contiguous and d.shape == (n, n)
    if d.dtype == np.int64:
        lib.oracle_fw_i64_steps(d, n, int(inf), int(k0), int(k1), _threads(threads))
    elif d.dtype == np.float64:
        lib.oracle_fw_f64_steps(d, n, int(k0), int(k1), _threads(threads))
    else:
        raise TypeError("fw_steps needs an int64 or float64 matrix")
    return d


def minplus(x: np.ndarray, y: np.ndarray, z: np.ndarray | None = None, inf: int = INF_I32,
            lib=None) -> np.ndarray:
    """(min,+) product of Eq. 2: x (M x K) (x) y (K x N), folded into z when z is given."""
    lib = lib or load()
    M, K = x.shape
    K2, N = y.shape
    assert K == K2
    if x.dtype.kind in "iu":
        X = np.ascontiguousarray(x, dtype=np.int64)
        Y = np.ascontiguousarray(y, dtype=np.int64)
        Z = np.full((M, N), inf, np.int64) if z is None else np.ascontiguousarray(z, dtype=np.int64).copy()
        lib.oracle_minplus_i64(Z, X, Y, M, N, K, int(inf), int(z is not None))
        return Z.astype(np.int32) if x.dtype == np.int32 else Z
    X = np.ascontiguousarray(x, dtype=np.float64)
    Y = np.ascontiguousarray(y, dtype=np.float64)
    Z = np.full((M, N), np.inf) if z is None else np.ascontiguousarray(z, dtype=np.float64).copy()
    lib.oracle_minplus_f64(Z, X, Y, M, N, K, int(z is not None))
    return Z


def minplus_rows(x: np.ndarray, y: np.ndarray, rows, z: np.ndarray | None = None, inf: int = INF_I32,
                 threads: int | None = None, lib=None) -> np.ndarray:
    """Rows ``rows`` of the (min,+) product of Eq. 2, x (M x K) (x) y (K x N), folded into z
    (len(rows) x N) when given.  int32 operands -> int32 result (int64 sums, >= inf reported as
    inf); float32 operands -> float64 result (fp64 sums)."""
    lib = lib or load()
    M, K = x.shape
    K2, N = y.shape
    assert K == K2
    src = np.ascontiguousarray(rows, dtype=np.int64)
    assert src.size == 0 or (src.min() >= 0 and src.max() < M)
    if x.dtype.kind in "iu":
        X = np.ascontiguousarray(x, dtype=np.int32)
        Y = np.ascontiguousarray(y, dtype=np.int32)
        Z = np.empty((len(src), N), np.int64) if z is None else np.ascontiguousarray(z, dtype=np.int64).copy()
        lib.oracle_minplus_rows_i32(Z, X, Y, N, K, src, len(src), int(inf), int(z is not None), _threads(threads))
        return Z.astype(np.int32)
    X = np.ascontiguousarray(x, dtype=np.float32)
    Y = np.ascontiguousarray(y, dtype=np.float32)
    Z = np.empty((len(src), N), np.float64) if z is None else np.ascontiguousarray(z, dtype=np.float64).copy()
    lib.oracle_minplus_rows_f32(Z, X, Y, N, K, src, len(src), int(z is not None), _threads(threads))
    return Z


def squaring(h: np.ndarray, inf: int = INF_I32, max_iters: int | None = None, lib=None):
    """Sec. 3.2: repeat the (min,+) product of Eq. 2 of the matrix with itself until it stops
    changing, or for at most ``max_iters`` products.  Returns (d, number of products that
    changed something).  The diagonal is set to 0 first (a self-loop costs nothing)."""
    h = np.asarray(h)
    isint = h.dtype.kind in "iu"
    d = np.minimum(h.astype(np.int64), inf) if isint else h.astype(np.float64)
    np.fill_diagonal(d, 0)
    changed = 0
    t = 0
    while max_iters is None or t < max_iters:
        nxt = minplus(d, d, inf=inf, lib=lib)
        t += 1
        if np.array_equal(nxt, d):
            break
        d = nxt
        changed += 1
    if isint and h.dtype == np.int32:
        d = d.astype(np.int32)
    return d, changed


def dijkstra_rows(w: np.ndarray, sources, inf: int = INF_I32, threads: int | None = None,
                  lib=None) -> np.ndarray:
    """Distances from each source in ``sources`` (array Dijkstra; weights must be >= 0)."""
    lib = lib or load()
    n = w.shape[0]
    src = np.ascontiguousarray(sources, dtype=np.int64)
    if w.dtype.kind in "iu":
        W = np.ascontiguousarray(w, dtype=np.int64)
        out = np.empty((len(src), n), np.int64)
        lib.oracle_dijkstra_rows_i64(W, n, int(inf), src, len(src), out, _threads(threads))
        return out.astype(np.int32) if w.dtype == np.int32 else out
    W = np.ascontiguousarray(w, dtype=np.float64)
    out = np.empty((len(src), n), np.float64)
    lib.oracle_dijkstra_rows_f64(W, n, src, len(src), out, _threads(threads))
    return out


def fw_pred(h: np.ndarray, inf: int = INF_I32, lib=None):
    """(d, pred) by Eq. 1 with the predecessor indices of Sec. 2 (single thread)."""
    lib = lib or load()
    h = np.asarray(h)
    n = h.shape[0]
    pred = np.empty((n, n), np.int64)
    if h.dtype.kind in "iu":
        d = np.ascontiguousarray(h, dtype=np.int64).copy()
        lib.oracle_fw_pred_i64(d, pred, n, int(inf))
        return (d.astype(np.int32) if h.dtype == np.int32 else d), pred.astype(np.int32)
    d = np.ascontiguousarray(h, dtype=np.float64).copy()
    lib.oracle_fw_pred_f64(d, pred, n)
    return d, pred.astype(np.int32)


def last_hop(d: np.ndarray, w: np.ndarray, inf: int = INF_I32, threads: int | None = None, lib=None,
             rows=None) -> np.ndarray:
    """pred[i, j] = smallest k != j minimising d[i, k] + w[k, j]; -1 on the diagonal and where
    j is unreachable.  Integers: exact (int64), entries >= inf missing.  float32: the sums are
    formed in float32 (d and w are taken as float32), +inf missing.  With ``rows`` only those
    source rows are computed and returned (len(rows) x n); d may then hold just those rows."""
    lib = lib or load()
    n = w.shape[0]
    src = np.arange(n, dtype=np.int64) if rows is None else np.ascontiguousarray(rows, dtype=np.int64)
    if d.shape[0] != len(src):
        d = d[src]
    pred = np.empty((len(src), n), np.int64)
    if w.dtype.kind in "iu":
        D = np.ascontiguousarray(np.minimum(d.astype(np.int64), inf))
        W = np.ascontiguousarray(np.minimum(w.astype(np.int64), inf))
        lib.oracle_last_hop_i64(D, W, pred, n, src, len(src), int(inf), _threads(threads))
    else:
        D = np.ascontiguousarray(d, dtype=np.float32)
        W = np.ascontiguousarray(w, dtype=np.float32)
        lib.oracle_last_hop_f32(D, W, pred, n, src, len(src), _threads(threads))
    return pred.astype(np.int32)


def check_predecessors(pred: np.ndarray, d: np.ndarray, h: np.ndarray, inf: int = INF_I32, rtol: float = 0.0,
                       rows=None) -> list[str]:
    """Violations of the properties every valid predecessor matrix of the closure d of h has.

    For each checked source row i (all rows, or ``rows``): pred[i, i] = -1; pred[i, j] = -1
    exactly where j is unreachable; otherwise p = pred[i, j] is a vertex != j with an edge
    p -> j and d[i, p] + w[p, j] = d[i, j] (within rtol for floats); and walking back from
    every j reaches i within n steps along edges whose costs sum to d[i, j].
    """
    bad = []
    n = h.shape[0]
    isint = h.dtype.kind in "iu"
    W = np.minimum(h.astype(np.int64), inf) if isint else h.astype(np.float64)
    D = d.astype(np.int64) if isint else d.astype(np.float64)
    P = np.asarray(pred).astype(np.int64)
    fin = (lambda a: a < inf) if isint else np.isfinite
    close = (lambda a, b: a == b) if isint else (lambda a, b: np.abs(a - b) <= rtol * np.abs(b))
    for i in (range(n) if rows is None else rows):
        reach = fin(D[i])
        reach[i] = False
        p = P[i]
        if p[i] != -1:
            bad.append(f"pred[{i},{i}] != -1")
        if np.any(p[~reach] != -1):
            bad.append(f"row {i}: unreachable or diagonal entry with a predecessor")
        js = np.nonzero(reach)[0]
        if js.size == 0:
            continue
        pj = p[js]
        if np.any((pj < 0) | (pj >= n) | (pj == js)):
            bad.append(f"row {i}: predecessor out of range or equal to its vertex")
            continue
        wl = W[pj, js]
        if not np.all(fin(wl)):
            bad.append(f"row {i}: predecessor without an edge to its vertex")
            continue
        if not np.all(close(D[i, pj] + wl, D[i, js])):
            bad.append(f"row {i}: last edge not tight (d[i,p] + w[p,j] != d[i,j])")
            continue
        cur, cost = js.copy(), np.zeros(js.size, W.dtype)
        for _ in range(n):
            live = cur != i
            if not live.any():
                break
            prev = P[i, cur[live]]
            cost[live] += W[prev, cur[live]]
            cur[live] = prev
        if np.any(cur != i):
            bad.append(f"row {i}: a predecessor walk does not reach the source")
        elif not np.all(close(cost, D[i, js])):
            bad.append(f"row {i}: a walked path's cost differs from d[i,j]")
    return bad


def bellman_ford_rows(w: np.ndarray, sources, inf: int = INF_I32, threads: int | None = None, lib=None):
    """(distances from each source, negative-cycle flag per source) by Bellman-Ford.  Negative
    weights allowed; int32/int64 -> exact int64 arithmetic, float -> fp64."""
    lib = lib or load()
    n = w.shape[0]
    src = np.ascontiguousarray(sources, dtype=np.int64)
    neg = np.zeros(len(src), np.int32)
    if w.dtype.kind in "iu":
        W = np.ascontiguousarray(np.minimum(w.astype(np.int64), inf))
        out = np.empty((len(src), n), np.int64)
        lib.oracle_bellman_ford_rows_i64(W, n, int(inf), src, len(src), out, neg, _threads(threads))
        return (out.astype(np.int32) if w.dtype == np.int32 else out), neg.astype(bool)
    W = np.ascontiguousarray(w, dtype=np.float64)
    out = np.empty((len(src), n), np.float64)
    lib.oracle_bellman_ford_rows_f64(W, n, src, len(src), out, neg, _threads(threads))
    return out, neg.astype(bool)


def edge_mask(h: np.ndarray, inf: int = INF_I32) -> np.ndarray:
    """Boolean adjacency (i != j and h[i, j] is an edge)."""
    m = (h < inf) if h.dtype.kind in "iu" else np.isfinite(h)
    m = m.copy()
    np.fill_diagonal(m, False)
    return m


def reachability(h: np.ndarray, inf: int = INF_I32) -> np.ndarray:
    """reach[i, j] = True iff j is reachable from i (every i reaches itself): BFS per source."""
    adj = edge_mask(h, inf)
    n = adj.shape[0]
    reach = np.zeros((n, n), dtype=bool)
    nbrs = [np.nonzero(adj[i])[0] for i in range(n)]
    for s in range(n):
        seen = reach[s]
        seen[s] = True
        frontier = [s]
        while frontier:
            nxt = []
            for u in frontier:
                for v in nbrs[u]:
                    if not seen[v]:
                        seen[v] = True
                        nxt.append(v)
            frontier = nxt
    return reach


def check_invariants(d: np.ndarray, h: np.ndarray, inf: int = INF_I32, rtol: float = 0.0,
                     sample_k: int | None = None, seed: int = 0) -> list[str]:
    """Return the list of violated properties of a claimed closure d of cost matrix h.

    rtol = 0 demands exact relations (integers); floats allow rtol relative slack.
    The triangle inequality is checked for every k, or for ``sample_k`` random k.
    """
    bad = []
    n = h.shape[0]
    if n == 0:
        return bad
    isint = h.dtype.kind in "iu"
    D = d.astype(np.int64) if isint else d.astype(np.float64)
    H = h.astype(np.int64) if isint else h.astype(np.float64)
    if isint:
        H = np.minimum(H, inf)
    if np.any(np.diagonal(D) != 0):
        bad.append("diagonal not zero")
    Hn = H.copy()
    np.fill_diagonal(Hn, 0)
    slack = (lambda a: a * (1 + rtol)) if not isint else (lambda a: a)
    fin = Hn < inf if isint else np.isfinite(Hn)
    if np.any(D[fin] > slack(Hn[fin])):
        bad.append("d > w on some edge")
    ks = range(n) if sample_k is None else np.random.default_rng(seed).choice(n, size=min(n, sample_k), replace=False)
    for k in ks:
        via = D[:, k:k + 1] + D[k:k + 1, :]
        if isint:
            via = np.minimum(via, inf)
        if np.any(D > slack(via)):
            bad.append(f"triangle inequality fails through k={int(k)}")
            break
    reach = reachability(h, inf)
    got = D < inf if isint else np.isfinite(D)
    if not np.array_equal(reach, got):
        bad.append("reachability pattern differs from BFS closure")
    return bad
