"""a8: choosing how to close a graph -- exhaustive autotuning and a learned cost model.

A closure can run as blocked Floyd-Warshall (many launches over all SMs), as R-Kleene with a
leaf cutoff (Sec. 3.3), as repeated (min,+) squaring (Sec. 3.2; a few products when the graph's
diameter is small), or on a single CTA in one launch (the batched kernel on a batch of one);
which is fastest depends on the size, density and type of the graph.  Two planners pick the
configuration from the graph's features (vertex count, edge density, dtype):

* ``Autotuner`` times every candidate on the GPU (median of a few runs) and keeps the fastest.
  Every timing it takes is appended, as one JSON row, to a log.  It is the fallback and the
  judge of the learned model's regret.
* ``CostModel`` is a 2 x 64 ReLU perceptron (fp32) that predicts the log run time of a
  (graph, configuration) pair and chooses the candidate with the smallest prediction.  It is
  trained on the autotuner's logs, on the GPU, by the library's own forward, loss, backward and
  Adam kernels (apsp_mlp_*); nothing here calls a framework optimiser or autograd.

Results do not depend on the choice: every candidate computes the same closure (int32
bit-identical, float32 up to summation order).
"""
from __future__ import annotations

import json
import math
import os
import statistics
import time

import numpy as np
import torch

from . import (apsp_close_cta, apsp_fw, apsp_mlp_adam, apsp_mlp_backward, apsp_mlp_forward, apsp_mlp_loss, apsp_mlp_param_count,
               apsp_rkleene, apsp_rkleene_workspace_bytes, apsp_squaring, apsp_squaring_workspace_bytes, lib)

CANDIDATES = (("fw", 0), ("rkleene", 128), ("rkleene", 256), ("rkleene", 512), ("rkleene", 1024), ("rkleene", 4096),
              ("cta", 0), ("squaring", 0))
CTA_MAX_N = 1024  # beyond this one SM is far too slow to be worth timing
IN_DIM = 12
FW16_MIN_N = 4096  # apsp_fw runs phase 3 on packed 16-bit pairs for int32 graphs this large
HIDDEN = 64
SMS = 152  # streaming multiprocessors of the GB300 the timing log was recorded on


def squaring_products(n: int, density: float, dtype: str = "int32") -> float:
    """About how many (min,+) squarings close a directed Erdos-Renyi graph: t squarings reach
    shortest paths of up to 2^t edges, and one more product confirms that nothing changes.  The
    edge count of the longest shortest path is estimated from the mean degree d = n p.  With
    integer weights uniform in [1, 100] a path can stay on the d / 100 lightest edges of each
    vertex when there are enough of them (about 1.5 ln n / ln(1 + d / 100) edges), and is never
    much longer than the sparse-graph bound 7 ln n / ln d.  With continuous (lognormal) weights
    it is about 1.2 ln n on dense graphs and 1.8 ln n on sparse ones (both measured on these
    generators by Dijkstra's hop counts)."""
    n = max(n, 2)
    deg = max(n * density, 1e-9)
    ln_n = math.log(n)
    if dtype == "int32":
        hops = 7.0 * ln_n / math.log(max(deg, 1.5))
        if deg > 1.0:
            hops = min(hops, 1.5 * ln_n / math.log1p(deg / 100.0))
    else:
        hops = (1.2 if deg >= 50.0 else 1.8) * ln_n
    hops = min(max(hops, 1.0), float(n - 1))
    return math.ceil(math.log2(hops)) + 1.0


def full_product_waves(n: int) -> int:
    """Waves of 128 x 128 output tiles of one full n x n product over the SMs (one tile per SM
    at a time): a product of 13 x 13 tiles takes two waves of work on 152 SMs, 12 x 12 one."""
    t = -(-max(n, 1) // 128)
    return -(-t * t // SMS)


def features(n: int, density: float, dtype: str, algo: str, param: int) -> list[float]:
    """Feature vector of a (graph, configuration) pair, each entry scaled to about [0, 1]."""
    rk = algo == "rkleene"
    sq = algo == "squaring"
    return [math.log2(max(n, 1)) / 15.0, float(density), 1.0 if dtype == "float32" else 0.0,
            1.0 if algo == "fw" else 0.0, 1.0 if rk else 0.0, 1.0 if algo == "cta" else 0.0,
            math.log2(param) / 11.0 if rk else 0.0,
            (math.log2(max(n, 1)) - math.log2(param)) / 8.0 if rk and param else 0.0,
            1.0 if sq else 0.0,
            1.0 if algo == "fw" and dtype == "int32" and n >= FW16_MIN_N else 0.0,
            min(squaring_products(n, density, dtype), 15.0) / 15.0 if sq else 0.0,
            math.log2(full_product_waves(n)) / 8.0]


def applicable(n: int):
    """Candidates worth considering for an n-vertex graph."""
    return [(a, p) for a, p in CANDIDATES
            if not (a == "rkleene" and p >= n) and not (a == "cta" and n > CTA_MAX_N)]


def density_of(h: np.ndarray, inf: int = 0x3FFFFFFF) -> float:
    """Directed edge density m / (n (n - 1)) of a cost matrix (diagonal excluded)."""
    n = h.shape[0]
    if n < 2:
        return 0.0
    edges = np.count_nonzero(h < inf) if h.dtype.kind in "iu" else np.count_nonzero(np.isfinite(h))
    return (edges - n) / float(n * (n - 1))


def run_config(d: torch.Tensor, algo: str, param: int, ws: torch.Tensor | None = None):
    if algo == "fw":
        apsp_fw(d, ws=ws)
    elif algo == "cta":
        apsp_close_cta(d)
    elif algo == "squaring":
        apsp_squaring(d, ws=ws)
    else:
        apsp_rkleene(d, cutoff=param, ws=ws)


def time_config(d0: torch.Tensor, algo: str, param: int, reps: int = 3) -> float:
    """Median milliseconds of one closure of a fresh copy of d0 (CUDA events)."""
    n = d0.shape[0]
    ws = torch.empty(max(256, apsp_rkleene_workspace_bytes(n, n, d0.dtype, param or 256),
                         apsp_squaring_workspace_bytes(n, n, d0.dtype)), dtype=torch.uint8, device=d0.device)
    work = d0.clone()
    run_config(work, algo, param, ws)  # warm-up (first-launch set-up)
    out = []
    for _ in range(reps):
        work.copy_(d0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        run_config(work, algo, param, ws)
        e1.record()
        torch.cuda.synchronize()
        out.append(e0.elapsed_time(e1))
    return statistics.median(out)


class Autotuner:
    """Exhaustive search over CANDIDATES; every measurement is logged as a JSON row."""

    def __init__(self, log_path: str | None = None, reps: int = 3):
        self.log_path = log_path
        self.reps = reps
        self.rows: list[dict] = []

    def measure(self, h: np.ndarray, tag: str = "") -> list[dict]:
        n = h.shape[0]
        dtype = "float32" if h.dtype == np.float32 else "int32"
        dens = density_of(h)
        d0 = torch.from_numpy(h).cuda()
        rows = []
        for algo, param in applicable(n):
            ms = time_config(d0, algo, param, self.reps)
            rows.append({"n": n, "density": round(dens, 6), "dtype": dtype, "algo": algo, "param": param,
                         "ms": round(ms, 5), "tag": tag, "gpu": torch.cuda.get_device_name()})
        self.rows.extend(rows)
        if self.log_path:
            with open(self.log_path, "a") as f:
                for r in rows:
                    f.write(json.dumps(r) + "\n")
        return rows

    def best(self, h: np.ndarray) -> tuple[str, int]:
        rows = self.measure(h)
        r = min(rows, key=lambda r: r["ms"])
        return r["algo"], r["param"]


def load_rows(path: str) -> list[dict]:
    with open(path) as f:
        return [json.loads(line) for line in f if line.strip()]


class CostModel:
    """Perceptron predicting log(ms) of a closure configuration; trained with apsp_mlp_*."""

    def __init__(self, seed: int = 0, device=None):
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.np = apsp_mlp_param_count(IN_DIM)
        rng = np.random.default_rng(seed)  # He initialisation
        W1 = rng.normal(0, math.sqrt(2.0 / IN_DIM), (IN_DIM, HIDDEN))
        W2 = rng.normal(0, math.sqrt(2.0 / HIDDEN), (HIDDEN, HIDDEN))
        w3 = rng.normal(0, math.sqrt(1.0 / HIDDEN), HIDDEN)
        p = np.concatenate([W1.ravel(), np.full(HIDDEN, 0.01), W2.ravel(), np.full(HIDDEN, 0.01), w3, [0.0]])
        assert p.size == self.np
        self.params = torch.tensor(p, dtype=torch.float32, device=self.device)
        self.y_shift = 0.0

    # -- training ------------------------------------------------------------------------
    def fit(self, rows: list[dict], epochs: int = 3000, lr: float = 3e-3) -> list[float]:
        """Full-batch Adam on log(ms); returns the loss every 100 epochs."""
        X = torch.tensor([features(r["n"], r["density"], r["dtype"], r["algo"], r["param"]) for r in rows],
                         dtype=torch.float32, device=self.device)
        y = np.log(np.array([r["ms"] for r in rows], dtype=np.float64))
        self.y_shift = float(y.mean())
        Y = torch.tensor(y - self.y_shift, dtype=torch.float32, device=self.device)
        B = X.shape[0]
        out = torch.empty(B, dtype=torch.float32, device=self.device)
        acts = torch.empty(B * 2 * HIDDEN, dtype=torch.float32, device=self.device)
        dout = torch.empty_like(out)
        loss = torch.zeros(1, dtype=torch.float32, device=self.device)
        grads = torch.zeros_like(self.params)
        m = torch.zeros_like(self.params)
        v = torch.zeros_like(self.params)
        ws = torch.empty(int(lib().apsp_mlp_backward_workspace_bytes(IN_DIM, B)), dtype=torch.uint8, device=self.device)
        hist = []
        for step in range(1, epochs + 1):
            apsp_mlp_forward(self.params, X, out, acts)
            apsp_mlp_loss(out, Y, dout, loss)
            apsp_mlp_backward(self.params, X, acts, dout, grads, ws)
            apsp_mlp_adam(self.params, grads, m, v, lr, step)
            if step % 100 == 0 or step == 1:
                hist.append(float(loss.item()))
        return hist

    # -- inference -----------------------------------------------------------------------
    def predict_ms(self, n: int, density: float, dtype: str) -> dict:
        cands = applicable(n)
        X = torch.tensor([features(n, density, dtype, a, p) for a, p in cands], dtype=torch.float32,
                         device=self.device)
        out = torch.empty(len(cands), dtype=torch.float32, device=self.device)
        apsp_mlp_forward(self.params, X, out)
        pred = np.exp(out.cpu().numpy().astype(np.float64) + self.y_shift)
        return {c: float(t) for c, t in zip(cands, pred)}

    def choose(self, n: int, density: float, dtype: str) -> tuple[str, int]:
        pred = self.predict_ms(n, density, dtype)
        return min(pred, key=pred.get)

    # -- persistence ---------------------------------------------------------------------
    def save(self, path: str):
        with open(path, "w") as f:
            json.dump({"in_dim": IN_DIM, "hidden": HIDDEN, "y_shift": self.y_shift,
                       "params": self.params.cpu().tolist()}, f)

    @classmethod
    def load(cls, path: str, device=None) -> "CostModel":
        with open(path) as f:
            d = json.load(f)
        if d.get("in_dim") != IN_DIM or d.get("hidden") != HIDDEN:
            raise ValueError(f"{path}: a network of {d.get('in_dim')} features x {d.get('hidden')} units, "
                             f"not {IN_DIM} x {HIDDEN}; retrain it with planner.main()")
        m = cls(device=device)
        m.y_shift = d["y_shift"]
        m.params = torch.tensor(d["params"], dtype=torch.float32, device=m.device)
        return m


DEFAULT_MODEL = os.path.join(os.path.dirname(os.path.abspath(__file__)), "cost_model.json")
DEFAULT_LOG = os.path.join(os.path.dirname(os.path.abspath(__file__)), "timings_gb300.jsonl")


def sweep_graphs(seed: int = 0):
    """The autotuning sweep: sizes 32..16384 (log-spaced), both dtypes, sparse and dense, and
    denser int32 graphs (p = 0.6 and 0.8, shortest paths of 4 to 6 edges) between 362 and 2896
    vertices, where a few full-size products of repeated squaring compete with Floyd-Warshall's
    block steps."""
    import workloads
    sizes = sorted({int(round(2 ** e)) for e in np.arange(5.0, 14.01, 0.5)})
    for i, n in enumerate(sizes):
        for dt in ("int32", "float32"):
            for p in ((0.02, 0.4, 0.6, 0.8) if dt == "int32" and 362 <= n <= 2896 else (0.02, 0.4)):
                kw = {"lo": 1, "hi": 100} if dt == "int32" else {"dist": "lognormal", "lo": 0.0, "hi": 1.0}
                yield workloads.er_graph(n, p, dt, seed=seed * 100000 + 10 * n + (p > 0.1) + (p > 0.5) + (p > 0.7), **kw)


def main(log_path: str = DEFAULT_LOG, model_path: str = DEFAULT_MODEL, reps: int = 5):
    """Record a timing log on this GPU with the exhaustive autotuner and fit the cost model."""
    if os.path.exists(log_path):
        os.remove(log_path)
    tuner = Autotuner(log_path=log_path, reps=reps)
    for h in sweep_graphs():
        tuner.measure(h, tag="sweep")
    model = CostModel(seed=0)
    hist = model.fit(load_rows(log_path), epochs=4000)
    model.save(model_path)
    return hist


def default_plan(n: int, density: float, dtype: str) -> tuple[str, int]:
    """The plan without a model: blocked Floyd-Warshall."""
    return ("fw", 0)


def paper_rule(n: int) -> tuple[str, int]:
    """The paper's guidance (Sec. 4): R-Kleene for graphs above 1000 vertices, FW below."""
    return ("rkleene", 256) if n > 1000 else ("fw", 0)
