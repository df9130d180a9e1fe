"""a9 host logic without a GPU: the arena allocator and the admission/batching policy."""
import time

import numpy as np

from paper_2310_03983_gb300.serve import Arena, Request, Scheduler, percentiles


def test_arena_first_fit_coalesces_and_tracks_peak():
    a = Arena(1000, align=10)
    x = a.alloc(95)    # rounds to 100
    y = a.alloc(300)
    z = a.alloc(500)
    assert (x, y, z) == (0, 100, 400)
    assert a.alloc(200) is None
    a.free(y)
    assert a.alloc(250) == 100           # first fit into the hole
    a.free(100)
    a.free(x)
    a.free(z)
    assert a.free_list == [(0, 1000)] and a.used == 0 and a.peak == 900


def test_arena_random_sequence_never_overlaps():
    rng = np.random.default_rng(0)
    a = Arena(1 << 16, align=64)
    live = {}
    for _ in range(3000):
        if live and rng.random() < 0.45:
            off = rng.choice(list(live))
            a.free(off)
            live.pop(off)
        else:
            size = int(rng.integers(1, 5000))
            off = a.alloc(size)
            if off is not None:
                live[off] = -(-size // 64) * 64
        spans = sorted(live.items())
        for (o1, s1), (o2, _) in zip(spans, spans[1:]):
            assert o1 + s1 <= o2
        assert a.used == sum(live.values()) <= a.capacity


def _req(i, n, dtype="int32", t=0.0):
    return Request(rid=i, n=n, dtype=dtype, arrival=t)


def test_admission_lets_small_requests_pass_a_blocked_large_one():
    # room for two 64 x 64 graphs (4096 elements each) plus 512 elements
    s = Scheduler(Arena(2 * 4096 + 512, align=64), small_max=32)
    for i, n in enumerate([64, 64, 64, 64, 16, 16]):
        s.arrive(_req(i, n))
    admitted = [r.rid for r in s.admit(0.0)]
    assert admitted == [0, 1, 4, 5]                    # the 16 x 16 graphs pass the blocked head
    assert [r.rid for r in s.waiting] == [2, 3]        # large ones keep their arrival order
    for r in [r for w in (s.ready_small["int32"], list(s.ready_large)) for r in w]:
        s.release(r)
    assert [r.rid for r in s.admit(1.0)] == [2, 3]


def test_launch_grouping_by_dtype_and_large_first():
    s = Scheduler(Arena(1 << 20), small_max=100)
    for i, (n, dt) in enumerate([(50, "int32"), (60, "float32"), (500, "int32"), (70, "int32")]):
        s.arrive(_req(i, n, dt))
    s.admit(0.0)
    w1 = s.next_launch()
    assert w1[0] == "solo" and w1[1].n == 500
    w2 = s.next_launch()
    assert w2[0] == "batch" and w2[1] == "int32" and [r.n for r in w2[2]] == [50, 70]
    w3 = s.next_launch()
    assert w3[0] == "batch" and w3[1] == "float32"
    assert s.next_launch() is None
    for r in w2[2] + w3[2] + [w1[1]]:
        s.release(r)
    assert s.arena.used == 0


def test_very_large_requests_do_not_share_the_gpu():
    s = Scheduler(Arena(1 << 30), small_max=100, big_n=2048, big_slots=1)
    for i, n in enumerate([4096, 3000, 500, 50]):
        s.arrive(_req(i, n))
    s.admit(0.0)
    w = s.next_launch(big_inflight=0)
    assert w[0] == "solo" and w[1].n == 4096
    w = s.next_launch(big_inflight=1)      # 3000 must wait: the mid-size one goes around it
    assert w[0] == "solo" and w[1].n == 500
    w = s.next_launch(big_inflight=1)
    assert w[0] == "batch" and [r.n for r in w[2]] == [50]
    assert s.next_launch(big_inflight=1) is None
    w = s.next_launch(big_inflight=0)
    assert w[0] == "solo" and w[1].n == 3000


def test_percentiles():
    p = percentiles(list(range(1, 101)))
    assert abs(p["p50"] - 50.5) < 1e-9 and abs(p["p99"] - 99.01) < 1e-9


class _NumpyHostArena:
    """The HostArena interface over plain numpy memory (no GPU needed)."""

    def __init__(self, elems):
        import torch
        self.buf = torch.zeros(elems, dtype=torch.int32)
        self.arena = Arena(elems)

    def view(self, off, n, dtype):
        import torch
        t = self.buf[off:off + n * n].view(n, n)
        return t.view(torch.float32) if dtype == "float32" else t


def test_feeder_makes_every_request_within_the_arena():
    """The feeder makes each request's matrix (in arrival order, on worker threads) into the
    host arena, waits for room when the arena is full, and the matrices are the request's own."""
    import workloads
    from paper_2310_03983_gb300.serve import Feeder, stream_requests
    pool = workloads.RequestPool(seed=1, size_u=1 << 20, size_w=1 << 18, threads=2)
    t = np.linspace(0.0, 0.05, 40)
    ns = np.array([8 + (7 * k) % 90 for k in range(40)])
    ps = np.linspace(0.05, 0.5, 40)
    dts = np.where(np.arange(40) % 2 == 0, "int32", "float32")
    reqs = stream_requests(t, ns, ps, dts)
    host = _NumpyHostArena(4 * 96 * 96)  # room for about four matrices at a time
    make = lambda k, n, p, dt, out: workloads.request_matrix(pool, k, n, p, dt, out=out)  # noqa: E731
    f = Feeder(reqs, host, make, threads=3, lead=None)
    f.start(time.perf_counter())
    seen, peak = 0, 0
    deadline = time.perf_counter() + 60
    while seen < len(reqs) and time.perf_counter() < deadline:
        for r in reqs:
            if r.ready and r.host is not None:
                want = workloads.request_matrix(pool, r.rid, r.n, r.density, r.dtype)
                assert np.array_equal(r.host.numpy(), want), r.rid
                peak = max(peak, host.arena.used)
                f.release(r)
                seen += 1
        time.sleep(0.001)
    f.close()
    assert seen == len(reqs)
    assert host.arena.used == 0 and peak <= host.arena.capacity
    assert all(r.ready for r in reqs)


def test_request_matrix_is_an_er_graph_of_its_own_parameters():
    import workloads
    pool = workloads.RequestPool(seed=2, size_u=1 << 22, size_w=1 << 20, threads=2)
    m = workloads.request_matrix(pool, 5, 600, 0.2, "int32")
    off = ~np.eye(600, dtype=bool)
    e = m[off] < workloads.INF_I32
    assert abs(e.mean() - 0.2) < 0.01 and np.all(np.diagonal(m) == 0)
    assert m[off][e].min() == 1 and m[off][e].max() == 100
    assert np.array_equal(m, workloads.request_matrix(pool, 5, 600, 0.2, "int32"))  # deterministic per k
    assert not np.array_equal(m, workloads.request_matrix(pool, 6, 600, 0.2, "int32"))
    f = workloads.request_matrix(pool, 7, 300, 0.4, "float32")
    ef = np.isfinite(f[~np.eye(300, dtype=bool)])
    assert abs(ef.mean() - 0.4) < 0.02 and np.all(f[~np.eye(300, dtype=bool)][ef] > 0)
    big = np.zeros((50, 64), np.int32)  # in place, with a row stride past n
    workloads.request_matrix(pool, 8, 50, 0.3, "int32", out=big[:, :50])
    assert np.array_equal(big[:, :50], workloads.request_matrix(pool, 8, 50, 0.3, "int32"))
    assert np.all(big[:, 50:] == 0)


def test_recorded_cost_model_matches_the_feature_vector():
    """The trained network shipped with the package takes the planner's current feature vector,
    and the derived features behave as documented."""
    import json

    from paper_2310_03983_gb300 import planner
    with open(planner.DEFAULT_MODEL) as f:
        d = json.load(f)
    assert d["in_dim"] == planner.IN_DIM and d["hidden"] == planner.HIDDEN
    assert len(d["params"]) == planner.IN_DIM * 64 + 64 + 64 * 64 + 64 + 64 + 1
    for n in (32, 1000, 4096, 32768):
        for algo, param in planner.applicable(n):
            assert len(planner.features(n, 0.1, "int32", algo, param)) == planner.IN_DIM
    # 12 x 12 output tiles fill one wave of 152 SMs, 13 x 13 need two
    assert planner.full_product_waves(1536) == 1 and planner.full_product_waves(1537) == 2
    # denser graphs settle in no more squarings than sparser ones of the same size
    for dt in ("int32", "float32"):
        ks = [planner.squaring_products(2048, p, dt) for p in (0.01, 0.05, 0.2, 0.8)]
        assert ks == sorted(ks, reverse=True) and 2 <= ks[-1] <= ks[0] <= 6
