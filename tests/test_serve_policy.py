"""a9 host logic without a GPU: the arena allocator and the admission/batching policy."""
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
