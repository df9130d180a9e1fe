"""The argument behind the 16-bit paths, checked on the CPU with small caps.

The int32 closures run Eq. 1 partly in the (min,+) semiring truncated at a cap C (values at or
above C all mean "at least C"): truncation t(v) = min(v, C) satisfies t(min(a, b)) =
min(t(a), t(b)) and t(a + b) = t(t(a) + t(b)) for a, b >= 0, so a closure that mixes exact and
truncated relaxations keeps t(stored) = t(exact distance) for every entry.  The library then
certifies the result: if (largest stored value below C) + (largest weight) < C, every entry at
or above C is unreachable and becomes the sentinel, giving the exact closure; otherwise the
same mapping leaves a matrix between the distances and the weights (every weight is below C),
and an exact closure of it is the exact answer.

Here a plain numpy Floyd-Warshall chooses, for every (k, i, j) relaxation at random, one of
the three forms the closures use: exact, min(d, a + b); truncated with the old entry kept,
min(d, min(C, t(a) + t(b))) (the 16-bit phase 3, which folds into the exact old entry); and
fully truncated, min(t(d), t(a) + t(b)) capped (the 16-bit panel products and diagonal
closures, whose operands and results are all capped).  The three claims are checked against
the oracle on hundreds of small graphs, including paths whose lengths straddle the cap.  None
of this touches the GPU code.
"""
import numpy as np

import oracle

INF = oracle.INF_I32


def _mixed_fw(h, cap, rng):
    d = h.astype(np.int64)
    n = d.shape[0]
    t = lambda v: np.minimum(v, cap)
    for k in range(n):
        a = d[:, k][:, None]
        b = d[k, :][None, :]
        exact = np.minimum(d, a + b)
        keep_old = np.minimum(d, np.minimum(cap, t(a) + t(b)))
        capped = np.minimum(t(d), np.minimum(cap, t(a) + t(b)))
        pick = rng.integers(0, 3, d.shape)
        d = np.where(pick == 0, exact, np.where(pick == 1, keep_old, capped))
        d = np.minimum(d, INF)  # int32 storage saturates at the sentinel
    return d


def _certify(d, cap, wmax):
    below = d[d < cap]
    largest = int(below.max()) if below.size else 0
    mapped = np.where(d >= cap, INF, d)
    return largest + wmax < cap, mapped


def _graphs(rng):
    for trial in range(600):
        cap = int(rng.choice([20, 64, 200]))
        n = int(rng.integers(2, 24))
        p = float(rng.uniform(0.05, 0.9))
        hi = max(1, cap // 4)
        h = np.where(rng.random((n, n)) < p, rng.integers(0, hi + 1, (n, n)), INF).astype(np.int64)
        np.fill_diagonal(h, 0)
        yield cap, h
    for cap in (20, 64, 200):  # directed paths whose far ends pass the cap
        for w in (1, cap // 8, cap // 4):
            n = min(40, cap // max(w, 1) + 3)
            h = np.full((n, n), INF, np.int64)
            np.fill_diagonal(h, 0)
            h[np.arange(n - 1), np.arange(1, n)] = w
            yield cap, h


def test_truncated_mix_keeps_truncated_distances_and_the_certificate_is_sound():
    rng = np.random.default_rng(17)
    held = failed = 0
    for cap, h in _graphs(rng):
        exact = oracle.fw(h.astype(np.int32), threads=1).astype(np.int64)
        d = _mixed_fw(h, cap, rng)
        # invariant: truncation of every stored entry equals truncation of the distance
        assert np.array_equal(np.minimum(d, cap), np.minimum(exact, cap))
        finite = h[(h < INF) & ~np.eye(h.shape[0], dtype=bool)]
        wmax = int(finite.max()) if finite.size else 0
        ok, mapped = _certify(d, cap, wmax)
        if ok:
            held += 1
            assert np.array_equal(mapped, exact)  # the certified mapping is the exact closure
        else:
            failed += 1
        # the int32 pass from the mapped matrix closes it exactly, certified or not
        assert np.all(mapped >= exact)
        assert np.array_equal(oracle.fw(mapped.astype(np.int32), threads=1).astype(np.int64), exact)
    assert held > 100 and failed > 20  # both sides of the certificate were exercised


def test_certificate_would_be_unsound_without_the_weight_term():
    """The weight term matters: on a path of weight-15 hops (within the 16-bit pass's limit of
    cap / 4 for cap 64) the distances 15, 30, 45, 60 stay below the cap and 75 jumps over it.
    A test without the weight would accept the result and map the reachable 75 to the
    sentinel; the certificate (60 + 15 >= 64) refuses it."""
    cap = 64
    n = 6
    h = np.full((n, n), INF, np.int64)
    np.fill_diagonal(h, 0)
    h[np.arange(n - 1), np.arange(1, n)] = 15
    exact = oracle.fw(h.astype(np.int32), threads=1).astype(np.int64)
    assert exact[0, n - 1] == 75
    d = _mixed_fw(h, cap, np.random.default_rng(0))
    below = d[d < cap]
    assert int(below.max()) == 60
    ok, mapped = _certify(d, cap, wmax=15)
    assert not ok                             # the certificate refuses ...
    assert mapped[0, n - 1] == INF            # ... the mapping that would lose d(0, 5) = 75
    assert np.array_equal(oracle.fw(mapped.astype(np.int32), threads=1).astype(np.int64), exact)
