"""Pins of the oracle's event consumers and scoring (oracle/consumers_oracle.c).

Each pin takes an oracle library handle (the default build, or a copy with a
planted mistake in the mutation test) and raises AssertionError when the
oracle disagrees with:
  - closed forms of the time surface of the RL appendix (S <- S e^{-dt/tau} + 1),
  - hand-counted event frames over fixed windows,
  - the defining properties of the F1 score (identical streams, halves,
    flipped polarities, shifted times),
  - a maximum one-to-one matching found by brute force (augmenting paths),
    which the oracle's greedy time-ordered matching must reach exactly.
"""
from __future__ import annotations

import math

import numpy as np

import oracle


def pin_time_surface(library):
    # one cell updated at t = 0, 10 ms, 20 ms with tau = 10 ms:
    # S = ((1 e^-1) + 1) e^-1 + 1 = 1 + e^-1 + e^-2
    ev = oracle.pack([0, 10_000, 20_000, 5_000], [2, 2, 2, 2], [1, 1, 1, 1], [1, 1, 1, 0])
    order = np.argsort(ev, kind="stable")
    S, last = oracle.time_surface(4, 3, ev[order], tau_us=10_000.0, library=library)
    assert math.isclose(S[1, 1, 2], 1 + math.exp(-1) + math.exp(-2), rel_tol=1e-14)
    assert S[0, 1, 2] == 1.0 and last[0, 1, 2] == 5_000 and last[1, 1, 2] == 20_000
    assert S.sum() == S[1, 1, 2] + 1.0
    # two updates tau ln 2 apart: 1/2 + 1
    ev = oracle.pack([1000, 1000 + round(10_000 * math.log(2))], [0, 0], [0, 0], [0, 0])
    S, _ = oracle.time_surface(1, 1, ev, tau_us=10_000.0, library=library)
    assert abs(S[0, 0, 0] - 1.5) < 1e-4


def pin_event_frames(library):
    t = [0, 19_999, 20_000, 45_000, 60_000]
    ev = oracle.pack(t, [0, 0, 1, 1, 0], [0, 0, 0, 2, 0], [1, 0, 1, 1, 1])
    fr = oracle.event_frames(3, 3, ev, 0, 20_000, 3, library=library)
    assert fr[0, 1, 0, 0] == 1 and fr[0, 0, 0, 0] == 1
    assert fr[1, 1, 0, 1] == 1 and fr[2, 1, 2, 1] == 1
    assert fr.sum() == 4          # the event at 60 ms is past the 3 windows
    fr = oracle.event_frames(3, 3, ev, 19_999, 1, 2, library=library)
    assert fr.sum() == 2 and fr[0, 0, 0, 0] == 1 and fr[1, 1, 0, 1] == 1


def pin_match_f1(library):
    rng = np.random.default_rng(0)
    n = 2000
    t = np.sort(rng.integers(0, 100_000, n))
    x = rng.integers(0, 16, n)
    y = rng.integers(0, 12, n)
    p = (x + y) % 2            # one polarity per pixel, so flipping never re-matches
    ref = oracle.pack(t, x, y, p)
    r = oracle.match_f1(16, 12, ref, ref, library=library)
    assert r["f1"] == 1.0 and r["count_err"] == 0.0
    far = oracle.pack(t + 5000, x, y, p)
    r = oracle.match_f1(16, 12, far, ref, tol_us=1000, library=library)
    assert r["matched"] < 0.2 * n
    half = ref[::2]
    r = oracle.match_f1(16, 12, half, ref, library=library)
    assert r["precision"] == 1.0 and abs(r["recall"] - len(half) / n) < 1e-12
    assert abs(r["f1"] - 2 * r["recall"] / (1 + r["recall"])) < 1e-12
    assert r["count_abs_err"] == n - len(half)
    flipped = oracle.pack(t, x, y, 1 - p)
    r = oracle.match_f1(16, 12, flipped, ref, library=library)
    assert r["matched"] == 0


def _max_matching(ta, tb, tol):
    """Size of a maximum one-to-one matching with |ta - tb| <= tol (Kuhn's
    augmenting paths: plain, independent of any ordering argument)."""
    adj = [[j for j, b in enumerate(tb) if abs(a - b) <= tol] for a in ta]
    owner = [-1] * len(tb)

    def augment(i, seen):
        for j in adj[i]:
            if not seen[j]:
                seen[j] = True
                if owner[j] < 0 or augment(owner[j], seen):
                    owner[j] = i
                    return True
        return False

    return sum(augment(i, [False] * len(tb)) for i in range(len(ta)))


def pin_match_f1_is_maximum(library):
    rng = np.random.default_rng(42)
    for trial in range(40):
        n_a, n_b = rng.integers(0, 25, 2)
        cells = int(rng.integers(1, 4))
        tol = int(rng.integers(0, 40))
        ta = rng.integers(0, 200, n_a)
        tb = rng.integers(0, 200, n_b)
        ca = rng.integers(0, cells, n_a)
        cb = rng.integers(0, cells, n_b)
        a = oracle.pack(ta, ca // 2, np.zeros(n_a, int), ca % 2)
        b = oracle.pack(tb, cb // 2, np.zeros(n_b, int), cb % 2)
        want = sum(_max_matching(ta[ca == c].tolist(), tb[cb == c].tolist(), tol) for c in range(cells))
        r = oracle.match_f1(4, 1, a, b, tol_us=tol, library=library)
        assert r["matched"] == want, (trial, r["matched"], want)
        want_cnt = sum(abs(int((ca == c).sum()) - int((cb == c).sum())) for c in range(cells))
        assert r["count_abs_err"] == want_cnt


ALL_CONSUMER_PINS = [pin_time_surface, pin_event_frames, pin_match_f1, pin_match_f1_is_maximum]
