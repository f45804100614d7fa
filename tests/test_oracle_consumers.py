"""CPU pins of the oracle's event consumers and scoring (closed forms)."""
import math

import numpy as np

import oracle


def test_time_surface_closed_form():
    # one cell updated at t = 0, 10 ms, 20 ms with tau = 10 ms:
    # S = ((1 * e^-1) + 1) * e^-1 + 1 = 1 + e^-1 + e^-2
    ev = oracle.pack([0, 10_000, 20_000, 5_000], [2, 2, 2, 2], [1, 1, 1, 1], [1, 1, 1, 0])
    order = np.argsort(ev, kind="stable")
    S, last = oracle.time_surface(4, 3, ev[order], tau_us=10_000.0)
    assert math.isclose(S[1, 1, 2], 1 + math.exp(-1) + math.exp(-2), rel_tol=1e-14)
    assert S[0, 1, 2] == 1.0 and last[0, 1, 2] == 5_000 and last[1, 1, 2] == 20_000
    assert S.sum() == S[1, 1, 2] + 1.0


def test_event_frames_counts():
    t = [0, 19_999, 20_000, 45_000, 60_000]
    ev = oracle.pack(t, [0, 0, 1, 1, 0], [0, 0, 0, 2, 0], [1, 0, 1, 1, 1])
    fr = oracle.event_frames(3, 3, ev, 0, 20_000, 3)
    assert fr[0, 1, 0, 0] == 1 and fr[0, 0, 0, 0] == 1
    assert fr[1, 1, 0, 1] == 1 and fr[2, 1, 2, 1] == 1
    assert fr.sum() == 4          # the event at 60 ms is past the 3 windows


def test_match_f1_cases():
    rng = np.random.default_rng(0)
    n = 2000
    t = np.sort(rng.integers(0, 100_000, n))
    x = rng.integers(0, 16, n)
    y = rng.integers(0, 12, n)
    p = (x + y) % 2            # one polarity per pixel, so flipping never re-matches
    ref = oracle.pack(t, x, y, p)
    r = oracle.match_f1(16, 12, ref, ref)
    assert r["f1"] == 1.0 and r["count_err"] == 0.0
    far = oracle.pack(t + 5000, x, y, p)
    r = oracle.match_f1(16, 12, far, ref, tol_us=1000)
    assert r["matched"] < 0.2 * n
    half = ref[::2]
    r = oracle.match_f1(16, 12, half, ref)
    assert r["precision"] == 1.0 and abs(r["recall"] - len(half) / n) < 1e-12
    assert abs(r["f1"] - 2 * r["recall"] / (1 + r["recall"])) < 1e-12
    assert r["count_abs_err"] == n - len(half)
    flipped = oracle.pack(t, x, y, 1 - p)
    r = oracle.match_f1(16, 12, flipped, ref)
    assert r["matched"] == 0
