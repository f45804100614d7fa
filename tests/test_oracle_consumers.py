"""CPU pins of the oracle's event consumers and scoring (closed forms)."""
import math

import numpy as np
import pytest

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


def test_library_f1_agrees_with_the_oracle():
    """The library's event scoring (host code, no GPU) against the oracle's, on
    random streams with jitter, drops, extras and flipped polarities."""
    import oracle as orc
    from paper_2602_15018_gb300 import build, event_f1
    try:
        build._nvcc()
    except RuntimeError:
        pytest.skip("nvcc not available")
    build.build()
    rng = np.random.default_rng(7)
    for trial in range(5):
        n = 3000
        t = rng.integers(0, 200000, n)
        x = rng.integers(0, 40, n)
        y = rng.integers(0, 30, n)
        p = rng.integers(0, 2, n)
        ref = orc.pack(t, x, y, p)
        keep = rng.random(n) > 0.1
        tp = np.clip(t + rng.integers(-1500, 1500, n), 0, None)
        pp = np.where(rng.random(n) < 0.05, 1 - p, p)
        pred = np.concatenate([orc.pack(tp, x, y, pp)[keep],
                               orc.pack(rng.integers(0, 200000, 300), rng.integers(0, 40, 300),
                                        rng.integers(0, 30, 300), rng.integers(0, 2, 300))])
        pred = pred[rng.permutation(len(pred))]
        for tol in (0, 500, 1000):
            a = orc.match_f1(40, 30, pred, ref, tol)
            b = event_f1(pred, ref, tol)
            for k in ("matched", "n_pred", "n_ref", "count_abs_err"):
                assert a[k] == b[k], (trial, tol, k, a[k], b[k])
            assert abs(a["f1"] - b["f1"]) < 1e-12
