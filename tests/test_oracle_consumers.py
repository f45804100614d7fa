"""CPU pins of the oracle's event consumers and scoring (pins in consumer_pins.py)."""
import numpy as np
import pytest

import consumer_pins as CP
import oracle


def test_time_surface_closed_form():
    CP.pin_time_surface(oracle.lib())


def test_event_frames_counts():
    CP.pin_event_frames(oracle.lib())


def test_match_f1_cases():
    CP.pin_match_f1(oracle.lib())


def test_match_f1_is_a_maximum_matching():
    CP.pin_match_f1_is_maximum(oracle.lib())


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
