"""The seeded synthetic inputs (scenes/) hold the recipe the measurements state:
deterministic per seed, the texture scene's intensities in [0.02, 1], chunked
rendering equal to one-shot rendering, and the HD texture workload's event
rate near 0.0085 events per pixel-frame under its sensor settings (checked on
the oracle over the first frames)."""
import numpy as np

import oracle
import scenes


def test_seeded_and_chunk_invariant():
    sc = scenes.TextureScene(96, 64, seed=3)
    a = scenes.render_frames(sc, 9, device="cpu", chunk=4).numpy()
    b = scenes.TextureScene(96, 64, seed=3).render(np.arange(9)).numpy()
    c = scenes.TextureScene(96, 64, seed=4).render(np.arange(9)).numpy()
    assert np.array_equal(a, b) and not np.array_equal(b, c)
    assert a.dtype == np.float32 and 0.02 <= a.min() and a.max() <= 1.0
    s1 = scenes.SinusoidScene(40, 30, seed=1).render(np.arange(3)).numpy()
    s2 = scenes.SinusoidScene(40, 30, seed=1).render(np.arange(3)).numpy()
    assert np.array_equal(s1, s2) and np.abs(s1 - 0.5).max() <= 8 * 0.2 + 1e-6


def test_hd_texture_event_rate():
    fr = scenes.render_frames(scenes.TextureScene(1280, 720, seed=0), 21, device="cpu").numpy()
    sim = oracle.OracleSim(1280, 720, c_pos=0.2, c_neg=0.25, sigma_c=0.03, c_min=0.01, refractory_us=100, seed=1)
    ev, _ = sim.step(fr, 0, 1000)
    rate = len(ev) / (20 * 1280 * 720)
    assert 0.004 < rate < 0.02, rate
