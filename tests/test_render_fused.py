"""Render-fused event simulation against the oracle.

The paper argues for producing event data on the fly, without storing the
rendered frames (Sec. 1).  neurosim_evsim_step_texture renders a procedural
texture scene inside the emission kernel.  Its events must equal, bit for
bit, those of the FP32 oracle run on the frames the library's stand-alone
renderer (neurosim_render_texture) writes for the same scene and times; and
the renderer must draw the scene its definition states, which the seeded
scene generator of the tests computes independently in float64.
"""
import numpy as np
import pytest
import torch

import oracle
import scenes

pytestmark = pytest.mark.gpu

DT = 1000
SIM = dict(c_pos=0.2, c_neg=0.25, sigma_c=0.03, refractory_us=100, seed=11)


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import __graft_entry__
    __graft_entry__.build()


def _scene(W, H, seed, speed=(300.0, 600.0)):
    from paper_2602_15018_gb300 import texture_scene
    sc = scenes.TextureScene(W, H, seed=seed, speed=speed)
    return sc, texture_scene(**sc.params())


@pytest.mark.parametrize("W,H", [(320, 181), (1280, 720)])
def test_renderer_draws_the_scene_definition(W, H):
    """FP32 library renderer against the float64 scene generator: the texture
    agrees within the rounding of FP32 texture coordinates (|x| up to about
    1e4 px, so about 1e-3 px), and at most a few pixels right on a rectangle
    edge may fall on the other side of it."""
    from paper_2602_15018_gb300 import render_texture
    sc, ts = _scene(W, H, seed=W + 3)
    T = 6
    got = render_texture(ts, T, t0_us=123_000, dt_us=DT).cpu().numpy()
    want = sc.render(np.arange(T), t0_us=123_000, dt_us=DT, device="cuda").cpu().numpy()
    err = np.abs(got.astype(np.float64) - want.astype(np.float64))
    assert np.all((got >= 0.02 - 1e-6) & (got <= 1.0 + 1e-6))
    off = err > 2e-4
    assert off.sum() <= max(4, 1e-4 * err.size), (int(off.sum()), float(err.max()))
    assert np.median(err) < 2e-5


@pytest.mark.parametrize("W,H,T", [(320, 181, 40), (1280, 720, 48)])
def test_fused_step_matches_oracle_on_rendered_frames(W, H, T):
    """Two consecutive fused steps (an initialising one, then one that
    continues from the stored state after a gap) against the oracle on the
    renderer's frames for the same times."""
    from paper_2602_15018_gb300 import EventSim, render_texture
    _, ts = _scene(W, H, seed=W + H)
    g = EventSim(W, H, max_frames_per_step=T, **SIM)
    cp, cn = g.thresholds()
    o = oracle.OracleSim(W, H, c_pos_map=cp, c_neg_map=cn, refractory_us=100)
    t_starts = [5_000, 5_000 + T * DT + 1500]
    for k, t0 in enumerate(t_starts):
        g.step_texture(ts, T, t0, DT)
        ev, seg = g.drain()
        fr = render_texture(ts, T, t0_us=t0, dt_us=DT).cpu().numpy()
        rev, rseg = o.step(fr, t0, DT)
        assert np.array_equal(seg, rseg), f"step {k}: interval offsets differ"
        assert np.array_equal(ev, rev), f"step {k}: events differ ({len(ev)} vs {len(rev)})"
        assert len(rev) > 1000
    st = g.get_state()
    assert np.array_equal(st["ref"], o.ref) and np.array_equal(st["lprev"], o.lprev)
    g.close()


def test_fused_equals_unfused_step_and_replays_after_overflow():
    """The fused step gives the events of the plain step on the rendered
    frames, also when a tiny initial capacity makes the drain regrow the
    buffers and replay the pending fused steps."""
    from paper_2602_15018_gb300 import EventSim, render_texture
    W, H, T = 640, 360, 30
    _, ts = _scene(W, H, seed=77)
    a = EventSim(W, H, max_frames_per_step=T, event_capacity=500, **SIM)
    b = EventSim(W, H, max_frames_per_step=T, **SIM)
    for k in range(2):
        a.step_texture(ts, T, k * T * DT, DT)
        b.step(render_texture(ts, T, t0_us=k * T * DT, dt_us=DT), k * T * DT, DT)
    ea, sa = a.drain()
    eb, sb = b.drain()
    assert len(eb) > 5000
    assert np.array_equal(sa, sb) and np.array_equal(ea, eb)
    a.close()
    b.close()


def test_fused_step_rejects_bad_scenes():
    from paper_2602_15018_gb300 import EventSim, NeurosimError, render_texture
    g = EventSim(64, 48, max_frames_per_step=8, **SIM)
    _, ts = _scene(64, 40, seed=1)                  # other height
    with pytest.raises(NeurosimError):
        g.step_texture(ts, 4, 0, DT)
    _, ts = _scene(64, 48, seed=1)
    ts.octaves = 0
    with pytest.raises(NeurosimError):
        g.step_texture(ts, 4, 0, DT)
    with pytest.raises(NeurosimError):
        render_texture(ts, 2)
    ts.octaves = 4
    ts.n_rects = 17
    with pytest.raises(NeurosimError):
        g.step_texture(ts, 4, 0, DT)
    g.close()
