"""Sensor bandwidth filter on the GPU against the oracle (reading R13), bit for bit.

Shapes: 23 x 41 pixels (not a multiple of 4: the scalar kernel) and 64 x 48
(the 128-bit kernel), 37 frames (a ragged tail after the 4-frame groups),
split over two calls with the state carried, in place and out of place; and
the filtered frames through the event model against the oracle's events.
"""
import numpy as np
import pytest
import torch

import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import __graft_entry__
    __graft_entry__.build()


def _frames(seed, T, H, W):
    rng = np.random.default_rng(seed)
    base = rng.uniform(-4.0, 1.0, (H, W))
    walk = np.cumsum(rng.standard_normal((T, H, W)) * 0.08, axis=0)
    return (base + walk).astype(np.float32)


@pytest.mark.parametrize("H,W", [(23, 41), (64, 48)])
@pytest.mark.parametrize("cutoff_hz", [40.0, 400.0, 1e9])
def test_lowpass_matches_oracle(H, W, cutoff_hz):
    from paper_2602_15018_gb300 import lowpass_alpha, lowpass_log
    T = 37
    alpha = lowpass_alpha(cutoff_hz, 1000)            # the library's gain
    L = _frames(int(cutoff_hz) % 1000 + H, T, H, W)
    want, want_state = oracle.lowpass_log(L, oracle.lowpass_alpha(cutoff_hz, 1000))
    Ld = torch.from_numpy(L).cuda()
    got, st = lowpass_log(Ld, alpha)
    assert np.array_equal(got.cpu().numpy(), want)
    assert np.array_equal(st.cpu().numpy(), want_state)
    # two calls with the state carried, the second in place
    a, st2 = lowpass_log(Ld[:16].contiguous(), alpha)
    tail = Ld[16:].clone()
    b, st3 = lowpass_log(tail, alpha, state=st2, out=tail)
    assert b.data_ptr() == tail.data_ptr()
    assert np.array_equal(torch.cat([a, b]).cpu().numpy(), want)
    assert np.array_equal(st3.cpu().numpy(), want_state)


def test_filtered_frames_give_the_oracles_events():
    from paper_2602_15018_gb300 import EventSim, lowpass_alpha, lowpass_log
    H, W, T = 36, 52, 60
    alpha = lowpass_alpha(150.0, 1000)
    L = _frames(5, T, H, W)
    filt, _ = oracle.lowpass_log(L, oracle.lowpass_alpha(150.0, 1000))
    sim_o = oracle.OracleSim(W, H, c_pos=0.15, c_neg=0.15, sigma_c=0.03, refractory_us=100, input_is_log=True,
                             seed=9)
    ev_o, seg_o = sim_o.step(filt, 0, 1000)
    got, _ = lowpass_log(torch.from_numpy(L).cuda(), alpha)
    sim = EventSim(W, H, c_pos=0.15, c_neg=0.15, sigma_c=0.03, refractory_us=100, input_is_log=True, seed=9,
                   max_frames_per_step=T)
    sim.step(got, 0, 1000)
    ev, seg = sim.drain()
    sim.close()
    assert len(ev_o) > 100
    assert np.array_equal(ev, ev_o) and np.array_equal(seg, seg_o)


def test_lowpass_rejects_bad_arguments():
    from paper_2602_15018_gb300 import NeurosimError, lowpass_log
    L = torch.zeros((4, 8, 8), device="cuda")
    for alpha in (0.0, -0.5, 1.5, float("nan")):
        with pytest.raises(NeurosimError):
            lowpass_log(L, alpha)
    out = torch.zeros((5, 8, 8), device="cuda")
    with pytest.raises(NeurosimError):                 # partly overlapping buffers
        lowpass_log(out[:4], 0.5, out=out[1:])
