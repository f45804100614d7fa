"""Sensor leak and shot noise on the GPU against the oracle, bit for bit.

Sec. 2 of the paper lists noise among the non-idealities the simulator
models (and the user may turn off), with no model; the readings are the
oracle's R14 (leak: a reference drift, equal to a rising log input) and R15
(shot noise: Poisson events per 64-pixel tile and interval from
counter-based SplitMix64 draws, merged into the stream per interval).
"""
import numpy as np
import pytest
import torch

import oracle

pytestmark = pytest.mark.gpu

DT = 1000


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import __graft_entry__
    __graft_entry__.build()


def _log_frames(seed, T, H, W):
    rng = np.random.default_rng(seed)
    base = rng.uniform(-3.0, 0.0, (H, W))
    walk = np.cumsum(rng.standard_normal((T, H, W)) * 0.04, axis=0)
    return (base + walk).astype(np.float32)


@pytest.mark.parametrize("H,W,rate", [(23, 41, 40.0), (64, 48, 3.5), (8, 8, 0.0)])
def test_leak_matches_oracle_and_feeds_the_event_model(H, W, rate):
    from paper_2602_15018_gb300 import EventSim, leak_log
    T, t0, origin = 57, 3_000, 1_000
    L = _log_frames(H * W, T, H, W)
    sim = EventSim(W, H, c_pos=0.2, c_neg=0.25, sigma_c=0.03, refractory_us=100, input_is_log=True, seed=3,
                   max_frames_per_step=T)
    cp, cn = sim.thresholds()
    want = oracle.leak_log(L, t0, DT, origin, rate, cpos=cp)
    got = leak_log(torch.from_numpy(L).cuda(), t0, DT, origin, rate,
                   c_pos=torch.from_numpy(np.ascontiguousarray(cp.ravel())).cuda())
    assert np.array_equal(got.cpu().numpy(), want)
    uni = leak_log(torch.from_numpy(L).cuda(), t0, DT, origin, rate, c_pos=0.2)
    assert np.array_equal(uni.cpu().numpy(), oracle.leak_log(L, t0, DT, origin, rate, cpos_u=0.2))
    x = torch.from_numpy(L).cuda()
    assert leak_log(x, t0, DT, origin, rate, c_pos=0.2, out=x).data_ptr() == x.data_ptr()   # in place
    sim.step(got, t0, DT)
    ev, seg = sim.drain()
    o = oracle.OracleSim(W, H, c_pos_map=cp, c_neg_map=cn, refractory_us=100, input_is_log=True)
    rev, rseg = o.step(want, t0, DT)
    assert np.array_equal(seg, rseg) and np.array_equal(ev, rev)
    sim.close()


@pytest.mark.parametrize("W,H,rate,n_int,D0", [(37, 83, 40.0, 500, 700), (1280, 720, 1.0, 40, 1000),
                                              (5, 3, 60.0, 200, 333), (64, 48, 0.0, 10, 1000)])
def test_shot_noise_matches_oracle(W, H, rate, n_int, D0):
    from paper_2602_15018_gb300 import shot_noise
    seed, ta0 = 1234 + W, 40_000
    ev, seg = shot_noise(W, H, rate, seed, ta0, D0, DT, n_int)
    rev, rseg = oracle.shot_noise(W, H, rate, seed, ta0, D0, DT, n_int)
    assert np.array_equal(seg, rseg)
    assert np.array_equal(ev.cpu().numpy().view(np.uint64), rev)
    if rate > 0:
        assert len(rev) > 100


def test_shot_noise_merged_into_a_signal_stream():
    import scenes
    from paper_2602_15018_gb300 import EventSim, merge_events, shot_noise
    W, H, T = 160, 96, 30
    fr = scenes.render_frames(scenes.TextureScene(W, H, seed=5, speed=(300.0, 600.0)), T)
    sim = EventSim(W, H, c_pos=0.2, c_neg=0.25, sigma_c=0.03, refractory_us=100, seed=8, max_frames_per_step=T)
    sim.step(fr.cuda(), 0, DT)
    sig, sseg = sim.drain(to="cuda")
    noise, nseg = shot_noise(W, H, 20.0, 99, 1000, DT, DT, T - 1)     # the step's intervals
    got, gseg = merge_events(sig, sseg, noise, nseg)
    want, wseg = oracle.merge_events(sig.cpu().numpy().view(np.uint64), sseg, noise.cpu().numpy().view(np.uint64),
                                     nseg)
    assert np.array_equal(gseg, wseg) and np.array_equal(got.cpu().numpy().view(np.uint64), want)
    assert len(noise) > 100 and len(sig) > 1000
    sim.close()


def test_noise_calls_reject_bad_arguments():
    from paper_2602_15018_gb300 import NeurosimError, leak_log, shot_noise
    with pytest.raises(NeurosimError):
        shot_noise(64, 48, 100.0, 1, 0, DT, DT, 4)                     # tile mean 6.4 > 4
    with pytest.raises(NeurosimError):
        shot_noise(64, 48, 1.0, 1, 0, 0, DT, 4)                        # empty first interval
    L = torch.zeros((4, 8, 8), device="cuda")
    with pytest.raises(NeurosimError):
        leak_log(L, 0, DT, 10, 1.0)                                    # starts before the origin
    with pytest.raises(NeurosimError):
        leak_log(L, 0, DT, 0, -1.0)
