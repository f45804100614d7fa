"""CPU pins of the oracle (closed forms, brute force, libm, published vectors)."""
import numpy as np
import pytest

import oracle
import oracle_pins as P


@pytest.fixture(scope="module")
def L():
    return oracle.lib()


def test_ramps(L):
    P.pin_ramps(L)


def test_constant_and_first_frame(L):
    P.pin_constant_and_first_frame(L)


def test_uneven_interval(L):
    P.pin_uneven_interval(L)


def test_refractory(L):
    P.pin_refractory(L)


def test_brute_force(L):
    P.pin_brute_force(L)


def test_lowpass_filter(L):
    P.pin_lowpass(L)


def test_log_vs_libm(L):
    P.pin_log(L)


def test_splitmix64_published_vector(L):
    # SplitMix64 reference test vector (seed 1234567, first five outputs)
    exp = [6457827717110365317, 3203168211198807973, 9817491932198370423,
           4593380528125082431, 16408922859458223821]
    assert [oracle.splitmix64_at(1234567, i) for i in range(5)] == exp


def test_irwin_hall_moments(L):
    z = np.array([oracle.normal_ih12(42, i) for i in range(60000)])
    assert abs(z.mean()) < 0.02 and abs(z.var() - 1.0) < 0.02
    assert z.min() >= -6.0 and z.max() <= 6.0
    # Irwin-Hall(12) - 6 has excess kurtosis -0.1 (a Gaussian has 0)
    k = ((z - z.mean()) ** 4).mean() / z.var() ** 2 - 3.0
    assert -0.2 < k < 0.0
    assert np.all(np.round(z * 2**20) == z * 2**20)


def test_threshold_maps(L):
    P.pin_threshold_maps(L)


def test_band_and_order(L):
    P.pin_band_and_order(L)


def test_fp64_agreement(L):
    P.pin_fp64_agreement(L)


def test_step_composition(L):
    P.pin_step_composition(L)


def test_time_errors(L):
    sim = oracle.OracleSim(4, 4, input_is_log=True)
    sim.step(np.zeros((2, 4, 4), np.float32), 0, 1000)
    with pytest.raises(oracle.OracleError):
        sim.step(np.zeros((1, 4, 4), np.float32), 1000, 1000)   # not after 1000
    with pytest.raises(oracle.OracleError):
        sim.step(np.zeros((1, 4, 4), np.float32), 2000, 0)      # dt = 0
    with pytest.raises(oracle.OracleError):
        sim.step(np.zeros((2, 4, 4), np.float32), 2**32 - 2, 5)  # past 2^32 - 2


def test_intensity_clamp_and_nan(L):
    W, H = 3, 1
    sim = oracle.OracleSim(W, H, c_pos=0.2, c_neg=0.2)
    fr = np.array([[[0.5, 0.5, 0.5]], [[-3.0, np.nan, 2e9]]], np.float32)
    ev, seg = sim.step(fr, 0, 1000)
    Lexp = oracle.mylog(np.array([0.0, 0.0, 1e6], np.float32) + np.float32(1e-3))
    assert np.array_equal(sim.lprev, Lexp)
    t, x, y, p = oracle.unpack(ev)
    assert set(x[p == 0].tolist()) == {0, 1} and set(x[p == 1].tolist()) == {2}


def test_banded_oracle_equals_one_sensor(L):
    """The band-parallel oracle run (row bands on host threads, merged into the
    output order) equals one oracle sensor over the whole frame, bit for bit,
    on a textured scene with noise and refractory; with more bands than rows
    too."""
    import scenes
    W, H, T = 61, 37, 30
    fr = scenes.render_frames(scenes.TextureScene(W, H, seed=4, speed=(300.0, 600.0)), T).numpy()
    cp, cn = oracle.threshold_maps(W, H, 0.2, 0.25, 0.03, 0.01, 9, library=L)
    one = oracle.OracleSim(W, H, c_pos_map=cp, c_neg_map=cn, refractory_us=100, library=L)
    ev, seg = one.step(fr, 0, 1000)
    assert len(ev) > 500
    for threads in (1, 3, 8, 64):
        bev, bseg, used, st = oracle.banded_step(fr, W, H, 0, 1000, cp, cn, refractory_us=100, threads=threads,
                                                 library=L)
        assert used == min(threads, H)
        assert np.array_equal(bseg, seg) and np.array_equal(bev, ev), threads
        for k in ("ref", "lprev", "tlast"):
            assert np.array_equal(st[k], getattr(one, k)), (threads, k)


def test_leak_closed_form(L):
    P.pin_leak(L)


def test_shot_noise_statistics(L):
    P.pin_shot_noise(L)


def test_merge_streams(L):
    P.pin_merge(L)
