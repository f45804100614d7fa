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
