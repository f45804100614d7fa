"""Pins of the interpolator oracle (CPU); the pins are in interp_pins.py."""
import interp_pins as IP
from oracle import interp_oracle as io


def test_bf16_rounding_matches_torch():
    IP.pin_bf16_rounding(io)


def test_conv3_is_a_sum_of_2d_correlations():
    IP.pin_conv3(io)


def test_convT2_special_cases():
    IP.pin_convT2(io)


def test_untrained_network_is_linear_interpolation():
    IP.pin_untrained_is_linear(io)


def test_gradients_match_finite_differences():
    IP.pin_gradients(io)


def test_adamw_first_step_closed_form():
    IP.pin_adamw_first_step(io)


def test_bf16_rounded_gradients_stay_close():
    IP.pin_quantized_gradients(io)
