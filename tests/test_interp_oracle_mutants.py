"""Planted mistakes in a copy of the interpolator oracle must each fail a pin.

Each case rewrites one expression of oracle/interp_oracle.py in a temporary
copy, loads the copy as its own module, and runs the pins of interp_pins.py
against it: a flipped tap, transposed upsampling taps, a wrong interpolation
weight, a dropped ReLU mask, skip gradient or skip mask, a missing loss normalisation,
a missing AdamW bias correction, weight decay on biases, truncating BF16."""
import importlib.util
import os
import tempfile

import pytest

import interp_pins as IP

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle", "interp_oracle.py")

MUTANTS = [
    ("conv3_tap_flipped", "out += patch @ w[dy, dx]", "out += patch @ w[2 - dy, 2 - dx]"),
    ("convT2_taps_transposed", "out[:, a::2, b::2, :] = x @ w[:, a, b, :]", "out[:, a::2, b::2, :] = x @ w[:, b, a, :]"),
    ("interp_weight_shifted", "base = np.stack([L0 + (j / 4.0) * (L4 - L0) for j in (1, 2, 3)])",
     "base = np.stack([L0 + (j / 4.0) * (L4 - L0) for j in (0, 1, 2)])"),
    ("relu_mask_dropped", "gd1 = q(gd1 * (c[\"d1\"] > 0))", "gd1 = q(gd1)"),
    ("skip_gradient_dropped", "ge2 = q(ge2 + ge2b * (c[\"e2\"] > 0))", "ge2 = q(ge2b * (c[\"e2\"] > 0))"),
    ("skip_mask_dropped", "ge1 = q(gcat1[..., 32:] * (c[\"e1\"] > 0))", "ge1 = q(gcat1[..., 32:])"),
    ("loss_grad_not_averaged", "return d / np.sqrt(d * d + CHARB_EPS * CHARB_EPS) / d.size",
     "return d / np.sqrt(d * d + CHARB_EPS * CHARB_EPS)"),
    ("adam_no_bias_correction", "upd = (m / (1 - b1 ** t)) / (np.sqrt(v / (1 - b2 ** t)) + eps)",
     "upd = m / (np.sqrt(v) + eps)"),
    ("decay_on_biases", "if k.startswith(\"W\"):\n            upd = upd + wd * p[k]", "if True:\n            upd = upd + wd * p[k]"),
    ("bf16_truncates", "r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16", "r = (u >> 16) << 16"),
]


@pytest.fixture(scope="module")
def tmpdir_mut():
    with tempfile.TemporaryDirectory(prefix="interp_mut_") as d:
        yield d


def _mutant_module(tmp, name, old, new):
    src = open(SRC).read()
    assert src.count(old) >= 1, f"mutation site for {name} not found"
    path = os.path.join(tmp, f"interp_oracle_{name}.py")
    with open(path, "w") as f:
        f.write(src.replace(old, new, 1))
    spec = importlib.util.spec_from_file_location(f"interp_oracle_{name}", path)
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_interp_mutant_is_caught(tmpdir_mut, name, old, new):
    mod = _mutant_module(tmpdir_mut, name, old, new)
    for pin in IP.ALL_INTERP_PINS:
        try:
            pin(mod)
        except AssertionError:
            return
    pytest.fail(f"planted mistake {name} passed every interpolator pin")
