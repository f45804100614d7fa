"""Planted mistakes in a copy of the oracle must each fail at least one pin.

Each case rewrites one expression of oracle/evsim_oracle.c in a temporary
copy, builds it with the oracle's own flags, and runs the pins against it.
This checks that the pins are strong enough to catch a plausible slip (a tie
rule, a dropped state update, a transposed coordinate, a wrong rounding)."""
import os
import shutil
import subprocess
import tempfile

import pytest

import consumer_pins as CP
import oracle
import oracle_pins as P

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(os.path.dirname(HERE), "oracle")

# (name, original text, replacement, count of occurrences to replace)
MUTANTS = [
    ("tie_rule_strict", "if (!(lvl <= bb)) break;", "if (!(lvl < bb)) break;"),
    ("ref_to_frame_value", "                    r = lvl;\n                    if (refractory_us != 0 && tl != TLAST_NONE && t - tl < (int64_t)refractory_us)\n                        continue;                            /* R5 */",
     "                    r = bb;\n                    if (refractory_us != 0 && tl != TLAST_NONE && t - tl < (int64_t)refractory_us)\n                        continue;                            /* R5 */"),
    ("frac_flipped", "const float num = lvl - a;\n                    const float frac = num / den;\n                    float tf = floorf(frac * Df);            /* R4 */",
     "const float num = bb - lvl;\n                    const float frac = num / den;\n                    float tf = floorf(frac * Df);            /* R4 */"),
    ("round_not_floor", "float tf = floorf(frac * Df);            /* R4 */",
     "float tf = roundf(frac * Df);            /* R4 */"),
    ("refractory_le", "t - tl < (int64_t)refractory_us)\n                        continue;                            /* R5 */",
     "t - tl <= (int64_t)refractory_us)\n                        continue;                            /* R5 */"),
    ("tlast_not_updated", "eb_push(&b, pack(t, x, y, 1));\n                    tl = t;",
     "eb_push(&b, pack(t, x, y, 1));"),
    ("polarity_swapped", "eb_push(&b, pack(t, x, y, 0));", "eb_push(&b, pack(t, x, y, 1));"),
    ("xy_transposed", "eb_push(&b, pack(t, x, y, 1));", "eb_push(&b, pack(t, y, x, 1));"),
    ("interval_start_wrong", "const int64_t ta = *tau_prev;", "const int64_t ta = tb - dt;"),
    ("log_coeff", "static const float C_INV5 = 0x1.99999ap-3f;",
     "static const float C_INV5 = 0x1.555556p-3f;"),
    ("log_no_range_fold", "if (m > C_SQRT2) {", "if (m > 2.0f) {"),
    ("noise_same_draw", "float zn = oracle_normal_ih12(seed, (uint64_t)u * 2u + 1u);",
     "float zn = oracle_normal_ih12(seed, (uint64_t)u * 2u + 0u);"),
    ("noise_sign", "vp = c_pos + dp;", "vp = c_pos - dp;"),
    ("first_frame_lprev", "                ref[u] = L;\n                lprev[u] = L;\n                tlast[u] = TLAST_NONE;\n            }\n            *has_prev = 1;\n            *tau_prev = tb;\n            continue;\n        }\n        const int64_t ta = *tau_prev;\n        const int64_t D = tb - ta;\n        const float Df",
     "                ref[u] = L;\n                lprev[u] = 0.0f;\n                tlast[u] = TLAST_NONE;\n            }\n            *has_prev = 1;\n            *tau_prev = tb;\n            continue;\n        }\n        const int64_t ta = *tau_prev;\n        const int64_t D = tb - ta;\n        const float Df"),
    ("lowpass_sign", "const float d = L[(int64_t)k * n + i] - s;", "const float d = s - L[(int64_t)k * n + i];"),
    ("lowpass_state_ignored", "float s = init ? L[i] : state[i];", "float s = L[i];"),
    ("lowpass_starts_at_zero", "float s = init ? L[i] : state[i];", "float s = init ? 0.0f : state[i];"),
    ("lowpass_state_not_saved", "        state[i] = s;\n    }\n    return ORACLE_OK;", "    }\n    return ORACLE_OK;"),
    ("lowpass_gain_squared", "s = fmaf(alpha, d, s);", "s = fmaf(alpha * alpha, d, s);"),
    ("leak_sign", "out[(int64_t)f * n + i] = L[(int64_t)f * n + i] + delta;",
     "out[(int64_t)f * n + i] = L[(int64_t)f * n + i] - delta;"),
    ("leak_without_threshold", "const float k = (cpos ? cpos[i] : cpos_u) * rate_us;", "const float k = rate_us;"),
    ("shot_always_on", "(int)(d2 >> 63));", "1);"),
    ("shot_time_from_pixel_bits", "((d1 & 0xFFFFFFFFull) * (uint64_t)D) >> 32", "((d1 >> 32) * (uint64_t)D) >> 32"),
    ("shot_rate_without_pixels", "rate_hz * (double)len * (double)D * 1e-6", "rate_hz * 64.0 * (double)D * 1e-6 * 0.5"),
    ("shot_ragged_tile_full", "npix - tile * SHOT_TILE;", "SHOT_TILE;"),
    ("lowpass_alpha_no_two_pi", "exp(-two_pi * cutoff_hz", "exp(-cutoff_hz"),
    ("lowpass_alpha_kept_fraction", "return (float)(1.0 - keep);", "return (float)keep;"),
    ("lowpass_alpha_dt_in_ms", "((double)dt_us * 1e-6)", "((double)dt_us * 1e-3)"),
]


# mistakes in the consumers and the scoring (oracle/consumers_oracle.c); none of
# them writes outside its buffers
CONSUMER_MUTANTS = [
    ("surface_decay_sign", "decay = exp(-(double)(t - last[c]) / tau_us);",
     "decay = exp((double)(t - last[c]) / tau_us);"),
    ("surface_last_not_updated", "        S[c] = S[c] * decay + 1.0;\n        last[c] = t;",
     "        S[c] = S[c] * decay + 1.0;"),
    ("frames_window_from_zero", "const int64_t w = (t - t_start) / win_us;", "const int64_t w = t / win_us;"),
    ("match_tolerance_strict", "if (llabs(ta - tb) <= tol_us)", "if (llabs(ta - tb) < tol_us)"),
    ("match_wrong_advance", "else if (ta < tb) ++ii;", "else if (ta > tb) ++ii;"),
    ("cell_without_polarity", "return (y << 49) | (x << 33) | (p << 32) | t;", "return (y << 49) | (x << 33) | t;"),
    ("count_error_signed", "cnt_err += llabs((i1 - i) - (j1 - j));", "cnt_err += (i1 - i) - (j1 - j);"),
]


def _build_mutant(tmp, name, old, new, target="evsim_oracle.c"):
    other = "consumers_oracle.c" if target == "evsim_oracle.c" else "evsim_oracle.c"
    src = open(os.path.join(SRC, target)).read()
    assert old in src, f"mutation site for {name} not found"
    mutated = src.replace(old, new, 1)
    d = os.path.join(tmp, name)
    os.makedirs(d)
    open(os.path.join(d, target), "w").write(mutated)
    shutil.copy(os.path.join(SRC, other), d)
    so = os.path.join(d, "lib.so")
    subprocess.check_call(["gcc", *oracle.CFLAGS, "-o", so, os.path.join(d, "evsim_oracle.c"),
                           os.path.join(d, "consumers_oracle.c"), "-lm"])
    return oracle.load_library(so)


def _fails_some_pin(library):
    pins = P.ALL_PINS + [lambda L: P.pin_log(L, stride=257)]
    for pin in pins:
        try:
            pin(library)
        except (AssertionError, oracle.OracleError):
            return True
    return False


@pytest.fixture(scope="module")
def tmpdir_mut():
    d = tempfile.mkdtemp(prefix="oracle_mut_")
    yield d
    shutil.rmtree(d, ignore_errors=True)


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_mutant_is_caught(tmpdir_mut, name, old, new):
    lib = _build_mutant(tmpdir_mut, name, old, new)
    assert _fails_some_pin(lib), f"planted mistake {name} passed every pin"


@pytest.mark.parametrize("name,old,new", CONSUMER_MUTANTS, ids=[m[0] for m in CONSUMER_MUTANTS])
def test_consumer_mutant_is_caught(tmpdir_mut, name, old, new):
    lib = _build_mutant(tmpdir_mut, name, old, new, target="consumers_oracle.c")
    for pin in CP.ALL_CONSUMER_PINS:
        try:
            pin(lib)
        except (AssertionError, oracle.OracleError):
            return
    pytest.fail(f"planted mistake {name} passed every consumer pin")
