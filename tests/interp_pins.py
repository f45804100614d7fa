"""Pins of the interpolator oracle (oracle/interp_oracle.py): library
routines, closed forms and finite differences, so that a dropped term, a
wrong index or a transposed operand in the oracle fails before any GPU
comparison.  Each pin takes the oracle module (the real one, or a copy with
a planted mistake in the mutation test)."""
import numpy as np
import scipy.signal
import torch


def pin_bf16_rounding(io):
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.standard_normal(5000) * 10.0 ** rng.integers(-6, 6, 5000),
                        [1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, -1.0 - 2 ** -8, 0.0, 65504.0]])
    ref = torch.from_numpy(x.astype(np.float32)).to(torch.bfloat16).double().numpy()
    assert np.array_equal(io.bf16(x), ref)


def pin_conv3(io):
    rng = np.random.default_rng(1)
    x = rng.standard_normal((2, 7, 9, 3))
    w = rng.standard_normal((3, 3, 3, 4))
    out = io.conv3(x, w)
    ref = np.zeros_like(out)
    for n in range(2):
        for o in range(4):
            for c in range(3):
                ref[n, :, :, o] += scipy.signal.correlate2d(x[n, :, :, c], w[:, :, c, o], mode="same")
    assert np.allclose(out, ref, atol=1e-12)
    # stride 2 keeps the even positions of the stride-1 result
    x2 = rng.standard_normal((1, 8, 12, 3))
    assert np.allclose(io.conv3(x2, w, 2), io.conv3(x2, w)[:, ::2, ::2, :], atol=1e-12)


def pin_convT2(io):
    rng = np.random.default_rng(2)
    x = rng.standard_normal((2, 3, 5, 4))
    eye = np.zeros((4, 2, 2, 4))
    for a in range(2):
        for b in range(2):
            eye[:, a, b, :] = np.eye(4)
    assert np.allclose(io.convT2(x, eye), np.repeat(np.repeat(x, 2, axis=1), 2, axis=2))
    one = np.zeros((4, 2, 2, 4))
    one[:, 1, 0, :] = np.eye(4)                   # only (a, b) = (1, 0)
    up = io.convT2(x, one)
    assert np.allclose(up[:, 1::2, 0::2, :], x) and np.abs(up[:, 0::2, :, :]).max() == 0.0


def pin_untrained_is_linear(io):
    rng = np.random.default_rng(3)
    p = io.init_params(0)
    L0 = rng.standard_normal((2, 8, 12))
    L4 = rng.standard_normal((2, 8, 12))
    out, _ = io.forward(p, L0, L4)
    for j in range(3):
        assert np.allclose(out[j], L0 + (j + 1) / 4.0 * (L4 - L0), atol=1e-14)


def _rand_params(io, seed):
    p = io.init_params(seed)
    rng = np.random.default_rng(seed + 100)
    p["W9"] = rng.standard_normal(io.SHAPES["W9"]) * 0.3
    for k in io.BIAS:
        p[k] = rng.standard_normal(io.BIAS[k]) * 0.05
    return p


def pin_gradients(io):
    rng = np.random.default_rng(4)
    p = _rand_params(io, 4)
    N, H, W = 2, 8, 12
    L0 = rng.uniform(-4.0, 0.0, (N, H, W))
    L4 = L0 + rng.normal(0.0, 0.3, (N, H, W))
    T = rng.uniform(-4.0, 0.0, (3, N, H, W))
    loss, g, _ = io.loss_and_grads(p, L0, L4, T)
    h = 1e-6
    for k in list(io.SHAPES) + list(io.BIAS):
        flat = p[k].reshape(-1)
        idx = rng.choice(flat.size, size=min(6, flat.size), replace=False)
        if k == "W1":   # only the two real input channels carry gradient
            idx = [np.ravel_multi_index((1, 2, 1, 5), p[k].shape), np.ravel_multi_index((0, 0, 0, 0), p[k].shape)]
        for i in idx:
            old = flat[i]
            flat[i] = old + h
            lp = io.charbonnier(io.forward(p, L0, L4)[0], T)
            flat[i] = old - h
            lm = io.charbonnier(io.forward(p, L0, L4)[0], T)
            flat[i] = old
            fd = (lp - lm) / (2 * h)
            an = g[k].reshape(-1)[i]
            assert abs(fd - an) <= 1e-6 * max(1e-3, abs(fd)) + 1e-9, (k, i, fd, an)


def pin_adamw_first_step(io):
    rng = np.random.default_rng(5)
    p = {"W1": rng.standard_normal((3, 3, 8, 32)), "b1": rng.standard_normal(32)}
    g = {"W1": rng.standard_normal((3, 3, 8, 32)), "b1": rng.standard_normal(32)}
    st = io.adamw_init(p)
    lr, wd, eps = 1e-3, 1e-4, 1e-8
    q = io.adamw_step(p, g, st, lr, wd=wd, eps=eps)
    # the first step of Adam moves every coordinate by about lr: m_hat = g, v_hat = g^2
    # absolute tolerance only: a relative one (numpy's default 1e-5) would hide lr * wd * p
    assert np.allclose(q["W1"], p["W1"] - lr * (g["W1"] / (np.abs(g["W1"]) + eps) + wd * p["W1"]),
                       rtol=0.0, atol=1e-15)
    assert np.allclose(q["b1"], p["b1"] - lr * g["b1"] / (np.abs(g["b1"]) + eps), rtol=0.0, atol=1e-15)
    assert st["t"] == 1


def pin_quantized_gradients(io):
    """Rounding the activation gradients to BF16 (quantize_grads) changes each
    parameter gradient by no more than a chain of BF16 roundings allows: a few
    2^-8 relative in norm, far below what a wrong tap or channel would move;
    and it does change them (the rounding is applied)."""
    rng = np.random.default_rng(6)
    p = _rand_params(io, 6)
    N, H, W = 2, 8, 12
    L0 = rng.uniform(-4.0, 0.0, (N, H, W))
    L4 = L0 + rng.normal(0.0, 0.3, (N, H, W))
    T = rng.uniform(-4.0, 0.0, (3, N, H, W))
    _, g, _ = io.loss_and_grads(p, L0, L4, T, quantize=True)
    _, gq, _ = io.loss_and_grads(p, L0, L4, T, quantize=True, quantize_grads=True)
    moved = 0
    for k in list(io.SHAPES) + list(io.BIAS):
        a, b = gq[k].reshape(-1), g[k].reshape(-1)
        nb = np.linalg.norm(b)
        if nb == 0:
            assert np.linalg.norm(a) == 0, k
            continue
        rel = np.linalg.norm(a - b) / nb
        assert rel < 8 * 2.0 ** -8, (k, rel)
        moved += rel > 0
    assert moved >= 10


ALL_INTERP_PINS = [pin_bf16_rounding, pin_conv3, pin_convT2, pin_untrained_is_linear, pin_gradients,
                   pin_adamw_first_step, pin_quantized_gradients]
