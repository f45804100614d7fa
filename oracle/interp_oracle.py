"""Oracle of the learned temporal interpolator (TEST INFRASTRUCTURE ONLY).

Plain, slow FP64 numpy restatement of the small convolutional U-Net that
predicts three intermediate log-intensity frames between two keyframes
(L0 at tau, L4 at tau + 4 dt), its gradients, the Charbonnier loss and the
AdamW update.  Only the test suite, the smoke check and the benchmark's CPU
legs may import it; it shares nothing with the CUDA library.

The paper has no interpolator: it renders every frame (Sec. 2).  This part
follows the project's own definition, stated here so that it can be checked
by eye (no parity to the paper exists; see "parity unpinned" below):

  input    x = [L0, L4 - L0, 0 x 6]                       (8 channels)
  e1 = relu(conv3(x,  W1: 8 -> 32)  + b1)                  H   x W
  e2 = relu(conv3s2(e1, W2: 32 -> 64) + b2)                H/2 x W/2
  e3 = relu(conv3s2(e2, W3: 64 -> 128) + b3)               H/4 x W/4
  e4 = relu(conv3(e3, W4: 128 -> 128) + b4)                H/4 x W/4
  u1 = convT2(e4, W5: 128 -> 64) + b5                      H/2 x W/2
  d1 = relu(conv3([u1, e2], W6: 128 -> 64) + b6)           H/2 x W/2
  u2 = convT2(d1, W7: 64 -> 32) + b7                       H   x W
  d2 = relu(conv3([u2, e1], W8: 64 -> 32) + b8)            H   x W
  r  = d2 W9 (32 -> 3) + b9                                H   x W
  L_j = L0 + (j / 4) (L4 - L0) + r_{j-1},  j = 1, 2, 3

conv3: 3 x 3, zero padding 1, stride 1; conv3s2: the same at stride 2
(output (y, x) reads input (2y + dy - 1, 2x + dx - 1)); convT2: 2 x 2
transposed convolution at stride 2, out(2y + a, 2x + b) = in(y, x) W[a, b].
Layouts: activations [N, H, W, C]; W1..W4, W6, W8 as [3, 3, Cin, Cout];
W5, W7 as [Cin, 2, 2, Cout]; W9 as [32, 3].

loss = mean over (j, n, y, x) of sqrt((L_j - T_j)^2 + eps^2), eps = 1e-3
(Charbonnier), against target frames T_j of the plain 1000 FPS renderer.
AdamW (Loshchilov and Hutter, ICLR 2019): m = b1 m + (1 - b1) g,
v = b2 v + (1 - b2) g^2, w -= lr (m / (1 - b1^t) / (sqrt(v / (1 - b2^t)) + eps)
+ wd w), weight decay on the weight tensors only.

With quantize=True the oracle rounds what the GPU path stores in BF16 (the
weights and every activation it writes) to BF16 (round to nearest even), and
keeps all arithmetic in FP64; with quantize_grads=True (backward) it also
rounds the activation gradients the GPU path stores in BF16.  The CUDA path
then differs only by its FP32 accumulation order, and by the rare BF16
rounding that this order flips.

Parity unpinned against the paper (it has no interpolator); the oracle is
pinned to mathematics instead: finite differences of the loss, the direct
definitions of the convolutions, and a closed-form AdamW step.
"""
from __future__ import annotations

import numpy as np

LAYERS = ("W1", "W2", "W3", "W4", "W5", "W6", "W7", "W8", "W9")
SHAPES = {
    "W1": (3, 3, 8, 32), "W2": (3, 3, 32, 64), "W3": (3, 3, 64, 128), "W4": (3, 3, 128, 128),
    "W5": (128, 2, 2, 64), "W6": (3, 3, 128, 64), "W7": (64, 2, 2, 32), "W8": (3, 3, 64, 32),
    "W9": (32, 3),
}
BIAS = {"b1": 32, "b2": 64, "b3": 128, "b4": 128, "b5": 64, "b6": 64, "b7": 32, "b8": 32, "b9": 3}
CHARB_EPS = 1e-3


def bf16(x):
    """Round to the nearest BF16 value (ties to even), returned as float64."""
    a = np.ascontiguousarray(x, dtype=np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    out = r.astype(np.uint32).view(np.float32).astype(np.float64)
    nan = np.isnan(a)
    if nan.any():
        out[nan] = np.nan
    return out


def init_params(seed: int = 0):
    """He-normal weights (fan-in), zero biases, zero last layer: the untrained
    network is exactly linear interpolation."""
    rng = np.random.default_rng(seed)
    p = {}
    for k, shp in SHAPES.items():
        if k == "W9":
            p[k] = np.zeros(shp)
            continue
        fan_in = shp[0] * shp[1] * shp[2] if k not in ("W5", "W7") else shp[0]
        w = rng.standard_normal(shp) * np.sqrt(2.0 / fan_in)
        if k == "W1":
            w[:, :, 2:, :] = 0.0          # padded input channels
        p[k] = w
    for k, n in BIAS.items():
        p[k] = np.zeros(n)
    return p


# ---------------------------------------------------------------------------
# layers (forward)
# ---------------------------------------------------------------------------
def pad1(x):
    return np.pad(x, ((0, 0), (1, 1), (1, 1), (0, 0)))


def conv3(x, w, stride=1):
    """out[n, y, x, o] = sum_{dy, dx, c} in[n, s y + dy - 1, s x + dx - 1, c] w[dy, dx, c, o]."""
    N, H, W, C = x.shape
    Ho, Wo = H // stride, W // stride
    xp = pad1(x)
    out = np.zeros((N, Ho, Wo, w.shape[3]))
    for dy in range(3):
        for dx in range(3):
            patch = xp[:, dy: dy + stride * Ho: stride, dx: dx + stride * Wo: stride, :]
            out += patch @ w[dy, dx]
    return out


def convT2(x, w):
    """out[n, 2y + a, 2x + b, o] = sum_c in[n, y, x, c] w[c, a, b, o]."""
    N, H, W, C = x.shape
    out = np.zeros((N, 2 * H, 2 * W, w.shape[3]))
    for a in range(2):
        for b in range(2):
            out[:, a::2, b::2, :] = x @ w[:, a, b, :]
    return out


def relu(x):
    return np.maximum(x, 0.0)


def forward(p, L0, L4, quantize=False):
    """L0, L4: [N, H, W] log frames (H, W divisible by 4).  Returns the three
    predicted frames [3, N, H, W] and the cache for backward."""
    q = bf16 if quantize else (lambda v: v)
    w = {k: (q(v) if k.startswith("W") else v) for k, v in p.items()}
    L0 = np.asarray(L0, np.float64)
    L4 = np.asarray(L4, np.float64)
    N, H, W = L0.shape
    x = np.zeros((N, H, W, 8))
    x[..., 0] = L0
    x[..., 1] = L4 - L0
    x = q(x)
    c = {"x": x, "w": w}
    c["e1"] = q(relu(conv3(x, w["W1"]) + w["b1"]))
    c["e2"] = q(relu(conv3(c["e1"], w["W2"], 2) + w["b2"]))
    c["e3"] = q(relu(conv3(c["e2"], w["W3"], 2) + w["b3"]))
    c["e4"] = q(relu(conv3(c["e3"], w["W4"]) + w["b4"]))
    c["u1"] = q(convT2(c["e4"], w["W5"]) + w["b5"])
    c["cat2"] = np.concatenate([c["u1"], c["e2"]], axis=3)
    c["d1"] = q(relu(conv3(c["cat2"], w["W6"]) + w["b6"]))
    c["u2"] = q(convT2(c["d1"], w["W7"]) + w["b7"])
    c["cat1"] = np.concatenate([c["u2"], c["e1"]], axis=3)
    c["d2"] = q(relu(conv3(c["cat1"], w["W8"]) + w["b8"]))
    r = c["d2"] @ w["W9"] + w["b9"]                       # [N, H, W, 3]
    base = np.stack([L0 + (j / 4.0) * (L4 - L0) for j in (1, 2, 3)])
    out = base + np.moveaxis(r, 3, 0)
    return out, c


def charbonnier(out, target):
    d = out - target
    return float(np.mean(np.sqrt(d * d + CHARB_EPS * CHARB_EPS)))


def charbonnier_grad(out, target):
    d = out - target
    return d / np.sqrt(d * d + CHARB_EPS * CHARB_EPS) / d.size


# ---------------------------------------------------------------------------
# backward
# ---------------------------------------------------------------------------
def conv3_backward(x, w, gout, stride=1):
    """Gradients of conv3 with respect to its input and weights."""
    N, H, W, C = x.shape
    Ho, Wo = H // stride, W // stride
    xp = pad1(x)
    gxp = np.zeros_like(xp)
    gw = np.zeros_like(w)
    for dy in range(3):
        for dx in range(3):
            sl = (slice(None), slice(dy, dy + stride * Ho, stride), slice(dx, dx + stride * Wo, stride),
                  slice(None))
            patch = xp[sl]
            gw[dy, dx] = patch.reshape(-1, C).T @ gout.reshape(-1, gout.shape[3])
            gxp[sl] += gout @ w[dy, dx].T
    return gxp[:, 1:-1, 1:-1, :], gw


def convT2_backward(x, w, gout):
    gx = np.zeros_like(x)
    gw = np.zeros_like(w)
    for a in range(2):
        for b in range(2):
            g = gout[:, a::2, b::2, :]
            gx += g @ w[:, a, b, :].T
            gw[:, a, b, :] = x.reshape(-1, x.shape[3]).T @ g.reshape(-1, g.shape[3])
    return gx, gw


def backward(p, cache, gout, quantize_grads=False):
    """gout: d loss / d out [3, N, H, W].  Returns gradients for every
    parameter (same keys and shapes as p).

    With quantize_grads=True the gradients of the activations are rounded to
    BF16 where the GPU path stores them in BF16: the loss gradient; the
    gradient of d2; the gradient of the concatenation [u2, e1] after conv8
    (the e1 half masked by e1 > 0); that of d1; that of [u1, e2] after conv6
    (the e2 half masked); those of e4 and e3; and the e2 and e1 halves again
    after the stride-2 layers add their data gradients to them.  Every weight
    and bias gradient is then computed from those rounded values.  All
    arithmetic stays FP64."""
    q = bf16 if quantize_grads else (lambda v: v)
    w, c = cache["w"], cache
    g = {}
    gr = q(np.moveaxis(gout, 0, 3))                                    # [N, H, W, 3]
    g["W9"] = c["d2"].reshape(-1, 32).T @ gr.reshape(-1, 3)
    g["b9"] = gr.reshape(-1, 3).sum(0)
    gd2 = q((gr @ w["W9"].T) * (c["d2"] > 0))
    gcat1, g["W8"] = conv3_backward(c["cat1"], w["W8"], gd2)
    g["b8"] = gd2.reshape(-1, 32).sum(0)
    gu2 = q(gcat1[..., :32])
    ge1 = q(gcat1[..., 32:] * (c["e1"] > 0))
    g["b7"] = gu2.reshape(-1, 32).sum(0)
    gd1, g["W7"] = convT2_backward(c["d1"], w["W7"], gu2)
    gd1 = q(gd1 * (c["d1"] > 0))
    gcat2, g["W6"] = conv3_backward(c["cat2"], w["W6"], gd1)
    g["b6"] = gd1.reshape(-1, 64).sum(0)
    gu1 = q(gcat2[..., :64])
    ge2 = q(gcat2[..., 64:] * (c["e2"] > 0))
    g["b5"] = gu1.reshape(-1, 64).sum(0)
    ge4, g["W5"] = convT2_backward(c["e4"], w["W5"], gu1)
    ge4 = q(ge4 * (c["e4"] > 0))
    ge3, g["W4"] = conv3_backward(c["e3"], w["W4"], ge4)
    g["b4"] = ge4.reshape(-1, 128).sum(0)
    ge3 = q(ge3 * (c["e3"] > 0))
    ge2b, g["W3"] = conv3_backward(c["e2"], w["W3"], ge3, 2)
    g["b3"] = ge3.reshape(-1, 128).sum(0)
    ge2 = q(ge2 + ge2b * (c["e2"] > 0))
    ge1b, g["W2"] = conv3_backward(c["e1"], w["W2"], ge2, 2)
    g["b2"] = ge2.reshape(-1, 64).sum(0)
    ge1 = q(ge1 + ge1b * (c["e1"] > 0))
    _, g["W1"] = conv3_backward(c["x"], w["W1"], ge1)
    g["b1"] = ge1.reshape(-1, 32).sum(0)
    return g



def loss_and_grads(p, L0, L4, targets, quantize=False, quantize_grads=False):
    out, cache = forward(p, L0, L4, quantize)
    g = backward(p, cache, charbonnier_grad(out, targets), quantize_grads)
    return charbonnier(out, targets), g, out


# ---------------------------------------------------------------------------
# optimiser
# ---------------------------------------------------------------------------
def adamw_init(p):
    return {"t": 0, "m": {k: np.zeros_like(v) for k, v in p.items()},
            "v": {k: np.zeros_like(v) for k, v in p.items()}}


def adamw_step(p, g, state, lr, wd=1e-4, b1=0.9, b2=0.999, eps=1e-8):
    state["t"] += 1
    t = state["t"]
    out = {}
    for k in p:
        m = state["m"][k] = b1 * state["m"][k] + (1 - b1) * g[k]
        v = state["v"][k] = b2 * state["v"][k] + (1 - b2) * g[k] * g[k]
        upd = (m / (1 - b1 ** t)) / (np.sqrt(v / (1 - b2 ** t)) + eps)
        if k.startswith("W"):
            upd = upd + wd * p[k]
        out[k] = p[k] - lr * upd
    return out
