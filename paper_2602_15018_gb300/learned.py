"""Learned path: a renderer at a quarter of the event camera's frame rate, the
interpolator's intermediate frames, and the exact event model on the result.

The paper renders every frame for its event camera (Sec. 2, >2700 FPS); here
keyframes arrive every 4 dt, the U-Net (interp.py) predicts the three log
frames between them, and the unchanged FP32 event emission runs on the full
1000 FPS log sequence.  Training clips are 1000 FPS sequences of the seeded
procedural scenes the plain simulator is benchmarked on.
"""
from __future__ import annotations

import math

import numpy as np
import torch

import scenes

from .evsim import EventSim, event_f1, log_intensity
from .interp import Interpolator


def training_clips(batch: int, size: int, seed: int, speed=(150.0, 300.0), device="cuda") -> torch.Tensor:
    """[batch, 5, size, size] log frames (1000 FPS): crops of one seeded texture
    scene of 4 size x 4 size at a random time in a 2 s clip."""
    rng = np.random.default_rng(seed)
    big = 4 * size
    sc = scenes.TextureScene(big, big, seed=int(rng.integers(1 << 30)), speed=speed)
    t0 = int(rng.integers(0, 2_000_000)) // 1000 * 1000
    fr = scenes.render_frames(sc, 5, t0_us=t0, dt_us=1000, device=device)
    lg = log_intensity(fr.contiguous())
    out = torch.empty((batch, 5, size, size), dtype=torch.float32, device=device)
    for b in range(batch):
        y, x = rng.integers(0, big - size + 1, 2)
        out[b] = lg[:, y:y + size, x:x + size]
    return out


def train(net: Interpolator, steps: int, batch: int = 16, size: int = 256, lr: float = 1e-3,
          weight_decay: float = 1e-4, seed: int = 10000, speed=(150.0, 300.0), report: int = 0):
    """AdamW with a cosine learning-rate schedule over `steps` steps; returns
    the losses of the steps it reports (every `report` steps, 0 = none)."""
    losses = []
    for it in range(steps):
        clips = training_clips(batch, size, seed + it, speed)
        lr_t = lr * 0.5 * (1.0 + math.cos(math.pi * it / max(1, steps)))
        want = bool(report) and (it % report == 0 or it == steps - 1)
        loss = net.train_step(clips, lr_t, weight_decay, want_loss=want)
        if want:
            losses.append((it, loss))
    return losses


def interpolate_sequence(net: Interpolator, keys: torch.Tensor, chunk: int = 8) -> torch.Tensor:
    """Log keyframes [K, H, W] at spacing 4 dt -> log frames [4 (K - 1) + 1, H, W]
    at spacing dt (keyframes kept, three predicted frames per interval)."""
    K, H, W = keys.shape
    seq = torch.empty((4 * (K - 1) + 1, H, W), dtype=torch.float32, device=keys.device)
    seq[0::4] = keys
    for i in range(0, K - 1, chunk):
        b = min(chunk, K - 1 - i)
        mid = net.forward(keys[i:i + b].contiguous(), keys[i + 1:i + 1 + b].contiguous())   # [3, b, H, W]
        for j in range(3):
            seq[4 * i + 1 + j: 4 * (i + b): 4] = mid[j]
    return seq


def events_of(frames: torch.Tensor, input_is_log: bool, t0_us: int = 0, dt_us: int = 1000, launches=None, **sim):
    """Events (host uint64 records) of one sensor over `frames` [T, H, W].
    If `launches` is a list, the number of kernels the simulator launched is
    appended to it."""
    T, H, W = frames.shape
    s = EventSim(W, H, input_is_log=input_is_log, max_frames_per_step=T, **sim)
    s.step(frames.contiguous(), t0_us, dt_us)
    ev, _ = s.drain()
    if launches is not None:
        launches.append(int(s.stats()["kernel_launches"]))
    s.close()
    return ev


def evaluate(net: Interpolator, width: int, height: int, n_keys: int, scene_seed: int, tol_us: int = 1000,
             speed=(150.0, 300.0), **sim) -> dict:
    """F1 and count error of the events of the learned path (keyframes every
    4 ms + predicted frames) and of plain linear interpolation against the
    plain 1000 FPS path, on one seeded HD-like texture clip."""
    sc = scenes.TextureScene(width, height, seed=scene_seed, speed=speed)
    T = 4 * (n_keys - 1) + 1
    frames = scenes.render_frames(sc, T, device="cuda", chunk=32)
    ref = events_of(frames, False, **sim)
    keys = log_intensity(frames[0::4].contiguous())
    del frames
    lin_net = Interpolator(8, height, width, seed=0)          # untrained: r = 0, linear interpolation
    res = {"n_ref": int(len(ref)), "frames": T}
    for name, model in (("learned", net), ("linear", lin_net)):
        seq = interpolate_sequence(model, keys)
        ev = events_of(seq, True, **sim)
        sc_ = event_f1(ev, ref, tol_us)
        res[name] = {k: sc_[k] for k in ("f1", "precision", "recall", "count_err", "n_pred")}
        del seq
    lin_net.close()
    return res
