"""Learned path: a renderer at a quarter of the event camera's frame rate, the
interpolator's intermediate frames, and the exact event model on the result.

The paper renders every frame for its event camera (Sec. 2, >2700 FPS); here
keyframes arrive every 4 dt, the U-Net (interp.py) predicts the three log
frames between them, and the unchanged FP32 event emission runs on the full
1000 FPS log sequence.  The caller supplies the data: training clips of 1000
FPS log frames from a clip source, and rendered frames to score on.  This
module renders nothing itself.
"""
from __future__ import annotations

import math
from typing import Callable

import torch

from .evsim import EventSim, event_f1, log_intensity
from .interp import Interpolator


def train(net: Interpolator, steps: int, clip_source: Callable[[int], torch.Tensor], lr: float = 1e-3,
          weight_decay: float = 1e-4, report: int = 0):
    """AdamW with a cosine learning-rate schedule over `steps` steps.
    clip_source(it) returns step it's clips: DEVICE [batch, 5, H, W] log frames
    at 1000 FPS (frames 0 and 4 are the keyframes, 1..3 the targets).  Returns
    the losses of the steps it reports (every `report` steps, 0 = none)."""
    losses = []
    for it in range(steps):
        clips = clip_source(it)
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


def evaluate(net: Interpolator, frames: torch.Tensor, tol_us: int = 1000, **sim) -> dict:
    """F1 and count error of the events of the learned path (keyframes every
    4 frames + predicted frames) and of plain linear interpolation against the
    plain path on all of `frames` (DEVICE intensity frames [4 (K - 1) + 1, H, W]
    at 1000 FPS)."""
    T, H, W = frames.shape
    if (T - 1) % 4 != 0 or T < 5:
        raise ValueError("frames must hold 4 (K - 1) + 1 frames, K >= 2")
    ref = events_of(frames, False, **sim)
    keys = log_intensity(frames[0::4].contiguous())
    lin_net = Interpolator(8, H, W, seed=0)          # untrained: r = 0, linear interpolation
    res = {"n_ref": int(len(ref)), "frames": T}
    for name, model in (("learned", net), ("linear", lin_net)):
        seq = interpolate_sequence(model, keys)
        ev = events_of(seq, True, **sim)
        sc_ = event_f1(ev, ref, tol_us)
        res[name] = {k: sc_[k] for k in ("f1", "precision", "recall", "count_err", "n_pred")}
        del seq
    lin_net.close()
    return res
