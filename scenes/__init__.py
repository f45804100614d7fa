"""Seeded procedural intensity scenes (synthetic inputs for tests and benchmarks).

This module only renders linear intensity frames; it holds none of the event
model's arithmetic (no log, no thresholds, no crossings).  The same code runs
on the CPU (inputs for the oracle and the parity tests) and on a CUDA device
(large benchmark inputs); both the CUDA library and the oracle always consume
one rendered copy, so the two devices need not agree bit for bit.

The paper renders indoor scenes with Habitat-Sim (Sec. 2); those assets and
the graphics stack are not available, so seeded procedural scenes with the
same role stand in:

  SinusoidScene  sum of 8 seeded 2-D sinusoids (spatial frequency 0.01-0.1
                 cycles/px, amplitude 0.05-0.2, offset 0.5) translating at a
                 seeded 150-300 px/s.
  TextureScene   4-octave value noise (hashed lattice, smoothstep, base
                 period 64 px, lacunarity 2, gain 0.5) mapped to [0.02, 1],
                 seen through a smooth affine camera path (rotation rate up to
                 90 deg/s, zoom 0.9-1.1, translation 150-300 px/s), with 16
                 moving occluding rectangles of random intensity drawn
                 last-on-top.
  log_ramp       frames whose log intensity is an exact linear ramp (closed-
                 form cases).
"""
from __future__ import annotations

import math

import numpy as np
import torch

_M32 = 0xFFFFFFFF


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


def _times_s(frame_idx, t0_us: int, dt_us: int, device) -> torch.Tensor:
    f = torch.as_tensor(np.asarray(frame_idx, np.float64), device=device)
    return (t0_us + f * dt_us) * 1e-6


class SinusoidScene:
    """Sum of 8 seeded 2-D sinusoids translating at one seeded velocity."""

    def __init__(self, width: int, height: int, seed: int = 0, n_waves: int = 8,
                 freq=(0.01, 0.1), amp=(0.05, 0.2), speed=(150.0, 300.0)):
        self.W, self.H = int(width), int(height)
        g = _rng(seed)
        mag = g.uniform(*freq, n_waves)
        ang = g.uniform(0, 2 * math.pi, n_waves)
        self.fx = mag * np.cos(ang)
        self.fy = mag * np.sin(ang)
        self.a = g.uniform(*amp, n_waves)
        self.phi = g.uniform(0, 2 * math.pi, n_waves)
        sp = g.uniform(*speed)
        va = g.uniform(0, 2 * math.pi)
        self.vx, self.vy = sp * math.cos(va), sp * math.sin(va)

    def render(self, frame_idx, t0_us: int = 0, dt_us: int = 1000, device="cpu",
               out: torch.Tensor | None = None) -> torch.Tensor:
        t = _times_s(frame_idx, t0_us, dt_us, device).view(-1, 1, 1)
        y = torch.arange(self.H, device=device, dtype=torch.float64).view(1, -1, 1)
        x = torch.arange(self.W, device=device, dtype=torch.float64).view(1, 1, -1)
        acc = torch.full((t.shape[0], self.H, self.W), 0.5, dtype=torch.float64, device=device)
        for i in range(len(self.a)):
            ph = 2 * math.pi * (self.fx[i] * (x - self.vx * t) + self.fy[i] * (y - self.vy * t))
            acc += self.a[i] * torch.sin(ph + self.phi[i])
        res = acc.to(torch.float32)
        if out is not None:
            out.copy_(res)
            return out
        return res


def _hash2(ix: torch.Tensor, iy: torch.Tensor, salt: int) -> torch.Tensor:
    """32-bit integer hash of a lattice point, returned as float64 in [0, 1)."""
    h = ((ix * 0x8DA6B343) ^ (iy * 0xD8163841) ^ salt) & _M32
    h = h ^ (h >> 15)
    h = (h * 0x2C1B3C6D) & _M32
    h = h ^ (h >> 12)
    h = (h * 0x297A2D39) & _M32
    h = h ^ (h >> 15)
    return h.to(torch.float64) * (1.0 / 4294967296.0)


def _value_noise(px: torch.Tensor, py: torch.Tensor, period: float, salt: int) -> torch.Tensor:
    u = px / period
    v = py / period
    iu = torch.floor(u)
    iv = torch.floor(v)
    fu = u - iu
    fv = v - iv
    su = fu * fu * (3.0 - 2.0 * fu)
    sv = fv * fv * (3.0 - 2.0 * fv)
    i0 = iu.to(torch.int64)
    j0 = iv.to(torch.int64)
    h00 = _hash2(i0, j0, salt)
    h10 = _hash2(i0 + 1, j0, salt)
    h01 = _hash2(i0, j0 + 1, salt)
    h11 = _hash2(i0 + 1, j0 + 1, salt)
    top = h00 + (h10 - h00) * su
    bot = h01 + (h11 - h01) * su
    return top + (bot - top) * sv


class TextureScene:
    """Value-noise texture under a smooth affine camera path plus occluders."""

    def __init__(self, width: int, height: int, seed: int = 0, speed=(150.0, 300.0),
                 n_rects: int = 16, max_rot_dps: float = 90.0, octaves: int = 4,
                 base_period: float = 64.0, rect_speed_max: float = 300.0):
        self.W, self.H = int(width), int(height)
        g = _rng(seed)
        self.salt = int(g.integers(0, 2**31))
        self.octaves = octaves
        self.base_period = base_period
        sp = g.uniform(*speed)
        va = g.uniform(0, 2 * math.pi)
        self.vx, self.vy = sp * math.cos(va), sp * math.sin(va)
        self.off = g.uniform(-1e4, 1e4, 2)
        # rotation rate w(t) = A sin(2 pi t / P + phase), |w| <= max_rot_dps
        self.rot_a = math.radians(g.uniform(0.3, 1.0) * max_rot_dps)
        self.rot_p = g.uniform(0.5, 2.0)
        self.rot_ph = g.uniform(0, 2 * math.pi)
        # zoom z(t) = 1 + 0.1 sin(2 pi t / P + phase), in [0.9, 1.1]
        self.zoom_p = g.uniform(1.0, 3.0)
        self.zoom_ph = g.uniform(0, 2 * math.pi)
        n = n_rects
        self.rw = g.uniform(32, 256, n)
        self.rh = g.uniform(32, 256, n)
        self.rval = g.uniform(0.02, 1.0, n)
        self.rcx = g.uniform(0, self.W, n)
        self.rcy = g.uniform(0, self.H, n)
        rs = g.uniform(0, rect_speed_max, n)
        ra = g.uniform(0, 2 * math.pi, n)
        self.rvx = rs * np.cos(ra)
        self.rvy = rs * np.sin(ra)

    def params(self) -> dict:
        """The scene as keyword arguments of the library's texture_scene (the
        same camera, texture and rectangles; its renderer works in FP32)."""
        rects = [(self.rcx[k], self.rcy[k], self.rw[k], self.rh[k], self.rvx[k], self.rvy[k], self.rval[k])
                 for k in range(len(self.rw))]
        return dict(width=self.W, height=self.H, salt=self.salt, octaves=self.octaves,
                    base_period=self.base_period, gain=0.5, intensity=(0.02, 1.0), velocity=(self.vx, self.vy),
                    offset=(float(self.off[0]), float(self.off[1])),
                    rotation=(self.rot_a, self.rot_p, self.rot_ph), zoom=(0.1, self.zoom_p, self.zoom_ph),
                    rects=rects)

    def _theta(self, t: torch.Tensor) -> torch.Tensor:
        k = 2 * math.pi / self.rot_p
        return self.rot_a / k * (math.cos(self.rot_ph) - torch.cos(k * t + self.rot_ph))

    def render(self, frame_idx, t0_us: int = 0, dt_us: int = 1000, device="cpu",
               out: torch.Tensor | None = None) -> torch.Tensor:
        t = _times_s(frame_idx, t0_us, dt_us, device).view(-1, 1, 1)
        y = torch.arange(self.H, device=device, dtype=torch.float64).view(1, -1, 1)
        x = torch.arange(self.W, device=device, dtype=torch.float64).view(1, 1, -1)
        cx, cy = 0.5 * self.W, 0.5 * self.H
        th = self._theta(t)
        z = 1.0 + 0.1 * torch.sin(2 * math.pi * t / self.zoom_p + self.zoom_ph)
        c, s = torch.cos(th), torch.sin(th)
        dx, dy = (x - cx) / z, (y - cy) / z
        wx = c * dx - s * dy + cx + self.vx * t + self.off[0]
        wy = s * dx + c * dy + cy + self.vy * t + self.off[1]
        acc = torch.zeros(wx.shape, dtype=torch.float64, device=device)
        amp, norm, period = 1.0, 0.0, self.base_period
        for o in range(self.octaves):
            acc += amp * _value_noise(wx, wy, period, (self.salt + 0x9E3779B9 * (o + 1)) & _M32)
            norm += amp
            amp *= 0.5
            period *= 0.5
        img = 0.02 + 0.98 * (acc / norm)
        img = img.expand(t.shape[0], self.H, self.W).clone() if img.shape[0] != t.shape[0] else img
        for k in range(len(self.rw)):
            ex_w, ex_h = self.W + self.rw[k], self.H + self.rh[k]
            rcx = torch.remainder(self.rcx[k] + self.rvx[k] * t, ex_w) - 0.5 * self.rw[k]
            rcy = torch.remainder(self.rcy[k] + self.rvy[k] * t, ex_h) - 0.5 * self.rh[k]
            m = ((x - rcx).abs() < 0.5 * self.rw[k]) & ((y - rcy).abs() < 0.5 * self.rh[k])
            img = torch.where(m, torch.full_like(img, float(self.rval[k])), img)
        res = img.to(torch.float32)
        if out is not None:
            out.copy_(res)
            return out
        return res


def render_frames(scene, n_frames: int, t0_us: int = 0, dt_us: int = 1000, device="cpu",
                  chunk: int = 64, out: torch.Tensor | None = None) -> torch.Tensor:
    """Render frames 0..n_frames-1 (at t0 + f * dt) into a [T, H, W] FP32 tensor."""
    if out is None:
        out = torch.empty((n_frames, scene.H, scene.W), dtype=torch.float32, device=device)
    for f0 in range(0, n_frames, chunk):
        f1 = min(n_frames, f0 + chunk)
        scene.render(np.arange(f0, f1), t0_us, dt_us, device=device, out=out[f0:f1])
    return out


def log_ramp(width: int, height: int, n_frames: int, l0: float, slope: float) -> np.ndarray:
    """Log-domain frames L_f = l0 + f * slope at every pixel (closed-form inputs)."""
    f = np.arange(n_frames, dtype=np.float64)
    vals = (l0 + f * slope).astype(np.float32)
    return np.broadcast_to(vals[:, None, None], (n_frames, height, width)).copy()


def random_log_frames(width: int, height: int, n_frames: int, seed: int, lo=-2.0, hi=2.0,
                      step: float | None = None) -> np.ndarray:
    """Seeded random log-domain frames (uniform, or a random walk with `step`)."""
    g = _rng(seed)
    if step is None:
        return g.uniform(lo, hi, (n_frames, height, width)).astype(np.float32)
    walk = np.cumsum(g.normal(0, step, (n_frames, height, width)), axis=0)
    return (walk + g.uniform(lo, hi, (1, height, width))).astype(np.float32)
