"""Python face of the learned interpolator (C ABI "Learned interpolator").

Argument marshalling only: forward, training, gradients and the optimiser all
run in the CUDA library.  Parameters move as one flat FP32 array in the
layout the header documents; `to_dict` / `from_dict` convert it to named
tensors ([3, 3, Cin, Cout], [Cin, 2, 2, Cout], [32, 3] and biases).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np
import torch

from ._lib import check, lib

# (name, shape in the flat array) in storage order: weights, then biases
_W = [("W1", (3, 3, 8, 32)), ("W2", (3, 3, 32, 64)), ("W3", (3, 3, 64, 128)), ("W4", (3, 3, 128, 128)),
      ("W5", (128, 2, 2, 64)), ("W6", (3, 3, 128, 64)), ("W7", (64, 2, 2, 32)), ("W8", (3, 3, 64, 32)),
      ("W9", (32, 16))]
_B = [("b1", 32), ("b2", 64), ("b3", 128), ("b4", 128), ("b5", 64), ("b6", 64), ("b7", 32), ("b8", 32),
      ("b9", 16)]


def to_dict(flat: np.ndarray) -> dict:
    out, o = {}, 0
    for k, shp in _W:
        n = int(np.prod(shp))
        out[k] = flat[o:o + n].reshape(shp)
        o += n
    for k, n in _B:
        out[k] = flat[o:o + n]
        o += n
    out["W9"] = out["W9"][:, :3]
    out["b9"] = out["b9"][:3]
    return out


def from_dict(p: dict) -> np.ndarray:
    parts = []
    for k, shp in _W:
        v = np.asarray(p[k], np.float32)
        if k == "W9":
            v = np.concatenate([v, np.zeros((32, 13), np.float32)], axis=1)
        parts.append(v.reshape(-1))
    for k, n in _B:
        v = np.asarray(p[k], np.float32).reshape(-1)
        if k == "b9":
            v = np.concatenate([v, np.zeros(13, np.float32)])
        parts.append(v)
    return np.concatenate(parts).astype(np.float32)


class Interpolator:
    """U-Net that predicts the 3 log frames between two log keyframes."""

    def __init__(self, max_batch: int, max_height: int, max_width: int, seed: int = 0,
                 stream: torch.cuda.Stream | None = None):
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        h = C.c_void_p()
        check(lib().neurosim_interp_create(int(max_batch), int(max_height), int(max_width), int(seed),
                                           C.c_void_p(self.stream.cuda_stream), C.byref(h)))
        self._h = h
        self.n_params = int(lib().neurosim_interp_param_count())

    @staticmethod
    def _dev(t):
        if not (t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()):
            raise ValueError("expected a contiguous float32 CUDA tensor")
        return C.c_void_p(t.data_ptr())

    def forward(self, L0: torch.Tensor, L4: torch.Tensor, out: torch.Tensor | None = None) -> torch.Tensor:
        B, H, W = L0.shape
        if out is None:
            out = torch.empty((3, B, H, W), dtype=torch.float32, device=L0.device)
        check(lib().neurosim_interp_forward(self._h, self._dev(L0), self._dev(L4), B, H, W, self._dev(out)))
        return out

    def train_step(self, clips: torch.Tensor, lr: float, weight_decay: float = 1e-4, want_loss=True):
        B, F, H, W = clips.shape
        assert F == 5
        loss = C.c_float(0.0)
        check(lib().neurosim_interp_train_step(self._h, self._dev(clips), B, H, W, float(lr), float(weight_decay),
                                               C.byref(loss) if want_loss else None))
        return float(loss.value) if want_loss else None

    def gradients(self, clips: torch.Tensor):
        B, F, H, W = clips.shape
        g = np.empty(self.n_params, np.float32)
        loss = C.c_float(0.0)
        check(lib().neurosim_interp_gradients(self._h, self._dev(clips), B, H, W, C.c_void_p(g.ctypes.data),
                                              C.byref(loss)))
        return float(loss.value), g

    def get_params(self) -> np.ndarray:
        p = np.empty(self.n_params, np.float32)
        check(lib().neurosim_interp_get_params(self._h, C.c_void_p(p.ctypes.data), self.n_params))
        return p

    def set_params(self, flat: np.ndarray) -> None:
        flat = np.ascontiguousarray(flat, np.float32)
        check(lib().neurosim_interp_set_params(self._h, C.c_void_p(flat.ctypes.data), self.n_params))

    def save(self, path: str, with_optimizer: bool = True) -> None:
        """Checkpoint: parameters, and the AdamW state unless with_optimizer is False."""
        check(lib().neurosim_interp_save(self._h, os.fsencode(path), int(bool(with_optimizer))))

    def load(self, path: str) -> None:
        check(lib().neurosim_interp_load(self._h, os.fsencode(path)))

    def launches(self) -> int:
        n = C.c_uint64(0)
        check(lib().neurosim_interp_launches(self._h, C.byref(n)))
        return int(n.value)

    def close(self) -> None:
        if getattr(self, "_h", None):
            lib().neurosim_interp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
