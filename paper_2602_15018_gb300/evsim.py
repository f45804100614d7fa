"""Python face of the event simulator: one `EventSim` per sensor.

Thin wrapper over the C ABI (include/neurosim_evsim.h): it turns tensors into
pointers and sizes and keeps the frames of pending steps alive until the
drain (the library may replay them after a buffer overflow).  PyTorch only
supplies device memory and the CUDA stream.
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from ._lib import MAX_RECTS, BatchParams, Params, Stats, TextureScene, check, lib


def _params(width: int, height: int, c_pos: float = 0.2, c_neg: float = 0.2,
            sigma_c: float = 0.0, c_min: float = 0.01, refractory_us: int = 0,
            log_eps: float = 1e-3, input_is_log: bool = False, seed: int = 0,
            c_pos_map=None, c_neg_map=None, keep=None) -> Params:
    """neurosim_evsim_params of one sensor (host maps are kept alive in `keep`)."""
    p = Params()
    lib().neurosim_evsim_default_params(C.byref(p))
    p.width, p.height = int(width), int(height)
    p.c_pos, p.c_neg, p.sigma_c, p.c_min = c_pos, c_neg, sigma_c, c_min
    p.refractory_us = int(refractory_us)
    p.log_eps = log_eps
    p.input_is_log = int(bool(input_is_log))
    p.seed = int(seed)
    if c_pos_map is not None:
        cp = np.ascontiguousarray(c_pos_map, np.float32).reshape(-1)
        cn = np.ascontiguousarray(c_neg_map, np.float32).reshape(-1)
        if keep is not None:
            keep += [cp, cn]
        p.c_pos_map = cp.ctypes.data_as(C.POINTER(C.c_float))
        p.c_neg_map = cn.ctypes.data_as(C.POINTER(C.c_float))
    return p


class EventSim:
    """Contrast-threshold DVS simulator for one sensor (arXiv 2602.15018, Sec. 2).

    step(frames, t0_us, dt_us) enqueues frames [T, H, W] (FP32, CUDA, contiguous)
    at times t0 + f dt; drain() returns the events of all pending steps as
    packed uint64 records ([63:32] t | [31:17] y | [16:1] x | [0] p) in
    interval-major (t, y, x, p) order, plus per-interval offsets.
    """

    def __init__(self, width: int, height: int, c_pos: float = 0.2, c_neg: float = 0.2,
                 sigma_c: float = 0.0, c_min: float = 0.01, refractory_us: int = 0,
                 log_eps: float = 1e-3, input_is_log: bool = False, seed: int = 0,
                 c_pos_map=None, c_neg_map=None, event_capacity: int = 0,
                 max_frames_per_step: int = 0, max_pending_intervals: int = 0,
                 pixels_per_thread: int = 0, prefetch_frames: int = 0, ctas_per_sm: int = 0,
                 stream: torch.cuda.Stream | None = None, device=None):
        L = lib()
        self.W, self.H = int(width), int(height)
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None
                                   else torch.device(device).index or 0)
        p = Params()
        L.neurosim_evsim_default_params(C.byref(p))
        p.width, p.height = self.W, self.H
        p.c_pos, p.c_neg, p.sigma_c, p.c_min = c_pos, c_neg, sigma_c, c_min
        p.refractory_us = int(refractory_us)
        p.log_eps = log_eps
        p.input_is_log = int(bool(input_is_log))
        p.seed = int(seed)
        keep = []
        if c_pos_map is not None:
            cp = np.ascontiguousarray(c_pos_map, np.float32).reshape(-1)
            cn = np.ascontiguousarray(c_neg_map, np.float32).reshape(-1)
            keep += [cp, cn]
            p.c_pos_map = cp.ctypes.data_as(C.POINTER(C.c_float))
            p.c_neg_map = cn.ctypes.data_as(C.POINTER(C.c_float))
        p.event_capacity = int(event_capacity)
        p.max_frames_per_step = int(max_frames_per_step)
        p.max_pending_intervals = int(max_pending_intervals)
        p.pixels_per_thread = int(pixels_per_thread)
        p.prefetch_frames = int(prefetch_frames)
        p.ctas_per_sm = int(ctas_per_sm)
        with torch.cuda.device(self.device):
            self.stream = stream if stream is not None else torch.cuda.current_stream()
            h = C.c_void_p()
            check(L.neurosim_evsim_create(C.byref(p), C.c_void_p(self.stream.cuda_stream),
                                          C.byref(h)))
        self._h = h
        self._keep = []          # frames of pending steps (replayed on overflow)

    # ------------------------------------------------------------------ steps
    def step(self, frames: torch.Tensor, t0_us: int, dt_us: int) -> None:
        if not (frames.is_cuda and frames.dtype == torch.float32 and frames.is_contiguous()):
            raise ValueError("frames must be a contiguous float32 CUDA tensor [T, H, W]")
        T = frames.numel() // (self.W * self.H)
        if T * self.W * self.H != frames.numel():
            raise ValueError("frames size is not a multiple of H*W")
        check(lib().neurosim_evsim_step(self._h, C.c_void_p(frames.data_ptr()), T, int(t0_us),
                                        int(dt_us)))
        self._keep.append(frames)

    def step_texture(self, scene: TextureScene, n_frames: int, t0_us: int, dt_us: int) -> None:
        """Render-fused step (library call neurosim_evsim_step_texture): the
        emission kernel renders the texture scene's frames t0 + f dt itself."""
        check(lib().neurosim_evsim_step_texture(self._h, C.byref(scene), int(n_frames), int(t0_us), int(dt_us)))

    def step_host(self, frames, t0_us: int, dt_us: int) -> None:
        """Step from HOST frames (numpy or CPU tensor, float32, C-contiguous)."""
        if isinstance(frames, torch.Tensor):
            if frames.is_cuda or frames.dtype != torch.float32 or not frames.is_contiguous():
                raise ValueError("host frames must be a contiguous float32 CPU tensor")
            ptr = frames.data_ptr()
            n = frames.numel()
        else:
            if frames.dtype != np.float32 or not frames.flags["C_CONTIGUOUS"]:
                raise ValueError("host frames must be C-contiguous float32")
            ptr = frames.ctypes.data
            n = frames.size
        T = n // (self.W * self.H)
        check(lib().neurosim_evsim_step_host(self._h, C.c_void_p(ptr), T, int(t0_us), int(dt_us)))
        self._keep.append(frames)

    # ------------------------------------------------------------------ output
    def pending(self):
        n_ev, n_seg = C.c_uint64(0), C.c_int64(0)
        check(lib().neurosim_evsim_pending(self._h, C.byref(n_ev), C.byref(n_seg)))
        return int(n_ev.value), int(n_seg.value)

    def drain(self, to: str = "cpu", out: torch.Tensor | None = None):
        """Returns (events, seg_offsets).

        to="cpu": events as a numpy uint64 array (or `out`, a preallocated
        host buffer -- a numpy uint64 array or a 64-bit CPU tensor, pinned for
        the fastest copy -- sliced to the count); to="cuda": an int64 CUDA
        tensor holding the same 64-bit records (or `out`, a preallocated int64
        CUDA tensor, sliced to the count)."""
        n_ev, n_seg = self.pending()
        seg = np.zeros(n_seg + 1, np.int64)
        n_out, n_segs = C.c_uint64(0), C.c_int64(0)
        segp = seg.ctypes.data_as(C.POINTER(C.c_int64))
        if to == "cuda":
            if out is None:
                out = torch.empty(max(n_ev, 1), dtype=torch.int64, device=self.device)
            check(lib().neurosim_evsim_drain_events(
                self._h, C.c_void_p(out.data_ptr()), out.numel(), 1, C.byref(n_out), segp,
                seg.size, C.byref(n_segs)))
            ev = out[: n_out.value]
        else:
            if out is None:
                out = np.empty(max(n_ev, 1), np.uint64)
            if isinstance(out, torch.Tensor):
                if out.is_cuda or out.element_size() != 8 or not out.is_contiguous():
                    raise ValueError("out must be a contiguous 64-bit CPU tensor")
                ptr, size = out.data_ptr(), out.numel()
            else:
                if out.dtype != np.uint64 or not out.flags["C_CONTIGUOUS"]:
                    raise ValueError("out must be a C-contiguous uint64 array")
                ptr, size = out.ctypes.data, out.size
            check(lib().neurosim_evsim_drain_events(
                self._h, C.c_void_p(ptr), size, 0, C.byref(n_out), segp, seg.size, C.byref(n_segs)))
            ev = out[: n_out.value]
        self._keep = []
        return ev, seg

    # ------------------------------------------------------------ zero copy
    def events_view(self):
        """(events, seg_offsets) without a copy: events is a CUDA int64 tensor
        (the record bits) aliasing the library's record buffer (through
        DLPack), valid until the
        next step, drain, release or close of this simulator; the events stay
        pending until release()."""
        p = C.c_void_p()
        check(lib().neurosim_evsim_events_dlpack(self._h, C.byref(p)))
        new_capsule = C.pythonapi.PyCapsule_New
        new_capsule.restype = C.py_object
        new_capsule.argtypes = [C.c_void_p, C.c_char_p, C.c_void_p]
        from torch.utils.dlpack import from_dlpack
        ev = from_dlpack(new_capsule(p, b"dltensor", None))
        n_ev, n_seg = self.pending()
        seg = np.zeros(n_seg + 1, np.int64)
        evp, n_out, n_segs = C.c_void_p(), C.c_uint64(0), C.c_int64(0)
        check(lib().neurosim_evsim_peek_events(self._h, C.byref(evp), C.byref(n_out),
                                               C.c_void_p(seg.ctypes.data), seg.size, C.byref(n_segs)))
        return ev, seg

    def release(self) -> None:
        """Clears the pending events (after events_view), copying nothing."""
        check(lib().neurosim_evsim_release_events(self._h))

    # ------------------------------------------------------------------ state
    def get_state(self):
        n = self.W * self.H
        ref = np.empty(n, np.float32)
        lp = np.empty(n, np.float32)
        tl = np.empty(n, np.uint32)
        tau, has = C.c_int64(0), C.c_int32(0)
        check(lib().neurosim_evsim_get_state(
            self._h, ref.ctypes.data_as(C.POINTER(C.c_float)),
            lp.ctypes.data_as(C.POINTER(C.c_float)), tl.ctypes.data_as(C.POINTER(C.c_uint32)),
            C.byref(tau), C.byref(has)))
        return dict(ref=ref, lprev=lp, tlast=tl, tau_prev=int(tau.value), has_prev=bool(has.value))

    def set_state(self, ref, lprev, tlast, tau_prev: int, has_prev: bool = True) -> None:
        ref = np.ascontiguousarray(ref, np.float32).reshape(-1)
        lp = np.ascontiguousarray(lprev, np.float32).reshape(-1)
        tl = np.ascontiguousarray(tlast, np.uint32).reshape(-1)
        check(lib().neurosim_evsim_set_state(
            self._h, ref.ctypes.data_as(C.POINTER(C.c_float)),
            lp.ctypes.data_as(C.POINTER(C.c_float)), tl.ctypes.data_as(C.POINTER(C.c_uint32)),
            int(tau_prev), int(bool(has_prev))))

    def thresholds(self):
        n = self.W * self.H
        cp = np.empty(n, np.float32)
        cn = np.empty(n, np.float32)
        check(lib().neurosim_evsim_get_thresholds(
            self._h, cp.ctypes.data_as(C.POINTER(C.c_float)), cn.ctypes.data_as(C.POINTER(C.c_float))))
        return cp.reshape(self.H, self.W), cn.reshape(self.H, self.W)

    def set_profiling(self, enable: bool) -> None:
        check(lib().neurosim_evsim_set_profiling(self._h, int(bool(enable))))

    def stats(self) -> dict:
        st = Stats()
        check(lib().neurosim_evsim_get_stats(self._h, C.byref(st)))
        return {k: getattr(st, k) for k, _ in Stats._fields_}

    def close(self) -> None:
        if getattr(self, "_h", None):
            lib().neurosim_evsim_destroy(self._h)
            self._h = None
            self._keep = []

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def device_log(x: torch.Tensor) -> torch.Tensor:
    """The library's FP32 log on a CUDA tensor (verification of the model's log)."""
    if not (x.is_cuda and x.dtype == torch.float32 and x.is_contiguous()):
        raise ValueError("x must be a contiguous float32 CUDA tensor")
    y = torch.empty_like(x)
    check(lib().neurosim_debug_log(C.c_void_p(x.data_ptr()), C.c_void_p(y.data_ptr()), x.numel(),
                                   C.c_void_p(torch.cuda.current_stream().cuda_stream)))
    return y


def log_intensity(frames: torch.Tensor, log_eps: float = 1e-3, out: torch.Tensor | None = None) -> torch.Tensor:
    """The event model's log intensity of raw frames (library kernel): feeding
    the result with input_is_log=True gives the events of the raw frames."""
    if not (frames.is_cuda and frames.dtype == torch.float32 and frames.is_contiguous()):
        raise ValueError("frames must be a contiguous float32 CUDA tensor")
    if out is None:
        out = torch.empty_like(frames)
    check(lib().neurosim_log_intensity(C.c_void_p(frames.data_ptr()), C.c_void_p(out.data_ptr()), frames.numel(),
                                       float(log_eps), C.c_void_p(torch.cuda.current_stream().cuda_stream)))
    return out


def lowpass_alpha(cutoff_hz: float, dt_us: int) -> float:
    """Per-frame gain of the first-order bandwidth filter for a cutoff frequency
    (library call neurosim_lowpass_alpha: 1 - exp(-2 pi f_c dt), FP32)."""
    a = C.c_float(0.0)
    check(lib().neurosim_lowpass_alpha(float(cutoff_hz), int(dt_us), C.byref(a)))
    return float(a.value)


def lowpass_log(L: torch.Tensor, alpha: float, state: torch.Tensor | None = None,
                out: torch.Tensor | None = None):
    """Sensor bandwidth limit (library kernel): first-order low-pass of the log
    frames L [T, H, W] (or [T, n]), s <- s + alpha (L - s) per frame.  With
    state None the filter starts at frame 0; pass the returned state to the
    next call to continue the stream.  out may be L (in place).  Returns
    (filtered frames, state)."""
    if not (L.is_cuda and L.dtype == torch.float32 and L.is_contiguous() and L.dim() >= 2):
        raise ValueError("L must be a contiguous float32 CUDA tensor [T, ...]")
    T = L.shape[0]
    n = L[0].numel()
    init = state is None
    if init:
        state = torch.empty(n, dtype=torch.float32, device=L.device)
    elif not (state.is_cuda and state.dtype == torch.float32 and state.is_contiguous() and state.numel() == n):
        raise ValueError("state must be a contiguous float32 CUDA tensor of one frame's size")
    if out is None:
        out = torch.empty_like(L)
    elif not (out.is_cuda and out.dtype == torch.float32 and out.is_contiguous() and out.shape == L.shape):
        raise ValueError("out must match L")
    check(lib().neurosim_lowpass_log(C.c_void_p(L.data_ptr()), C.c_void_p(out.data_ptr()), T, n, float(alpha),
                                     C.c_void_p(state.data_ptr()), int(init),
                                     C.c_void_p(torch.cuda.current_stream().cuda_stream)))
    return out, state


def _ptr_array(tensors):
    arr = (C.c_void_p * len(tensors))()
    for i, t in enumerate(tensors):
        if not (t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()):
            raise ValueError("frames must be contiguous float32 CUDA tensors")
        arr[i] = t.data_ptr()
    return arr


class EventSimBatch:
    """Many independent sensors stepped together (C ABI "Batched sensors").

    sensors: list of dicts with EventSim's sensor keywords (width, height,
    c_pos, c_neg, sigma_c, c_min, refractory_us, log_eps, input_is_log,
    seed, c_pos_map, c_neg_map).  init(first) takes one [H, W] frame per
    sensor at t0_us; set_frames(bufs, slot) registers one [T, H, W] buffer
    per sensor in a frame slot that step(slot) reads (step() may be captured
    in a CUDA graph on `stream`, one graph per slot); drain() returns the
    committed records and the offsets of the (step, sensor, interval)
    segments.
    """

    def __init__(self, sensors, frames_per_step: int, dt_us: int = 1000, t0_us: int = 0,
                 event_capacity: int = 0, max_pending_steps: int = 0,
                 pixels_per_thread: int = 0, prefetch_frames: int = 0, frame_slots: int = 0, ctas_per_sm: int = 0,
                 stream: torch.cuda.Stream | None = None):
        L = lib()
        keep = []
        arr = (Params * len(sensors))()
        for i, kw in enumerate(sensors):
            arr[i] = _params(keep=keep, **kw)
        self.dims = [(int(kw["height"]), int(kw["width"])) for kw in sensors]
        bp = BatchParams()
        L.neurosim_evsim_batch_default_params(C.byref(bp))
        bp.n_streams = len(sensors)
        bp.frames_per_step = int(frames_per_step)
        bp.dt_us = int(dt_us)
        bp.t0_us = int(t0_us)
        bp.event_capacity = int(event_capacity)
        bp.max_pending_steps = int(max_pending_steps)
        bp.pixels_per_thread = int(pixels_per_thread)
        bp.prefetch_frames = int(prefetch_frames)
        bp.ctas_per_sm = int(ctas_per_sm)
        bp.frame_slots = int(frame_slots)
        self.T = int(frames_per_step)
        self.n = len(sensors)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        h = C.c_void_p()
        check(L.neurosim_evsim_batch_create(arr, C.byref(bp), C.c_void_p(self.stream.cuda_stream),
                                            C.byref(h)))
        self._h = h
        self._bufs = {}

    def init(self, first_frames) -> None:
        self._first = list(first_frames)
        check(lib().neurosim_evsim_batch_init(self._h, _ptr_array(self._first)))

    def set_frames(self, buffers, slot: int = 0) -> None:
        for (H, W), b in zip(self.dims, buffers):
            if b.numel() != self.T * H * W:
                raise ValueError("each buffer must hold frames_per_step frames of its sensor")
        self._bufs[slot] = list(buffers)
        check(lib().neurosim_evsim_batch_set_frames(self._h, int(slot), _ptr_array(self._bufs[slot])))

    def set_frames_strided(self, frames, strides, slot: int = 0) -> None:
        """Registers sensor i's frames as views frames[i] (a CUDA float32 tensor whose
        first element is frame 0) with consecutive frames strides[i] floats apart."""
        arr = (C.c_void_p * len(frames))()
        st = (C.c_int64 * len(frames))()
        for i, (t, s_) in enumerate(zip(frames, strides)):
            if not (t.is_cuda and t.dtype == torch.float32):
                raise ValueError("frames must be float32 CUDA tensors")
            arr[i] = t.data_ptr()
            st[i] = int(s_)
        self._bufs[slot] = list(frames)
        check(lib().neurosim_evsim_batch_set_frames_strided(self._h, int(slot), arr, st))

    def step(self, slot: int = 0) -> None:
        check(lib().neurosim_evsim_batch_step(self._h, int(slot)))

    def pending(self):
        n_ev, n_seg = C.c_uint64(0), C.c_int64(0)
        check(lib().neurosim_evsim_batch_pending(self._h, C.byref(n_ev), C.byref(n_seg)))
        return int(n_ev.value), int(n_seg.value)

    def drain(self, to: str = "cpu", out: torch.Tensor | None = None, strict: bool = True):
        """(events, seg_offsets): records of the committed steps in order
        step, sensor, interval; seg_offsets has one entry per segment + 1.
        With strict=False a dropped-step condition is returned as a third
        item (the NEUROSIM status) instead of raised, after the records of
        the committed steps."""
        n_ev, n_seg = self.pending()
        seg = np.zeros(n_seg + 1, np.int64)
        n_out, ns = C.c_uint64(0), C.c_int64(0)
        segp = seg.ctypes.data_as(C.POINTER(C.c_int64))
        if to == "cuda":
            if out is None:
                out = torch.empty(max(n_ev, 1), dtype=torch.int64, device=self.stream.device)
            rc = lib().neurosim_evsim_batch_drain(self._h, C.c_void_p(out.data_ptr()), out.numel(), 1,
                                                  C.byref(n_out), segp, seg.size, C.byref(ns))
            ev = out[: n_out.value]
        else:
            buf = np.empty(max(n_ev, 1), np.uint64)
            rc = lib().neurosim_evsim_batch_drain(self._h, C.c_void_p(buf.ctypes.data), buf.size, 0,
                                                  C.byref(n_out), segp, seg.size, C.byref(ns))
            ev = buf[: n_out.value]
        if strict:
            check(rc)
            return ev, seg
        return ev, seg, rc

    def split(self, events, seg):
        """Per sensor: list over sensors of (events, offsets) of its intervals,
        steps concatenated (offsets relative to the sensor's own events)."""
        n_steps = (len(seg) - 1) // (self.n * self.T) if self.n * self.T else 0
        res = []
        for i in range(self.n):
            parts, offs, base = [], [0], 0
            for k in range(n_steps):
                s0 = (k * self.n + i) * self.T
                a, b = seg[s0], seg[s0 + self.T]
                parts.append(events[a:b])
                offs.extend(list(seg[s0 + 1: s0 + self.T + 1] - a + base))
                base += b - a
            ev = np.concatenate(parts) if parts else np.empty(0, np.uint64)
            res.append((ev, np.asarray(offs, np.int64)))
        return res

    def get_state(self, i: int):
        H, W = self.dims[i]
        n = H * W
        ref = np.empty(n, np.float32)
        lp = np.empty(n, np.float32)
        tl = np.empty(n, np.uint32)
        tau = C.c_int64(0)
        check(lib().neurosim_evsim_batch_get_state(
            self._h, int(i), ref.ctypes.data_as(C.POINTER(C.c_float)),
            lp.ctypes.data_as(C.POINTER(C.c_float)), tl.ctypes.data_as(C.POINTER(C.c_uint32)),
            C.byref(tau)))
        return dict(ref=ref, lprev=lp, tlast=tl, tau=int(tau.value))

    def thresholds(self, i: int):
        H, W = self.dims[i]
        cp = np.empty(H * W, np.float32)
        cn = np.empty(H * W, np.float32)
        check(lib().neurosim_evsim_batch_get_thresholds(
            self._h, int(i), cp.ctypes.data_as(C.POINTER(C.c_float)),
            cn.ctypes.data_as(C.POINTER(C.c_float))))
        return cp.reshape(H, W), cn.reshape(H, W)

    def counters(self):
        la, st = C.c_uint64(0), C.c_uint64(0)
        check(lib().neurosim_evsim_batch_counters(self._h, C.byref(la), C.byref(st)))
        return int(la.value), int(st.value)

    def close(self) -> None:
        if getattr(self, "_h", None):
            lib().neurosim_evsim_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def autotune(frames: torch.Tensor, dt_us: int = 1000, repeats: int = 5, cache_path: str | None = None,
             **sensor):
    """Times every emission launch shape (warp tile x CTAs per SM) on `frames`
    [T, H, W] (FP32, CUDA) for one sensor (EventSim's keywords), the median of
    `repeats` steps each, and returns (pixels_per_thread, ctas_per_sm,
    median_ms) of the fastest; `cache_path` is a JSON-lines cache keyed by GPU
    model, width, height and T that also lists every variant's time."""
    H, W = frames.shape[-2], frames.shape[-1]
    if not (frames.is_cuda and frames.dtype == torch.float32 and frames.is_contiguous()):
        raise ValueError("frames must be a contiguous float32 CUDA tensor [T, H, W]")
    keep = []
    p = _params(W, H, keep=keep, **sensor)
    ppt, ctas, ms = C.c_int32(0), C.c_int32(0), C.c_double(0.0)
    T = frames.numel() // (H * W)
    check(lib().neurosim_evsim_autotune(C.byref(p), C.c_void_p(frames.data_ptr()), T, int(dt_us),
                                        int(repeats), cache_path.encode() if cache_path else None,
                                        C.byref(ppt), C.byref(ctas), C.byref(ms)))
    return int(ppt.value), int(ctas.value), float(ms.value)


def event_f1(pred, ref, tol_us: int = 1000) -> dict:
    """Event F1 and count error of `pred` against `ref` (uint64 records, any
    order), scored by the library (C ABI neurosim_event_f1)."""
    a = np.ascontiguousarray(np.asarray(pred).view(np.uint64) if np.asarray(pred).dtype == np.int64
                             else np.asarray(pred, np.uint64))
    b = np.ascontiguousarray(np.asarray(ref).view(np.uint64) if np.asarray(ref).dtype == np.int64
                             else np.asarray(ref, np.uint64))
    counts = (C.c_int64 * 4)()
    scores = (C.c_double * 4)()
    check(lib().neurosim_event_f1(C.c_void_p(a.ctypes.data), a.size, C.c_void_p(b.ctypes.data), b.size,
                                  int(tol_us), counts, scores))
    return dict(matched=int(counts[0]), n_pred=int(counts[1]), n_ref=int(counts[2]),
                count_abs_err=int(counts[3]), precision=float(scores[0]), recall=float(scores[1]),
                f1=float(scores[2]), count_err=float(scores[3]))


class TimeSurface:
    """Time surface of one sensor on the device (C ABI neurosim_time_surface):
    S[2, H, W] evaluated at `t_ref`; update(events, t_query) decays it to
    t_query and adds the events (int64 CUDA tensor of records, t <= t_query)."""

    def __init__(self, width: int, height: int, tau_us: float = 10_000.0, device="cuda"):
        self.W, self.H, self.tau = int(width), int(height), float(tau_us)
        self.S = torch.zeros((2, self.H, self.W), dtype=torch.float32, device=device)
        self.t_ref = 0

    def update(self, events: torch.Tensor, t_query_us: int) -> torch.Tensor:
        if events.numel() and not (events.is_cuda and events.dtype == torch.int64 and events.is_contiguous()):
            raise ValueError("events must be a contiguous int64 CUDA tensor of records")
        t = C.c_int64(self.t_ref)
        check(lib().neurosim_time_surface(C.c_void_p(self.S.data_ptr()), self.W, self.H, C.byref(t),
                                          C.c_void_p(events.data_ptr() if events.numel() else 0), events.numel(),
                                          int(t_query_us), self.tau,
                                          C.c_void_p(torch.cuda.current_stream().cuda_stream)))
        self.t_ref = int(t.value)
        return self.S


def event_frames(events: torch.Tensor, width: int, height: int, t_start_us: int, window_us: int,
                 n_windows: int) -> torch.Tensor:
    """Per-window polarity counts int32 [n_windows, 2, H, W] of records (int64 CUDA tensor)."""
    out = torch.zeros((n_windows, 2, height, width), dtype=torch.int32, device=events.device)
    check(lib().neurosim_event_frames(C.c_void_p(out.data_ptr()), int(width), int(height),
                                      C.c_void_p(events.data_ptr() if events.numel() else 0), events.numel(),
                                      int(t_start_us), int(window_us), int(n_windows),
                                      C.c_void_p(torch.cuda.current_stream().cuda_stream)))
    return out


def texture_scene(width: int, height: int, salt: int, octaves: int = 4, base_period: float = 64.0,
                  gain: float = 0.5, intensity=(0.02, 1.0), velocity=(0.0, 0.0), offset=(0.0, 0.0),
                  rotation=(0.0, 1.0, 0.0), zoom=(0.0, 1.0, 0.0), rects=()) -> TextureScene:
    """A neurosim_texture_scene: rotation = (rate amplitude rad/s, period s,
    phase), zoom = (amplitude, period s, phase), rects = up to 16 tuples
    (x, y, w, h, vx, vy, value) in pixels, px/s and intensity."""
    if len(rects) > MAX_RECTS:
        raise ValueError(f"at most {MAX_RECTS} rectangles")
    s = TextureScene()
    s.width, s.height, s.salt, s.octaves = int(width), int(height), int(salt) & 0xFFFFFFFF, int(octaves)
    s.base_period, s.gain = float(base_period), float(gain)
    s.intensity_lo, s.intensity_hi = float(intensity[0]), float(intensity[1])
    s.vx, s.vy = float(velocity[0]), float(velocity[1])
    s.offset_x, s.offset_y = float(offset[0]), float(offset[1])
    s.rot_amp_rad_s, s.rot_period_s, s.rot_phase = (float(v) for v in rotation)
    s.zoom_amp, s.zoom_period_s, s.zoom_phase = (float(v) for v in zoom)
    s.n_rects = len(rects)
    for i, (x, y, w, h, vx, vy, val) in enumerate(rects):
        s.rect_x[i], s.rect_y[i], s.rect_w[i], s.rect_h[i] = float(x), float(y), float(w), float(h)
        s.rect_vx[i], s.rect_vy[i], s.rect_value[i] = float(vx), float(vy), float(val)
    return s


def render_texture(scene: TextureScene, n_frames: int, t0_us: int = 0, dt_us: int = 1000,
                   out: torch.Tensor | None = None) -> torch.Tensor:
    """Frames t0 + f dt, f < n_frames, of the scene (library renderer) as a
    CUDA float32 tensor [n_frames, height, width]."""
    if out is None:
        out = torch.empty((int(n_frames), scene.height, scene.width), dtype=torch.float32, device="cuda")
    elif not (out.is_cuda and out.dtype == torch.float32 and out.is_contiguous()
              and out.numel() == int(n_frames) * scene.width * scene.height):
        raise ValueError("out must be a contiguous float32 CUDA tensor of n_frames frames")
    check(lib().neurosim_render_texture(C.byref(scene), C.c_void_p(out.data_ptr()), int(n_frames), int(t0_us),
                                        int(dt_us), C.c_void_p(torch.cuda.current_stream().cuda_stream)))
    return out


def drain_into(sims, out: torch.Tensor):
    """Variable-length batching: drains the sensors `sims` back to back into
    one preallocated int64 CUDA tensor `out` (device-to-device copies into its
    slices).  Returns (offsets, segs): sensor i's records are
    out[offsets[i]:offsets[i + 1]], segs[i] its interval offsets.  Raises if
    `out` is too small, before draining anything."""
    if not (out.is_cuda and out.dtype == torch.int64 and out.is_contiguous() and out.dim() == 1):
        raise ValueError("out must be a contiguous 1-D int64 CUDA tensor")
    counts = [s.pending()[0] for s in sims]
    offsets = np.zeros(len(sims) + 1, np.int64)
    offsets[1:] = np.cumsum(counts)
    if offsets[-1] > out.numel():
        raise ValueError(f"out holds {out.numel()} records, the sensors have {int(offsets[-1])} pending")
    segs = []
    for i, s in enumerate(sims):
        view = out[int(offsets[i]):]
        ev, seg = s.drain(to="cuda", out=view)
        assert ev.numel() == counts[i]
        segs.append(seg)
    return offsets, segs


def leak_log(L: torch.Tensor, t0_us: int, dt_us: int, origin_us: int, rate_hz: float,
             c_pos=0.2, out: torch.Tensor | None = None) -> torch.Tensor:
    """Sensor leak (library call neurosim_leak_log) on log frames L [T, ...] at
    t0 + f dt: the log input rises by C+ * rate * (t - origin).  c_pos: a CUDA
    float32 tensor of per-pixel ON thresholds (one frame's size) or a number.
    out may be L (in place)."""
    if not (L.is_cuda and L.dtype == torch.float32 and L.is_contiguous() and L.dim() >= 2):
        raise ValueError("L must be a contiguous float32 CUDA tensor [T, ...]")
    T, n = L.shape[0], L[0].numel()
    cp_ptr, cp_u = None, 0.0
    if isinstance(c_pos, torch.Tensor):
        if not (c_pos.is_cuda and c_pos.dtype == torch.float32 and c_pos.is_contiguous() and c_pos.numel() == n):
            raise ValueError("c_pos must be a contiguous float32 CUDA tensor of one frame's size")
        cp_ptr = c_pos.data_ptr()
    else:
        cp_u = float(c_pos)
    if out is None:
        out = torch.empty_like(L)
    check(lib().neurosim_leak_log(C.c_void_p(L.data_ptr()), C.c_void_p(out.data_ptr()), T, n, int(t0_us), int(dt_us),
                                  int(origin_us), float(rate_hz), C.c_void_p(cp_ptr), cp_u,
                                  C.c_void_p(torch.cuda.current_stream().cuda_stream)))
    return out


def shot_noise(width: int, height: int, rate_hz: float, seed: int, ta0_us: int, D0_us: int, dt_us: int,
               n_intervals: int):
    """Shot-noise events (library call neurosim_shot_noise) of a step's
    intervals: (records as an int64 CUDA tensor, host offsets)."""
    seg = np.zeros(int(n_intervals) + 1, np.int64)
    n = C.c_uint64(0)
    L = lib()
    st = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = L.neurosim_shot_noise(int(width), int(height), float(rate_hz), int(seed), int(ta0_us), int(D0_us),
                               int(dt_us), int(n_intervals), None, 0, C.c_void_p(seg.ctypes.data), C.byref(n), st)
    if rc not in (0, 4) or (rc == 4 and n.value == 0):
        check(rc)
    out = torch.empty(max(1, n.value), dtype=torch.int64, device="cuda")
    check(L.neurosim_shot_noise(int(width), int(height), float(rate_hz), int(seed), int(ta0_us), int(D0_us),
                                int(dt_us), int(n_intervals), C.c_void_p(out.data_ptr()), out.numel(),
                                C.c_void_p(seg.ctypes.data), C.byref(n), st))
    return out[: n.value], seg


def merge_events(a: torch.Tensor, seg_a, b: torch.Tensor, seg_b):
    """Two event streams with the same intervals merged per interval in the
    stream's order (library call neurosim_merge_events): (int64 CUDA tensor,
    host offsets)."""
    sa = np.ascontiguousarray(seg_a, np.int64)
    sb = np.ascontiguousarray(seg_b, np.int64)
    if len(sa) != len(sb):
        raise ValueError("the streams have different interval counts")
    for t in (a, b):
        if not (t.is_cuda and t.element_size() == 8 and t.is_contiguous()):
            raise ValueError("events must be contiguous 64-bit CUDA tensors")
    out = torch.empty(max(1, int(sa[-1] + sb[-1])), dtype=torch.int64, device="cuda")
    so = np.zeros(len(sa), np.int64)
    check(lib().neurosim_merge_events(C.c_void_p(a.data_ptr()), C.c_void_p(sa.ctypes.data), C.c_void_p(b.data_ptr()),
                                      C.c_void_p(sb.ctypes.data), len(sa) - 1, C.c_void_p(out.data_ptr()),
                                      C.c_void_p(so.ctypes.data), C.c_void_p(torch.cuda.current_stream().cuda_stream)))
    return out[: int(so[-1])], so
