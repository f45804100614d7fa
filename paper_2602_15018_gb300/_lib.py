"""ctypes declarations of libneurosim_evsim.so (C ABI: include/neurosim_evsim.h).

Argument marshalling only: every step of the event path runs in the CUDA
library.  Importing the binding never falls back to anything else: if the
shared library is missing, `lib()` raises.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libneurosim_evsim.so")

NEUROSIM_OK = 0
STATUS = {1: "E_INVALID", 2: "E_CUDA", 3: "E_TIME", 4: "E_OVERFLOW", 5: "E_TIMEOUT",
          6: "E_NOMEM", 7: "E_STATE", 8: "E_IO"}

# Every exported function of the C ABI, by header section.
EXPORTS = [
    "neurosim_evsim_default_params", "neurosim_evsim_create", "neurosim_evsim_step",
    "neurosim_evsim_step_host", "neurosim_evsim_pending", "neurosim_evsim_drain_events",
    "neurosim_evsim_get_state", "neurosim_evsim_set_state", "neurosim_evsim_get_thresholds",
    "neurosim_evsim_destroy", "neurosim_last_error", "neurosim_abi_version",
    "neurosim_debug_log", "neurosim_evsim_set_profiling", "neurosim_evsim_get_stats",
    "neurosim_evsim_step_noalloc",
    "neurosim_evsim_batch_default_params", "neurosim_evsim_batch_create",
    "neurosim_evsim_batch_set_frames", "neurosim_evsim_batch_set_frames_strided", "neurosim_evsim_batch_init", "neurosim_evsim_batch_step",
    "neurosim_evsim_batch_pending", "neurosim_evsim_batch_drain", "neurosim_evsim_batch_get_state",
    "neurosim_evsim_batch_get_thresholds", "neurosim_evsim_batch_counters",
    "neurosim_evsim_batch_destroy", "neurosim_evsim_autotune", "neurosim_debug_umma_gemm",
    "neurosim_interp_param_count", "neurosim_interp_create", "neurosim_interp_forward",
    "neurosim_interp_train_step", "neurosim_interp_gradients", "neurosim_interp_get_params",
    "neurosim_interp_set_params", "neurosim_interp_save", "neurosim_interp_load",
    "neurosim_interp_launches", "neurosim_interp_destroy",
    "neurosim_event_f1", "neurosim_log_intensity", "neurosim_time_surface", "neurosim_event_frames",
    "neurosim_lowpass_log", "neurosim_lowpass_alpha", "neurosim_debug_expiring_wait",
    "neurosim_render_texture", "neurosim_evsim_step_texture",
    "neurosim_evsim_peek_events", "neurosim_evsim_release_events", "neurosim_evsim_events_dlpack",
    "neurosim_leak_log", "neurosim_shot_noise", "neurosim_merge_events",
]

MAX_RECTS = 16


class NeurosimError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


class TextureScene(C.Structure):
    """Mirror of neurosim_texture_scene."""
    _fields_ = [
        ("width", C.c_int32), ("height", C.c_int32), ("salt", C.c_uint32), ("octaves", C.c_int32),
        ("base_period", C.c_float), ("gain", C.c_float), ("intensity_lo", C.c_float), ("intensity_hi", C.c_float),
        ("vx", C.c_double), ("vy", C.c_double), ("offset_x", C.c_double), ("offset_y", C.c_double),
        ("rot_amp_rad_s", C.c_double), ("rot_period_s", C.c_double), ("rot_phase", C.c_double),
        ("zoom_amp", C.c_double), ("zoom_period_s", C.c_double), ("zoom_phase", C.c_double),
        ("n_rects", C.c_int32), ("reserved", C.c_int32),
        ("rect_x", C.c_double * MAX_RECTS), ("rect_y", C.c_double * MAX_RECTS),
        ("rect_w", C.c_double * MAX_RECTS), ("rect_h", C.c_double * MAX_RECTS),
        ("rect_vx", C.c_double * MAX_RECTS), ("rect_vy", C.c_double * MAX_RECTS),
        ("rect_value", C.c_double * MAX_RECTS),
    ]


class Params(C.Structure):
    """Mirror of neurosim_evsim_params."""
    _fields_ = [
        ("width", C.c_int32), ("height", C.c_int32),
        ("c_pos", C.c_float), ("c_neg", C.c_float), ("sigma_c", C.c_float),
        ("c_min", C.c_float), ("refractory_us", C.c_uint32), ("log_eps", C.c_float),
        ("input_is_log", C.c_int32), ("seed", C.c_uint64),
        ("c_pos_map", C.POINTER(C.c_float)), ("c_neg_map", C.POINTER(C.c_float)),
        ("event_capacity", C.c_uint64), ("max_frames_per_step", C.c_int32),
        ("max_pending_intervals", C.c_int32), ("pixels_per_thread", C.c_int32),
        ("prefetch_frames", C.c_int32), ("ctas_per_sm", C.c_int32), ("reserved", C.c_int32 * 5),
    ]


class BatchParams(C.Structure):
    """Mirror of neurosim_evsim_batch_params."""
    _fields_ = [
        ("n_streams", C.c_int32), ("frames_per_step", C.c_int32), ("dt_us", C.c_int32),
        ("max_pending_steps", C.c_int32), ("t0_us", C.c_int64), ("event_capacity", C.c_uint64),
        ("pixels_per_thread", C.c_int32), ("prefetch_frames", C.c_int32),
        ("frame_slots", C.c_int32), ("ctas_per_sm", C.c_int32), ("reserved", C.c_int32 * 4),
    ]


class Stats(C.Structure):
    """Mirror of neurosim_evsim_stats."""
    _fields_ = [("steps", C.c_uint64), ("kernel_launches", C.c_uint64),
                ("px_frames", C.c_uint64), ("events_drained", C.c_uint64),
                ("timed_steps", C.c_uint64), ("emit_ms", C.c_double), ("sort_ms", C.c_double)]


_lock = threading.Lock()
_lib = None


def lib():
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise ImportError(
                    f"{LIB_PATH} is not built; run `python -c 'import __graft_entry__ as g; "
                    "g.build()'` (needs nvcc)")
            L = C.CDLL(LIB_PATH)
            vp, i32, i64, u64 = C.c_void_p, C.c_int32, C.c_int64, C.c_uint64
            f32p, u32p = C.POINTER(C.c_float), C.POINTER(C.c_uint32)
            L.neurosim_evsim_default_params.restype = None
            L.neurosim_evsim_default_params.argtypes = [C.POINTER(Params)]
            L.neurosim_evsim_create.restype = C.c_int
            L.neurosim_evsim_create.argtypes = [C.POINTER(Params), vp, C.POINTER(vp)]
            L.neurosim_evsim_step.restype = C.c_int
            L.neurosim_evsim_step.argtypes = [vp, vp, i32, i64, i32]
            L.neurosim_evsim_step_host.restype = C.c_int
            L.neurosim_evsim_step_host.argtypes = [vp, vp, i32, i64, i32]
            L.neurosim_evsim_pending.restype = C.c_int
            L.neurosim_evsim_pending.argtypes = [vp, C.POINTER(u64), C.POINTER(i64)]
            L.neurosim_evsim_drain_events.restype = C.c_int
            L.neurosim_evsim_drain_events.argtypes = [vp, vp, u64, i32, C.POINTER(u64),
                                                      C.POINTER(i64), i64, C.POINTER(i64)]
            L.neurosim_evsim_get_state.restype = C.c_int
            L.neurosim_evsim_get_state.argtypes = [vp, f32p, f32p, u32p, C.POINTER(i64),
                                                   C.POINTER(i32)]
            L.neurosim_evsim_set_state.restype = C.c_int
            L.neurosim_evsim_set_state.argtypes = [vp, f32p, f32p, u32p, i64, i32]
            L.neurosim_evsim_get_thresholds.restype = C.c_int
            L.neurosim_evsim_get_thresholds.argtypes = [vp, f32p, f32p]
            L.neurosim_evsim_destroy.restype = None
            L.neurosim_evsim_destroy.argtypes = [vp]
            L.neurosim_last_error.restype = C.c_char_p
            L.neurosim_last_error.argtypes = []
            L.neurosim_abi_version.restype = C.c_int32
            L.neurosim_abi_version.argtypes = []
            L.neurosim_debug_log.restype = C.c_int
            L.neurosim_debug_log.argtypes = [vp, vp, i64, vp]
            L.neurosim_evsim_set_profiling.restype = C.c_int
            L.neurosim_evsim_set_profiling.argtypes = [vp, i32]
            L.neurosim_evsim_get_stats.restype = C.c_int
            L.neurosim_evsim_get_stats.argtypes = [vp, C.POINTER(Stats)]
            L.neurosim_evsim_step_noalloc.restype = C.c_int
            L.neurosim_evsim_step_noalloc.argtypes = [
                vp, i32, i32, i32, i64, i32, vp, vp, C.c_float, C.c_float, C.c_uint32,
                C.c_float, i32, vp, vp, vp, vp, vp, vp, i32, i64, vp, u64, vp,
                C.POINTER(u64), vp]
            L.neurosim_evsim_batch_default_params.restype = None
            L.neurosim_evsim_batch_default_params.argtypes = [C.POINTER(BatchParams)]
            L.neurosim_evsim_batch_create.restype = C.c_int
            L.neurosim_evsim_batch_create.argtypes = [C.POINTER(Params), C.POINTER(BatchParams), vp,
                                                      C.POINTER(vp)]
            L.neurosim_evsim_batch_set_frames.restype = C.c_int
            L.neurosim_evsim_batch_set_frames.argtypes = [vp, i32, C.POINTER(vp)]
            L.neurosim_evsim_batch_set_frames_strided.restype = C.c_int
            L.neurosim_evsim_batch_set_frames_strided.argtypes = [vp, i32, C.POINTER(vp), C.POINTER(i64)]
            L.neurosim_evsim_batch_init.restype = C.c_int
            L.neurosim_evsim_batch_init.argtypes = [vp, C.POINTER(vp)]
            L.neurosim_evsim_batch_step.restype = C.c_int
            L.neurosim_evsim_batch_step.argtypes = [vp, i32]
            L.neurosim_evsim_batch_pending.restype = C.c_int
            L.neurosim_evsim_batch_pending.argtypes = [vp, C.POINTER(u64), C.POINTER(i64)]
            L.neurosim_evsim_batch_drain.restype = C.c_int
            L.neurosim_evsim_batch_drain.argtypes = [vp, vp, u64, i32, C.POINTER(u64),
                                                     C.POINTER(i64), i64, C.POINTER(i64)]
            L.neurosim_evsim_batch_get_state.restype = C.c_int
            L.neurosim_evsim_batch_get_state.argtypes = [vp, i32, f32p, f32p, u32p, C.POINTER(i64)]
            L.neurosim_evsim_batch_get_thresholds.restype = C.c_int
            L.neurosim_evsim_batch_get_thresholds.argtypes = [vp, i32, f32p, f32p]
            L.neurosim_evsim_batch_counters.restype = C.c_int
            L.neurosim_evsim_batch_counters.argtypes = [vp, C.POINTER(u64), C.POINTER(u64)]
            L.neurosim_evsim_batch_destroy.restype = None
            L.neurosim_evsim_batch_destroy.argtypes = [vp]
            L.neurosim_evsim_autotune.restype = C.c_int
            L.neurosim_evsim_autotune.argtypes = [C.POINTER(Params), vp, i32, i32, i32, C.c_char_p,
                                                  C.POINTER(i32), C.POINTER(i32),
                                                  C.POINTER(C.c_double)]
            L.neurosim_debug_umma_gemm.restype = C.c_int
            L.neurosim_debug_umma_gemm.argtypes = [i32, i32, i32, i32, vp, vp, vp, vp]
            L.neurosim_interp_param_count.restype = C.c_int64
            L.neurosim_interp_param_count.argtypes = []
            L.neurosim_interp_create.restype = C.c_int
            L.neurosim_interp_create.argtypes = [i32, i32, i32, u64, vp, C.POINTER(vp)]
            L.neurosim_interp_forward.restype = C.c_int
            L.neurosim_interp_forward.argtypes = [vp, vp, vp, i32, i32, i32, vp]
            L.neurosim_interp_train_step.restype = C.c_int
            L.neurosim_interp_train_step.argtypes = [vp, vp, i32, i32, i32, C.c_float, C.c_float,
                                                     C.POINTER(C.c_float)]
            L.neurosim_interp_gradients.restype = C.c_int
            L.neurosim_interp_gradients.argtypes = [vp, vp, i32, i32, i32, vp, C.POINTER(C.c_float)]
            L.neurosim_interp_get_params.restype = C.c_int
            L.neurosim_interp_get_params.argtypes = [vp, vp, i64]
            L.neurosim_interp_set_params.restype = C.c_int
            L.neurosim_interp_set_params.argtypes = [vp, vp, i64]
            L.neurosim_interp_save.restype = C.c_int
            L.neurosim_interp_save.argtypes = [vp, C.c_char_p, i32]
            L.neurosim_interp_load.restype = C.c_int
            L.neurosim_interp_load.argtypes = [vp, C.c_char_p]
            L.neurosim_interp_launches.restype = C.c_int
            L.neurosim_interp_launches.argtypes = [vp, C.POINTER(u64)]
            L.neurosim_interp_destroy.restype = None
            L.neurosim_interp_destroy.argtypes = [vp]
            L.neurosim_time_surface.restype = C.c_int
            L.neurosim_time_surface.argtypes = [vp, i32, i32, C.POINTER(i64), vp, i64, i64, C.c_float, vp]
            L.neurosim_event_frames.restype = C.c_int
            L.neurosim_event_frames.argtypes = [vp, i32, i32, vp, i64, i64, i64, i32, vp]
            L.neurosim_lowpass_log.restype = C.c_int
            L.neurosim_lowpass_log.argtypes = [vp, vp, i32, i64, C.c_float, vp, i32, vp]
            L.neurosim_leak_log.restype = C.c_int
            L.neurosim_leak_log.argtypes = [vp, vp, i32, i64, i64, i32, i64, C.c_double, vp, C.c_float, vp]
            L.neurosim_shot_noise.restype = C.c_int
            L.neurosim_shot_noise.argtypes = [i32, i32, C.c_double, u64, i64, i32, i32, i32, vp, u64, vp,
                                              C.POINTER(u64), vp]
            L.neurosim_merge_events.restype = C.c_int
            L.neurosim_merge_events.argtypes = [vp, vp, vp, vp, i32, vp, vp, vp]
            L.neurosim_evsim_peek_events.restype = C.c_int
            L.neurosim_evsim_peek_events.argtypes = [vp, C.POINTER(vp), C.POINTER(u64), vp, i64, C.POINTER(i64)]
            L.neurosim_evsim_release_events.restype = C.c_int
            L.neurosim_evsim_release_events.argtypes = [vp]
            L.neurosim_evsim_events_dlpack.restype = C.c_int
            L.neurosim_evsim_events_dlpack.argtypes = [vp, C.POINTER(vp)]
            L.neurosim_render_texture.restype = C.c_int
            L.neurosim_render_texture.argtypes = [C.POINTER(TextureScene), vp, i32, i64, i32, vp]
            L.neurosim_evsim_step_texture.restype = C.c_int
            L.neurosim_evsim_step_texture.argtypes = [vp, C.POINTER(TextureScene), i32, i64, i32]
            L.neurosim_debug_expiring_wait.restype = C.c_int
            L.neurosim_debug_expiring_wait.argtypes = [i32, u64, vp]
            L.neurosim_lowpass_alpha.restype = C.c_int
            L.neurosim_lowpass_alpha.argtypes = [C.c_double, i32, C.POINTER(C.c_float)]
            L.neurosim_log_intensity.restype = C.c_int
            L.neurosim_log_intensity.argtypes = [vp, vp, i64, C.c_float, vp]
            L.neurosim_event_f1.restype = C.c_int
            L.neurosim_event_f1.argtypes = [vp, i64, vp, i64, i64, C.POINTER(i64), C.POINTER(C.c_double)]
            _lib = L
    return _lib


def check(rc: int) -> None:
    if rc != NEUROSIM_OK:
        msg = lib().neurosim_last_error()
        raise NeurosimError(rc, msg.decode() if msg else "")
