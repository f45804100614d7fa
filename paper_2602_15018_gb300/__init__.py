"""GB300-native event-generation path of Neurosim (arXiv 2602.15018).

The compute path is the CUDA library libneurosim_evsim.so (C ABI in
include/neurosim_evsim.h); this package only binds it.
"""
from .evsim import (EventSim, EventSimBatch, TimeSurface, autotune, device_log, event_f1,  # noqa: F401
                    drain_into, event_frames, leak_log, log_intensity, lowpass_alpha, lowpass_log,
                    merge_events, render_texture, shot_noise, texture_scene)
from .interp import Interpolator  # noqa: F401
from ._lib import NeurosimError, lib  # noqa: F401

__all__ = ["EventSim", "EventSimBatch", "Interpolator", "autotune", "device_log", "event_f1", "drain_into", "leak_log", "log_intensity", "merge_events", "shot_noise", "lowpass_alpha", "lowpass_log", "render_texture", "texture_scene", "TimeSurface", "event_frames", "NeurosimError", "lib"]
