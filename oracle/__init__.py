"""Oracle for the Neurosim event-generation path (test infrastructure only).

A plain, slow, single-threaded CPU statement of the contrast-threshold event
model of arXiv 2602.15018 (Sec. 1 event tuple; Sec. 2, paragraph "Neurosim
simulates event cameras at multi-kilohertz rates"), written in C
(``evsim_oracle.c``) and wrapped here with ctypes.  Only the test suite, the
smoke check and the benchmark's CPU-baseline leg may import this package; the
CUDA library never does, and the two share no code.

Functions (each follows the passage and reading named in the C source):
  mylog                 project FP32 log (reading R1)
  lowpass_alpha         per-frame gain of the bandwidth filter (reading R13)
  lowpass_log           sensor bandwidth filter on log frames (reading R13)
  leak_log              sensor leak as the drift of the log input (reading R14)
  shot_noise            shot-noise events per tile and interval (reading R15)
  merge_events          two event streams merged per interval (reading R8)
  splitmix64_at         SplitMix64 output i of a seeded stream (reading R6)
  normal_ih12           Irwin-Hall(12) normal draw (reading R6)
  threshold_maps        per-pixel thresholds max(c_min, C + sigma z) (R6)
  OracleSim             stateful FP32-mirrored (or FP64) event simulator
  banded_step           OracleSim over row bands on several host threads
  time_surface          Eq. for the time surface in the supplementary RL
                        section (S <- S exp(-dt/tau) + 1)
  event_frames          per-pixel polarity histograms over fixed windows
  match_f1              event-stream F1 and count error (scoring reading)

Parity unpinned: none of the functions above lacks a pin; see tests/.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SRC = [os.path.join(_HERE, "evsim_oracle.c"), os.path.join(_HERE, "consumers_oracle.c")]
_LIB_PATH = os.path.join(_BUILD, "libevsim_oracle.so")
_lock = threading.Lock()
_lib = None

CFLAGS = ["-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared"]


def build(force: bool = False) -> str:
    """Compile the oracle into oracle/_build/libevsim_oracle.so (gcc, no FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    srcs = [s for s in _SRC if os.path.exists(s)]
    newest = max(os.path.getmtime(s) for s in srcs)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < newest:
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", *CFLAGS, "-o", tmp, *srcs, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _configure(L):
    """Declare the C signatures on a loaded oracle library."""
    f32p = C.POINTER(C.c_float)
    f64p = C.POINTER(C.c_double)
    i64p = C.POINTER(C.c_int64)
    i32p = C.POINTER(C.c_int32)
    u64p = C.POINTER(C.c_uint64)
    u64pp = C.POINTER(u64p)
    i64pp = C.POINTER(C.POINTER(C.c_int64))
    L.oracle_mylog.restype = C.c_float
    L.oracle_mylog.argtypes = [C.c_float]
    L.oracle_lowpass_log.restype = C.c_int
    L.oracle_lowpass_log.argtypes = [f32p, f32p, C.c_int32, C.c_int64, C.c_float, f32p, C.c_int32]
    L.oracle_leak_log.restype = C.c_int
    L.oracle_leak_log.argtypes = [f32p, f32p, C.c_int32, C.c_int64, C.c_int64, C.c_int32, C.c_int64,
                                  C.c_double, f32p, C.c_float]
    L.oracle_shot_noise.restype = C.c_int
    L.oracle_shot_noise.argtypes = [C.c_int32, C.c_int32, C.c_double, C.c_uint64, C.c_int64, C.c_int32,
                                    C.c_int32, C.c_int32, u64pp, i64p, i64pp]
    L.oracle_merge_events.restype = C.c_int
    L.oracle_merge_events.argtypes = [u64p, i64p, u64p, i64p, C.c_int32, u64p, i64p]
    L.oracle_lowpass_alpha.restype = C.c_float
    L.oracle_lowpass_alpha.argtypes = [C.c_double, C.c_int32]
    L.oracle_mylog_batch.restype = None
    L.oracle_mylog_batch.argtypes = [f32p, f32p, C.c_int64]
    L.oracle_mylog_max_ulp.restype = C.c_double
    L.oracle_mylog_max_ulp.argtypes = [C.c_uint32, C.c_uint32, C.c_uint32,
                                       C.POINTER(C.c_uint32)]
    L.oracle_splitmix64_at.restype = C.c_uint64
    L.oracle_splitmix64_at.argtypes = [C.c_uint64, C.c_uint64]
    L.oracle_normal_ih12.restype = C.c_float
    L.oracle_normal_ih12.argtypes = [C.c_uint64, C.c_uint64]
    L.oracle_threshold_maps.restype = None
    L.oracle_threshold_maps.argtypes = [C.c_int32, C.c_int32, C.c_float, C.c_float,
                                        C.c_float, C.c_float, C.c_uint64, f32p, f32p]
    common = [C.c_int32, C.c_int32, f32p, C.c_int32, C.c_int64, C.c_int32, f32p, f32p,
              C.c_uint32]
    L.oracle_evsim_step_f32.restype = C.c_int
    L.oracle_evsim_step_f32.argtypes = common + [
        C.c_float, C.c_int32, f32p, f32p, i64p, i32p, i64p, u64pp, i64p, i64pp, i32p]
    L.oracle_evsim_step_f64.restype = C.c_int
    L.oracle_evsim_step_f64.argtypes = common + [
        C.c_double, C.c_int32, f64p, f64p, i64p, i32p, i64p, u64pp, i64p, i64pp, i32p]
    L.oracle_free.restype = None
    L.oracle_free.argtypes = [C.c_void_p]
    L.oracle_time_surface.restype = C.c_int
    L.oracle_time_surface.argtypes = [C.c_int32, C.c_int32, u64p, C.c_int64, f64p, i64p,
                                      C.c_double]
    L.oracle_event_frames.restype = C.c_int
    L.oracle_event_frames.argtypes = [C.c_int32, C.c_int32, u64p, C.c_int64, C.c_int64,
                                      C.c_int64, C.c_int32, i32p]
    L.oracle_match_f1.restype = C.c_int
    L.oracle_match_f1.argtypes = [C.c_int32, C.c_int32, u64p, C.c_int64, u64p, C.c_int64,
                                  C.c_int64, i64p, f64p]
    return L


def load_library(path: str):
    """Load an oracle build from `path` (the default build, or a test's variant)."""
    return _configure(C.CDLL(path))


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = load_library(build())
    return _lib


def _p(a, ct):
    return a.ctypes.data_as(C.POINTER(ct))


# --------------------------------------------------------------------------
# log, random draws, thresholds
# --------------------------------------------------------------------------
def lowpass_log(L, alpha, state=None, library=None):
    """Sensor bandwidth filter (reading R13) over log frames L [T, ...]; returns
    (filtered frames, state).  state None starts the filter at frame 0."""
    x = np.ascontiguousarray(L, dtype=np.float32)
    T = x.shape[0]
    n = int(x[0].size) if T else (0 if state is None else int(np.asarray(state).size))
    init = state is None
    st = np.zeros(n, np.float32) if init else np.ascontiguousarray(state, np.float32).reshape(-1).copy()
    out = np.empty_like(x)
    rc = (library or lib()).oracle_lowpass_log(_p(x, C.c_float), _p(out, C.c_float), T, n, float(alpha),
                                               _p(st, C.c_float), int(init))
    if rc != 0:
        raise OracleError(_ERR.get(rc, f"error {rc}"))
    return out, st


def lowpass_alpha(cutoff_hz, dt_us, library=None) -> np.float32:
    """Per-frame gain of the bandwidth filter (reading R13), 1 - exp(-2 pi f_c dt),
    rounded once to FP32; raises for f_c <= 0, dt_us < 1 or a gain that rounds to 0."""
    a = np.float32((library or lib()).oracle_lowpass_alpha(float(cutoff_hz), int(dt_us)))
    if not a > 0:
        raise OracleError("invalid cutoff or frame spacing")
    return a


def leak_log(L, t0_us, dt_us, origin_us, rate_hz, cpos=None, cpos_u=0.2, library=None):
    """Sensor leak (reading R14) on log frames L [T, ...] at t0 + k dt: the log
    input rises by C+ * rate * (t - origin); cpos: per-pixel ON thresholds."""
    x = np.ascontiguousarray(L, dtype=np.float32)
    T = x.shape[0]
    n = int(x[0].size) if T else 0
    out = np.empty_like(x)
    cp = None if cpos is None else np.ascontiguousarray(cpos, np.float32).reshape(-1)
    rc = (library or lib()).oracle_leak_log(_p(x, C.c_float), _p(out, C.c_float), T, n, int(t0_us), int(dt_us),
                                            int(origin_us), float(rate_hz),
                                            None if cp is None else _p(cp, C.c_float), float(cpos_u))
    if rc != 0:
        raise OracleError(_ERR.get(rc, f"error {rc}"))
    return out


def shot_noise(width, height, rate_hz, seed, ta0_us, D0_us, dt_us, n_intervals, library=None):
    """Shot-noise events (reading R15) of n_intervals intervals (the first
    D0_us long from ta0_us, then dt_us each): (records uint64, offsets int64)."""
    L = library or lib()
    evp = C.POINTER(C.c_uint64)()
    segp = C.POINTER(C.c_int64)()
    n = C.c_int64(0)
    rc = L.oracle_shot_noise(int(width), int(height), float(rate_hz), int(seed), int(ta0_us), int(D0_us),
                             int(dt_us), int(n_intervals), C.byref(evp), C.byref(n), C.byref(segp))
    if rc != 0:
        raise OracleError(_ERR.get(rc, f"error {rc}"))
    try:
        ev = np.ctypeslib.as_array(evp, shape=(n.value,)).copy() if n.value else np.zeros(0, np.uint64)
        seg = np.ctypeslib.as_array(segp, shape=(int(n_intervals) + 1,)).copy()
    finally:
        L.oracle_free(C.cast(evp, C.c_void_p))
        L.oracle_free(C.cast(segp, C.c_void_p))
    return ev, seg


def merge_events(a, seg_a, b, seg_b, library=None):
    """Two interval-structured streams merged per interval in record order (R8)."""
    a = np.ascontiguousarray(a, np.uint64)
    b = np.ascontiguousarray(b, np.uint64)
    sa = np.ascontiguousarray(seg_a, np.int64)
    sb = np.ascontiguousarray(seg_b, np.int64)
    if len(sa) != len(sb):
        raise OracleError("streams have different interval counts")
    out = np.empty(a.size + b.size, np.uint64)
    so = np.empty(len(sa), np.int64)
    rc = (library or lib()).oracle_merge_events(_p(a, C.c_uint64), _p(sa, C.c_int64), _p(b, C.c_uint64),
                                                _p(sb, C.c_int64), len(sa) - 1, _p(out, C.c_uint64),
                                                _p(so, C.c_int64))
    if rc != 0:
        raise OracleError(_ERR.get(rc, f"error {rc}"))
    return out, so


def mylog(x, library=None) -> np.ndarray:
    x = np.ascontiguousarray(x, dtype=np.float32)
    y = np.empty_like(x)
    (library or lib()).oracle_mylog_batch(_p(x, C.c_float), _p(y, C.c_float), x.size)
    return y


def mylog_max_ulp(lo_bits: int, hi_bits: int, stride: int = 1, library=None):
    wb = C.c_uint32(0)
    e = (library or lib()).oracle_mylog_max_ulp(lo_bits, hi_bits, stride, C.byref(wb))
    return e, wb.value


def splitmix64_at(seed: int, index: int) -> int:
    return int(lib().oracle_splitmix64_at(seed, index))


def normal_ih12(seed: int, slot: int) -> float:
    return float(lib().oracle_normal_ih12(seed, slot))


def threshold_maps(width, height, c_pos, c_neg, sigma, c_min, seed, library=None):
    n = width * height
    cp = np.empty(n, np.float32)
    cn = np.empty(n, np.float32)
    (library or lib()).oracle_threshold_maps(width, height, c_pos, c_neg, sigma, c_min, seed,
                                _p(cp, C.c_float), _p(cn, C.c_float))
    return cp.reshape(height, width), cn.reshape(height, width)


# --------------------------------------------------------------------------
# Packed records: [63:32] t | [31:17] y | [16:1] x | [0] p
# --------------------------------------------------------------------------
def unpack(ev: np.ndarray):
    ev = np.asarray(ev, dtype=np.uint64)
    t = (ev >> np.uint64(32)).astype(np.int64)
    y = ((ev >> np.uint64(17)) & np.uint64(0x7FFF)).astype(np.int32)
    x = ((ev >> np.uint64(1)) & np.uint64(0xFFFF)).astype(np.int32)
    p = (ev & np.uint64(1)).astype(np.int8)
    return t, x, y, p


def pack(t, x, y, p) -> np.ndarray:
    t = np.asarray(t, np.uint64)
    return ((t << np.uint64(32)) | (np.asarray(y, np.uint64) << np.uint64(17))
            | (np.asarray(x, np.uint64) << np.uint64(1)) | np.asarray(p, np.uint64))


class OracleError(RuntimeError):
    pass


_ERR = {1: "invalid argument", 2: "out of memory", 3: "time error"}


class OracleSim:
    """Stateful oracle event simulator for one sensor (FP32-mirrored or FP64).

    step(frames, t0, dt) returns (events uint64[n], seg_offsets int64[n_seg+1])
    for the intervals that step closes, in output order (reading R8).
    """

    def __init__(self, width, height, c_pos=0.2, c_neg=0.2, sigma_c=0.0, c_min=0.01,
                 refractory_us=0, log_eps=1e-3, input_is_log=False, seed=0,
                 c_pos_map=None, c_neg_map=None, precision="f32", library=None):
        self.W, self.H = int(width), int(height)
        self._L = library
        n = self.W * self.H
        if c_pos_map is not None:
            self.cpos = np.ascontiguousarray(c_pos_map, np.float32).reshape(-1).copy()
            self.cneg = np.ascontiguousarray(c_neg_map, np.float32).reshape(-1).copy()
        else:
            cp, cn = threshold_maps(self.W, self.H, c_pos, c_neg, sigma_c, c_min, seed,
                                    library=library)
            self.cpos, self.cneg = cp.reshape(-1), cn.reshape(-1)
        self.refractory_us = int(refractory_us)
        self.log_eps = float(log_eps)
        self.input_is_log = int(bool(input_is_log))
        self.precision = precision
        ft = np.float32 if precision == "f32" else np.float64
        self.ref = np.zeros(n, ft)
        self.lprev = np.zeros(n, ft)
        self.tlast = np.full(n, -1, np.int64)
        self.has_prev = C.c_int32(0)
        self.tau_prev = C.c_int64(0)

    def step(self, frames, t0: int, dt: int):
        L = self._L or lib()
        fr = np.ascontiguousarray(frames, dtype=np.float32)
        T = 0 if fr.size == 0 else fr.reshape(-1, self.H * self.W).shape[0]
        evp = C.POINTER(C.c_uint64)()
        segp = C.POINTER(C.c_int64)()
        n_ev = C.c_int64(0)
        n_seg = C.c_int32(0)
        if self.precision == "f32":
            fn, ct, eps = L.oracle_evsim_step_f32, C.c_float, C.c_float(self.log_eps)
        else:
            fn, ct, eps = L.oracle_evsim_step_f64, C.c_double, C.c_double(self.log_eps)
        rc = fn(self.W, self.H, _p(fr, C.c_float), T, int(t0), int(dt),
                _p(self.cpos, C.c_float), _p(self.cneg, C.c_float), self.refractory_us,
                eps, self.input_is_log, _p(self.ref, ct), _p(self.lprev, ct),
                _p(self.tlast, C.c_int64), C.byref(self.has_prev), C.byref(self.tau_prev),
                C.byref(evp), C.byref(n_ev), C.byref(segp), C.byref(n_seg))
        if rc != 0:
            raise OracleError(_ERR.get(rc, f"error {rc}"))
        try:
            ev = np.ctypeslib.as_array(evp, shape=(n_ev.value,)).copy() if n_ev.value else \
                np.zeros(0, np.uint64)
            seg = np.ctypeslib.as_array(segp, shape=(n_seg.value + 1,)).copy()
        finally:
            L.oracle_free(C.cast(evp, C.c_void_p))
            L.oracle_free(C.cast(segp, C.c_void_p))
        return ev, seg

    @property
    def tau(self) -> int:
        return int(self.tau_prev.value)


def banded_step(frames, width, height, t0: int, dt: int, c_pos_map, c_neg_map, refractory_us=0,
                log_eps=1e-3, input_is_log=False, threads=None, library=None):
    """One step of fresh sensors' oracle (FP32), run band-parallel: the frames'
    rows are split into bands, each band is simulated by its own OracleSim on
    its own host thread (the ctypes call releases the interpreter lock), and
    the bands' records are merged into the output order of reading R8.
    Pixels are independent in the model, so the result equals one OracleSim
    over the whole frame (checked in the oracle's tests).  Returns (events,
    seg_offsets, threads used, final state: dict of ref, lprev (FP32) and
    tlast (int64, -1 = none) over all pixels)."""
    from concurrent.futures import ThreadPoolExecutor
    fr = np.asarray(frames, dtype=np.float32).reshape(-1, height, width)
    T = fr.shape[0]
    cp = np.ascontiguousarray(c_pos_map, np.float32).reshape(height, width)
    cn = np.ascontiguousarray(c_neg_map, np.float32).reshape(height, width)
    n_thr = max(1, min(int(threads or os.cpu_count() or 1), height))
    edges = np.linspace(0, height, n_thr + 1).astype(int)
    L = library or lib()

    def band(b):
        y0, y1 = int(edges[b]), int(edges[b + 1])
        sim = OracleSim(width, y1 - y0, c_pos_map=cp[y0:y1], c_neg_map=cn[y0:y1], refractory_us=refractory_us,
                        log_eps=log_eps, input_is_log=input_is_log, library=L)
        ev, seg = sim.step(np.ascontiguousarray(fr[:, y0:y1, :]), t0, dt)
        return ev + (np.uint64(y0) << np.uint64(17)), seg, sim

    with ThreadPoolExecutor(max_workers=n_thr) as ex:
        parts = list(ex.map(band, range(n_thr)))
    state = {k: np.concatenate([getattr(sim, k) for _, _, sim in parts]) for k in ("ref", "lprev", "tlast")}
    parts = [(ev, seg) for ev, seg, _ in parts]
    n_seg = len(parts[0][1]) - 1
    rec = np.concatenate([ev for ev, _ in parts]) if parts else np.zeros(0, np.uint64)
    j = np.concatenate([np.repeat(np.arange(n_seg), np.diff(seg)) for _, seg in parts])
    order = np.lexsort((rec, j))
    seg = np.zeros(n_seg + 1, np.int64)
    seg[1:] = np.cumsum(np.bincount(j, minlength=n_seg))
    return rec[order], seg, n_thr, state


# --------------------------------------------------------------------------
# Consumers and scoring
# --------------------------------------------------------------------------
def time_surface(width, height, events, tau_us=10_000.0, S=None, last=None, library=None):
    """Time surface of the supplementary RL section; returns (S[2,H,W], last[2,H,W])."""
    ev = np.ascontiguousarray(events, np.uint64)
    if S is None:
        S = np.zeros((2, height, width), np.float64)
        last = np.full((2, height, width), -1, np.int64)
    rc = (library or lib()).oracle_time_surface(width, height, _p(ev, C.c_uint64), ev.size,
                                   _p(S, C.c_double), _p(last, C.c_int64), float(tau_us))
    if rc:
        raise OracleError("time_surface: bad argument")
    return S, last


def event_frames(width, height, events, t_start, win_us, n_win, library=None):
    """Per-pixel polarity counts over n_win windows: int32[n_win, 2, H, W]."""
    ev = np.ascontiguousarray(events, np.uint64)
    out = np.zeros((n_win, 2, height, width), np.int32)
    rc = (library or lib()).oracle_event_frames(width, height, _p(ev, C.c_uint64), ev.size, int(t_start),
                                   int(win_us), int(n_win), _p(out, C.c_int32))
    if rc:
        raise OracleError("event_frames: bad argument")
    return out


def match_f1(width, height, pred, ref, tol_us=1000, library=None):
    """Event F1 and count error of `pred` against `ref` (scoring reading)."""
    a = np.ascontiguousarray(pred, np.uint64)
    b = np.ascontiguousarray(ref, np.uint64)
    counts = np.zeros(4, np.int64)
    scores = np.zeros(4, np.float64)
    rc = (library or lib()).oracle_match_f1(width, height, _p(a, C.c_uint64), a.size, _p(b, C.c_uint64),
                               b.size, int(tol_us), _p(counts, C.c_int64),
                               _p(scores, C.c_double))
    if rc:
        raise OracleError("match_f1 failed")
    return dict(matched=int(counts[0]), n_pred=int(counts[1]), n_ref=int(counts[2]),
                count_abs_err=int(counts[3]), precision=float(scores[0]),
                recall=float(scores[1]), f1=float(scores[2]), count_err=float(scores[3]))
