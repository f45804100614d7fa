#!/usr/bin/env python
"""Benchmark of the event-generation path on GB300 (one JSON line on stdout).

Workload (default, "hd"): 1280x720 FP32 intensity frames, 2000 frames at
1000 FPS per step; value-noise texture under an affine camera path with 16
moving occluders; C+ 0.2, C- 0.25, per-pixel threshold sigma 0.03, refractory
100 us.  One step = emission + interval sort + drain of the step's events to
a device buffer, over frames already resident in HBM (7.4 GB per step, far
larger than L2, so no L2 flush is needed between steps).

Metric: Mpixel-frames/s (whole job, all ranks) with events/s alongside.
Roofline: the emission kernel (the dominant one), algorithmic bytes per
launch = 4 B per pixel-frame read + 32 B per pixel of state and thresholds
+ 4 B per event key written, over its CUDA-event duration on the library's
stream, against the measured HBM copy bandwidth.

--impl reference runs the oracle (the plain CPU restatement of the model) on
a bounded sample of the same workload on the host cores.

Multi-GPU (torchrun): independent replicas, one sensor stream per rank with
its own seed; no collective on the data path (the barrier and the max over
ranks of the timed region use torch.distributed only for timing).
"""
from __future__ import annotations

import argparse
import ctypes as C
import datetime as _dt
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402
import torch  # noqa: E402

import scenes  # noqa: E402

DT = 1000
HD = dict(W=1280, H=720, T=2000)
CONFIG2_SIM = dict(c_pos=0.2, c_neg=0.25, sigma_c=0.03, c_min=0.01, refractory_us=100, seed=1)
C1 = dict(W=240, H=180, T=200)
CONFIG1_SIM = dict(c_pos=0.2, c_neg=0.2, sigma_c=0.0, c_min=0.01, refractory_us=0, seed=0)
FALLBACK_HBM_GBS = 6800.0
METRIC = "Mpixel-frames/s (events/s alongside), plain event simulation"


def render_config2(seed: int = 0, device="cuda", n_frames: int = HD["T"]) -> torch.Tensor:
    sc = scenes.TextureScene(HD["W"], HD["H"], seed=seed)
    return scenes.render_frames(sc, n_frames, device=device, chunk=32)


# Batched workload: 256 independent sensors, resolutions 346x260 / 640x480 /
# 1280x720 by index mod 3, texture scenes as the HD workload, per-sensor
# C+ and C- drawn from U[0.15, 0.35], sigma 0.03, refractory 100 us; steps of
# 125 frames at 1000 FPS (a 500-frame clip is 4 steps), each a CUDA-graph
# replay of one batched step.
BATCH = dict(n=256, sizes=((346, 260), (640, 480), (1280, 720)), T=125)


def batch_sensors(seed: int = 0, n: int = BATCH["n"]):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        W, H = BATCH["sizes"][i % 3]
        cp, cn = rng.uniform(0.15, 0.35, 2)
        out.append(dict(width=W, height=H, c_pos=float(cp), c_neg=float(cn), sigma_c=0.03,
                        c_min=0.01, refractory_us=100, seed=seed * 100003 + i))
    return out


def render_config1(seed: int = 0, device="cuda", n_frames: int = C1["T"]) -> torch.Tensor:
    return scenes.render_frames(scenes.SinusoidScene(C1["W"], C1["H"], seed=seed), n_frames,
                                device=device)


WORKLOADS = {
    "hd": dict(dims=HD, sim=CONFIG2_SIM, render=render_config2,
               name="plain HD: 1280x720 FP32, 2000 frames @1000 FPS, value-noise texture + "
                    "affine camera + 16 occluders, C+0.2 C-0.25 sigma0.03 refractory 100us"),
    "c1": dict(dims=C1, sim=CONFIG1_SIM, render=render_config1,
               name="plain 240x180 FP32, 200 frames @1000 FPS, 8 translating sinusoids, "
                    "C+-0.2, no noise, no refractory"),
    "learned": dict(dims=None, sim=None, render=None,
                    name="learned: HD 1280x720 texture clip, keyframes at 250 FPS, U-Net predicts 3 log frames "
                         "per interval, exact event emission at 1000 FPS; C+0.2 C-0.25 sigma0.03 refractory 100us"),
    "batched_learned": dict(dims=None, sim=None, render=None,
                            name="batched + learned: 1024 sensors at 320x240 and 64 at 1280x720, keyframes at "
                                 "250 FPS, U-Net predicts 3 log frames per interval, one batched event step of 4 "
                                 "frames per interval; texture scenes up to 600 px/s, C+0.2 C-0.25 sigma0.03 "
                                 "refractory 100us"),
    "hd_fused": dict(dims=HD, sim=CONFIG2_SIM, render=None,
                     name="render-fused HD: 1280x720, 2000 frames @1000 FPS per step of the library's texture scene "
                          "(4-octave value noise, affine camera, 16 occluders) rendered inside the emission kernel; "
                          "C+0.2 C-0.25 sigma0.03 refractory 100us"),
    "batch": dict(dims=None, sim=None, render=None,
                  name="batched: 256 sensors (346x260 / 640x480 / 1280x720 by index mod 3), "
                       "125 frames @1000 FPS per step (500-frame clips in 4 steps), texture scenes, C+- ~ U[0.15,0.35], "
                       "sigma 0.03, refractory 100us, one CUDA-graph replay per step"),
}


# --------------------------------------------------------------------------
# helpers
# --------------------------------------------------------------------------
def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def combine_ranks(dist, device, ms: float, n_events: int = 0):
    """Whole-job timing over the ranks of a replica run: the slowest rank's
    time (every rank's work counts only when all have finished) and the events
    of all ranks.  With dist None (one process) the inputs come back."""
    if dist is None:
        return ms, n_events
    t = torch.tensor([ms], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    e = torch.tensor([float(n_events)], device=device, dtype=torch.float64)
    dist.all_reduce(e, op=dist.ReduceOp.SUM)
    return float(t.item()), int(e.item())


def job_value(px_frames_per_rank: int, ws: int, ms: float) -> float:
    """Whole-job Mpixel-frames/s: every rank's pixel-frames over the slowest rank's time."""
    return px_frames_per_rank * ws / (ms / 1e3) / 1e6


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2602_15018_gb300", "csrc")
    for f in ("evsim_emit.cuh", "evsim_kernels.cu", "evsim_internal.h"):
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profiled_traffic(px_frames_per_launch: int, workload: str):
    """DRAM bytes per emission launch from the committed ncu summary, scaled by
    pixel-frames; None when absent or taken on a different kernel source."""
    path = os.path.join(ROOT, "profiles", f"emit_kernel_{workload}.md")
    try:
        txt = open(path).read()
    except OSError:
        return None
    m = re.search(r"bench: dram_bytes_per_px_frame=([0-9.eE+-]+) source=([0-9a-f]+)", txt)
    if not m or m.group(2) != kernel_source_hash():
        return None
    return float(m.group(1)) * px_frames_per_launch


class ClockSampler:
    """nvidia-smi samples (200 ms) of SM clock and throttle reasons during a region."""

    FIELDS = ("timestamp,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")
    NAMES = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")

    def __init__(self, local_rank: int):
        vis = os.environ.get("CUDA_VISIBLE_DEVICES")
        self.sel = vis.split(",")[local_rank].strip() if vis else str(local_rank)
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", self.sel], stdout=subprocess.PIPE,
                stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        threading.Thread(target=self._read, daemon=True).start()

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append((time.time(), [c.strip() for c in line.split(",")]))

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self, t0: float, t1: float):
        rows = [r for (t, r) in self.rows if t0 - 0.25 <= t <= t1 + 0.25 and len(r) >= 8]
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        reasons = sorted({n for r in rows for n, v in zip(self.NAMES, r[4:8]) if v == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows)}


# --------------------------------------------------------------------------
# our arm
# --------------------------------------------------------------------------
def run_ours(args):
    from paper_2602_15018_gb300 import EventSim

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    wl = WORKLOADS[args.workload]
    W, H, T = wl["dims"]["W"], wl["dims"]["H"], wl["dims"]["T"]
    if args.frames:
        T = args.frames     # shorter clip of the same scene (small profiling cases)
    npix = W * H
    frames = wl["render"](seed=args.seed + rank, device=dev, n_frames=T)
    # Steps alternate forward and time-reversed playback of the rendered clip,
    # so that every step continues the previous one without a scene cut.
    frames_rev = frames.flip(0).contiguous()
    torch.cuda.synchronize()

    sim = EventSim(W, H, **wl["sim"], max_frames_per_step=T)
    span = T * DT
    cap = npix * T // 8
    out = torch.empty(cap, dtype=torch.int64, device=dev)

    def drain():
        nonlocal out
        n, _ = sim.pending()
        if n > out.numel():
            out = torch.empty(int(n * 1.25), dtype=torch.int64, device=dev)
        ev, _ = sim.drain(to="cuda", out=out)
        return int(ev.numel())

    def one_step(k, drain_now=True):
        sim.step(frames if k % 2 == 0 else frames_rev, k * span, DT)
        return drain() if drain_now else 0

    k = 0
    for j in range(args.warmup):                # same drain cadence as the timed steps
        one_step(k, drain_now=(j + 1) % 4 == 0 or j + 1 == args.warmup)
        k += 1
    # the stream-time budget of timestamps (2^32 us) bounds the number of steps
    if (k + args.steps + 1) * span > 0xFFFFFFFE:
        raise SystemExit("too many steps for the 2^32 us timestamp range")
    sim.set_profiling(True)
    st0 = sim.stats()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    stream = sim.stream
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    tw0 = time.time()
    e0.record(stream)
    n_events = 0
    # steps run back to back; the records of every 4 steps are drained at once
    for j in range(args.steps):
        n_events += one_step(k, drain_now=(j + 1) % 4 == 0 or j + 1 == args.steps)
        k += 1
    e1.record(stream)
    torch.cuda.synchronize()
    tw1 = time.time()
    if dist:
        dist.barrier()
    clocks.stop()
    ms = e0.elapsed_time(e1)
    st1 = sim.stats()
    sim.set_profiling(False)
    ms, n_events_all = combine_ranks(dist, dev, ms, n_events)

    px_frames_step = T * npix
    value = job_value(px_frames_step * args.steps, ws, ms)
    launches = int(st1["kernel_launches"] - st0["kernel_launches"])
    timed = st1["timed_steps"] - st0["timed_steps"]
    emit_ms = (st1["emit_ms"] - st0["emit_ms"]) / max(1, timed)
    sort_ms = (st1["sort_ms"] - st0["sort_ms"]) / max(1, timed)
    ev_per_step = n_events / max(1, args.steps)
    alg_bytes = 4.0 * px_frames_step + 32.0 * npix + 4.0 * ev_per_step
    peak, peak_src = measured_peaks()
    achieved = alg_bytes / (emit_ms / 1e3) / 1e9
    traffic = profiled_traffic(px_frames_step, args.workload)

    # end to end through the C ABI with host buffers (pinned frames in, host events out)
    e2e = None
    if args.e2e_steps > 0:
        host_frames = frames.cpu().pin_memory()
        host_frames_rev = frames_rev.cpu().pin_memory()
        del frames, frames_rev
        torch.cuda.empty_cache()
        host_out = torch.empty(max(1 << 20, int(ev_per_step * 1.5)), dtype=torch.int64).pin_memory()
        sim2 = EventSim(W, H, **wl["sim"], max_frames_per_step=T)
        d2h = 0

        def e2e_step(kk):
            nonlocal host_out
            sim2.step_host(host_frames if kk % 2 == 0 else host_frames_rev, kk * span, DT)
            n, _ = sim2.pending()
            if n > host_out.numel():
                host_out = torch.empty(int(n * 1.25), dtype=torch.int64).pin_memory()
            ev, _ = sim2.drain(to="cpu", out=host_out)
            return ev.numel() * 8

        for kk in range(min(args.warmup, 2)):
            e2e_step(kk)
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for kk in range(args.e2e_steps):
            d2h += e2e_step(kk + 2)
        torch.cuda.synchronize()
        e2e_ms, _ = combine_ranks(dist, dev, (time.perf_counter() - t0) * 1e3)
        e2e = {"value": round(job_value(px_frames_step * args.e2e_steps, ws, e2e_ms), 1),
               "unit": "Mpixel-frames/s",
               "h2d_bytes_per_step": 4 * px_frames_step,
               "d2h_bytes_per_step": int(d2h / args.e2e_steps)}
        sim2.close()

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(args, dev)

    secondary = None
    if rank == 0 and ws == 1 and args.workload == "hd" and not args.frames and not args.no_secondary:
        sim.close()
        sim = None
        torch.cuda.empty_cache()
        secondary = run_secondary()

    if rank == 0:
        clk = clocks.summary(tw0, tw1)
        line = {
            "metric": METRIC,
            "value": round(value, 1),
            "unit": "Mpixel-frames/s",
            "n_gpus": ws,
            "steps": args.steps,
            "warmup": args.warmup,
            "ms_per_step": round(ms / args.steps, 4),
            "higher_is_better": True,
            "scaling": "weak",
            "vs_baseline": None,
            "dtype": "f32",
            "data": "synthetic (seeded procedural scenes rendered on the device)",
            "config": {"workload": wl["name"], "width": W, "height": H, "frames_per_step": T,
                       "dt_us": DT, "streams_per_gpu": 1,
                       "parallelism": f"replicas x{ws} (independent sensor streams)",
                       "l2": "inputs 4*T*H*W bytes per step, far larger than L2; no flush"},
            "events_per_s": round(n_events_all / (ms / 1e3), 1),
            "events_per_step": round(ev_per_step, 1),
            "gpu_launches": launches,
            "kernel_ms": {"emit": round(emit_ms, 4), "sort": round(sort_ms, 4)},
            "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak,
                         "unit": "GB/s", "frac": round(achieved / peak, 4),
                         "traffic": None if traffic is None else int(traffic),
                         "kernel": "emit_kernel", "peak_source": peak_src},
            "e2e": e2e,
            "cpu_baseline": cpu,
            "clocks": clk,
        }
        if secondary is not None:
            line["secondary"] = secondary
        print(json.dumps(line), flush=True)
    if sim is not None:
        sim.close()
    if dist:
        dist.destroy_process_group()


# Algorithmic operations of one rendered pixel-frame (scene_render.cuh): the
# camera map (4 FMA) and 4 octaves of 81 operations each (coordinates 2,
# floor 2, fractions 2, smoothsteps 6, conversions 2, four lattice hashes of
# 14 integer and conversion operations, interpolation 7, octave updates 4),
# the normalisation (2) and the emission filter's two compares.
RENDER_OPS_PER_PX_FRAME = 4 + 4 * 81 + 2 + 2


def alu_peak_tops() -> float:
    """One thread instruction per lane per cycle: SMs x 4 schedulers x 32 lanes
    x the maximum SM clock (Tops/s)."""
    p = torch.cuda.get_device_properties(torch.cuda.current_device())
    mhz = 2070.0
    try:
        mhz = float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["sm_max_mhz"])
    except (OSError, KeyError, ValueError):
        pass
    return p.multi_processor_count * 128 * mhz * 1e6 / 1e12


def fused_cpu_baseline(gen, n_frames: int = 12):
    """Render + simulate on the host, for a bounded sample: the seeded scene
    generator on the CPU (float64 torch, all host threads) for the first
    frames, then the oracle band-parallel on all host cores."""
    import oracle
    W, H = gen.W, gen.H
    t0 = time.perf_counter()
    fr = scenes.render_frames(gen, n_frames, device="cpu").numpy()
    t_render = time.perf_counter() - t0
    cp, cn = oracle.threshold_maps(W, H, 0.2, 0.25, 0.03, 0.01, CONFIG2_SIM["seed"])
    t0 = time.perf_counter()
    ev, _, used, _ = oracle.banded_step(fr, W, H, 0, DT, cp, cn, refractory_us=100, threads=host_cores())
    t_sim = time.perf_counter() - t0
    px = n_frames * W * H
    return {"value": round(px / (t_render + t_sim) / 1e6, 2), "unit": "Mpixel-frames/s", "cores": used,
            "kind": "oracle",
            "sample": f"first {n_frames} frames: the scene generator on the host ({t_render:.1f} s, torch float64, "
                      f"{torch.get_num_threads()} threads) then the C oracle on {used} row bands ({t_sim:.1f} s, "
                      f"{len(ev)} events)"}


def run_fused(args):
    """Render-fused HD steps: the emission kernel renders the library's texture
    scene itself (no frame bytes through HBM).  Timed beside the unfused path
    on the same scene and times: the stand-alone renderer writing the frames
    to HBM, then the plain step reading them."""
    from paper_2602_15018_gb300 import EventSim, render_texture, texture_scene
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    W, H, T = HD["W"], HD["H"], args.frames or HD["T"]
    npix = W * H
    span = T * DT
    gen = scenes.TextureScene(W, H, seed=args.seed + rank)
    ts = texture_scene(**gen.params())
    sim = EventSim(W, H, **CONFIG2_SIM, max_frames_per_step=T)
    out = torch.empty(npix * T // 8, dtype=torch.int64, device=dev)

    def drain(s):
        nonlocal out
        n, _ = s.pending()
        if n > out.numel():
            out = torch.empty(int(n * 1.25), dtype=torch.int64, device=dev)
        ev, _ = s.drain(to="cuda", out=out)
        return int(ev.numel())

    k = 0
    for j in range(args.warmup):
        sim.step_texture(ts, T, k * span, DT)
        if (j + 1) % 4 == 0 or j + 1 == args.warmup:
            drain(sim)
        k += 1
    sim.set_profiling(True)
    st0 = sim.stats()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    tw0 = time.time()
    e0.record(sim.stream)
    n_events = 0
    for j in range(args.steps):
        sim.step_texture(ts, T, k * span, DT)
        if (j + 1) % 4 == 0 or j + 1 == args.steps:
            n_events += drain(sim)
        k += 1
    e1.record(sim.stream)
    torch.cuda.synchronize()
    tw1 = time.time()
    if dist:
        dist.barrier()
    clocks.stop()
    ms = e0.elapsed_time(e1)
    st1 = sim.stats()
    ms, n_events_all = combine_ranks(dist, dev, ms, n_events)
    timed = st1["timed_steps"] - st0["timed_steps"]
    emit_ms = (st1["emit_ms"] - st0["emit_ms"]) / max(1, timed)
    sort_ms = (st1["sort_ms"] - st0["sort_ms"]) / max(1, timed)
    launches = int(st1["kernel_launches"] - st0["kernel_launches"])
    sim.close()

    # unfused: the renderer writes the frames to HBM, the plain step reads them
    frames = torch.empty((T, H, W), dtype=torch.float32, device=dev)
    simu = EventSim(W, H, **CONFIG2_SIM, max_frames_per_step=T)
    cur = torch.cuda.current_stream()
    n_u = max(1, min(args.steps, 4))
    ku = 0
    for _ in range(2):
        render_texture(ts, T, ku * span, DT, out=frames)
        simu.step(frames, ku * span, DT)
        drain(simu)
        ku += 1
    torch.cuda.synchronize()
    rt, stp = 0.0, 0.0
    for _ in range(n_u):
        a, b, c = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        a.record(cur)
        render_texture(ts, T, ku * span, DT, out=frames)
        b.record(cur)
        simu.step(frames, ku * span, DT)
        drain(simu)
        c.record(cur)
        torch.cuda.synchronize()
        rt += a.elapsed_time(b)
        stp += b.elapsed_time(c)
        ku += 1
    simu.close()
    del frames
    torch.cuda.empty_cache()

    # end to end through the C ABI: the scene (host struct) in, the events out
    # to pinned host memory, every step
    e2e = None
    if args.e2e_steps > 0:
        sim2 = EventSim(W, H, **CONFIG2_SIM, max_frames_per_step=T)
        host_out = torch.empty(max(1 << 20, int(n_events / max(1, args.steps) * 1.5)), dtype=torch.int64).pin_memory()
        d2h, k2 = 0, 0

        def e2e_step():
            nonlocal host_out, k2
            sim2.step_texture(ts, T, k2 * span, DT)
            k2 += 1
            n, _ = sim2.pending()
            if n > host_out.numel():
                host_out = torch.empty(int(n * 1.25), dtype=torch.int64).pin_memory()
            ev, _ = sim2.drain(to="cpu", out=host_out)
            return ev.numel() * 8

        for _ in range(2):
            e2e_step()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            d2h += e2e_step()
        torch.cuda.synchronize()
        e2e_ms, _ = combine_ranks(dist, dev, (time.perf_counter() - t0) * 1e3)
        e2e = {"value": round(job_value(T * npix * args.e2e_steps, ws, e2e_ms), 1), "unit": "Mpixel-frames/s",
               "h2d_bytes_per_step": C.sizeof(ts), "d2h_bytes_per_step": int(d2h / args.e2e_steps)}
        sim2.close()

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu = fused_cpu_baseline(gen)

    px = T * npix
    peak = alu_peak_tops()
    achieved = RENDER_OPS_PER_PX_FRAME * px / (emit_ms / 1e3) / 1e12
    if rank == 0:
        line = {
            "metric": METRIC, "value": round(job_value(px * args.steps, ws, ms), 1), "unit": "Mpixel-frames/s",
            "n_gpus": ws, "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms / args.steps, 4),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (the library's seeded texture scene, rendered inside the emission kernel)",
            "config": {"workload": WORKLOADS["hd_fused"]["name"], "width": W, "height": H, "frames_per_step": T,
                       "dt_us": DT, "streams_per_gpu": 1,
                       "parallelism": f"replicas x{ws} (independent sensor streams)",
                       "l2": "no frames in memory; event buffers only"},
            "events_per_s": round(n_events_all / (ms / 1e3), 1),
            "events_per_step": round(n_events / max(1, args.steps), 1),
            "gpu_launches": launches,
            "kernel_ms": {"emit_fused": round(emit_ms, 4), "sort": round(sort_ms, 4)},
            "unfused": {"render_ms": round(rt / n_u, 4), "step_ms": round(stp / n_u, 4),
                        "value": round(px / ((rt + stp) / n_u / 1e3) / 1e6, 1), "unit": "Mpixel-frames/s",
                        "frame_bytes_per_step": 4 * px},
            "roofline": {"bound": "alu", "achieved": round(achieved, 3), "peak": round(peak, 2),
                         "unit": "Tops/s", "frac": round(achieved / peak, 4), "traffic": None,
                         "kernel": "emit_kernel (render-fused)",
                         "ops_per_px_frame": RENDER_OPS_PER_PX_FRAME,
                         "peak_source": "SMs x 128 lanes x max SM clock"},
            "e2e": e2e, "cpu_baseline": cpu, "clocks": clocks.summary(tw0, tw1),
        }
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def run_batch(args):
    """Batched sensors: one CUDA-graph replay of the batched step per step."""
    from paper_2602_15018_gb300 import EventSimBatch
    ws, rank, local = dist_env()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    T = args.frames or BATCH["T"]
    sensors = batch_sensors(args.seed + rank)
    first, slot0, slot1 = [], [], []
    for i, sn in enumerate(sensors):
        sc = scenes.TextureScene(sn["width"], sn["height"], seed=args.seed * 100003 + 7 * i + rank)
        fr = scenes.render_frames(sc, T + 1, device=dev, chunk=T + 1)
        first.append(fr[0].contiguous())
        slot0.append(fr[1:].contiguous())                 # forward
        slot1.append(fr[:T].flip(0).contiguous())         # back again: no scene cut
        del fr
    npix = sum(sn["width"] * sn["height"] for sn in sensors)
    # the project's autotuner on one sensor of each resolution (its step of T
    # frames); the batch's single launch takes the shape tuned for the
    # resolution that holds the most pixels of the batch
    from paper_2602_15018_gb300 import autotune
    tuned, px_of = {}, {}
    for i, sn in enumerate(sensors):
        key = f"{sn['width']}x{sn['height']}"
        px_of[key] = px_of.get(key, 0) + sn["width"] * sn["height"]
        if key not in tuned:
            kw = {k: sn[k] for k in ("c_pos", "c_neg", "sigma_c", "c_min", "refractory_us", "seed")}
            ppt, ctas, tms = autotune(slot0[i], dt_us=DT, repeats=5, **kw)
            tuned[key] = {"pixels_per_thread": ppt, "ctas_per_sm": ctas, "median_ms": round(tms, 4)}
    main_res = max(px_of, key=px_of.get)
    shape = tuned[main_res]
    pend = 4
    st = torch.cuda.Stream(device=dev)
    batch = EventSimBatch(sensors, frames_per_step=T, dt_us=DT, t0_us=0, max_pending_steps=pend,
                          stream=st, pixels_per_thread=shape["pixels_per_thread"],
                          ctas_per_sm=shape["ctas_per_sm"])
    with torch.cuda.stream(st):
        batch.init(first)
        batch.set_frames(slot0, slot=0)
        batch.set_frames(slot1, slot=1)
    torch.cuda.synchronize()
    graphs = [torch.cuda.CUDAGraph(), torch.cuda.CUDAGraph()]
    for k in range(2):
        with torch.cuda.graph(graphs[k], stream=st):
            batch.step(slot=k)
    out = torch.empty(1, dtype=torch.int64, device=dev)
    n_events = 0

    def drain():
        nonlocal out, n_events
        n, _ = batch.pending()
        if n > out.numel():
            out = torch.empty(int(n * 1.25), dtype=torch.int64, device=dev)
        ev, _ = batch.drain(to="cuda", out=out)
        n_events += int(ev.numel())

    k = 0
    with torch.cuda.stream(st):
        for _ in range(args.warmup):
            graphs[k % 2].replay()
            k += 1
            if k % pend == 0:
                drain()
        drain()
    if (k + args.steps + 1) * T * DT > 0xFFFFFFFE:
        raise SystemExit("too many steps for the 2^32 us timestamp range")
    n_events = 0
    la0, _ = batch.counters()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    tw0 = time.time()
    with torch.cuda.stream(st):
        e0.record(st)
        for j in range(args.steps):
            graphs[k % 2].replay()
            k += 1
            if (j + 1) % pend == 0:
                drain()
        drain()
        e1.record(st)
    torch.cuda.synchronize()
    tw1 = time.time()
    if dist:
        dist.barrier()
    clocks.stop()
    ms = e0.elapsed_time(e1)
    la1, _ = batch.counters()
    launches = (la1 - la0) + 5 * args.steps    # graph replays are not counted by the library
    ms, n_events_all = combine_ranks(dist, dev, ms, n_events)
    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu = batch_cpu_baseline(sensors[:6], first[:6], slot0[:6], T)
    px_step = T * npix
    value = job_value(px_step * args.steps, ws, ms)
    ev_step = n_events / max(1, args.steps)
    alg = 4.0 * px_step + 32.0 * npix + 4.0 * ev_step
    peak, peak_src = measured_peaks()
    achieved = alg / (ms / args.steps / 1e3) / 1e9
    if rank == 0:
        line = {
            "metric": METRIC, "value": round(value, 1), "unit": "Mpixel-frames/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms / args.steps, 4),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded procedural scenes rendered on the device)",
            "config": {"workload": WORKLOADS["batch"]["name"], "streams": len(sensors),
                       "pixels_per_frame_step": npix, "frames_per_step": T, "dt_us": DT,
                       "parallelism": f"replicas x{ws} (independent batches)",
                       "l2": "inputs 4*T*sum(H*W) bytes per step, far larger than L2; no flush",
                       "autotuned": tuned, "launch_shape_from": main_res},
            "events_per_s": round(n_events_all / (ms / 1e3), 1),
            "events_per_step": round(ev_step, 1),
            "gpu_launches": int(launches),
            "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                         "frac": round(achieved / peak, 4), "traffic": None,
                         "kernel": "whole step (emission + interval sort + clock), graph replay",
                         "peak_source": peak_src},
            "e2e": None, "cpu_baseline": cpu,
            "clocks": clocks.summary(tw0, tw1),
        }
        print(json.dumps(line), flush=True)
    batch.close()
    if dist:
        dist.destroy_process_group()


UNET_FLOP_PER_PX = 2 * (9 * 8 * 32 + 9 * 32 * 64 // 4 + 9 * 64 * 128 // 16 + 9 * 128 * 128 // 16
                        + 128 * 256 // 16 + 9 * 128 * 64 // 4 + 64 * 128 // 4 + 9 * 64 * 32 + 32 * 16)


def measured_bf16_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["bf16_tflops"]), "measured"
    except Exception:
        return 1900.0, "fallback"


def training_clips(batch: int, size: int, seed: int, speed, device) -> torch.Tensor:
    """[batch, 5, size, size] log frames at 1000 FPS for the interpolator's
    training: crops of one seeded texture scene of 4 size x 4 size at a random
    time in a 2 s clip, generated on the fly (never stored)."""
    from paper_2602_15018_gb300 import log_intensity
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


def clip_source(batch: int, size: int, seed: int, speed, device):
    """Clip source for learned.train: step `it` gets training_clips(seed + it)."""
    return lambda it: training_clips(batch, size, seed + it, speed, device)


def run_learned(args):
    """Learned path at HD: train the interpolator on 1000 FPS clips, score its
    events against the plain 1000 FPS path, and time both pipelines."""
    from paper_2602_15018_gb300 import EventSim, Interpolator, log_intensity
    from paper_2602_15018_gb300 import learned
    ws, rank, local = dist_env()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    W, H = HD["W"], HD["H"]
    K = args.keys
    T = 4 * (K - 1) + 1
    npix = W * H
    net = Interpolator(8, H, W, seed=args.seed)
    t_tr = time.time()
    losses = learned.train(net, args.train_steps, clip_source(16, 256, 10000 + 7919 * rank, (150.0, 600.0), dev),
                           lr=1e-3, report=max(1, args.train_steps // 8))
    torch.cuda.synchronize()
    train_s = time.time() - t_tr
    ev_frames = scenes.render_frames(scenes.TextureScene(W, H, seed=args.seed + rank), T, device=dev, chunk=32)
    score = learned.evaluate(net, ev_frames, **CONFIG2_SIM)
    del ev_frames

    sc = scenes.TextureScene(W, H, seed=args.seed + 100 + rank)
    st = torch.cuda.current_stream()

    def ev():
        return torch.cuda.Event(enable_timing=True)

    def plain_once():
        a, b, c = ev(), ev(), ev()
        a.record(st)
        fr = scenes.render_frames(sc, T, device=dev, chunk=32)
        b.record(st)
        n = len(learned.events_of(fr, False, launches=ev_launches, **CONFIG2_SIM))
        c.record(st)
        torch.cuda.synchronize()
        return a.elapsed_time(b), b.elapsed_time(c), n

    def learned_once():
        a, b, c, d = ev(), ev(), ev(), ev()
        a.record(st)
        keys = sc.render(np.arange(0, T, 4), device=dev).contiguous()
        b.record(st)
        seq = learned.interpolate_sequence(net, log_intensity(keys))
        c.record(st)
        n = len(learned.events_of(seq, True, launches=ev_launches, **CONFIG2_SIM))
        d.record(st)
        torch.cuda.synchronize()
        return a.elapsed_time(b), b.elapsed_time(c), c.elapsed_time(d), n

    def unet_only():
        L0 = torch.randn((8, H, W), device=dev) * 0.3 - 2.0
        L4 = L0 + torch.randn((8, H, W), device=dev) * 0.05
        out = torch.empty((3, 8, H, W), device=dev)
        a, b = ev(), ev()
        a.record(st)
        net.forward(L0, L4, out)
        b.record(st)
        torch.cuda.synchronize()
        return a.elapsed_time(b)

    ev_launches = []                # kernels of each event simulation
    for _ in range(args.warmup):
        plain_once()
        learned_once()
        unet_only()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    ev_launches.clear()
    net_l0 = net.launches()
    tw0 = time.time()
    pl = [plain_once() for _ in range(args.steps)]
    le = [learned_once() for _ in range(args.steps)]
    un = [unet_only() for _ in range(args.steps)]
    tw1 = time.time()
    clocks.stop()
    launches = net.launches() - net_l0 + sum(ev_launches)
    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        keys0 = sc.render(np.array([0, 4]), device=dev).cpu().numpy()
        cpu = learned_cpu_baseline(net, [keys0], [CONFIG2_SIM], "one keyframe interval of the HD clip")
    med = lambda xs: float(statistics.median(xs))
    r_all, e_plain = med([x[0] for x in pl]), med([x[1] for x in pl])
    r_keys, u_ms, e_learn = med([x[0] for x in le]), med([x[1] for x in le]), med([x[2] for x in le])
    unet_ms = med(un)
    px = T * npix
    value = px / ((u_ms + e_learn) / 1e3) / 1e6
    tflops = 8 * npix * UNET_FLOP_PER_PX / (unet_ms / 1e3) / 1e12
    peak, peak_src = measured_bf16_peak()
    if rank == 0:
        line = {
            "metric": METRIC, "value": round(value, 1), "unit": "Mpixel-frames/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(u_ms + e_learn, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16 (U-Net), f32 (events)",
            "data": "synthetic (seeded procedural scenes rendered on the device)",
            "config": {"workload": WORKLOADS["learned"]["name"], "width": W, "height": H, "keyframes": K,
                       "frames": T, "dt_us": DT, "parallelism": f"replicas x{ws}",
                       "l2": "frames and activations far larger than L2; no flush"},
            "f1": round(score["learned"]["f1"], 4), "f1_linear": round(score["linear"]["f1"], 4),
            "count_err": round(score["learned"]["count_err"], 4),
            "count_err_linear": round(score["linear"]["count_err"], 4),
            "plain_value": round(px / (e_plain / 1e3) / 1e6, 1),
            "ms": {"render_all": round(r_all, 3), "events_plain": round(e_plain, 3), "render_keys": round(r_keys, 3),
                   "unet_all_intervals": round(u_ms, 3), "events_learned": round(e_learn, 3)},
            "e2e_speedup_vs_plain": round((r_all + e_plain) / (r_keys + u_ms + e_learn), 3),
            "train": {"steps": args.train_steps, "seconds": round(train_s, 1), "crops": "16 x 256x256",
                      "loss": [[int(i), round(float(l), 6)] for i, l in losses]},
            "gpu_launches": int(launches),
            "roofline": {"bound": "tensor", "achieved": round(tflops, 1), "peak": peak, "unit": "TFLOP/s",
                         "frac": round(tflops / peak, 4), "traffic": None,
                         "kernel": "U-Net forward, 8 HD intervals (9 tcgen05 GEMMs)", "peak_source": peak_src},
            "e2e": None, "cpu_baseline": cpu,
            "clocks": clocks.summary(tw0, tw1),
        }
        print(json.dumps(line), flush=True)
    net.close()


def run_batched_learned(args):
    """Batched + learned: every interval, the interpolator predicts 3 log frames
    for each of 1088 sensors from their keyframes, and one batched event step
    consumes them; scored (F1) and timed against the plain batched path on
    the rendered 1000 FPS frames."""
    from paper_2602_15018_gb300 import EventSimBatch, Interpolator, event_f1, log_intensity
    from paper_2602_15018_gb300 import learned
    ws, rank, local = dist_env()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    groups = [((320, 240), args.bl_small, 64), ((1280, 720), args.bl_big, 8)]    # (size, sensors, U-Net chunk)
    sim = dict(c_pos=0.2, c_neg=0.25, sigma_c=0.03, c_min=0.01, refractory_us=100, input_is_log=True)
    sensors = []
    for gi, ((W, H), n, _) in enumerate(groups):
        for i in range(n):
            sensors.append(dict(width=W, height=H, seed=rank * 100003 + gi * 10007 + i, **sim))
    net = Interpolator(8, 720, 1280, seed=args.seed)
    t_tr = time.time()
    learned.train(net, args.train_steps, clip_source(16, 256, 10000 + 7919 * rank, (150.0, 600.0), dev), lr=1e-3)
    torch.cuda.synchronize()
    train_s = time.time() - t_tr

    # log frames at 1000 FPS, t = 0..4 ms, per group: [5][n][H][W]; keys are frames 0 and 4
    t_r = time.time()
    logs = []
    for gi, ((W, H), n, _) in enumerate(groups):
        L = torch.empty((5, n, H, W), dtype=torch.float32, device=dev)
        for i in range(n):
            sc = scenes.TextureScene(W, H, seed=args.seed * 7 + gi * 100003 + i + 1000 * rank, speed=(150.0, 600.0))
            fr = sc.render(np.arange(5), device=dev).contiguous()
            L[:, i] = log_intensity(fr)
        logs.append(L)
    torch.cuda.synchronize()
    render_s = time.time() - t_r
    npix = sum(n * W * H for (W, H), n, _ in groups)

    # interval buffers [4][n][H][W]: planes 0..2 predicted, plane 3 the next key;
    # slot 0 interpolates key A (t 0) -> B (t 4), slot 1 B -> A (ping-pong)
    bufs = [[torch.empty((4, n, H, W), dtype=torch.float32, device=dev) for (W, H), n, _ in groups]
            for _ in range(2)]

    def predict(slot, model=None):
        model = model or net
        for gi, ((W, H), n, ch) in enumerate(groups):
            a, b = (logs[gi][0], logs[gi][4]) if slot == 0 else (logs[gi][4], logs[gi][0])
            buf = bufs[slot][gi]
            for c0 in range(0, n, ch):
                c1 = min(n, c0 + ch)
                tmp = model.forward(a[c0:c1].contiguous(), b[c0:c1].contiguous())
                buf[0:3, c0:c1] = tmp
            buf[3] = b

    def make_batch(plain):
        bt = EventSimBatch(sensors, frames_per_step=4, dt_us=DT, t0_us=0, max_pending_steps=4)
        bt.init([logs[gi][0, i] .contiguous() for gi, (_, n, _) in enumerate(groups) for i in range(n)])
        for slot in range(2):
            frames, strides = [], []
            for gi, ((W, H), n, _) in enumerate(groups):
                src = (plain_fwd[gi] if slot == 0 else plain_rev[gi]) if plain else bufs[slot][gi]
                for i in range(n):
                    frames.append(src[0, i])
                    strides.append(n * W * H)
            bt.set_frames_strided(frames, strides, slot=slot)
        return bt

    plain_fwd = [L[1:5].contiguous() for L in logs]                      # t 1..4 ms
    plain_rev = [torch.flip(L[0:4], dims=[0]).contiguous() for L in logs]  # t 3..0 ms

    # ---- score: 4 intervals of the plain, learned and linear (untrained) pipelines
    n_score = 4
    lin_net = Interpolator(8, 720, 1280, seed=0)
    per_pipe = []
    for plain, model in ((True, None), (False, net), (False, lin_net)):
        bt = make_batch(plain)
        for k in range(n_score):
            if not plain:
                predict(k % 2, model)
            bt.step(slot=k % 2)
        ev, seg = bt.drain()
        per_pipe.append(bt.split(ev, seg))
        bt.close()
    lin_net.close()

    def f1_of(pred):
        c = np.zeros(3, np.int64)
        for (ev_p, _), (ev_l, _) in zip(per_pipe[0], pred):
            r = event_f1(ev_l, ev_p, 1000)
            c += [r["matched"], r["n_pred"], r["n_ref"]]
        P_, R_ = c[0] / max(1, c[1]), c[0] / max(1, c[2])
        return 2 * P_ * R_ / max(1e-12, P_ + R_), c

    f1, counts = f1_of(per_pipe[1])
    f1_lin, _ = f1_of(per_pipe[2])

    # ---- timing
    st = torch.cuda.current_stream()

    timed_launches = {}             # library kernels inside each timed loop

    def timed(plain, steps):
        bt = make_batch(plain)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        # at most 4 intervals pend between drains (max_pending_steps)
        for k in range(args.warmup):
            if not plain:
                predict(k % 2)
            bt.step(slot=k % 2)
            if (k + 1) % 4 == 0:
                bt.drain(to="cuda")
        bt.drain(to="cuda")
        torch.cuda.synchronize()
        l0 = bt.counters()[0] + net.launches()
        e0.record(st)
        for j in range(steps):
            k = args.warmup + j
            if not plain:
                predict(k % 2)
            bt.step(slot=k % 2)
            if (j + 1) % 4 == 0:
                bt.drain(to="cuda")
        bt.drain(to="cuda")
        e1.record(st)
        torch.cuda.synchronize()
        timed_launches[plain] = bt.counters()[0] + net.launches() - l0
        bt.close()
        return e0.elapsed_time(e1) / steps

    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    tw0 = time.time()
    ms_plain = timed(True, args.steps)
    ms_learn = timed(False, args.steps)
    tw1 = time.time()
    clocks.stop()
    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        keys, sims = [], []
        for gi, ((W, H), n, _) in enumerate(groups):
            sc = scenes.TextureScene(W, H, seed=args.seed * 7 + gi * 100003 + 1000 * rank, speed=(150.0, 600.0))
            keys.append(sc.render(np.array([0, 4]), device=dev).cpu().numpy())
            sims.append({k: v for k, v in sensors[sum(m for _, m, _ in groups[:gi])].items()
                         if k not in ("width", "height", "input_is_log")})
        cpu = learned_cpu_baseline(net, keys, sims, "one keyframe interval of one 320x240 and one 1280x720 sensor")
    # renderer stand-in cost: one keyframe set vs four frame sets per interval
    r0 = time.time()
    for gi, ((W, H), n, _) in enumerate(groups):
        for i in range(min(n, 32)):
            scenes.TextureScene(W, H, seed=i).render(np.arange(4), device=dev)
    torch.cuda.synchronize()
    render_4_ms = (time.time() - r0) * 1e3 * sum(n for _, n, _ in groups) / sum(min(n, 32) for _, n, _ in groups)
    px = 4 * npix
    value = px / (ms_learn / 1e3) / 1e6
    peak, peak_src = measured_bf16_peak()
    unet_ms = ms_learn - ms_plain
    tflops = npix * UNET_FLOP_PER_PX / (max(unet_ms, 1e-3) / 1e3) / 1e12
    if rank == 0:
        line = {
            "metric": METRIC, "value": round(value, 1), "unit": "Mpixel-frames/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_learn, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "bf16 (U-Net), f32 (events)", "data": "synthetic (seeded procedural scenes rendered on the device)",
            "config": {"workload": WORKLOADS["batched_learned"]["name"], "sensors": len(sensors),
                       "pixels_per_interval": npix, "frames_per_interval": 4, "dt_us": DT,
                       "parallelism": f"replicas x{ws}",
                       "l2": "frames and activations far larger than L2; no flush"},
            "f1": round(float(f1), 4), "f1_linear": round(float(f1_lin), 4),
            "f1_counts": [int(c) for c in counts], "f1_intervals": n_score,
            "plain_value": round(px / (ms_plain / 1e3) / 1e6, 1),
            "ms": {"plain_events_per_interval": round(ms_plain, 3), "learned_per_interval": round(ms_learn, 3),
                   "render_4_frames_per_interval_est": round(render_4_ms, 1),
                   "render_1_keyframe_per_interval_est": round(render_4_ms / 4, 1)},
            "e2e_speedup_vs_plain_with_render": round((render_4_ms + ms_plain) / (render_4_ms / 4 + ms_learn), 3),
            "train": {"steps": args.train_steps, "seconds": round(train_s, 1)},
            "setup_render_s": round(render_s, 1),
            "gpu_launches": int(sum(timed_launches.values())),
            "roofline": {"bound": "tensor", "achieved": round(tflops, 1), "peak": peak, "unit": "TFLOP/s",
                         "frac": round(tflops / peak, 4), "traffic": None,
                         "kernel": "U-Net forward over all sensors of one interval (learned minus plain step)",
                         "peak_source": peak_src},
            "e2e": None, "cpu_baseline": cpu,
            "clocks": clocks.summary(tw0, tw1),
        }
        print(json.dumps(line), flush=True)
    net.close()


def _oracle_sample_frames(args, dev):
    wl = WORKLOADS[args.workload]
    n = min(args.cpu_frames, wl["dims"]["T"])
    fr = wl["render"](seed=args.seed, device=dev if dev is not None else "cpu", n_frames=n)
    return fr.cpu().numpy(), n


SECONDARY = (
    ("batch", ["--steps", "4"]),
    ("learned", ["--steps", "2", "--train-steps", "1000"]),
    ("batched_learned", ["--steps", "2", "--train-steps", "1000"]),
)
SECONDARY_KEYS = ("value", "unit", "ms_per_step", "events_per_s", "f1", "f1_linear", "count_err",
                  "count_err_linear", "plain_value", "e2e_speedup_vs_plain", "e2e_speedup_vs_plain_with_render",
                  "roofline", "clocks", "gpu_launches")


def run_secondary():
    """The batched and learned workloads, each in a child process after the
    headline measurement (short: 4 batched steps; the interpolator trained for
    1000 steps), so that one default run records the plain, batched and learned
    paths side by side.  A failure is recorded, not raised."""
    res = {}
    for name, extra in SECONDARY:
        cmd = [sys.executable, os.path.abspath(__file__), "--workload", name, "--warmup", "3", "--no-cpu-baseline",
               "--no-secondary", *extra]
        t0 = time.time()
        try:
            p = subprocess.run(cmd, capture_output=True, text=True, timeout=900)
            lines = [ln for ln in p.stdout.strip().splitlines() if ln.startswith("{")]
            if p.returncode != 0 or not lines:
                res[name] = {"error": f"exit {p.returncode}: {(p.stderr or p.stdout)[-300:]}"}
                continue
            d = json.loads(lines[-1])
            res[name] = {k: d[k] for k in SECONDARY_KEYS if k in d}
            res[name]["config"] = d.get("config", {}).get("workload")
            res[name]["args"] = " ".join(extra)
        except (subprocess.TimeoutExpired, OSError, ValueError) as e:
            res[name] = {"error": str(e)[-300:]}
        res[name]["wall_s"] = round(time.time() - t0, 1)
    return res


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def cpu_baseline(args, dev):
    """The oracle as it stands on the first frames of the workload: run
    band-parallel over all host cores (the same C oracle on row bands, one
    host thread each; pixels are independent, so the events are the same),
    and single-threaded beside it."""
    import oracle
    wl = WORKLOADS[args.workload]
    W, H = wl["dims"]["W"], wl["dims"]["H"]
    fr, n = _oracle_sample_frames(args, dev)
    sim = oracle.OracleSim(W, H, **{k: v for k, v in wl["sim"].items()})
    t0 = time.perf_counter()
    ev, _ = sim.step(fr, 0, DT)
    s1 = time.perf_counter() - t0
    px = n * W * H
    cores = host_cores()
    t0 = time.perf_counter()
    bev, _, used, _ = oracle.banded_step(fr, W, H, 0, DT, sim.cpos, sim.cneg, refractory_us=wl["sim"].get(
        "refractory_us", 0), log_eps=wl["sim"].get("log_eps", 1e-3), threads=cores)
    sn = time.perf_counter() - t0
    return {"value": round(px / sn / 1e6, 2), "unit": "Mpixel-frames/s", "cores": used,
            "kind": "oracle",
            "sample": f"first {n} frames of the workload ({px} pixel-frames, {len(bev)} events), "
                      f"C oracle on {used} row bands, one host thread each, {sn:.1f} s",
            "single_core": {"value": round(px / s1 / 1e6, 2), "cores": 1, "seconds": round(s1, 2),
                            "events": int(len(ev))}}


def batch_cpu_baseline(sensors, first, frames, T):
    """The event oracle (single thread) on a bounded sample of the batched
    workload: the first `len(first)` sensors over one whole step."""
    import oracle
    px, n_ev, s = 0, 0, 0.0
    for sn, f0, fr in zip(sensors, first, frames):
        kw = dict(c_pos=sn["c_pos"], c_neg=sn["c_neg"], sigma_c=sn["sigma_c"], c_min=sn["c_min"],
                  refractory_us=sn["refractory_us"], seed=sn["seed"])
        sim = oracle.OracleSim(sn["width"], sn["height"], **kw)
        seq = np.concatenate([f0.cpu().numpy()[None], fr.cpu().numpy()])
        t0 = time.perf_counter()
        ev, _ = sim.step(seq, 0, DT)
        s += time.perf_counter() - t0
        n_ev += len(ev)
        px += T * sn["width"] * sn["height"]
    sizes = ", ".join(f"{sn['width']}x{sn['height']}" for sn in sensors)
    return {"value": round(px / s / 1e6, 2), "unit": "Mpixel-frames/s", "cores": 1, "kind": "oracle",
            "sample": f"sensors {sizes} over one {T}-frame step ({px} pixel-frames, {n_ev} events), "
                      f"single-threaded C oracle, {s:.1f} s"}


def learned_cpu_baseline(net, keys, sims, what):
    """The learned pipeline's oracle on a bounded sample: per sensor, the
    oracle log of its intensity keyframes [K, H, W] (host), the FP64 U-Net
    oracle (BF16 storage mirrored) on the trained parameters, and the event
    oracle on the resulting log sequence.  Runs in a child process with one
    BLAS / OpenMP thread, so that it uses exactly one core."""
    import tempfile
    from paper_2602_15018_gb300.interp import to_dict
    params = {k: np.asarray(v, np.float64) for k, v in to_dict(net.get_params()).items()}
    with tempfile.TemporaryDirectory() as tmp:
        src = os.path.join(tmp, "sample.npz")
        arrays = {f"keys{i}": np.ascontiguousarray(k, np.float32) for i, k in enumerate(keys)}
        arrays.update({f"p_{k}": v for k, v in params.items()})
        np.savez(src, **arrays)
        with open(os.path.join(tmp, "sims.json"), "w") as f:
            json.dump(sims, f)
        env = dict(os.environ, OPENBLAS_NUM_THREADS="1", OMP_NUM_THREADS="1", MKL_NUM_THREADS="1")
        r = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-learned-sample", tmp],
                           env=env, capture_output=True, text=True, timeout=900)
    if r.returncode != 0:
        raise RuntimeError("learned oracle sample failed: " + r.stderr[-2000:])
    res = json.loads(r.stdout.strip().splitlines()[-1])
    s = res["unet_s"] + res["events_s"]
    return {"value": round(res["px"] / s / 1e6, 3), "unit": "Mpixel-frames/s", "cores": 1, "kind": "oracle",
            "sample": f"{what}: {res['px']} pixel-frames, {res['events']} events; FP64 U-Net oracle "
                      f"{res['unet_s']:.1f} s + C event oracle {res['events_s']:.1f} s, one thread"}


def oracle_learned_sample(tmp):
    """Child of learned_cpu_baseline: time the oracles on the saved sample."""
    import oracle
    from oracle import interp_oracle as io
    z = np.load(os.path.join(tmp, "sample.npz"))
    with open(os.path.join(tmp, "sims.json")) as f:
        sims = json.load(f)
    p = {k[2:]: z[k] for k in z.files if k.startswith("p_")}
    px, n_ev, t_unet, t_ev = 0, 0, 0.0, 0.0
    for i, sim_kw in enumerate(sims):
        keys = z[f"keys{i}"]
        K, H, W = keys.shape
        t0 = time.perf_counter()
        clamped = (np.minimum(np.maximum(keys, np.float32(0)), np.float32(1e6)) + np.float32(1e-3)).astype(np.float32)
        L = oracle.mylog(clamped)
        mid, _ = io.forward(p, L[:-1], L[1:], quantize=True)              # [3, K - 1, H, W]
        seq = np.empty((4 * (K - 1) + 1, H, W), np.float32)
        seq[0::4] = L
        for j in range(3):
            seq[1 + j::4] = mid[j]
        t1 = time.perf_counter()
        ev, _ = oracle.OracleSim(W, H, input_is_log=True, **sim_kw).step(seq, 0, DT)
        t2 = time.perf_counter()
        t_unet += t1 - t0
        t_ev += t2 - t1
        n_ev += len(ev)
        px += 4 * (K - 1) * H * W
    print(json.dumps({"px": px, "events": n_ev, "unet_s": t_unet, "events_s": t_ev}), flush=True)


# --------------------------------------------------------------------------
# reference arm: the oracle on the host cores
# --------------------------------------------------------------------------
def run_reference(args):
    ws, rank, local = dist_env()
    if rank != 0:
        return
    import oracle
    wl = WORKLOADS[args.workload]
    W, H = wl["dims"]["W"], wl["dims"]["H"]
    dev = None
    if torch.cuda.is_available():
        dev = torch.device("cuda", local)
    fr, n = _oracle_sample_frames(args, dev)
    cores = host_cores()
    cal = oracle.OracleSim(W, H, **wl["sim"])
    cp, cn = cal.cpos, cal.cneg
    kw = dict(refractory_us=wl["sim"].get("refractory_us", 0), log_eps=wl["sim"].get("log_eps", 1e-3),
              threads=cores)
    # size each step so that warm-up + timed steps take about two minutes
    t0 = time.perf_counter()
    oracle.banded_step(fr[: min(n, 17)], W, H, 0, DT, cp, cn, **kw)
    per_frame = (time.perf_counter() - t0) / max(1, min(n, 17) - 1)
    n = int(max(2, min(n, 120.0 / (args.steps + args.warmup) / max(per_frame, 1e-4))))
    fr = np.ascontiguousarray(fr[:n])
    for _ in range(args.warmup):
        oracle.banded_step(fr, W, H, 0, DT, cp, cn, **kw)
    times, n_ev, used = [], 0, 1
    for _ in range(args.steps):
        t0 = time.perf_counter()
        ev, _, used, _ = oracle.banded_step(fr, W, H, 0, DT, cp, cn, **kw)
        times.append(time.perf_counter() - t0)
        n_ev += len(ev)
    s = sum(times)
    px = n * W * H * args.steps
    val = px / s / 1e6
    line = {
        "impl": "reference", "metric": METRIC, "value": round(val, 2), "unit": "Mpixel-frames/s",
        "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(1e3 * s / args.steps, 2), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded procedural scenes)",
        "config": {"workload": wl["name"], "width": W, "height": H,
                   "frames_per_step": n, "dt_us": DT,
                   "sample": f"each step: {n} frames of the workload (bounded sample)"},
        "events_per_s": round(n_ev / s, 1),
        "cpu_baseline": {"value": round(val, 2), "unit": "Mpixel-frames/s", "cores": used,
                         "kind": "oracle",
                         "sample": f"{n} frames x {args.steps} steps from a fresh sensor, C oracle on {used} "
                                   f"row bands, one host thread each"},
        "e2e": {"value": round(val, 2), "unit": "Mpixel-frames/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="hd")
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--cpu-frames", type=int, default=480)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-secondary", action="store_true",
                    help="default workload: skip the batched and learned child runs")
    ap.add_argument("--keys", type=int, default=126, help="learned workload: keyframes per clip")
    ap.add_argument("--bl-small", type=int, default=1024, help="batched_learned: 320x240 sensors")
    ap.add_argument("--bl-big", type=int, default=64, help="batched_learned: 1280x720 sensors")
    ap.add_argument("--train-steps", type=int, default=8000, help="learned workload: training steps")
    ap.add_argument("--frames", type=int, default=0,
                    help="frames per step (default: the workload's); for small profiling cases")
    ap.add_argument("--oracle-learned-sample", default=None, help=argparse.SUPPRESS)
    args = ap.parse_args()
    if args.oracle_learned_sample:
        oracle_learned_sample(args.oracle_learned_sample)
        return
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        if args.workload in ("batch", "learned", "batched_learned", "hd_fused"):
            ap.error("the reference arm runs the plain workloads only")
        run_reference(args)
    elif args.workload == "batch":
        run_batch(args)
    elif args.workload == "hd_fused":
        run_fused(args)
    elif args.workload == "learned":
        run_learned(args)
    elif args.workload == "batched_learned":
        run_batched_learned(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
