"""Batched sensors: every stream of a batch gives exactly the events of the
FP32-mirrored oracle run on that stream alone, eagerly and when the step is
captured once in a CUDA graph and replayed; failed steps are dropped on the
device and reported by the drain.

Streams of mixed, ragged resolutions and different parameters share one
launch, as the concurrent simulation instances of the paper's RL setup do
(arXiv 2602.15018, Sec. 4 and the RL appendix).
"""
import numpy as np
import pytest
import torch

import oracle
import scenes

pytestmark = pytest.mark.gpu

DT = 1000

SENSORS = [
    dict(width=37, height=23, c_pos=0.15, c_neg=0.3, sigma_c=0.02, refractory_us=100, seed=1),
    dict(width=64, height=48, c_pos=0.25, c_neg=0.2, seed=2),
    dict(width=200, height=120, c_pos=0.2, c_neg=0.25, sigma_c=0.03, refractory_us=100, seed=3),
    dict(width=5, height=3, c_pos=0.1, c_neg=0.1, seed=4),
    dict(width=333, height=77, c_pos=0.2, c_neg=0.2, sigma_c=0.01, seed=5),
]


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import __graft_entry__
    __graft_entry__.build()


def _frames(n_frames):
    out = []
    for i, s in enumerate(SENSORS):
        sc = scenes.TextureScene(s["width"], s["height"], seed=40 + i, speed=(300.0, 600.0))
        out.append(scenes.render_frames(sc, n_frames))
    return out


def _oracles(batch):
    res = []
    for i, s in enumerate(SENSORS):
        cp, cn = batch.thresholds(i)
        res.append(oracle.OracleSim(s["width"], s["height"], c_pos_map=cp, c_neg_map=cn,
                                    refractory_us=s.get("refractory_us", 0)))
    return res


def _check_stream(batch, i, o, ev, offs, what):
    rev, rseg = o.step_result
    assert np.array_equal(offs, rseg), f"{what}: stream {i} offsets differ"
    assert np.array_equal(ev, rev), f"{what}: stream {i} events differ ({len(ev)} vs {len(rev)})"
    st = batch.get_state(i)
    assert np.array_equal(st["ref"], o.ref) and np.array_equal(st["lprev"], o.lprev)
    tl = o.tlast.copy()
    tl[tl < 0] = 0xFFFFFFFF
    assert np.array_equal(st["tlast"].astype(np.int64), tl)
    assert st["tau"] == o.tau


def _run_oracles(orcs, frames, k0, k1, T, t0):
    """Oracle steps k0..k1-1 (frames 1 + k T .. 1 + (k+1) T); step_result holds
    the concatenated events and offsets."""
    for i, o in enumerate(orcs):
        evs, offs = [], [0]
        for k in range(k0, k1):
            chunk = np.ascontiguousarray(frames[i][1 + k * T: 1 + (k + 1) * T].numpy())
            ev, seg = o.step(chunk, t0 + (1 + k * T) * DT, DT)
            evs.append(ev)
            offs.extend((seg[1:] + offs[-1]).tolist())
        o.step_result = (np.concatenate(evs), np.array(offs, np.int64))


def _init(batch, orcs, frames, t0):
    first = [f[0].contiguous().cuda() for f in frames]
    batch.init(first)
    for i, o in enumerate(orcs):
        o.step(np.ascontiguousarray(frames[i][:1].numpy()), t0, DT)
    return first


def test_batch_eager_matches_oracle_per_stream():
    from paper_2602_15018_gb300 import EventSimBatch
    T, steps, t0 = 6, 4, 5000
    frames = _frames(1 + steps * T)
    batch = EventSimBatch(SENSORS, frames_per_step=T, dt_us=DT, t0_us=t0)
    orcs = _oracles(batch)
    first = _init(batch, orcs, frames, t0)
    # two frame slots, used alternately
    bufs = [[torch.empty((T, s["height"], s["width"]), dtype=torch.float32, device="cuda") for s in SENSORS]
            for _ in range(2)]
    batch.set_frames(bufs[0], slot=0)
    batch.set_frames(bufs[1], slot=1)
    for drain_after in ((0, 2), (2, 3), (3, 4)):     # two steps between the first drain
        for k in range(*drain_after):
            for i in range(len(SENSORS)):
                bufs[k % 2][i].copy_(frames[i][1 + k * T: 1 + (k + 1) * T])
            batch.step(slot=k % 2)
        ev, seg = batch.drain()
        _run_oracles(orcs, frames, drain_after[0], drain_after[1], T, t0)
        per = batch.split(ev, seg)
        for i, o in enumerate(orcs):
            _check_stream(batch, i, o, per[i][0], per[i][1], f"steps {drain_after}")
    launches, n_steps = batch.counters()
    assert n_steps == 1 + steps and launches == 2 + 5 * steps   # init: emission + clock
    del first
    batch.close()


def test_batch_graph_replay_matches_oracle():
    """One step captured in a CUDA graph, replayed with refilled buffers."""
    from paper_2602_15018_gb300 import EventSimBatch
    T, steps, t0 = 8, 5, 0
    frames = _frames(1 + steps * T)
    s = torch.cuda.Stream()
    batch = EventSimBatch(SENSORS, frames_per_step=T, dt_us=DT, t0_us=t0, stream=s, pixels_per_thread=8,
                          max_pending_steps=steps)
    orcs = _oracles(batch)
    bufs = [torch.empty((T, q["height"], q["width"]), dtype=torch.float32, device="cuda") for q in SENSORS]
    with torch.cuda.stream(s):
        first = _init(batch, orcs, frames, t0)
        batch.set_frames(bufs)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        batch.step()
    with torch.cuda.stream(s):
        for k in range(steps):
            for i in range(len(SENSORS)):
                bufs[i].copy_(frames[i][1 + k * T: 1 + (k + 1) * T], non_blocking=True)
            g.replay()
    s.synchronize()
    ev, seg = batch.drain()
    _run_oracles(orcs, frames, 0, steps, T, t0)
    per = batch.split(ev, seg)
    for i, o in enumerate(orcs):
        _check_stream(batch, i, o, per[i][0], per[i][1], "graph")
    del first, g
    batch.close()


def test_batch_overflow_drops_the_step_and_later_ones():
    """A step over the event capacity is dropped with every later one; the
    drain delivers the committed steps, reports the overflow and the batch
    continues from the last good state."""
    from paper_2602_15018_gb300 import EventSimBatch
    from paper_2602_15018_gb300._lib import NeurosimError
    T, t0 = 6, 0
    frames = _frames(1 + 3 * T)
    # step 0 fits, step 1 (scene moving faster) does not: capacity between the two
    batch = EventSimBatch(SENSORS, frames_per_step=T, dt_us=DT, t0_us=t0)
    orcs = _oracles(batch)
    _init(batch, orcs, frames, t0)
    bufs = [torch.empty((T, q["height"], q["width"]), dtype=torch.float32, device="cuda") for q in SENSORS]
    batch.set_frames(bufs)
    for i in range(len(SENSORS)):
        bufs[i].copy_(frames[i][1:1 + T])
    batch.step()
    n0, _ = batch.pending()
    batch.close()
    assert n0 > 0

    batch = EventSimBatch(SENSORS, frames_per_step=T, dt_us=DT, t0_us=t0, event_capacity=n0)
    orcs = _oracles(batch)
    _init(batch, orcs, frames, t0)
    batch.set_frames(bufs)
    for k in range(3):
        for i in range(len(SENSORS)):
            bufs[i].copy_(frames[i][1 + k * T: 1 + (k + 1) * T])
        batch.step()
    ev, seg, rc = batch.drain(strict=False)
    assert rc == 4, rc                       # NEUROSIM_E_OVERFLOW
    _run_oracles(orcs, frames, 0, 1, T, t0)  # only step 0 was committed
    per = batch.split(ev, seg)
    for i, o in enumerate(orcs):
        _check_stream(batch, i, o, per[i][0], per[i][1], "overflow")
    # the condition is cleared: an empty drain succeeds and the state stays
    ev2, seg2 = batch.drain()
    assert len(ev2) == 0 and len(seg2) == 1
    with pytest.raises(NeurosimError):
        batch.init([f[0].contiguous().cuda() for f in frames])   # already initialised
    batch.close()


def test_batch_pending_capacity_is_enforced():
    from paper_2602_15018_gb300 import EventSimBatch
    T, t0 = 4, 0
    frames = _frames(1 + 2 * T)
    batch = EventSimBatch(SENSORS, frames_per_step=T, dt_us=DT, t0_us=t0, max_pending_steps=1)
    orcs = _oracles(batch)
    _init(batch, orcs, frames, t0)
    bufs = [torch.empty((T, q["height"], q["width"]), dtype=torch.float32, device="cuda") for q in SENSORS]
    batch.set_frames(bufs)
    for k in range(2):
        for i in range(len(SENSORS)):
            bufs[i].copy_(frames[i][1 + k * T: 1 + (k + 1) * T])
        batch.step()
    ev, seg, rc = batch.drain(strict=False)
    assert rc == 4 and len(seg) == len(SENSORS) * T + 1
    _run_oracles(orcs, frames, 0, 1, T, t0)
    per = batch.split(ev, seg)
    for i, o in enumerate(orcs):
        _check_stream(batch, i, o, per[i][0], per[i][1], "pending")
    batch.close()


def test_autotune_picks_the_fastest_timed_variant_and_caches_it(tmp_path):
    """The tuner times every launch shape (warp tile 256 or 512 pixels x 1 up
    to the resident CTAs per SM), keeps the one with the smallest median
    time, caches it with every variant's time, and the picked shape computes
    the default shape's events."""
    import json

    from paper_2602_15018_gb300 import EventSim, autotune
    W, H, T = 320, 180, 40
    fr = scenes.render_frames(scenes.TextureScene(W, H, seed=9), T).cuda()
    cache = str(tmp_path / "tune.jsonl")
    kw = dict(c_pos=0.2, c_neg=0.25, sigma_c=0.03, refractory_us=100, seed=1)
    ppt, ctas, ms = autotune(fr, dt_us=DT, repeats=5, cache_path=cache, **kw)
    lines = open(cache).read().strip().split("\n")
    assert len(lines) == 1
    rec = json.loads(lines[0])
    timings = rec["timings"]
    shapes = {(p, c) for p, c, _ in timings}
    assert {(8, 1), (16, 1)} <= shapes and len(shapes) == len(timings) >= 4
    fastest = min(timings, key=lambda v: v[2])
    assert (ppt, ctas) == (fastest[0], fastest[1]) == (rec["pixels_per_thread"], rec["ctas_per_sm"])
    assert abs(ms - fastest[2]) < 1e-3 and ms > 0
    again = autotune(fr, dt_us=DT, repeats=5, cache_path=cache, **kw)
    assert again[:2] == (ppt, ctas) and len(open(cache).read().strip().split("\n")) == 1
    res = []
    for shape in (dict(), dict(pixels_per_thread=ppt, ctas_per_sm=ctas)):
        sim = EventSim(W, H, max_frames_per_step=T, **kw, **shape)
        sim.step(fr, 0, DT)
        res.append(sim.drain())
        sim.close()
    assert np.array_equal(res[0][0], res[1][0]) and np.array_equal(res[0][1], res[1][1])


def test_batch_strided_frames_match_oracle():
    """Three equal-size sensors whose frames interleave in one [T][3][H][W]
    array (frame stride 3 H W), as the interpolator's output is laid out."""
    from paper_2602_15018_gb300 import EventSimBatch
    T, t0, W, H = 5, 0, 48, 40
    sensors = [dict(width=W, height=H, c_pos=0.2, c_neg=0.25, sigma_c=0.02, refractory_us=50, seed=60 + i)
               for i in range(3)]
    clips = [scenes.render_frames(scenes.TextureScene(W, H, seed=80 + i, speed=(300.0, 600.0)), 1 + 2 * T)
             for i in range(3)]
    batch = EventSimBatch(sensors, frames_per_step=T, dt_us=DT, t0_us=t0)
    orcs = []
    for i, s in enumerate(sensors):
        cp, cn = batch.thresholds(i)
        orcs.append(oracle.OracleSim(W, H, c_pos_map=cp, c_neg_map=cn, refractory_us=50))
    batch.init([c[0].contiguous().cuda() for c in clips])
    for i, o in enumerate(orcs):
        o.step(np.ascontiguousarray(clips[i][:1].numpy()), t0, DT)
    inter = torch.empty((T, 3, H, W), dtype=torch.float32, device="cuda")
    batch.set_frames_strided([inter[0, i] for i in range(3)], [3 * H * W] * 3, slot=0)
    for k in range(2):
        for i in range(3):
            inter[:, i] = clips[i][1 + k * T: 1 + (k + 1) * T].cuda()
        batch.step(slot=0)
        ev, seg = batch.drain()
        per = batch.split(ev, seg)
        for i, o in enumerate(orcs):
            rev, rseg = o.step(np.ascontiguousarray(clips[i][1 + k * T: 1 + (k + 1) * T].numpy()),
                               t0 + (1 + k * T) * DT, DT)
            assert np.array_equal(per[i][0], rev), (k, i)
            assert np.array_equal(per[i][1], rseg), (k, i)
    batch.close()


def test_batch_at_benchmark_shapes_graph_replay():
    """24 sensors cycling 346x260 / 640x480 / 1280x720 with the batched
    benchmark's parameters (C+- from U[0.15, 0.35], sigma 0.03, refractory
    100 us, texture scenes), 16 frames per step, 3 steps from one captured
    CUDA graph over two frame slots: every sensor's records, offsets and state
    equal the oracle's on that sensor alone, bit for bit.  This reaches the
    descriptor search and the per-sensor chunk tables at several hundred
    tiles per sensor."""
    from concurrent.futures import ThreadPoolExecutor

    import bench
    from paper_2602_15018_gb300 import EventSimBatch
    T, steps, t0 = 16, 3, 0
    sensors = bench.batch_sensors(seed=3, n=24)
    frames = []
    for i, s in enumerate(sensors):
        sc = scenes.TextureScene(s["width"], s["height"], seed=500 + i, speed=(150.0, 600.0))
        frames.append(scenes.render_frames(sc, 1 + steps * T, device="cuda", chunk=17).cpu())
    st = torch.cuda.Stream()
    batch = EventSimBatch(sensors, frames_per_step=T, dt_us=DT, t0_us=t0, stream=st, max_pending_steps=steps)
    orcs = []
    for i, s in enumerate(sensors):
        cp, cn = batch.thresholds(i)
        ocp, ocn = oracle.threshold_maps(s["width"], s["height"], s["c_pos"], s["c_neg"], 0.03, 0.01, s["seed"])
        assert np.array_equal(cp, ocp) and np.array_equal(cn, ocn)
        orcs.append(oracle.OracleSim(s["width"], s["height"], c_pos_map=cp, c_neg_map=cn, refractory_us=100))
    bufs = [[torch.empty((T, s["height"], s["width"]), dtype=torch.float32, device="cuda") for s in sensors]
            for _ in range(2)]
    with torch.cuda.stream(st):
        first = [f[0].contiguous().cuda() for f in frames]
        batch.init(first)
        batch.set_frames(bufs[0], slot=0)
        batch.set_frames(bufs[1], slot=1)
    torch.cuda.synchronize()
    graphs = []
    for slot in range(2):
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=st):
            batch.step(slot=slot)
        graphs.append(g)
    for k in range(steps):
        for i in range(len(sensors)):
            bufs[k % 2][i].copy_(frames[i][1 + k * T: 1 + (k + 1) * T])
        torch.cuda.synchronize()
        graphs[k % 2].replay()
    torch.cuda.synchronize()
    ev, seg = batch.drain()

    def run(i):
        o = orcs[i]
        o.step(np.ascontiguousarray(frames[i][:1].numpy()), t0, DT)
        evs, offs = [], [0]
        for k in range(steps):
            e, sg = o.step(np.ascontiguousarray(frames[i][1 + k * T: 1 + (k + 1) * T].numpy()),
                           t0 + (1 + k * T) * DT, DT)
            evs.append(e)
            offs.extend((sg[1:] + offs[-1]).tolist())
        o.step_result = (np.concatenate(evs), np.array(offs, np.int64))

    with ThreadPoolExecutor(max_workers=8) as ex:
        list(ex.map(run, range(len(sensors))))
    per = batch.split(ev, seg)
    total = 0
    for i, o in enumerate(orcs):
        _check_stream(batch, i, o, per[i][0], per[i][1], "benchmark shapes")
        total += len(per[i][0])
    assert total > 100_000
    del first
    batch.close()
