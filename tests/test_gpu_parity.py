"""GPU parity: the CUDA event path against the FP32-mirrored oracle, bit for bit.

The event set, its order and the interval offsets must be identical (the
oracle mirrors the FP32 operation order, so the tolerance is zero); the
per-pixel state after a step must be identical too.  Inputs are seeded
synthetic scenes with the shapes of the workloads: 240x180 sinusoids, HD
value-noise texture with occluders, mixed odd sizes.
"""
import numpy as np
import pytest
import torch

import oracle
import scenes

pytestmark = pytest.mark.gpu

DT = 1000


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import __graft_entry__
    __graft_entry__.build()


def _sims(W, H, **kw):
    from paper_2602_15018_gb300 import EventSim
    gkw = {k: v for k, v in kw.items() if k not in ("precision",)}
    g = EventSim(W, H, **gkw)
    cp, cn = g.thresholds()
    okw = {k: v for k, v in kw.items() if k in ("refractory_us", "log_eps", "input_is_log")}
    o = oracle.OracleSim(W, H, c_pos_map=cp, c_neg_map=cn, **okw)
    return g, o


def _first_diff(a, b):
    n = min(len(a), len(b))
    d = np.nonzero(a[:n] != b[:n])[0]
    i = int(d[0]) if len(d) else n
    return i, (oracle.unpack(a[i:i + 1]) if i < len(a) else None), \
        (oracle.unpack(b[i:i + 1]) if i < len(b) else None)


def assert_same(ev, seg, rev, rseg, what=""):
    assert np.array_equal(seg, rseg), f"{what}: interval offsets differ"
    if not np.array_equal(ev, rev):
        i, ga, ob = _first_diff(ev, rev)
        raise AssertionError(f"{what}: events differ (gpu {len(ev)}, oracle {len(rev)}); first at "
                             f"{i}: gpu {ga} oracle {ob}")


def _check_state(g, o):
    st = g.get_state()
    assert np.array_equal(st["ref"], o.ref), "ref differs"
    assert np.array_equal(st["lprev"], o.lprev), "lprev differs"
    tl = o.tlast.copy()
    tl[tl < 0] = 0xFFFFFFFF
    assert np.array_equal(st["tlast"].astype(np.int64), tl), "tlast differs"
    assert st["tau_prev"] == o.tau


def test_log_bit_exact_domain():
    """Device log == oracle log on every FP32 value of [1e-8, 1e6 + 1]."""
    from paper_2602_15018_gb300 import device_log
    lo = int(np.float32(1e-8).view(np.uint32))
    hi = int(np.float32(1e6 + 1).view(np.uint32))
    chunk = 1 << 26
    for b0 in range(lo, hi + 1, chunk):
        bits = np.arange(b0, min(hi + 1, b0 + chunk), dtype=np.uint32)
        x = bits.view(np.float32)
        y = device_log(torch.from_numpy(x).cuda()).cpu().numpy()
        assert np.array_equal(y.view(np.uint32), oracle.mylog(x).view(np.uint32)), hex(b0)


def test_log_bit_exact_sampled_full_range():
    """Every 17th positive float (subnormals to max) and the special values."""
    from paper_2602_15018_gb300 import device_log
    bits = np.arange(1, 0x7F800000, 17, dtype=np.uint32)
    x = np.concatenate([bits.view(np.float32),
                        np.array([0.0, np.inf, -1.0, np.nan, -0.0], np.float32)])
    y = device_log(torch.from_numpy(x).cuda()).cpu().numpy()
    r = oracle.mylog(x)
    assert np.array_equal(np.isnan(y), np.isnan(r))
    m = ~np.isnan(r)
    assert np.array_equal(y[m].view(np.uint32), r[m].view(np.uint32))


@pytest.mark.parametrize("C", [0.1, 0.2, 0.25])
def test_random_log_8x8(C):
    fr = scenes.random_log_frames(8, 8, 6, seed=int(C * 100), lo=-1.0, hi=1.0)
    g, o = _sims(8, 8, c_pos=C, c_neg=C, input_is_log=True)
    g.step(torch.from_numpy(fr).cuda(), 0, DT)
    ev, seg = g.drain()
    rev, rseg = o.step(fr, 0, DT)
    assert_same(ev, seg, rev, rseg, f"8x8 C={C}")
    _check_state(g, o)
    g.close()


def test_ramps_closed_form_on_gpu():
    for s in (0.0625, 0.09375, -0.0625, 0.75):
        fr = scenes.log_ramp(5, 3, 41, 0.0, s)
        g, o = _sims(5, 3, c_pos=0.25, c_neg=0.25, input_is_log=True)
        g.step(torch.from_numpy(fr).cuda(), 0, DT)
        ev, seg = g.drain()
        rev, rseg = o.step(fr, 0, DT)
        assert_same(ev, seg, rev, rseg, f"ramp {s}")
        g.close()


def test_config1_sinusoids_240x180_full():
    """240x180, 200 frames at 1000 FPS, C+ = C- = 0.2, no noise, no refractory."""
    W, H, T = 240, 180, 200
    for seed in (0, 1):
        fr = scenes.render_frames(scenes.SinusoidScene(W, H, seed=seed), T)
        g, o = _sims(W, H, c_pos=0.2, c_neg=0.2, max_frames_per_step=T)
        g.step(fr.cuda(), 0, DT)
        ev, seg = g.drain()
        rev, rseg = o.step(fr.numpy(), 0, DT)
        assert_same(ev, seg, rev, rseg, f"config1 seed {seed}")
        assert len(ev) > 100000
        _check_state(g, o)
        g.close()


@pytest.mark.parametrize("W,H,ppt,pf", [(320, 181, 16, 2), (346, 260, 8, 3), (33, 17, 16, 3),
                                         (7, 5, 8, 2), (1024, 1, 16, 2), (1, 700, 8, 2)])
def test_texture_odd_sizes(W, H, ppt, pf):
    """Ragged tiles, frames that are not 16-byte aligned per row (W*H % 4 != 0)."""
    T = 40
    fr = scenes.render_frames(scenes.TextureScene(W, H, seed=W + H, speed=(300., 600.)), T)
    kw = dict(c_pos=0.2, c_neg=0.25, sigma_c=0.03, refractory_us=100, seed=W * 7 + H,
              max_frames_per_step=T, pixels_per_thread=ppt, prefetch_frames=pf)
    g, o = _sims(W, H, **kw)
    g.step(fr.cuda(), 5000, DT)
    ev, seg = g.drain()
    rev, rseg = o.step(fr.numpy(), 5000, DT)
    assert_same(ev, seg, rev, rseg, f"{W}x{H}")
    _check_state(g, o)
    g.close()


@pytest.mark.parametrize("ppt,win", [(16, 2), (16, 3), (8, 3)])
def test_exact_paths_crowded_tiles_and_many_events(ppt, win):
    """Log-domain frames built to reach every path of the emission kernel:
    quiet tiles, pairs of frames with a few pixels out of their band (one
    pass of the exact path), pixels with many events in one frame (keys
    regenerated from the saved state), frames where most pixels of a tile
    leave their band (more listed pixels than lanes: the general path), a
    pixel leaving its band again soon after its first events, and a
    continuing step whose first interval starts from the stored state."""
    W, H, T = 512, 4, 23
    rng = np.random.default_rng(ppt * 10 + win)
    base = rng.uniform(-3.0, 0.0, (H, W))
    fr = np.repeat(base[None], T, axis=0).astype(np.float64)
    # row 0: quiet.  row 1: a few pixels drift slowly (single events, retriggers)
    drift = rng.choice(W, 24, replace=False)
    fr[:, 1, drift] += np.arange(T)[:, None] * rng.uniform(0.05, 0.3, 24)
    # row 2: steps of +-3 (about 15 events in one frame) at random frames
    jump = rng.choice(W, 12, replace=False)
    at = rng.integers(1, T, 12)
    for x, f in zip(jump, at):
        fr[f:, 2, x] += rng.choice([-3.0, 3.0])
    # row 3: every pixel moves at frames 6..9 (crowded windows)
    fr[6:10, 3, :] += rng.uniform(-0.6, 0.6, (4, W)).cumsum(axis=0)
    fr = fr.astype(np.float32)
    kw = dict(c_pos=0.2, c_neg=0.2, sigma_c=0.02, refractory_us=30, seed=9, input_is_log=True,
              max_frames_per_step=T, pixels_per_thread=ppt, prefetch_frames=win)
    g, o = _sims(W, H, **kw)
    g.step(torch.from_numpy(fr).cuda(), 0, DT)
    ev, seg = g.drain()
    rev, rseg = o.step(fr, 0, DT)
    assert_same(ev, seg, rev, rseg, "crowded tiles")
    assert len(rev) > 1000
    _check_state(g, o)
    # a second, continuing step (the first interval's L_a comes from the state)
    fr2 = (fr[::-1] + np.float32(0.05)).copy()
    g.step(torch.from_numpy(fr2).cuda(), T * DT + 700, DT)
    ev, seg = g.drain()
    rev, rseg = o.step(fr2, T * DT + 700, DT)
    assert_same(ev, seg, rev, rseg, "crowded tiles, continuing step")
    _check_state(g, o)
    g.close()


def test_threshold_maps_match_oracle():
    W, H = 300, 200
    from paper_2602_15018_gb300 import EventSim
    g = EventSim(W, H, c_pos=0.2, c_neg=0.25, sigma_c=0.03, c_min=0.01, seed=12345)
    cp, cn = g.thresholds()
    ocp, ocn = oracle.threshold_maps(W, H, 0.2, 0.25, 0.03, 0.01, 12345)
    assert np.array_equal(cp, ocp) and np.array_equal(cn, ocn)
    g.close()


def test_multi_step_gaps_host_and_device_drain():
    """Steps with uneven gaps between them, host-memory frames, several steps
    between drains, drains to device memory; state identical after each drain."""
    W, H = 160, 96
    sc = scenes.TextureScene(W, H, seed=4, speed=(300., 600.))
    fr = scenes.render_frames(sc, 60).numpy()
    g, o = _sims(W, H, c_pos=0.2, c_neg=0.25, sigma_c=0.02, refractory_us=150, seed=8,
                 max_frames_per_step=32)
    plan = [(0, 1, 0), (1, 9, 2500), (9, 10, 13000), (10, 30, 20000), (30, 31, 41500),
            (31, 60, 43000)]
    batches = [[0, 1], [2, 3], [4, 5]]
    for b, idx in enumerate(batches):
        rev_all, rseg_all = [], [0]
        for k in idx:
            f0, f1, t0 = plan[k]
            chunk = np.ascontiguousarray(fr[f0:f1])
            if k % 2:
                g.step_host(chunk, t0, DT)
            else:
                g.step(torch.from_numpy(chunk).cuda(), t0, DT)
            rev, rseg = o.step(chunk, t0, DT)
            rev_all.append(rev)
            rseg_all.extend((rseg[1:] + rseg_all[-1]).tolist())
        if b == 1:
            ev_t, seg = g.drain(to="cuda")
            ev = ev_t.cpu().numpy().view(np.uint64)
        else:
            ev, seg = g.drain()
        assert_same(ev, seg, np.concatenate(rev_all), np.array(rseg_all), f"batch {b}")
        _check_state(g, o)
    g.close()


def test_pinned_host_frames_read_in_place_and_replayed():
    """Pinned host frames (read in place by the emission kernel) and pageable
    ones (copied to the staging buffer) give the oracle's events, also when an
    overflow makes the drain replay both steps from the host frames."""
    W, H, T = 240, 180, 40
    fr = scenes.render_frames(scenes.SinusoidScene(W, H, seed=5), T)
    g, o = _sims(W, H, c_pos=0.2, c_neg=0.2, max_frames_per_step=T, event_capacity=1000)
    pinned = fr[:20].contiguous().pin_memory()
    g.step_host(pinned, 0, DT)
    g.step_host(np.ascontiguousarray(fr[20:].numpy()), 20 * DT, DT)
    host_out = torch.empty(1 << 20, dtype=torch.int64).pin_memory()
    ev, seg = g.drain(to="cpu", out=host_out)
    rev, rseg = o.step(fr.numpy(), 0, DT)
    assert_same(ev.numpy().view(np.uint64), seg, rev, rseg, "host frames")
    _check_state(g, o)
    g.close()


def test_overflow_regrowth_is_exact():
    """A tiny initial capacity must regrow and replay without changing a bit."""
    W, H, T = 240, 180, 60
    fr = scenes.render_frames(scenes.SinusoidScene(W, H, seed=3), T)
    g, o = _sims(W, H, c_pos=0.2, c_neg=0.2, max_frames_per_step=T, event_capacity=1000)
    g.step(fr[:30].contiguous().cuda(), 0, DT)
    g.step(fr[30:].contiguous().cuda(), 30 * DT, DT)
    n, nseg = g.pending()
    ev, seg = g.drain()
    rev, rseg = o.step(fr.numpy(), 0, DT)
    assert n == len(rev) and nseg == T - 1
    assert_same(ev, seg, rev, rseg, "overflow")
    g.close()


def test_checkpoint_resume_bit_identical():
    W, H = 128, 72
    fr = scenes.render_frames(scenes.TextureScene(W, H, seed=9, speed=(300., 600.)), 40)
    kw = dict(c_pos=0.2, c_neg=0.25, sigma_c=0.03, refractory_us=100, seed=1,
              max_frames_per_step=40)
    from paper_2602_15018_gb300 import EventSim
    a = EventSim(W, H, **kw)
    a.step(fr.cuda(), 0, DT)
    ea, sa = a.drain()
    b = EventSim(W, H, **kw)
    b.step(fr[:17].contiguous().cuda(), 0, DT)
    e1, s1 = b.drain()
    st = b.get_state()
    b.close()
    c = EventSim(W, H, **kw)
    c.set_state(st["ref"], st["lprev"], st["tlast"], st["tau_prev"], st["has_prev"])
    c.step(fr[17:].contiguous().cuda(), 17 * DT, DT)
    e2, s2 = c.drain()
    assert np.array_equal(np.concatenate([e1, e2]), ea)
    assert np.array_equal(np.concatenate([s1, s2[1:] + s1[-1]]), sa)
    a.close()
    c.close()


def test_error_codes():
    from paper_2602_15018_gb300 import EventSim, NeurosimError
    with pytest.raises(NeurosimError, match="E_INVALID"):
        EventSim(0, 10)
    with pytest.raises(NeurosimError, match="E_INVALID"):
        EventSim(10, 10, c_pos=0.0)
    g = EventSim(8, 8, max_frames_per_step=4, input_is_log=True)
    fr = torch.zeros(2, 8, 8, device="cuda")
    g.step(fr, 1000, DT)
    with pytest.raises(NeurosimError, match="E_TIME"):
        g.step(fr, 1500, DT)          # not after the last frame (2000)
    with pytest.raises(NeurosimError, match="E_TIME"):
        g.step(fr, 5000, 0)
    with pytest.raises(NeurosimError, match="E_INVALID"):
        g.step(torch.zeros(5, 8, 8, device="cuda"), 9000, DT)   # more than max frames
    with pytest.raises(NeurosimError, match="E_STATE"):
        g.set_state(np.zeros(64), np.zeros(64), np.zeros(64), 0)
    g.step(torch.full((1, 8, 8), float("nan"), device="cuda"), 3000, DT)
    ev, seg = g.drain()            # NaN log input clamps to -32: OFF events, no fault
    assert len(ev) > 0 and np.all(oracle.unpack(ev)[3] == 0)
    g.close()


def test_hd_full_size_whole_stream():
    """The HD workload at full size (1280x720, 2000 frames, C+ 0.2, C- 0.25,
    sigma 0.03, refractory 100 us) in the benchmark's launch configuration:
    every record (about 15.6 M) and every interval offset of the step against
    the FP32 oracle over the whole frame, bit for bit, plus the final state.
    The oracle runs band-parallel on the host cores (pixels are independent;
    banded_step equals one oracle sensor, a CPU test checks)."""
    import bench
    W, H, T = 1280, 720, 2000
    frames = bench.render_config2(seed=0, device="cuda")
    from paper_2602_15018_gb300 import EventSim
    g = EventSim(W, H, **bench.CONFIG2_SIM, max_frames_per_step=T)
    g.step(frames, 0, DT)
    ev, seg = g.drain()
    st = g.get_state()
    cp, cn = g.thresholds()
    g.close()
    ocp, ocn = oracle.threshold_maps(W, H, 0.2, 0.25, 0.03, 0.01, bench.CONFIG2_SIM["seed"])
    assert np.array_equal(cp, ocp) and np.array_equal(cn, ocn)
    host = frames.cpu().numpy()
    del frames
    torch.cuda.empty_cache()
    rev, rseg, _, ost = oracle.banded_step(host, W, H, 0, DT, ocp, ocn, refractory_us=100)
    assert len(seg) == T and len(rev) > 10_000_000
    assert np.array_equal(seg, rseg)
    assert np.array_equal(ev, rev)
    assert np.array_equal(st["ref"], ost["ref"]) and np.array_equal(st["lprev"], ost["lprev"])
    assert np.array_equal(st["tlast"].astype(np.int64), np.where(ost["tlast"] < 0, 0xFFFFFFFF, ost["tlast"]))


@pytest.mark.parametrize("W,H", [(65535, 64), (65, 32767)])
def test_maximum_sizes_and_64_bit_keys(W, H):
    """The largest sensors the library accepts (2^22 pixels, x up to 65534 and
    y up to 32766 in the record): 22 pixel bits + 10 time bits + polarity take
    the 64-bit keys of the emission kernel and the interval sort, and the
    record's coordinates reach their extremes."""
    T = 6
    fr = scenes.random_log_frames(W, H, T, seed=W + H, step=0.15)
    g, o = _sims(W, H, c_pos=0.2, c_neg=0.25, sigma_c=0.03, refractory_us=100, seed=3, input_is_log=True,
                 max_frames_per_step=T)
    g.step(torch.from_numpy(fr).cuda(), 0, DT)
    ev, seg = g.drain()
    rev, rseg = o.step(fr, 0, DT)
    assert_same(ev, seg, rev, rseg, f"{W}x{H}")
    _check_state(g, o)
    x = (rev >> np.uint64(1)) & np.uint64(0xFFFF)
    y = (rev >> np.uint64(17)) & np.uint64(0x7FFF)
    assert int(x.max()) == W - 1 and int(y.max()) == H - 1
    g.close()


def test_long_gap_takes_64_bit_keys():
    """A step that continues after a 5 s gap: its first interval needs 23 time
    bits, so a 1000x700 sensor (20 pixel bits) switches to 64-bit keys for
    that step and back for the next."""
    W, H, T = 1000, 700, 8
    fr = scenes.random_log_frames(W, H, 3 * T, seed=11, step=0.12)
    g, o = _sims(W, H, c_pos=0.2, c_neg=0.2, sigma_c=0.02, refractory_us=50, seed=5, input_is_log=True,
                 max_frames_per_step=T)
    starts = [0, 5_000_000 + T * DT, 5_000_000 + 2 * T * DT]
    for k, t0 in enumerate(starts):
        chunk = np.ascontiguousarray(fr[k * T:(k + 1) * T])
        g.step(torch.from_numpy(chunk).cuda(), t0, DT)
        ev, seg = g.drain()
        rev, rseg = o.step(chunk, t0, DT)
        assert_same(ev, seg, rev, rseg, f"step {k}")
        assert len(rev) > 1000
    _check_state(g, o)
    g.close()
