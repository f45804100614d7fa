"""Pins that tie the oracle to facts outside itself.

Each pin takes an oracle library handle (the default build, or a copy of the
oracle with a planted mistake in the mutation test) and raises AssertionError
when the oracle disagrees with:
  - closed forms (exact linear log ramps, Sec. 2 model with readings R2-R4),
  - an analytically derived refractory sequence (reading R5),
  - brute-force time sampling of the linear interpolant (reading R2),
  - the double-precision libm log (reading R1),
  - the published SplitMix64 test vector and Irwin-Hall moments (reading R6),
  - invariants of the model (reference band, ordering, time range),
  - closed forms of the first-order bandwidth filter (reading R13).
"""
from __future__ import annotations

import math
from fractions import Fraction

import numpy as np

import oracle
import scenes

DT = 1000


def _sim(library, W, H, c=0.25, cneg=None, **kw):
    cp = np.full((H, W), c, np.float32)
    cn = np.full((H, W), c if cneg is None else cneg, np.float32)
    return oracle.OracleSim(W, H, c_pos_map=cp, c_neg_map=cn, library=library, **kw)


def _ramp_expected(l0, s, C, n_frames, up=True, R=0):
    """Analytic events of an exact ramp L_f = l0 +- f s, threshold C, one pixel.

    The k-th crossing is at level k C from the start; it lies in interval
    j = ceil(k C / s) - 1 (frame j to j+1) at t = j dt + floor((k C - j s) / s * dt).
    Returns a list of (interval, t, polarity)."""
    s_, C_ = Fraction(s), Fraction(C)
    total = Fraction(n_frames - 1) * s_
    out, last = [], None
    k = 1
    while k * C_ <= total:
        j = math.ceil(k * C_ / s_) - 1
        frac = (k * C_ - j * s_) / s_
        t = j * DT + math.floor(frac * DT)
        if R == 0 or last is None or t - last >= R:
            out.append((j, t, 1 if up else 0))
            last = t
        k += 1
    return out


def _events_with_interval(ev, seg):
    t, x, y, p = oracle.unpack(ev)
    j = np.repeat(np.arange(len(seg) - 1), np.diff(seg))
    return j, t, x, y, p


def pin_ramps(library):
    """Exact ramps: counts, intervals and times of every event (readings R2-R4)."""
    W, H = 3, 2
    for s, up in [(0.0625, True), (0.09375, True), (0.0625, False), (0.09375, False),
                  (0.75, True), (0.75, False)]:
        n = 41
        sign = 1 if up else -1
        frames = scenes.log_ramp(W, H, n, 0.0, sign * s)
        sim = _sim(library, W, H, input_is_log=True)
        ev, seg = sim.step(frames, 0, DT)
        assert len(seg) == n, "one interval per frame after the first"
        j, t, x, y, p = _events_with_interval(ev, seg)
        exp = _ramp_expected(0.0, s, 0.25, n, up)
        assert len(ev) == len(exp) * W * H, (s, up, len(ev), len(exp) * W * H)
        for px in range(W * H):
            xx, yy = px % W, px // W
            m = (x == xx) & (y == yy)
            got = list(zip(j[m].tolist(), t[m].tolist(), p[m].tolist()))
            assert got == exp, (s, up, px, got[:5], exp[:5])


def pin_constant_and_first_frame(library):
    """No change, no events; the first frame ever emits nothing (reading R7)."""
    W, H = 5, 4
    sim = _sim(library, W, H, input_is_log=True)
    ev, seg = sim.step(np.full((1, H, W), 0.3, np.float32), 0, DT)
    assert len(ev) == 0 and len(seg) == 1
    ev, seg = sim.step(np.full((6, H, W), 0.3, np.float32), 1000, DT)
    assert len(ev) == 0 and len(seg) == 7
    # a jump of exactly 3 C in one interval after a flat start: 3 events per pixel
    fr = np.full((1, H, W), 0.3 + 0.75, np.float32)
    ev, seg = sim.step(fr, 7000, DT)
    assert len(ev) == 3 * W * H, len(ev)


def pin_refractory(library):
    """Steep ramp, 4 crossings per interval at 250 us spacing; refractory R."""
    W, H = 2, 2
    for R in (300, 500, 1000):
        n = 12
        frames = scenes.log_ramp(W, H, n, 0.0, 1.0)
        sim = _sim(library, W, H, input_is_log=True, refractory_us=R)
        ev, seg = sim.step(frames, 0, DT)
        j, t, x, y, p = _events_with_interval(ev, seg)
        exp = _ramp_expected(0.0, 1.0, 0.25, n, True, R=R)
        m = (x == 1) & (y == 1)
        got = list(zip(j[m].tolist(), t[m].tolist(), p[m].tolist()))
        assert got == exp, (R, got[:6], exp[:6])
        # ref still advances through suppressed crossings: the band holds
        L = np.float32(11.0)
        assert np.all(sim.ref + np.float32(0.25) > L) and np.all(sim.ref - np.float32(0.25) < L)


def _brute_force_pixel(vals, C, D=DT, sub=16):
    """Sample the linear interpolant every 1/sub us; an event fires at the first
    sample at or past ref + C (or ref - C), after which ref moves by C."""
    ref = float(vals[0])
    out = []
    ts = np.arange(1, D * sub + 1) / sub
    for j in range(len(vals) - 1):
        a, b = float(vals[j]), float(vals[j + 1])
        Ls = a + (b - a) * ts / D          # monotone in the interval
        if b > a:
            while Ls[-1] >= ref + C:
                k = int(np.searchsorted(Ls, ref + C, side="left"))
                ref += C
                out.append((j, j * D + math.floor(ts[k]), 1))
        elif b < a:
            while Ls[-1] <= ref - C:
                k = int(np.searchsorted(-Ls, -(ref - C), side="left"))
                ref -= C
                out.append((j, j * D + math.floor(ts[k]), 0))
    return out


def pin_brute_force(library, seed=7):
    """8x6 pixels x 6 frames of random log values vs brute-force time sampling."""
    W, H, T = 8, 6, 6
    rng = np.random.default_rng(seed)
    for C in (0.1, 0.2, 0.25):
        fr = rng.uniform(-1.0, 1.0, (T, H, W)).astype(np.float32)
        sim = _sim(library, W, H, c=C, input_is_log=True)
        ev, seg = sim.step(fr, 0, DT)
        j, t, x, y, p = _events_with_interval(ev, seg)
        Cf = float(np.float32(C))
        for yy in range(H):
            for xx in range(W):
                exp = _brute_force_pixel(fr[:, yy, xx].astype(np.float64), Cf)
                m = (x == xx) & (y == yy)
                got = list(zip(j[m].tolist(), t[m].tolist(), p[m].tolist()))
                assert len(got) == len(exp), (C, xx, yy, len(got), len(exp))
                for (gj, gt, gp), (ej, et, ep) in zip(got, exp):
                    assert gj == ej and gp == ep and abs(gt - et) <= 1, (C, xx, yy, got, exp)


def pin_log(library, stride=1):
    """Project log vs libm double log: <= 2 ulp over the intensity domain [1e-8, 1e6+1]."""
    lo = int(np.float32(1e-8).view(np.uint32))
    hi = int(np.float32(1e6 + 1).view(np.uint32))
    err, wb = oracle.mylog_max_ulp(lo, hi, stride, library=library)
    assert err <= 2.0, (err, hex(wb))
    # sparse sweep over every positive float, subnormals included
    err2, wb2 = oracle.mylog_max_ulp(1, 0x7F7FFFFF, 4099, library=library)
    assert err2 <= 2.0, (err2, hex(wb2))
    sp = oracle.mylog(np.array([1.0, 0.0, np.inf, -1.0, np.nan], np.float32), library=library)
    assert sp[0] == 0.0 and sp[1] == -np.inf and sp[2] == np.inf
    assert np.isnan(sp[3]) and np.isnan(sp[4])


def pin_threshold_maps(library):
    """Per-pixel thresholds: clamp, independence of ON/OFF draws, moments (R6)."""
    W, H = 200, 150
    cp, cn = oracle.threshold_maps(W, H, 0.2, 0.25, 0.0, 0.01, 3, library=library)
    assert np.all(cp == np.float32(0.2)) and np.all(cn == np.float32(0.25))
    cp, cn = oracle.threshold_maps(W, H, 0.2, 0.25, 0.03, 0.01, 3, library=library)
    assert abs(cp.mean() - 0.2) < 1e-3 and abs(cn.mean() - 0.25) < 1e-3
    assert abs(cp.std() - 0.03) < 1e-3 and abs(cn.std() - 0.03) < 1e-3
    assert abs(np.corrcoef(cp.ravel(), cn.ravel())[0, 1]) < 0.02
    assert abs(np.corrcoef(cp[:, :-1].ravel(), cp[:, 1:].ravel())[0, 1]) < 0.02
    cp, cn = oracle.threshold_maps(W, H, 0.2, 0.25, 0.5, 0.05, 3, library=library)
    assert cp.min() == np.float32(0.05) and (cp == np.float32(0.05)).mean() > 0.2
    cp2, _ = oracle.threshold_maps(W, H, 0.2, 0.25, 0.5, 0.05, 4, library=library)
    assert not np.array_equal(cp, cp2)
    # realisation convention: pixel u uses normal slot 2u (ON) and 2u + 1 (OFF),
    # added with a + sign (the slots themselves are pinned by the SplitMix64
    # vector and the Irwin-Hall moments)
    cp, cn = oracle.threshold_maps(W, H, 0.2, 0.25, 0.03, 0.01, 9, library=library)
    for u in (0, 1, 777, W * H - 1):
        zp = np.float32(oracle.normal_ih12(9, 2 * u))
        zn = np.float32(oracle.normal_ih12(9, 2 * u + 1))
        assert cp.ravel()[u] == max(np.float32(0.01), np.float32(0.2) + np.float32(0.03) * zp)
        assert cn.ravel()[u] == max(np.float32(0.01), np.float32(0.25) + np.float32(0.03) * zn)


def pin_band_and_order(library, seed=11):
    """Invariants on a seeded texture scene: band, order, time range, count bound."""
    W, H, T = 96, 64, 40
    sc = scenes.TextureScene(W, H, seed=seed, speed=(300.0, 600.0))
    fr = scenes.render_frames(sc, T).numpy()
    sim = oracle.OracleSim(W, H, c_pos=0.2, c_neg=0.25, sigma_c=0.03, refractory_us=0,
                           seed=seed, library=library)
    ev0, _ = sim.step(fr[:1], 0, DT)
    assert len(ev0) == 0
    allL = []
    for f in range(1, T):
        ev, seg = sim.step(fr[f:f + 1], f * DT, DT)
        t, x, y, p = oracle.unpack(ev)
        assert np.all(t >= (f - 1) * DT) and np.all(t <= f * DT)
        assert np.all(np.diff(ev.astype(np.uint64)) >= 0) if len(ev) > 1 else True
        if len(ev) > 1:
            assert np.all(ev[1:] >= ev[:-1])
        L = oracle.mylog(np.minimum(np.maximum(fr[f], 0), 1e6) + np.float32(1e-3)).ravel()
        assert np.all(sim.ref + sim.cpos > L) and np.all(sim.ref - sim.cneg < L)
        allL.append(len(ev))
    assert sum(allL) > 100


def pin_fp64_agreement(library, seed=5):
    """FP32-mirrored vs FP64: <= 1e-4 of events unmatched, matched times within 1 us."""
    W, H, T = 160, 120, 50
    sc = scenes.TextureScene(W, H, seed=seed, speed=(300.0, 600.0))
    fr = scenes.render_frames(sc, T).numpy()
    kw = dict(c_pos=0.2, c_neg=0.25, sigma_c=0.03, refractory_us=100, seed=seed,
              library=library)
    e32, s32 = oracle.OracleSim(W, H, precision="f32", **kw).step(fr, 0, DT)
    e64, s64 = oracle.OracleSim(W, H, precision="f64", **kw).step(fr, 0, DT)
    assert len(e64) > 5000
    r = oracle.match_f1(W, H, e32, e64, tol_us=1)
    unmatched = (r["n_pred"] - r["matched"]) + (r["n_ref"] - r["matched"])
    assert unmatched <= 1e-4 * r["n_ref"] + 2, r


def pin_step_composition(library, seed=3):
    """One step over T frames equals the same frames split over several steps."""
    W, H, T = 40, 30, 24
    fr = scenes.random_log_frames(W, H, T, seed, step=0.15)
    a = _sim(library, W, H, c=0.2, input_is_log=True, refractory_us=50)
    ea, sa = a.step(fr, 100, DT)
    b = _sim(library, W, H, c=0.2, input_is_log=True, refractory_us=50)
    parts, segs = [], [0]
    for f0, f1 in [(0, 1), (1, 9), (9, 10), (10, 24)]:
        e, s = b.step(fr[f0:f1], 100 + f0 * DT, DT)
        parts.append(e)
        segs.extend((s[1:] + segs[-1]).tolist())
    eb = np.concatenate(parts)
    assert np.array_equal(ea, eb)
    assert np.array_equal(sa, np.array(segs))
    assert np.array_equal(a.ref, b.ref) and np.array_equal(a.tlast, b.tlast)


def pin_uneven_interval(library):
    """A step that starts 2500 us after the previous frame (dt = 1000): the first
    interval spans the gap.  A 0.75 rise with C = 0.25 crosses at 1/3, 2/3 and 1
    of the gap: t = 833, 1666, 2500; the next interval is a normal 1000 us one
    with a 0.5 rise: t = 3000, 3500."""
    W, H = 2, 1
    sim = _sim(library, W, H, input_is_log=True)
    sim.step(np.zeros((1, H, W), np.float32), 0, DT)
    fr = np.stack([np.full((H, W), 0.75, np.float32), np.full((H, W), 1.25, np.float32)])
    ev, seg = sim.step(fr, 2500, DT)
    j, t, x, y, p = _events_with_interval(ev, seg)
    m = x == 1
    assert t[m].tolist() == [833, 1666, 2500, 3000, 3500], t[m].tolist()
    assert j[m].tolist() == [0, 0, 0, 1, 1] and np.all(p == 1)


def pin_lowpass(library):
    """Sensor bandwidth filter (reading R13): s_k = s_{k-1} + alpha (L_k - s_{k-1}).

    Closed forms: alpha = 1 follows the frames (within two roundings); a constant input stays
    constant; a unit step reaches 1 - (1 - alpha)^k after k frames, and with
    alpha = 1 - exp(-2 pi f_c dt) it reaches 1 - 1/e after 1 / (2 pi f_c dt)
    frames (the time constant of the continuous first-order filter).
    Invariants: splitting the frames over two calls with the state carried
    gives the same bits; pixels are independent."""
    rng = np.random.default_rng(21)
    L = (rng.standard_normal((12, 3, 5)) * 0.7 - 2.0).astype(np.float32)
    out, st = oracle.lowpass_log(L, 1.0, library=library)
    # alpha = 1: fl(s + fl(L - s)) is L up to the rounding of the difference and of the sum
    prev = np.concatenate([L[:1], out[:-1]])
    bound = np.spacing(np.abs(L - prev)) / 2 + np.spacing(np.maximum(np.abs(L), np.abs(out))) / 2
    assert np.all(np.abs(out - L) <= bound) and np.array_equal(st, out[-1].reshape(-1))
    c = np.full((9, 4), -1.3, np.float32)
    out, _ = oracle.lowpass_log(c, 0.37, library=library)
    assert np.array_equal(out, c)
    n = 20                                            # frames per time constant
    alpha = np.float32(1.0 - math.exp(-1.0 / n))      # f_c = 1 / (2 pi n dt)
    step = np.ones((3 * n + 1, 2), np.float32)
    step[0] = 0.0
    out, _ = oracle.lowpass_log(step, alpha, library=library)
    k = np.arange(3 * n + 1)
    want = 1.0 - (1.0 - np.float64(alpha)) ** k
    assert np.max(np.abs(out[:, 0] - want)) < 2e-6, np.max(np.abs(out[:, 0] - want))
    assert abs(out[n, 0] - (1.0 - math.exp(-1.0))) < 4e-6
    assert np.all(np.diff(out[:, 0]) >= 0) and out[-1, 0] <= 1.0
    a = np.float32(0.23)
    full, st_full = oracle.lowpass_log(L, a, library=library)
    head, st_head = oracle.lowpass_log(L[:5], a, library=library)
    tail, st_tail = oracle.lowpass_log(L[5:], a, state=st_head, library=library)
    assert np.array_equal(np.concatenate([head, tail]), full) and np.array_equal(st_tail, st_full)
    perm = rng.permutation(15)
    flat = L.reshape(12, 15)
    pout, _ = oracle.lowpass_log(flat[:, perm], a, library=library)
    assert np.array_equal(pout, full.reshape(12, 15)[:, perm])
    pin_lowpass_alpha(library)


def pin_lowpass_alpha(library):
    """Gain of the bandwidth filter from its cutoff (reading R13).

    A first-order filter with cutoff f_c has time constant 1 / (2 pi f_c): a unit step
    sampled every dt must reach 1 - 1/e after that many frames.  With f_c dt = 1 / (2 pi n)
    the filter, run with the oracle's own gain, is checked there for several n.  Small
    f_c dt gives alpha ~ 2 pi f_c dt (first order of the series); a very high cutoff gives a
    gain that rounds to 1 (the filter follows the frames); doubling dt gives the square of
    the kept fraction."""
    for n in (5, 20, 64):
        fc = 1.0 / (2.0 * math.pi * n * 1e-3)          # dt = 1000 us
        alpha = oracle.lowpass_alpha(fc, 1000, library=library)
        step = np.ones((n + 1, 1), np.float32)
        step[0] = 0.0
        out, _ = oracle.lowpass_log(step, alpha, library=library)
        assert abs(out[n, 0] - (1.0 - math.exp(-1.0))) < 4e-6, (n, out[n, 0])
    x = 2.0 * math.pi * 1.0 * 10e-6                    # f_c = 1 Hz, dt = 10 us
    a = oracle.lowpass_alpha(1.0, 10, library=library)
    assert abs(a - x) <= x * x, (a, x)
    assert oracle.lowpass_alpha(1e9, 1000, library=library) == np.float32(1.0)
    a1 = np.float64(oracle.lowpass_alpha(37.0, 1000, library=library))
    a2 = np.float64(oracle.lowpass_alpha(37.0, 2000, library=library))
    assert abs((1.0 - a2) - (1.0 - a1) ** 2) < 1e-6
    for bad in ((0.0, 1000), (-5.0, 1000), (10.0, 0), (float("inf"), 1000)):
        try:
            oracle.lowpass_alpha(*bad, library=library)
        except oracle.OracleError:
            continue
        raise AssertionError(f"lowpass_alpha{bad} accepted")


def pin_leak(library):
    """Sensor leak (reading R14): the log input rises by C+ r (t - origin).

    Closed form: a still pixel with C+ = 0.2 and r = 40 Hz fires ON events
    every 1/r = 25 ms (40 in 1 s), all ON, at k * 25000 us within the model's
    rounding; the event rate does not depend on the pixel's threshold (the
    drift scales with C+); r = 0 changes nothing; frames starting later than
    the origin are the matching frames of a run from the origin."""
    T, n = 1001, 3
    L = np.full((T, 1, n), -1.0, np.float32)
    assert np.array_equal(oracle.leak_log(L, 0, DT, 0, 0.0, cpos_u=0.2, library=library), L)
    cp = np.array([0.2, 0.4, 0.1], np.float32)
    out = oracle.leak_log(L, 0, DT, 0, 40.0, cpos=cp, library=library)
    assert abs(out[-1, 0, 0] - 7.0) < 1e-5 and abs(out[-1, 0, 1] - 15.0) < 1e-5 and abs(out[500, 0, 2] - 1.0) < 1e-5
    sim = oracle.OracleSim(n, 1, c_pos_map=cp, c_neg_map=cp, input_is_log=True, library=library)
    ev, _ = sim.step(out, 0, DT)
    t, x, _, p = oracle.unpack(ev)
    assert np.all(p == 1)
    for u in range(n):
        tu = np.sort(t[x == u]).astype(np.int64)
        assert len(tu) in (39, 40), (u, len(tu))
        k = np.arange(1, len(tu) + 1)
        assert np.all(np.abs(tu - k * 25000) <= 2), (u, np.abs(tu - k * 25000).max())
    tail = oracle.leak_log(L[:400], 600 * DT, DT, 0, 40.0, cpos=cp, library=library)
    full = oracle.leak_log(np.full((1000, 1, n), -1.0, np.float32), 0, DT, 0, 40.0, cpos=cp, library=library)
    assert np.array_equal(tail, full[600:1000])


def pin_shot_noise(library):
    """Shot noise (reading R15), against Poisson statistics and its structure:
    the count matches the mean rate * pixels * time (4 sigma), counts per
    tile-interval have variance equal to their mean (Poisson), times are
    uniform in their interval and independent of the pixel, pixels uniform
    (also in a ragged last tile), polarities balanced, every interval sorted;
    an interval's events depend only on its start time (not on how many
    intervals are drawn); zero rate gives nothing; other seeds other events."""
    W, H, r, n_int = 37, 83, 40.0, 500          # 3071 px: 47 full tiles and one of 63
    ev, seg = oracle.shot_noise(W, H, r, 5, 0, 700, DT, n_int, library=library)
    npix = W * H
    expect = r * npix * (700 + (n_int - 1) * DT) * 1e-6
    assert abs(len(ev) - expect) < 4 * np.sqrt(expect), (len(ev), expect)
    t, x, y, p = oracle.unpack(ev)
    pix = y.astype(np.int64) * W + x
    assert np.all((x < W) & (y < H))
    j = np.repeat(np.arange(n_int), np.diff(seg))
    ta = np.where(j == 0, 0, 700 + (j - 1) * DT)
    D = np.where(j == 0, 700, DT)
    off = t.astype(np.int64) - ta
    assert np.all((off >= 0) & (off < D))
    assert abs(np.mean(off[j > 0]) / DT - 0.5) < 0.01
    assert abs(np.mean(p) - 0.5) < 0.01
    for jj in range(n_int):
        e = ev[seg[jj]:seg[jj + 1]]
        assert np.all(e[1:] >= e[:-1])
    tile = pix // 64
    counts = np.bincount((j[j > 0] - 1) * 48 + tile[j > 0], minlength=(n_int - 1) * 48).reshape(n_int - 1, 48)[:, :47]
    m, v = counts.mean(), counts.var()
    assert abs(v / m - 1.0) < 0.05, (m, v)
    per_px = np.bincount(pix, minlength=npix)
    last = per_px[47 * 64:].mean() / per_px[: 47 * 64].mean()
    assert abs(last - 1.0) < 0.1, last
    inner = (pix % 64)[j > 0] / 64.0
    rho = np.corrcoef(inner, off[j > 0] / DT)[0, 1]
    assert abs(rho) < 0.03, rho
    hist = np.bincount(pix % 64, minlength=64)
    assert hist.min() > 0.8 * hist.mean() and hist.max() < 1.2 * hist.mean()
    e5, s5 = oracle.shot_noise(W, H, r, 5, 0, 700, DT, 5, library=library)
    assert np.array_equal(e5, ev[: seg[5]]) and np.array_equal(s5, seg[:6])
    e_shift, s_shift = oracle.shot_noise(W, H, r, 5, 700 + 4 * DT, DT, DT, 3, library=library)
    assert np.array_equal(e_shift, ev[seg[5]:seg[8]])
    z, zs = oracle.shot_noise(W, H, 0.0, 5, 0, 700, DT, 10, library=library)
    assert len(z) == 0 and np.all(zs == 0)
    o, _ = oracle.shot_noise(W, H, r, 6, 0, 700, DT, 5, library=library)
    assert not np.array_equal(o[: min(len(o), len(e5))], e5[: min(len(o), len(e5))])
    try:
        oracle.shot_noise(W, H, 100.0, 5, 0, DT, DT, 2, library=library)   # mean 6.4 per tile: refused
    except oracle.OracleError:
        pass
    else:
        raise AssertionError("a tile mean above 4 was accepted")


def pin_merge(library):
    """Merging interval-structured streams: a permutation of their union,
    sorted per interval; merging with an empty stream changes nothing."""
    a, sa = oracle.shot_noise(40, 30, 20.0, 1, 0, DT, DT, 30, library=library)
    b, sb = oracle.shot_noise(40, 30, 20.0, 2, 0, DT, DT, 30, library=library)
    m, sm = oracle.merge_events(a, sa, b, sb, library=library)
    assert np.array_equal(sm, sa + sb)
    for j in range(30):
        seg = m[sm[j]:sm[j + 1]]
        assert np.all(seg[1:] >= seg[:-1])
        assert np.array_equal(np.sort(seg), np.sort(np.concatenate([a[sa[j]:sa[j + 1]], b[sb[j]:sb[j + 1]]])))
    e, se = oracle.merge_events(a, sa, np.zeros(0, np.uint64), np.zeros(31, np.int64), library=library)
    assert np.array_equal(e, a) and np.array_equal(se, sa)


ALL_PINS = [pin_ramps, pin_uneven_interval, pin_constant_and_first_frame, pin_refractory, pin_brute_force,
            pin_threshold_maps, pin_band_and_order, pin_fp64_agreement, pin_step_composition, pin_lowpass,
            pin_leak, pin_shot_noise, pin_merge]
