"""The no-allocation step entry point gives the same events as the regular one.

neurosim_evsim_step_noalloc is meant for callers that cannot call cudaMalloc
(real-time loops that must not enter the device allocator, hosts that only
borrow device buffers from another runtime): every buffer is the caller's,
and the library's intermediates live in one fixed device array.  This test
runs two consecutive steps through it, carrying the per-pixel state in
caller-owned buffers, and compares events, interval offsets and state with
the regular handle API (neurosim_evsim_step + drain) on the same frames; the
two must agree bit for bit, as every GPU parity test here requires.  It also
reads the device's free memory (cudaMemGetInfo) around the calls: the second
call must leave it unchanged, and the first may lower it by no more than the
fixed array and the code of the module that holds it, which the driver loads
on first use.

The file name sorts last so that a run stopping at the first failure has run
every other test already; it also passes on its own in a fresh process.
"""
import ctypes as C

import numpy as np
import pytest
import torch

import scenes

pytestmark = pytest.mark.gpu

DT = 1000


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import __graft_entry__
    __graft_entry__.build()


def _ptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None else C.c_void_p(0)


def test_noalloc_matches_regular_entry_point_two_calls():
    from paper_2602_15018_gb300 import EventSim, _lib
    W, H, T = 320, 181, 40
    fr = scenes.render_frames(scenes.TextureScene(W, H, seed=21, speed=(300.0, 600.0)), 2 * T)
    fr = fr.cuda()
    kw = dict(c_pos=0.2, c_neg=0.25, sigma_c=0.03, refractory_us=100, seed=5)

    # regular entry point: two steps, drained separately
    ref_sim = EventSim(W, H, max_frames_per_step=T, **kw)
    ref_ev, ref_seg = [], []
    for s in range(2):
        ref_sim.step(fr[s * T:(s + 1) * T].contiguous(), s * T * DT, DT)
        ev, seg = ref_sim.drain()
        ref_ev.append(ev)
        ref_seg.append(seg)
    st = ref_sim.get_state()
    cp, cn = ref_sim.thresholds()
    ref_sim.close()

    L = _lib.lib()
    dev = torch.device("cuda")
    npix = W * H
    cp_d = torch.from_numpy(np.ascontiguousarray(cp.ravel())).to(dev)
    cn_d = torch.from_numpy(np.ascontiguousarray(cn.ravel())).to(dev)
    ref_a = torch.empty(npix, dtype=torch.float32, device=dev)
    lp_a = torch.empty_like(ref_a)
    tl_a = torch.empty(npix, dtype=torch.int32, device=dev)
    ref_b = torch.empty_like(ref_a)
    lp_b = torch.empty_like(ref_a)
    tl_b = torch.empty_like(tl_a)
    cap = 2_000_000
    events = [torch.empty(cap, dtype=torch.int64, device=dev) for _ in range(2)]
    offs = [torch.empty(T, dtype=torch.int64, device=dev), torch.empty(T + 1, dtype=torch.int64, device=dev)]
    frames = [fr[s * T:(s + 1) * T].contiguous() for s in range(2)]
    stream = torch.cuda.current_stream().cuda_stream
    counts = []
    tau = -1
    torch.cuda.synchronize()
    free = [torch.cuda.mem_get_info()[0]]
    for s in range(2):
        n = C.c_uint64(0)
        src = (ref_a, lp_a, tl_a) if s == 1 else (None, None, None)
        dst = (ref_a, lp_a, tl_a) if s == 0 else (ref_b, lp_b, tl_b)
        rc = L.neurosim_evsim_step_noalloc(
            _ptr(frames[s]), T, W, H, s * T * DT, DT, _ptr(cp_d), _ptr(cn_d), 0.2, 0.25, 100, 1e-3, 0,
            _ptr(src[0]), _ptr(src[1]), _ptr(src[2]), _ptr(dst[0]), _ptr(dst[1]), _ptr(dst[2]),
            1 if s == 1 else 0, tau, _ptr(events[s]), cap, _ptr(offs[s]), C.byref(n), C.c_void_p(stream))
        _lib.check(rc)
        counts.append(n.value)
        free.append(torch.cuda.mem_get_info()[0])
        tau = s * T * DT + (T - 1) * DT
    # nothing allocated: the second call leaves the free memory as it was; the
    # first may only add the fixed 32 MiB array and its module's code
    assert free[2] == free[1], f"the second call changed free device memory by {free[1] - free[2]} bytes"
    assert 0 <= free[0] - free[1] <= (32 << 20) + (16 << 20), f"first call: {free[0] - free[1]} bytes"
    for s in range(2):
        got = events[s][: counts[s]].cpu().numpy().view(np.uint64)
        assert counts[s] == len(ref_ev[s]) > 0
        assert np.array_equal(got, ref_ev[s]), f"events of call {s} differ"
        assert np.array_equal(offs[s].cpu().numpy(), ref_seg[s]), f"offsets of call {s} differ"
    assert np.array_equal(ref_b.cpu().numpy(), st["ref"])
    assert np.array_equal(lp_b.cpu().numpy(), st["lprev"])
    assert np.array_equal(tl_b.cpu().numpy().view(np.uint32), st["tlast"])


def test_noalloc_rejects_steps_beyond_the_fixed_scratch():
    from paper_2602_15018_gb300 import _lib
    L = _lib.lib()
    W, H, T = 1280, 720, 2000          # chunk table alone: 1999 x 1800 x 8 bytes > 16 MiB
    dev = torch.device("cuda")
    frames = torch.zeros(4, dtype=torch.float32, device=dev)   # never read: rejected first
    state = torch.zeros(W * H, dtype=torch.float32, device=dev)
    tl = torch.zeros(W * H, dtype=torch.int32, device=dev)
    offs = torch.zeros(T + 1, dtype=torch.int64, device=dev)
    n = C.c_uint64(0)
    rc = L.neurosim_evsim_step_noalloc(
        _ptr(frames), T, W, H, 0, DT, C.c_void_p(0), C.c_void_p(0), 0.2, 0.2, 0, 1e-3, 0,
        C.c_void_p(0), C.c_void_p(0), C.c_void_p(0), _ptr(state), _ptr(state), _ptr(tl), 0, 0,
        C.c_void_p(0), 0, _ptr(offs), C.byref(n), C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 1, rc       # NEUROSIM_E_INVALID
    assert b"scratch" in L.neurosim_last_error()
