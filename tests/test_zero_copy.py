"""Zero-copy hand-off of events to PyTorch and variable-length batching.

The paper hands sensor data to NumPy and PyTorch consumers without copies
(Sec. 3, the Cortex paragraph).  In process, the simulator's pending events
can be viewed through DLPack: the torch tensor must alias the library's
record buffer (no copy) and hold exactly what a drain returns; releasing them
must continue the stream as a drain does.  Several sensors' variable-length
drains packed into one preallocated tensor must equal their separate drains.
"""
import ctypes as C

import numpy as np
import pytest
import torch

import scenes

pytestmark = pytest.mark.gpu

DT = 1000
KW = dict(c_pos=0.2, c_neg=0.25, sigma_c=0.03, refractory_us=100, seed=4)


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import __graft_entry__
    __graft_entry__.build()


def _frames(W, H, T, seed):
    return scenes.render_frames(scenes.TextureScene(W, H, seed=seed, speed=(300.0, 600.0)), T).cuda()


def test_dlpack_view_aliases_the_library_buffer_and_equals_drain():
    from paper_2602_15018_gb300 import EventSim, _lib
    W, H, T = 320, 181, 24
    fr = _frames(W, H, 2 * T, 8)
    a = EventSim(W, H, max_frames_per_step=T, **KW)
    b = EventSim(W, H, max_frames_per_step=T, **KW)
    for k in range(2):
        a.step(fr[k * T:(k + 1) * T].contiguous(), k * T * DT, DT)
        b.step(fr[k * T:(k + 1) * T].contiguous(), k * T * DT, DT)
        view, seg = a.events_view()
        ptr, n = C.c_void_p(), C.c_uint64(0)
        _lib.check(_lib.lib().neurosim_evsim_peek_events(a._h, C.byref(ptr), C.byref(n), None, 0, None))
        assert view.is_cuda and view.dtype == torch.int64 and view.numel() == n.value > 0
        assert view.data_ptr() == ptr.value                 # no copy: the library's own buffer
        got = view.cpu().numpy().view(np.uint64).copy()
        del view
        a.release()
        assert a.pending() == (0, 0)
        ev, sb = b.drain()
        assert np.array_equal(got, ev) and np.array_equal(seg, sb), f"step {k}"
    sa, sb = a.get_state(), b.get_state()
    assert all(np.array_equal(sa[k], sb[k]) for k in ("ref", "lprev", "tlast"))
    a.close()
    b.close()


def test_drain_into_packs_variable_length_drains():
    from paper_2602_15018_gb300 import EventSim, drain_into
    dims = [(64, 48), (200, 120), (33, 17)]
    T = 20
    sims, singles, refs = [], [], []
    for i, (W, H) in enumerate(dims):
        fr = _frames(W, H, T, 30 + i)
        s = EventSim(W, H, max_frames_per_step=T, **KW)
        r = EventSim(W, H, max_frames_per_step=T, **KW)
        s.step(fr, 0, DT)
        r.step(fr, 0, DT)
        sims.append(s)
        refs.append(r)
    small = torch.empty(10, dtype=torch.int64, device="cuda")
    with pytest.raises(ValueError):
        drain_into(sims, small)
    assert sum(s.pending()[0] for s in sims) > 10            # nothing was drained
    out = torch.full((10 ** 6,), -1, dtype=torch.int64, device="cuda")
    offsets, segs = drain_into(sims, out)
    packed = out.cpu().numpy().view(np.uint64)
    for i, r in enumerate(refs):
        ev, seg = r.drain()
        assert np.array_equal(packed[offsets[i]:offsets[i + 1]], ev), i
        assert np.array_equal(segs[i], seg), i
    assert np.all(out.cpu().numpy()[offsets[-1]:offsets[-1] + 5] == -1)
    for s in sims + refs:
        s.close()
