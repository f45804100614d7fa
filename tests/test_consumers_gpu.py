"""Time surface and polarity event frames on the GPU against the oracle, on
the events of a simulated texture clip."""
import numpy as np
import pytest
import torch

import oracle
import scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import __graft_entry__
    __graft_entry__.build()


def _events(W=160, H=96, T=80):
    from paper_2602_15018_gb300 import EventSim
    fr = scenes.render_frames(scenes.TextureScene(W, H, seed=31, speed=(300.0, 600.0)), T).cuda()
    s = EventSim(W, H, c_pos=0.2, c_neg=0.25, max_frames_per_step=T)
    s.step(fr, 0, 1000)
    ev, seg = s.drain()
    s.close()
    return ev, seg


def test_time_surface_matches_oracle():
    from paper_2602_15018_gb300 import TimeSurface
    W, H = 160, 96
    ev, seg = _events(W, H)
    assert len(ev) > 1000
    ts = TimeSurface(W, H, tau_us=10_000.0)
    S_o, last = None, None
    # three updates at interval boundaries, events of each chunk after the previous query
    for a, b, tq in ((0, 20, 20_000), (20, 50, 50_500), (50, 79, 79_000)):
        chunk = ev[seg[a]:seg[b]]
        ts.update(torch.from_numpy(chunk.view(np.int64)).cuda(), tq)
        S_o, last = oracle.time_surface(W, H, chunk, 10_000.0, S_o, last)
        ref = np.where(last >= 0, S_o * np.exp(-(tq - last) / 10_000.0), 0.0)
        got = ts.S.cpu().numpy().astype(np.float64)
        assert np.abs(got - ref).max() <= 1e-5 * max(1.0, ref.max()), np.abs(got - ref).max()
    assert ref.max() > 1.0


def test_event_frames_exact():
    from paper_2602_15018_gb300 import event_frames
    W, H = 160, 96
    ev, _ = _events(W, H)
    got = event_frames(torch.from_numpy(ev.view(np.int64)).cuda(), W, H, 3000, 20_000, 4).cpu().numpy()
    ref = oracle.event_frames(W, H, ev, 3000, 20_000, 4)
    assert np.array_equal(got, ref) and ref.sum() > 0
