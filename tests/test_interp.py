"""The learned interpolator on the tensor cores against its FP64 oracle.

The oracle rounds to BF16 exactly what the GPU stores in BF16 (weights and
activations), so the two differ by FP32 accumulation order and by the BF16
rounding of gradients the GPU keeps between layers; the tolerances below are
derived from that: outputs within 1 % of the residual scale; gradients, against
the oracle that also rounds the activation gradients the GPU stores in BF16,
element by element within 2^-7 (one BF16 ulp) of the tensor's largest entry
plus 2^-6 of the entry (measured differences reach 2^-9 of the largest entry
on these shapes).  Shapes: batch 2, 16 x 24 (several 128-row tiles at full size, ragged
tails at the quarter size), and 1 x 8 x 128 and 1 x 8 x 160, whose full-size
3x3 layers run from halo tiles (rows of 128 pixels; at width 160 the second
tile of a row reaches past the image), 1 x 8 x 256, whose half-size
128-channel layers stream their weights, 1 x 8 x 320 (halo tiles past the
image at 2.5 tiles per row), 1 x 8 x 512 (the quarter-size 128-channel layer
on the streamed-weight kernel) and 1 x 8 x 1280 (every layer at HD widths).
Checkpoints are checked against their documented byte layout.
"""
import numpy as np
import pytest
import torch

from oracle import interp_oracle as io

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import __graft_entry__
    __graft_entry__.build()


def _params(seed):
    p = io.init_params(seed)
    rng = np.random.default_rng(seed + 7)
    p["W9"] = rng.standard_normal((32, 3)) * 0.2
    for k, n in io.BIAS.items():
        p[k] = rng.standard_normal(n) * 0.05
    return p


def _clips(seed, N, H, W):
    """Smooth log-intensity clips [N, 5, H, W]: moving sinusoid patterns."""
    rng = np.random.default_rng(seed)
    y, x = np.mgrid[0:H, 0:W].astype(np.float64)
    out = np.zeros((N, 5, H, W))
    for n in range(N):
        for _ in range(3):
            fx, fy = rng.uniform(0.05, 0.3, 2)
            vx, vy = rng.uniform(-1.5, 1.5, 2)
            ph, a = rng.uniform(0, 6.28), rng.uniform(0.2, 0.6)
            for f in range(5):
                out[n, f] += a * np.sin(fx * (x - vx * f) + fy * (y - vy * f) + ph)
        out[n] += rng.uniform(-3.0, -1.0)
    return out


def _net(p, N=2, H=16, W=24):
    from paper_2602_15018_gb300 import Interpolator
    from paper_2602_15018_gb300.interp import from_dict
    net = Interpolator(N, H, W, seed=1)
    net.set_params(from_dict({k: np.asarray(v, np.float32) for k, v in p.items()}))
    return net


def test_param_roundtrip_and_untrained_is_linear():
    from paper_2602_15018_gb300 import Interpolator
    from paper_2602_15018_gb300.interp import to_dict
    net = Interpolator(2, 16, 24, seed=3)
    p = to_dict(net.get_params())
    assert np.all(p["W9"] == 0) and np.all(p["b9"] == 0) and np.all(p["W1"][:, :, 2:, :] == 0)
    assert 0.5 < np.std(p["W4"]) * np.sqrt(9 * 128 / 2.0) < 1.5        # He-normal scale
    c = torch.from_numpy(_clips(0, 2, 16, 24)).float().cuda()
    out = net.forward(c[:, 0].contiguous(), c[:, 4].contiguous())
    L0, L4 = c[:, 0], c[:, 4]
    for j in range(3):
        assert torch.allclose(out[j], L0 + (j + 1) / 4 * (L4 - L0), atol=1e-6)
    net.close()


# (1, 8, 320): full-size rows of 2.5 halo tiles (the last one past the image),
# as the 320 x 240 sensors of the batched learned path run them; (1, 8, 512):
# the quarter-size 128 -> 128 layer (conv4) and its data gradient take the
# streamed-weight halo kernel (128-pixel rows); (1, 8, 1280): every layer at
# the widths of an HD frame (conv4 on 320-pixel rows, conv6 on 640).
SHAPES = [(2, 16, 24), (1, 8, 128), (1, 8, 160), (1, 8, 256), (1, 8, 320), (1, 8, 512), (1, 8, 1280)]


@pytest.mark.parametrize("N,H,W", SHAPES)
def test_forward_matches_oracle(N, H, W):
    p = _params(11)
    clips = _clips(1, N, H, W)
    net = _net(p, N, H, W)
    c = torch.from_numpy(clips).float().cuda()
    out = net.forward(c[:, 0].contiguous(), c[:, 4].contiguous()).cpu().numpy()
    ref, _ = io.forward(p, clips[:, 0].astype(np.float32), clips[:, 4].astype(np.float32), quantize=True)
    base = np.stack([clips[:, 0] + (j + 1) / 4 * (clips[:, 4] - clips[:, 0]) for j in range(3)])
    r_ref = ref - base
    scale = np.abs(r_ref).max()
    assert scale > 0.05
    assert np.abs(out - ref).max() <= 0.01 * scale + 1e-4, np.abs(out - ref).max()
    net.close()


GRAD_ABS = 2.0 ** -7
GRAD_REL = 2.0 ** -6


@pytest.mark.parametrize("N,H,W", SHAPES)
def test_gradients_match_oracle(N, H, W):
    p = _params(12)
    clips = _clips(2, N, H, W).astype(np.float32)
    net = _net(p, N, H, W)
    loss, g = net.gradients(torch.from_numpy(clips).cuda())
    from paper_2602_15018_gb300.interp import to_dict
    gd = to_dict(g)
    ref_loss, ref_g, _ = io.loss_and_grads(p, clips[:, 0], clips[:, 4], np.moveaxis(clips[:, 1:4], 1, 0),
                                           quantize=True, quantize_grads=True)
    assert abs(loss - ref_loss) <= 1e-3 * ref_loss
    for k in list(io.SHAPES) + list(io.BIAS):
        a, b = np.asarray(gd[k], np.float64).reshape(-1), ref_g[k].reshape(-1)
        nb = np.linalg.norm(b)
        if nb == 0:
            assert np.linalg.norm(a) == 0, k
            continue
        # element by element: the oracle rounds to BF16 every activation and
        # activation gradient the GPU stores in BF16, so the two differ by
        # FP32 accumulation order (relative ~1e-6), by the few BF16 roundings
        # that order flips (one BF16 ulp, 2^-7 relative, of one stored value
        # each), by the rare ReLU mask a flipped activation turns (it passes
        # or stops one pixel-channel's gradient), and through the loss
        # gradient by the forward output's own rounding: GRAD_ABS (one BF16
        # ulp) of the tensor's largest entry plus GRAD_REL of the entry
        bound = GRAD_ABS * np.abs(b).max() + GRAD_REL * np.abs(b)
        bad = np.abs(a - b) > bound
        assert not bad.any(), (k, int(bad.sum()), float(np.abs(a - b).max() / np.abs(b).max()))
        rel = np.linalg.norm(a - b) / nb                    # summary in norm
        assert rel < 2.0 ** -7, (k, rel)
    net.close()


def test_train_step_applies_adamw():
    from paper_2602_15018_gb300.interp import to_dict
    p = _params(13)
    clips = torch.from_numpy(_clips(3, 2, 16, 24)).float().cuda()
    net = _net(p)
    p0 = net.get_params().astype(np.float64)
    _, g = net.gradients(clips)
    net.set_params(p0.astype(np.float32))            # resets the optimiser state
    lr, wd = 1e-3, 1e-4
    net.train_step(clips, lr, wd)
    p1 = net.get_params().astype(np.float64)
    st = io.adamw_init(to_dict(p0))
    want = io.adamw_step(to_dict(p0), to_dict(g.astype(np.float64)), st, lr, wd=wd)
    got = to_dict(p1)
    for k in want:
        assert np.allclose(got[k], want[k], atol=2e-6, rtol=1e-5), k
    net.close()


def test_training_beats_linear_interpolation():
    """A few hundred steps on moving patterns: the trained network predicts the
    intermediate frames of held-out clips better than linear interpolation
    (the untrained network), by at least 10 % in mean absolute log error, and
    the training loss falls."""
    from paper_2602_15018_gb300 import Interpolator
    N, H, W = 8, 32, 32
    net = Interpolator(N, H, W, seed=5)
    held = torch.from_numpy(_clips(999, N, H, W)).float().cuda()

    def err(model):
        out = model.forward(held[:, 0].contiguous(), held[:, 4].contiguous())
        return (out - held[:, 1:4].permute(1, 0, 2, 3)).abs().mean().item()

    e0 = err(net)
    losses = []
    for it in range(300):
        clips = torch.from_numpy(_clips(it, N, H, W)).float().cuda()
        loss = net.train_step(clips, 2e-3 * (0.5 + 0.5 * np.cos(np.pi * it / 300)), 1e-4,
                              want_loss=(it < 10 or it >= 290))
        if loss is not None:
            losses.append(loss)
    e1 = err(net)
    assert np.mean(losses[-10:]) < 0.9 * np.mean(losses[:10]), losses
    assert e1 < 0.9 * e0, (e0, e1)
    net.close()


def _fnv1a(b: bytes) -> int:
    x = 0xcbf29ce484222325
    for c in b:
        x = ((x ^ c) * 0x100000001b3) & 0xFFFFFFFFFFFFFFFF
    return x


def test_checkpoint_layout_and_resume(tmp_path):
    """save/load: the file holds the documented layout (parsed here byte by
    byte); a network of other max sizes loads it bit-exactly (parameters and
    forward output); and a resumed AdamW step matches the uninterrupted one,
    while a parameters-only checkpoint (moments reset) does not."""
    from paper_2602_15018_gb300 import Interpolator
    a = _net(_params(21))
    for it in range(3):
        a.train_step(torch.from_numpy(_clips(40 + it, 2, 16, 24)).float().cuda(), 1e-3, 1e-4, want_loss=False)
    full, bare = str(tmp_path / "full.ckpt"), str(tmp_path / "bare.ckpt")
    a.save(full)
    a.save(bare, with_optimizer=False)
    pa = a.get_params()
    n = pa.size
    raw = open(full, "rb").read()
    assert raw[:8] == b"NSIMUNT1" and len(raw) == 32 + 3 * 4 * n + 8
    version, flags = np.frombuffer(raw[8:16], "<u4")
    count, step = np.frombuffer(raw[16:32], "<i8")
    assert (version, flags, count, step) == (1, 1, n, 3)
    assert np.array_equal(np.frombuffer(raw[32:32 + 4 * n], "<f4"), pa)
    assert int(np.frombuffer(raw[-8:], "<u8")[0]) == _fnv1a(raw[:-8])
    assert len(open(bare, "rb").read()) == 32 + 4 * n + 8

    b = Interpolator(1, 32, 32, seed=9)
    b.load(full)
    assert np.array_equal(b.get_params(), pa)
    c = torch.from_numpy(_clips(77, 1, 16, 24)).float().cuda()
    assert torch.equal(a.forward(c[:, 0].contiguous(), c[:, 4].contiguous()),
                       b.forward(c[:, 0].contiguous(), c[:, 4].contiguous()))
    r = Interpolator(2, 16, 24, seed=9)
    r.load(bare)
    clips = torch.from_numpy(_clips(50, 2, 16, 24)).float().cuda()
    b.close()
    b = Interpolator(2, 16, 24, seed=9)
    b.load(full)
    for net in (a, b, r):
        net.train_step(clips, 1e-3, 1e-4, want_loss=False)
    pa, pb, pr = a.get_params(), b.get_params(), r.get_params()
    d_ab, d_ar = np.abs(pa - pb).max(), np.abs(pa - pr).max()
    assert d_ar > 1e-4 and d_ab < 0.01 * d_ar, (d_ab, d_ar)
    for net in (a, b, r):
        net.close()


def test_checkpoint_rejects_bad_files(tmp_path):
    from paper_2602_15018_gb300 import Interpolator
    from paper_2602_15018_gb300._lib import NeurosimError
    a = _net(_params(22))
    path = str(tmp_path / "a.ckpt")
    a.save(path, with_optimizer=False)
    raw = bytearray(open(path, "rb").read())
    b = Interpolator(2, 16, 24, seed=4)
    p0 = b.get_params()

    def rejects(data, code, what):
        bad = str(tmp_path / "bad.ckpt")
        open(bad, "wb").write(bytes(data))
        with pytest.raises(NeurosimError) as e:
            b.load(bad)
        assert e.value.code == code and what in str(e.value), str(e.value)
        assert np.array_equal(b.get_params(), p0)          # unchanged

    with pytest.raises(NeurosimError) as e:
        b.load(str(tmp_path / "missing.ckpt"))
    assert e.value.code == 8
    rejects(raw[:-100], 1, "truncated")
    flipped = bytearray(raw)
    flipped[1000] ^= 0x40
    rejects(flipped, 1, "checksum")
    rejects(b"NOTACKPT" + raw[8:], 1, "not an interpolator checkpoint")
    other = bytearray(raw[:-8])
    other[16:24] = np.array([12345], "<i8").tobytes()      # another parameter count, valid hash
    rejects(other + np.array([_fnv1a(bytes(other))], "<u8").tobytes(), 1, "parameters")
    assert not (tmp_path / "a.ckpt.tmp").exists()
    a.close()
    b.close()
