"""Pins for the oracle's U-Net fine stage (Sec. 3.2: a two-stage U-Net after feature
extraction, two upsampling stages, Sec. 4.2): 2x2 max pooling, nearest upsampling, the
skip concatenation and the level structure, each against PyTorch's routines; the windowed
forward against the whole frame; the receptive-radius bound against an impulse response."""
import numpy as np
import pytest
import torch
import torch.nn.functional as F

import oracle
from paper_2410_02314_gb300 import synth


@pytest.mark.parametrize("H,W", [(8, 8), (7, 9), (1, 5), (13, 2)])
def test_pool2_matches_torch_max_pool_ceil_mode(H, W):
    a = np.random.default_rng(H * 31 + W).normal(0.0, 1.0, (3, H, W))
    ref = F.max_pool2d(torch.from_numpy(a)[None], 2, 2, ceil_mode=True)[0].numpy()
    got = oracle.pool2(a)
    assert got.shape == (3, (H + 1) // 2, (W + 1) // 2) and np.array_equal(got, ref)


@pytest.mark.parametrize("h,w,H,W", [(4, 4, 8, 8), (4, 5, 7, 9), (1, 3, 1, 5), (7, 1, 13, 2)])
def test_upsample2_is_nearest_and_cropped(h, w, H, W):
    a = np.random.default_rng(h * 7 + w).normal(0.0, 1.0, (2, h, w))
    got = oracle.upsample2(a, H, W)
    ref = F.interpolate(torch.from_numpy(a)[None], scale_factor=2, mode="nearest")[0].numpy()[:, :H, :W]
    assert np.array_equal(got, ref)
    i, j = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
    assert np.array_equal(got, a[:, i // 2, j // 2])


def _unet_net(levels, dcd=None, C=8, dil=(1, 2, 1), seed=19, n_heads=5):
    spec = synth.NetSpec(in_ch=1, channels=C, dilations=tuple(dil), unet=levels, dcd=dcd, n_heads=n_heads)
    blob = synth.pack_blob(spec, synth.init_weights(spec, seed))
    return spec, oracle.Net(spec.to_json(), blob), synth.blob_f32_weights(blob, spec)


def _torch_unet(spec, w, x0):
    """The same net through torch conv2d, max_pool2d (ceil_mode), interpolate (nearest) and cat."""
    li = 0

    def conv(t, d):
        nonlocal li
        out = torch.relu(F.conv2d(t, torch.from_numpy(w.conv_w[li]), torch.from_numpy(w.conv_b[li]), padding=d,
                                  dilation=d))
        li += 1
        return out

    a = torch.from_numpy(x0)
    if spec.dcd:
        a = conv(a, spec.dilations[0])
        for block in spec.dcd["blocks"]:
            feats = [a]
            for d in block:
                feats.append(conv(torch.cat(feats, 1), d))
            a = conv(torch.cat(feats, 1), 1)
        feat_dil = spec.dilations[1:-1]
    else:
        feat_dil = spec.dilations[:-1]
    for d in feat_dil:
        a = conv(a, d)
    skips = [a]
    for _ in range(spec.unet):
        skips.append(conv(F.max_pool2d(skips[-1], 2, 2, ceil_mode=True), 1))
    up = skips.pop()
    while skips:
        skip = skips.pop()
        u = F.interpolate(up, scale_factor=2, mode="nearest")[:, :, : skip.shape[2], : skip.shape[3]]
        up = conv(torch.cat([skip, u], 1), 1)
    a = conv(up, spec.dilations[-1])
    return F.conv2d(a, torch.from_numpy(w.head_w)[:, :, None, None], torch.from_numpy(w.head_b)).numpy()


@pytest.mark.parametrize("levels,dcd,H,W", [(1, None, 9, 11), (2, None, 13, 10), (2, None, 16, 16),
                                             (2, {"growth": 16, "blocks": [[2, 3]]}, 11, 14)])
def test_unet_net_matches_torch_composition(levels, dcd, H, W):
    spec, net, w = _unet_net(levels, dcd)
    assert net.L == spec.L and [c for c, _, _, _ in net.layers] == [c for c, _, _ in spec.layers()]
    x0 = np.random.default_rng(H + W).normal(0.5, 0.5, (2, 1, H, W))
    got = oracle.forward_x(net, x0)
    ref = _torch_unet(spec, w, x0)
    assert np.max(np.abs(got - ref)) <= 1e-12 * max(1.0, np.abs(ref).max())


def test_unet_nine_heads_and_bf16_mode_round_only_conv_outputs():
    """The bf16 mode equals a torch emulation that rounds every conv output but the last to bf16
    (pooling and upsampling move the rounded values unchanged) with bf16-rounded weights."""
    spec, net, w = _unet_net(2, n_heads=9)
    q = oracle.quantized(net, "bf16")
    x0 = np.random.default_rng(3).normal(0.5, 0.5, (1, 1, 12, 13))
    got = oracle.forward_x(q, x0, quant="bf16")
    bf = lambda t: t.to(torch.float32).to(torch.bfloat16).to(torch.float64)
    wq = synth.Weights([w.conv_w[0]] + [bf(torch.from_numpy(a)).numpy() for a in w.conv_w[1:]], w.conv_b, None, 1e-5,
                       w.head_w, w.head_b)
    li = 0

    def conv(t, d, last=False):
        nonlocal li
        out = torch.relu(F.conv2d(t, torch.from_numpy(wq.conv_w[li]), torch.from_numpy(wq.conv_b[li]), padding=d,
                                  dilation=d))
        li += 1
        return out if last else bf(out)

    a = torch.from_numpy(x0)
    for d in spec.dilations[:-1]:
        a = conv(a, d)
    s1 = conv(F.max_pool2d(a, 2, 2, ceil_mode=True), 1)
    s2 = conv(F.max_pool2d(s1, 2, 2, ceil_mode=True), 1)
    u = conv(torch.cat([s1, F.interpolate(s2, scale_factor=2, mode="nearest")[:, :, : s1.shape[2], : s1.shape[3]]], 1), 1)
    u = conv(torch.cat([a, F.interpolate(u, scale_factor=2, mode="nearest")[:, :, : a.shape[2], : a.shape[3]]], 1), 1)
    a = conv(u, spec.dilations[-1], last=True)
    ref = F.conv2d(a, torch.from_numpy(w.head_w)[:, :, None, None], torch.from_numpy(w.head_b)).numpy()
    assert got.shape[1] == 9 and np.max(np.abs(got - ref)) <= 1e-12 * max(1.0, np.abs(ref).max())


def test_unet_window_equals_whole_frame():
    spec, net, _ = _unet_net(2, dil=(1, 2, 3, 1))
    rng = np.random.default_rng(5)
    frames = rng.integers(95, 700, (1, 90, 97)).astype(np.uint16)
    whole = oracle.forward(net, frames)
    for i0, j0 in [(0, 0), (37, 41), (66, 73), (45, 3)]:
        blk = oracle.forward_window(net, frames, i0, i0 + 17, j0, j0 + 19)
        assert np.max(np.abs(blk - whole[:, :, i0 : i0 + 17, j0 : j0 + 19])) <= 1e-12 * np.abs(whole).max()


def test_unet_receptive_radius_bounds_the_impulse_response():
    """A net with positive weights and zero biases: the heads respond to an input impulse
    exactly on a box around it, which R bounds."""
    spec = synth.NetSpec(in_ch=1, channels=4, dilations=(1, 2, 1), unet=2)
    w = synth.init_weights(spec, 7)
    w.conv_w = [np.abs(a) for a in w.conv_w]
    w.conv_b = [np.zeros_like(b) for b in w.conv_b]
    w.head_w, w.head_b = np.abs(w.head_w), np.zeros_like(w.head_b)
    net = oracle.Net(spec.to_json(), synth.pack_blob(spec, w))
    H = W = 2 * net.R + 41
    for c in (H // 2, H // 2 + 1):  # both pooling phases
        x0 = np.zeros((1, 1, H, W))
        x0[0, 0, c, c] = 1.0
        h = oracle.forward_x(net, x0)[0, 0]
        ii, jj = np.nonzero(h)
        assert len(ii) > 0 and np.abs(ii - c).max() <= net.R and np.abs(jj - c).max() <= net.R
    assert net.R == spec.R == 1 + 2 + 1 + 24
