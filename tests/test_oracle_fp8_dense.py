"""Pins of the oracle's e4m3 mode for nets with dense connection dilated blocks (Sec. 3.2.1)
and the U-Net fine stage (Sec. 3.2).

Their layers read channels written by several layers, each stored with its own activation
scale, so the oracle folds every input channel's scale into the weights before the
per-output-channel rounding.  Pinned by:
  * the channel provenance of a hand-counted net;
  * a net with dense blocks of no layers, which is a plain stack: with power-of-two scales the
    fold changes no rounding, so it must equal the plain-stack e4m3 oracle (the C forward);
  * an independent torch emulation of a dense + U-Net net: torch's own e4m3 cast at the same
    points, torch conv2d, max_pool2d, interpolate and cat;
  * the activation scales: each layer's largest output in an independent torch forward.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_2410_02314_gb300 import synth

torch = pytest.importorskip("torch")
F = torch.nn.functional


def test_input_producers_of_a_dense_block_and_unet():
    spec = synth.NetSpec(in_ch=1, channels=16, dilations=(1, 2, 1), unet=2, dcd={"growth": 16, "blocks": [[2, 4]]})
    net = oracle.Net(spec.to_json(), synth.pack_blob(spec, synth.init_weights(spec, 1)))
    kinds = [k for _, _, _, k in net.layers]
    assert kinds == ["stem", "dense", "dense", "transition", "plain", "down", "down", "up", "up", "plain"]
    pr = [list(p) for p in oracle.input_producers(net)]
    assert pr[0] == [-1]                                   # the stem reads the frames
    assert pr[1] == [0] * 16                               # first dense layer: the block input
    assert pr[2] == [0] * 16 + [1] * 16                    # block input, then dense layer 1
    assert pr[3] == [0] * 16 + [1] * 16 + [2] * 16         # the transition reads it all
    assert pr[4] == [3] * 16                               # plain layer after the block
    assert pr[5] == [4] * 16                               # level 1 down: pooled layer-4 features
    assert pr[6] == [5] * 16                               # level 2 down
    assert pr[7] == [5] * 16 + [6] * 16                    # level 1 up: skip, then upsampled level 2
    assert pr[8] == [4] * 16 + [7] * 16                    # level 0 up: skip, then upsampled level 1
    assert pr[9] == [8] * 16                               # the last layer


def test_empty_dense_blocks_equal_the_plain_stack_in_e4m3():
    dil = (1, 2, 4, 1)
    plain = synth.NetSpec(in_ch=1, channels=16, dilations=dil)
    dense = synth.NetSpec(in_ch=1, channels=16, dilations=dil, dcd={"growth": 16, "blocks": []})
    wts = synth.init_weights(plain, 5)
    net_p = oracle.Net(plain.to_json(), synth.pack_blob(plain, wts))
    net_d = oracle.Net(dense.to_json(), synth.pack_blob(dense, wts))
    assert [k for _, _, _, k in net_d.layers] == ["stem", "plain", "plain", "plain"]
    frames = np.random.default_rng(2).integers(100, 900, (2, 19, 23)).astype(np.uint16)
    x0 = oracle.ingest(frames, 1.0, 100.0, in_scale=net_p.in_scale)[:, None]
    # powers of two near amax / 448: scaling by them is exact, so the fold rounds nothing new
    sc = [1.0] + [2.0 ** np.round(np.log2(s)) for s in oracle.act_scales(net_p, frames)[1:]]
    got = oracle.forward_x(oracle.quantized(net_d, "fp8", sc), x0, quant="fp8", scales=sc)
    ref = oracle.forward_x(oracle.quantized(net_p, "fp8"), x0, quant="fp8", scales=sc)
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()
    # and e4m3 did round: the result is not the float64 one
    assert np.abs(ref - oracle.forward_x(net_p, x0)).max() > 1e-4 * np.abs(ref).max()


def _e4m3(t):
    return t.to(torch.float32).to(torch.float8_e4m3fn).to(torch.float64)


def test_dense_unet_e4m3_matches_torch_emulation():
    spec = synth.NetSpec(in_ch=1, channels=16, dilations=(1, 2, 1), unet=2, dcd={"growth": 16, "blocks": [[2, 4]]})
    blob = synth.pack_blob(spec, synth.init_weights(spec, 7))
    net = oracle.Net(spec.to_json(), blob)
    w = synth.blob_f32_weights(blob, spec)
    frames = np.random.default_rng(4).integers(100, 900, (1, 13, 14)).astype(np.uint16)
    x0 = oracle.ingest(frames, 1.0, 100.0, in_scale=net.in_scale)[:, None]
    sc = oracle.act_scales(net, frames)
    assert len(sc) == net.L and all(s > 0 for s in sc)
    got = oracle.forward_x(oracle.quantized(net, "fp8", sc), x0, quant="fp8", scales=sc)

    li = 0

    def conv(parts, d, last=False):
        """parts: list of (stored tensor, producing layer) concatenated along channels."""
        nonlocal li
        t = torch.cat([p for p, _ in parts], 1)
        wl = torch.from_numpy(w.conv_w[li])
        if li > 0:
            s_in = torch.cat([torch.full((p.shape[1],), sc[src + 1], dtype=torch.float32) for p, src in parts])
            wf = wl.to(torch.float32) * s_in[None, :, None, None]
            sw = wf.abs().amax(dim=(1, 2, 3)) / 448.0
            wl = _e4m3(wf / sw[:, None, None, None]) * sw.to(torch.float64)[:, None, None, None] \
                / s_in.to(torch.float64)[None, :, None, None]
        out = torch.relu(F.conv2d(t, wl, torch.from_numpy(w.conv_b[li]), padding=d, dilation=d))
        if not last:
            inv = torch.tensor(1.0 / sc[li + 1], dtype=torch.float32)
            out = _e4m3(out.to(torch.float32) * inv) * sc[li + 1]
        li += 1
        return out, li - 1

    def pool(p):
        return F.max_pool2d(p[0], 2, 2, ceil_mode=True), p[1]

    def up(p, like):
        return F.interpolate(p[0], scale_factor=2, mode="nearest")[:, :, : like[0].shape[2], : like[0].shape[3]], p[1]

    stem = conv([(torch.from_numpy(x0), -1)], 1)
    d1 = conv([stem], 2)
    d2 = conv([stem, d1], 4)
    tr = conv([stem, d1, d2], 1)
    a = conv([tr], 2)
    s1 = conv([pool(a)], 1)
    s2 = conv([pool(s1)], 1)
    u1 = conv([s1, up(s2, s1)], 1)
    u0 = conv([a, up(u1, a)], 1)
    last, _ = conv([u0], 1, last=True)
    ref = F.conv2d(last, torch.from_numpy(w.head_w)[:, :, None, None], torch.from_numpy(w.head_b)).numpy()
    assert np.abs(got - ref).max() <= 1e-9 * np.abs(ref).max()


def test_dense_fp8_mode_needs_the_scales():
    spec = synth.NetSpec(in_ch=1, channels=16, dilations=(1, 1), dcd={"growth": 16, "blocks": [[2]]})
    net = oracle.Net(spec.to_json(), synth.pack_blob(spec, synth.init_weights(spec, 3)))
    with pytest.raises(ValueError):
        oracle.quantized(net, "fp8")
    with pytest.raises(ValueError):
        oracle.forward_x(net, np.zeros((1, 1, 5, 5)), quant="fp8")


def test_dense_unet_activation_scales_are_the_layer_output_maxima():
    """act_scales of a dense + U-Net net: 1 for the frames, then each conv layer's largest
    stored output / 448, in execution order (layers 0..L-2), from an independent torch
    forward of the same net."""
    spec = synth.NetSpec(in_ch=1, channels=16, dilations=(1, 2, 1), unet=2, dcd={"growth": 16, "blocks": [[2, 4]]})
    blob = synth.pack_blob(spec, synth.init_weights(spec, 9))
    net = oracle.Net(spec.to_json(), blob)
    w = synth.blob_f32_weights(blob, spec)
    frames = np.random.default_rng(6).integers(100, 900, (2, 13, 14)).astype(np.uint16)
    x0 = torch.from_numpy(oracle.ingest(frames, 1.0, 100.0, in_scale=net.in_scale)[:, None])
    outs = []

    def conv(t, d):
        li = len(outs)
        out = torch.relu(F.conv2d(t, torch.from_numpy(w.conv_w[li]), torch.from_numpy(w.conv_b[li]), padding=d,
                                  dilation=d))
        outs.append(out)
        return out

    stem = conv(x0, 1)
    d1 = conv(stem, 2)
    d2 = conv(torch.cat([stem, d1], 1), 4)
    a = conv(conv(torch.cat([stem, d1, d2], 1), 1), 2)
    s1 = conv(F.max_pool2d(a, 2, 2, ceil_mode=True), 1)
    s2 = conv(F.max_pool2d(s1, 2, 2, ceil_mode=True), 1)
    up = lambda t, like: F.interpolate(t, scale_factor=2, mode="nearest")[:, :, : like.shape[2], : like.shape[3]]
    u1 = conv(torch.cat([s1, up(s2, s1)], 1), 1)
    conv(conv(torch.cat([a, up(u1, a)], 1), 1), 1)
    assert len(outs) == net.L
    want = [1.0] + [float(o.max()) / 448.0 for o in outs[:-1]]
    got = oracle.act_scales(net, frames, 1.0, 100.0)
    np.testing.assert_allclose(got, want, rtol=1e-12)
