"""Pins for the oracle's float64 forward (dilated conv stack + heads).

Each test checks the oracle against something other than itself: PyTorch's and SciPy's
convolution routines, the polyphase identity of dilated convolution, the receptive-field
support, translation equivariance, BatchNorm folding, and an analytic network whose
output is known in closed form.
"""
import math

import numpy as np
import pytest
import torch
import torch.nn.functional as F
from scipy.signal import correlate2d

import oracle
from paper_2410_02314_gb300 import synth


def make_net(C, dil, seed=7, in_ch=1, bn=False, positive=False, zero_bias=False):
    spec = synth.NetSpec(in_ch=in_ch, channels=C, dilations=tuple(dil))
    w = synth.init_weights(spec, seed, bn=bn)
    if positive:
        w.conv_w = [np.abs(a) for a in w.conv_w]
        w.head_w = np.abs(w.head_w)
    if zero_bias:
        w.conv_b = [np.zeros_like(b) for b in w.conv_b]
        w.head_b = np.zeros_like(w.head_b)
    blob = synth.pack_blob(spec, w)
    return spec, blob, oracle.Net(spec.to_json(), blob), synth.blob_f32_weights(blob, spec)


def torch_reference(x0, w, dil, bn=None, eps=1e-5):
    """The same network through torch.nn.functional.conv2d (float64, padding = dilation)."""
    a = torch.from_numpy(x0)
    for layer, d in enumerate(dil):
        a = F.conv2d(a, torch.from_numpy(w.conv_w[layer]), torch.from_numpy(w.conv_b[layer]),
                     padding=d, dilation=d)
        if bn is not None:
            g, be, mu, var = (torch.from_numpy(v) for v in bn[layer])
            a = F.batch_norm(a, mu, var, g, be, training=False, eps=eps)
        a = torch.relu(a)
    h = F.conv2d(a, torch.from_numpy(w.head_w)[:, :, None, None], torch.from_numpy(w.head_b))
    return h.numpy()


@pytest.mark.parametrize(
    "C,dil,H,W",
    [(3, (1, 2, 4), 9, 11), (4, (1, 2, 4, 8, 4, 1), 13, 12), (2, (3, 5), 7, 16), (3, (16, 1), 10, 9),
     # a plain stack of 20 layers: the version-2 blob of stacks beyond 16 layers
     (2, (1, 2, 1, 3) * 5, 9, 10)],
)
def test_forward_matches_torch_conv2d(C, dil, H, W):
    _, _, net, w = make_net(C, dil)
    rng = np.random.default_rng(11)
    x0 = rng.normal(0.5, 0.5, (2, 1, H, W))
    got = oracle.forward_x(net, x0)
    ref = torch_reference(x0, w, dil)
    assert np.max(np.abs(got - ref)) <= 1e-12 * max(1.0, np.max(np.abs(ref)))


def test_bn_unfolded_matches_torch_batch_norm():
    dil = (1, 2, 4)
    _, _, net, w = make_net(3, dil, bn=True)
    rng = np.random.default_rng(12)
    x0 = rng.normal(0.5, 0.5, (2, 1, 10, 10))
    got = oracle.forward_x(net, x0)
    ref = torch_reference(x0, w, dil, bn=w.bn, eps=w.bn_eps)
    assert np.max(np.abs(got - ref)) <= 1e-12


def test_bn_fold_invariance():
    """BN applied unfolded equals a plain net with W' = W g/sqrt(v+e), b' = (b-m) g/sqrt(v+e) + beta."""
    dil = (1, 2, 4)
    spec, _, net_bn, w = make_net(3, dil, bn=True)
    folded = synth.Weights([], [], None, 0.0, w.head_w, w.head_b)
    for layer in range(len(dil)):
        g, be, mu, var = w.bn[layer]
        s = g / np.sqrt(var + w.bn_eps)
        folded.conv_w.append(w.conv_w[layer] * s[:, None, None, None])
        folded.conv_b.append((w.conv_b[layer] - mu) * s + be)
    # float64 copy of the folded weights, bypassing the float32 blob
    net_f = oracle.Net(spec.to_json(), synth.pack_blob(spec, folded))
    net_f.conv_w = np.concatenate([a.ravel() for a in folded.conv_w])
    net_f.conv_b = np.concatenate(folded.conv_b)
    x0 = np.random.default_rng(13).normal(0.5, 0.5, (1, 1, 12, 12))
    np.testing.assert_allclose(oracle.forward_x(net_bn, x0), oracle.forward_x(net_f, x0), rtol=0, atol=1e-12)


@pytest.mark.parametrize("d", [1, 2, 3, 5])
def test_single_channel_layer_matches_scipy_correlate(d):
    """One channel, one layer: conv = correlate2d with the kernel dilated by zero insertion."""
    _, _, net, w = make_net(1, (d,), seed=21)
    x0 = np.random.default_rng(d).normal(0.0, 1.0, (1, 1, 12, 14))
    k = np.zeros((2 * d + 1, 2 * d + 1))
    k[::d, ::d] = w.conv_w[0][0, 0]
    a = np.maximum(correlate2d(x0[0, 0], k, mode="same", boundary="fill") + w.conv_b[0][0], 0.0)
    ref = w.head_w[:, 0][:, None, None] * a[None] + w.head_b[:, None, None]
    np.testing.assert_allclose(oracle.forward_x(net, x0)[0], ref, rtol=0, atol=1e-12)


@pytest.mark.parametrize("d", [2, 3])
def test_polyphase_identity(d):
    """A dilation-d layer equals an undilated layer applied to each of the d*d sub-grids."""
    spec_d, blob, net_d, w = make_net(3, (d,), seed=31)
    spec_1 = synth.NetSpec(in_ch=1, channels=3, dilations=(1,))
    net_1 = oracle.Net(spec_1.to_json(), synth.pack_blob(spec_1, w))
    x0 = np.random.default_rng(32).normal(0.0, 1.0, (1, 1, 13, 17))
    full = oracle.forward_x(net_d, x0)
    for a in range(d):
        for b in range(d):
            sub = oracle.forward_x(net_1, np.ascontiguousarray(x0[:, :, a::d, b::d]))
            np.testing.assert_allclose(full[:, :, a::d, b::d], sub, rtol=0, atol=1e-12)


@pytest.mark.parametrize("dil", [(1, 2, 4, 8, 4, 1), (1, 2, 4, 8, 16, 8, 4, 1)])
def test_receptive_field_is_exact_box(dil):
    """Positive weights, zero biases, one positive input pixel: the heads are nonzero exactly
    on the (2R+1)^2 box around it (every offset in [-R, R] is a sum of +-d_l)."""
    R = sum(dil)
    _, _, net, _ = make_net(2, dil, positive=True, zero_bias=True)
    S = 2 * R + 9
    x0 = np.zeros((1, 1, S, S))
    c = S // 2
    x0[0, 0, c, c] = 1.0
    h = oracle.forward_x(net, x0)[0, 0]
    support = np.argwhere(h != 0.0)
    assert support[:, 0].min() == c - R and support[:, 0].max() == c + R
    assert support[:, 1].min() == c - R and support[:, 1].max() == c + R
    assert len(support) == (2 * R + 1) ** 2


def test_translation_equivariance():
    dil = (1, 2, 4)
    R = sum(dil)
    _, _, net, _ = make_net(3, dil)
    x0 = np.random.default_rng(41).normal(0.5, 0.5, (1, 1, 40, 40))
    shifted = np.zeros_like(x0)
    shifted[:, :, 3:, 5:] = x0[:, :, :-3, :-5]
    h = oracle.forward_x(net, x0)
    hs = oracle.forward_x(net, shifted)
    inner = (slice(None), slice(None), slice(R + 3, 40 - R), slice(R + 5, 40 - R))
    inner_src = (slice(None), slice(None), slice(R, 40 - R - 3), slice(R, 40 - R - 5))
    np.testing.assert_allclose(hs[inner], h[inner_src], rtol=0, atol=1e-12)


def test_forward_window_equals_whole_frame():
    spec = synth.spec_small()
    w = synth.init_weights(spec, 5)
    blob = synth.pack_blob(spec, w)
    net = oracle.Net(spec.to_json(), blob)
    frames = np.random.default_rng(3).integers(90, 400, (1, 70, 66)).astype(np.uint16)
    full = oracle.forward(net, frames)
    for (i0, i1, j0, j1) in [(0, 9, 0, 7), (30, 41, 20, 33), (60, 70, 50, 66)]:
        part = oracle.forward_window(net, frames, i0, i1, j0, j1)
        np.testing.assert_array_equal(part, full[:, :, i0:i1, j0:j1])


def test_ingest_camera_transform():
    """x = (adu - offset)/gain * in_scale, checked on hand-picked values."""
    f = np.array([[[100, 350], [1100, 0]]], dtype=np.uint16)
    x = oracle.ingest(f, gain=2.0, offset=100.0, in_scale=1e-3)
    np.testing.assert_allclose(x[0], [[0.0, 0.125], [0.5, -0.05]], rtol=0, atol=1e-15)
    gm = np.array([[1.0, 2.0], [4.0, 0.5]])
    om = np.array([[100.0, 50.0], [100.0, 0.0]])
    x = oracle.ingest(f, gain_map=gm, offset_map=om, in_scale=1.0)
    np.testing.assert_allclose(x[0], [[0.0, 150.0], [250.0, 0.0]], rtol=0, atol=1e-12)


def test_sigmoid_matches_scipy_expit():
    from scipy.special import expit

    h = np.linspace(-30, 30, 1001)
    np.testing.assert_allclose(oracle.sigmoid(h), expit(h), rtol=1e-15, atol=0)


def analytic_net(L, dil, smooth_layer, a, b):
    """Channel 0 carries the image: every layer is the identity (centre tap 1) except one
    layer, which is a 3x3 box filter (all taps 1/9) at its dilation.  The p head is a*x - b,
    the offset, z and photon heads are 0.  Other channels are zero."""
    C = 2
    spec = synth.NetSpec(in_ch=1, channels=C, dilations=tuple(dil))
    ws, bs = [], []
    for layer in range(L):
        cin = 1 if layer == 0 else C
        w = np.zeros((C, cin, 3, 3))
        if layer == smooth_layer:
            w[0, 0] = 1.0 / 9.0
        else:
            w[0, 0, 1, 1] = 1.0
        ws.append(w)
        bs.append(np.zeros(C))
    hw = np.zeros((5, C))
    hw[0, 0] = a
    hb = np.array([-b, 0.0, 0.0, 0.0, 0.0])
    return spec, synth.pack_blob(spec, synth.Weights(ws, bs, None, 0.0, hw, hb))


def test_analytic_network_recovers_emitter_grid():
    """Noise-free emitters centred on pixels of a grid (spacing > 2R+3) come back exactly
    at their positions: the smoothed PSF peaks at the emitter pixel and offsets are 0."""
    dil = (1, 2, 1)
    R = sum(dil)
    spec, blob = analytic_net(3, dil, 1, a=200.0, b=20.0)
    net = oracle.Net(spec.to_json(), blob)
    T, H, W = 2, 60, 64
    sp = 2 * R + 5
    ys, xs = np.meshgrid(np.arange(6, H - 6, sp), np.arange(6, W - 6, sp), indexing="ij")
    n = ys.size
    em = synth.Emitters(frame=np.repeat(np.arange(T, dtype=np.int32), n), x=np.tile(xs.ravel(), T).astype(float),
                        y=np.tile(ys.ravel(), T).astype(float), z=np.zeros(T * n),
                        photons=np.full(T * n, 4000.0), bg=np.full(T, 50.0))
    frames = synth.simulate(em, T, H, W, synth.Camera(1.0, 100.0), False, None, noise=False)
    recs, heads, maps = oracle.localize(net, frames, p_min=0.5)
    got = sorted(zip(recs["frame"].tolist(), recs["y"].tolist(), recs["x"].tolist()))
    want = sorted(zip(em.frame.tolist(), em.y.tolist(), em.x.tolist()))
    assert got == want
    assert np.all(recs["z"] == 0.0) and np.all(recs["photons"] == 0.0)


# ----------------------------------------------------------------------------- narrow formats


def test_bf16_rounding_matches_torch_cast():
    rng = np.random.default_rng(1)
    v = np.concatenate([rng.normal(0, 1, 20000), rng.normal(0, 1e-3, 5000), rng.normal(0, 1e4, 5000),
                        [0.0, 1.0, -1.0, 1.00390625, 1.01171875, 3.0e38]])
    got = oracle.round_to(v, "bf16")
    ref = torch.from_numpy(v.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(got, ref)


def test_e4m3_rounding_matches_torch_cast_and_saturates():
    rng = np.random.default_rng(2)
    v = np.concatenate([rng.uniform(-448, 448, 20000), rng.normal(0, 1e-2, 5000), rng.normal(0, 3e-3, 5000),
                        [0.0, 2.0 ** -9, 3 * 2.0 ** -10, 2.0 ** -6, 448.0, -448.0, 17.0, 18.0, 19.0]])
    got = oracle.round_to(v, "fp8")
    ref = torch.from_numpy(v.astype(np.float32)).to(torch.float8_e4m3fn).to(torch.float64).numpy()
    np.testing.assert_array_equal(got, ref)
    # beyond the largest finite value: saturate (by the definition of the format's finite range)
    np.testing.assert_array_equal(oracle.round_to(np.array([460.0, 1e6, -500.0]), "fp8"), [448.0, 448.0, -448.0])
    # ties go to the even mantissa: 3*2^-10 lies halfway between 2^-9 and 2^-8
    assert oracle.round_to(np.array([3 * 2.0 ** -10]), "fp8")[0] == 2.0 ** -8


def test_quantized_forward_matches_torch_emulation():
    """The quantized oracle equals an independent torch emulation: e4m3 / bf16 casts at the
    same points, torch conv2d in float64."""
    spec = synth.spec_small()
    blob = synth.pack_blob(spec, synth.init_weights(spec, 4))
    net = oracle.Net(spec.to_json(), blob)
    w = synth.blob_f32_weights(blob)
    frames = np.random.default_rng(3).integers(100, 900, (2, 30, 34)).astype(np.uint16)
    x0 = oracle.ingest(frames, 1.0, 100.0, in_scale=net.in_scale)[:, None]
    scales = oracle.act_scales(net, frames)
    for fmt in ("bf16", "fp8"):
        got = oracle.forward_x(oracle.quantized(net, fmt), x0, quant=fmt, scales=scales)
        a = torch.from_numpy(x0)
        for layer, d in enumerate(net.dil):
            wl = torch.from_numpy(w.conv_w[layer])
            if layer > 0:
                if fmt == "bf16":
                    a = a.to(torch.float32).to(torch.bfloat16).to(torch.float64)
                    wl = wl.to(torch.float32).to(torch.bfloat16).to(torch.float64)
                else:
                    inv = np.float32(1.0 / scales[layer])
                    a = (a.to(torch.float32) * inv).to(torch.float8_e4m3fn).to(torch.float64) * scales[layer]
                    s = (wl.abs().amax(dim=(1, 2, 3)).to(torch.float32) / 448.0)
                    wl = (wl.to(torch.float32) / s[:, None, None, None]).to(torch.float8_e4m3fn).to(torch.float64) \
                        * s.to(torch.float64)[:, None, None, None]
            a = torch.relu(F.conv2d(a, wl, torch.from_numpy(w.conv_b[layer]), padding=d, dilation=d))
        ref = F.conv2d(a, torch.from_numpy(w.head_w)[:, :, None, None], torch.from_numpy(w.head_b)).numpy()
        assert np.abs(got - ref).max() <= 1e-9 * np.abs(ref).max(), fmt


# ----------------------------------------------------------------------------- three-frame context


def test_context_net_matches_torch_conv2d_with_three_input_channels():
    """in_ch = 3: the first layer convolves (frame t-1, t, t+1) as three input channels."""
    _, _, net, w = make_net(3, (1, 2, 4), in_ch=3)
    rng = np.random.default_rng(21)
    x0 = rng.normal(0.5, 0.5, (4, 3, 9, 10))
    got = oracle.forward_x(net, x0)
    ref = torch_reference(x0, w, (1, 2, 4))
    assert np.max(np.abs(got - ref)) <= 1e-12 * max(1.0, np.max(np.abs(ref)))


def _summed_first_layer(spec3, w3, channels):
    """The in_ch = 1 net whose first-layer weights are w3 summed over the given input channels."""
    spec1 = synth.NetSpec(in_ch=1, channels=spec3.channels, dilations=spec3.dilations)
    w1 = synth.init_weights(spec1, 0)
    w1.conv_w = [w3.conv_w[0][:, channels].sum(axis=1, keepdims=True)] + [a.copy() for a in w3.conv_w[1:]]
    w1.conv_b = [b.copy() for b in w3.conv_b]
    w1.head_w, w1.head_b = w3.head_w.copy(), w3.head_b.copy()
    blob = synth.pack_blob(spec1, w1)
    return oracle.Net(spec1.to_json(), blob)


def test_context_of_a_constant_stack_is_linear_in_the_frame_weights():
    """On a stack of identical frames the three input channels are equal inside the stack, so
    the net equals the one-frame net with first-layer weights summed over t-1, t, t+1; at the
    stack's first and last frame the missing neighbour is zero, which leaves only two of the
    three weight slices (zero padding in time, not replication)."""
    spec3 = synth.NetSpec(in_ch=3, channels=4, dilations=(1, 2, 4, 1))
    w3 = synth.init_weights(spec3, 9)
    w3.conv_w[0] = np.round(w3.conv_w[0] * 256.0) / 256.0  # sums of these stay exact in float32
    blob3 = synth.pack_blob(spec3, w3)
    net3, w3 = oracle.Net(spec3.to_json(), blob3), synth.blob_f32_weights(blob3)
    rng = np.random.default_rng(5)
    frame = rng.integers(90, 400, (1, 12, 13)).astype(np.uint16)
    stack = np.repeat(frame, 4, axis=0)
    got = oracle.forward(net3, stack, 1.0, 100.0)
    inner = oracle.forward(_summed_first_layer(spec3, w3, [0, 1, 2]), frame, 1.0, 100.0)[0]
    first = oracle.forward(_summed_first_layer(spec3, w3, [1, 2]), frame, 1.0, 100.0)[0]
    last = oracle.forward(_summed_first_layer(spec3, w3, [0, 1]), frame, 1.0, 100.0)[0]
    tol = 1e-11 * max(1.0, np.abs(inner).max())
    for t in (1, 2):
        assert np.max(np.abs(got[t] - inner)) <= tol
    assert np.max(np.abs(got[0] - first)) <= tol
    assert np.max(np.abs(got[3] - last)) <= tol
    assert np.max(np.abs(first - inner)) > 1e3 * tol  # the edge rule is visible in the output


def test_context_input_order_and_edges():
    x = np.arange(3 * 2 * 2, dtype=np.float64).reshape(3, 2, 2)
    c = oracle.context_input(x, 3)
    assert c.shape == (3, 3, 2, 2)
    assert np.array_equal(c[1, 0], x[0]) and np.array_equal(c[1, 1], x[1]) and np.array_equal(c[1, 2], x[2])
    assert not c[0, 0].any() and not c[2, 2].any()
    assert np.array_equal(oracle.context_input(x, 1)[:, 0], x)
    with pytest.raises(ValueError):
        oracle.context_input(x, 2)


# ----------------------------------------------------------------------------- dense blocks


def _dcd_net(C=8, g=16, blocks=((2, 4), (3,)), plain=(1, 1), seed=13, zero_dense=False):
    spec = synth.NetSpec(in_ch=1, channels=C, dilations=tuple(plain), dcd={"growth": g, "blocks": [list(b) for b in blocks]})
    w = synth.init_weights(spec, seed)
    if zero_dense:
        k = 0
        for b in blocks:
            k += 1  # skip the stem / previous transition
            for _ in b:
                w.conv_w[k] = np.zeros_like(w.conv_w[k])
                w.conv_b[k] = np.zeros_like(w.conv_b[k])
                k += 1
    blob = synth.pack_blob(spec, w)
    return spec, oracle.Net(spec.to_json(), blob), synth.blob_f32_weights(blob, spec)


def test_dense_blocks_match_torch_concatenation():
    """Dense connection dilated blocks: every dense layer convolves the concatenation of the
    block input and the block's earlier outputs; a transition conv maps back to C channels."""
    spec, net, w = _dcd_net()
    rng = np.random.default_rng(17)
    x0 = rng.normal(0.5, 0.5, (2, 1, 11, 13))
    got = oracle.forward_x(net, x0)
    a = torch.from_numpy(x0)
    li = 0

    def conv(t, d):
        nonlocal li
        out = torch.relu(F.conv2d(t, torch.from_numpy(w.conv_w[li]), torch.from_numpy(w.conv_b[li]), padding=d, dilation=d))
        li += 1
        return out

    a = conv(a, spec.dilations[0])
    for block in spec.dcd["blocks"]:
        feats = [a]
        for d in block:
            feats.append(conv(torch.cat(feats, 1), d))
        a = conv(torch.cat(feats, 1), 1)
    for d in spec.dilations[1:]:
        a = conv(a, d)
    ref = F.conv2d(a, torch.from_numpy(w.head_w)[:, :, None, None], torch.from_numpy(w.head_b)).numpy()
    assert np.max(np.abs(got - ref)) <= 1e-12 * max(1.0, np.abs(ref).max())


def test_dense_blocks_with_silent_dense_layers_reduce_to_the_plain_stack():
    """With all dense layers zero (weights and biases), their outputs are ReLU(0) = 0, so each
    transition sees the block input padded with zeros: the net equals the plain stack whose
    transition weights are their first C input channels (computed by the plain forward)."""
    C = 8
    spec, net, w = _dcd_net(C=C, zero_dense=True)
    plain_spec = synth.NetSpec(in_ch=1, channels=C, dilations=(1, 1, 1, 1))  # stem, 2 transitions, last
    pw = synth.init_weights(plain_spec, 0)
    keep = [0, 3, 5, 6]  # stem, transition 1, transition 2, last plain layer
    pw.conv_w = [w.conv_w[k][:, :C] if k in (3, 5) else w.conv_w[k] for k in keep]
    pw.conv_b = [w.conv_b[k] for k in keep]
    pw.head_w, pw.head_b = w.head_w, w.head_b
    plain = oracle.Net(plain_spec.to_json(), synth.pack_blob(plain_spec, pw))
    rng = np.random.default_rng(3)
    frames = rng.integers(90, 500, (2, 14, 15)).astype(np.uint16)
    got = oracle.forward(net, frames, 1.0, 100.0)
    want = oracle.forward(plain, frames, 1.0, 100.0)
    assert np.max(np.abs(got - want)) <= 1e-12 * max(1.0, np.abs(want).max())


def test_dense_blocks_window_equals_whole_frame():
    spec, net, _ = _dcd_net()
    assert net.R == sum(d for _, _, d in spec.layers())
    rng = np.random.default_rng(9)
    frames = rng.integers(90, 500, (1, 40, 44)).astype(np.uint16)
    whole = oracle.forward(net, frames, 1.0, 100.0)
    win = oracle.forward_window(net, frames, 18, 24, 20, 27, 1.0, 100.0)
    assert np.array_equal(win, whole[:, :, 18:24, 20:27])
