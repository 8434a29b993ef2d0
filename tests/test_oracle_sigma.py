"""Pins for the oracle's uncertainty heads (Sec. 3.2: DECODE-style outputs with the offset
uncertainties): the four extra 1x1 heads, their softplus activation and their readout in
the decode.  Each is checked against something other than the oracle itself: PyTorch's
softplus and conv2d, the identity softplus(h) - softplus(-h) = h, and the record's own
pixel found by numpy indexing."""
import numpy as np
import torch
import torch.nn.functional as F

import oracle
from paper_2410_02314_gb300 import synth


def test_softplus_matches_torch_and_its_identities():
    h = np.concatenate([np.linspace(-60.0, 60.0, 4001), [-800.0, -30.5, 0.0, 1e-9, 33.0, 700.0]])
    got = oracle.softplus(h)
    ref = F.softplus(torch.from_numpy(h), beta=1.0, threshold=1e9).numpy()  # log(1 + exp(h)), no linear cut-off
    finite = np.isfinite(ref)
    assert np.allclose(got[finite], ref[finite], rtol=1e-14, atol=1e-300)
    assert got[np.where(h == 0.0)[0][0]] == np.log(2.0)
    # softplus(h) - softplus(-h) = h; softplus > 0 wherever exp(h) does not underflow
    assert np.allclose(got - oracle.softplus(-h), h, rtol=1e-13, atol=1e-13)
    assert np.all(got >= 0.0) and np.all(got[h > -700.0] > 0.0)
    assert got[np.where(h == 700.0)[0][0]] == 700.0


def test_nine_head_forward_matches_torch_and_keeps_the_position_heads():
    """A 9-head net equals torch conv2d with a 9-output 1x1 head; its first five heads equal
    those of the 5-head net with the same conv weights and the first five head rows."""
    spec9 = synth.NetSpec(in_ch=1, channels=4, dilations=(1, 2, 3), n_heads=9)
    w9 = synth.init_weights(spec9, 21)
    blob9 = synth.pack_blob(spec9, w9)
    net9 = oracle.Net(spec9.to_json(), blob9)
    w = synth.blob_f32_weights(blob9)
    rng = np.random.default_rng(3)
    x0 = rng.normal(0.5, 0.5, (2, 1, 9, 12))
    got = oracle.forward_x(net9, x0)
    assert got.shape == (2, 9, 9, 12)
    a = torch.from_numpy(x0)
    for layer, d in enumerate(spec9.dilations):
        a = torch.relu(F.conv2d(a, torch.from_numpy(w.conv_w[layer]), torch.from_numpy(w.conv_b[layer]), padding=d,
                                dilation=d))
    ref = F.conv2d(a, torch.from_numpy(w.head_w)[:, :, None, None], torch.from_numpy(w.head_b)).numpy()
    assert np.max(np.abs(got - ref)) <= 1e-12 * max(1.0, np.abs(ref).max())
    spec5 = synth.NetSpec(in_ch=1, channels=4, dilations=(1, 2, 3))
    w5 = synth.Weights(w9.conv_w, w9.conv_b, None, 1e-5, w9.head_w[:5], w9.head_b[:5])
    net5 = oracle.Net(spec5.to_json(), synth.pack_blob(spec5, w5))
    assert np.array_equal(oracle.forward_x(net5, x0), got[:, :5])


def test_nine_head_dense_block_net_matches_torch():
    spec = synth.NetSpec(in_ch=1, channels=8, dilations=(1, 1), n_heads=9, dcd={"growth": 16, "blocks": [[2, 3]]})
    blob = synth.pack_blob(spec, synth.init_weights(spec, 4))
    net = oracle.Net(spec.to_json(), blob)
    w = synth.blob_f32_weights(blob, spec)
    x0 = np.random.default_rng(5).normal(0.5, 0.5, (1, 1, 10, 11))
    got = oracle.forward_x(net, x0)
    li = 0

    def conv(t, d):
        nonlocal li
        out = torch.relu(F.conv2d(t, torch.from_numpy(w.conv_w[li]), torch.from_numpy(w.conv_b[li]), padding=d,
                                  dilation=d))
        li += 1
        return out

    a = conv(torch.from_numpy(x0), 1)
    feats = [a]
    for d in (2, 3):
        feats.append(conv(torch.cat(feats, 1), d))
    a = conv(conv(torch.cat(feats, 1), 1), 1)
    ref = F.conv2d(a, torch.from_numpy(w.head_w)[:, :, None, None], torch.from_numpy(w.head_b)).numpy()
    assert got.shape[1] == 9 and np.max(np.abs(got - ref)) <= 1e-12 * max(1.0, np.abs(ref).max())


def test_maps_apply_sigmoid_to_p_and_softplus_to_the_uncertainty_heads():
    h = np.random.default_rng(8).normal(0.0, 4.0, (2, 9, 5, 6))
    m = oracle.maps_f32(h)
    assert m.dtype == np.float32 and m.shape == h.shape
    assert np.array_equal(m[:, 0], (1.0 / (1.0 + np.exp(-h[:, 0]))).astype(np.float32))
    assert np.array_equal(m[:, 1:5], h[:, 1:5].astype(np.float32))
    assert np.array_equal(m[:, 5:], F.softplus(torch.from_numpy(h[:, 5:]), threshold=1e9).numpy().astype(np.float32))


def test_sigma_readout_at_the_record_pixel():
    """Records of 9-channel maps equal those of their first five channels; each record's
    uncertainties are the sigma maps at its pixel (offsets 0, so x and y are the pixel
    indices), z and photons scaled by one float32 product."""
    rng = np.random.default_rng(9)
    T, H, W = 3, 17, 21
    maps = rng.uniform(0.05, 2.0, (T, 9, H, W)).astype(np.float32)
    maps[:, 0] = ((rng.permutation(T * H * W) + 0.5) / (T * H * W)).reshape(T, H, W).astype(np.float32)
    maps[:, 1:3] = 0.0
    zs, ps = np.float32(987.654), np.float32(12345.678)
    recs, sig = oracle.decode(maps, 0.3, float(zs), float(ps), with_sigma=True)
    assert len(recs) > 10 and len(sig) == len(recs)
    assert recs.tobytes() == oracle.decode(np.ascontiguousarray(maps[:, :5]), 0.3, float(zs), float(ps)).tobytes()
    for r, s in zip(recs, sig):
        t, i, j = int(r["frame"]), int(r["y"]), int(r["x"])
        assert (r["x"], r["y"]) == (j, i)
        assert s["sigma_x"] == maps[t, 5, i, j] and s["sigma_y"] == maps[t, 6, i, j]
        assert s["sigma_z"] == zs * maps[t, 7, i, j] and s["sigma_photons"] == ps * maps[t, 8, i, j]
