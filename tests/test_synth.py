"""Checks of the seeded input generators (not of the method)."""
import math

import numpy as np

from paper_2410_02314_gb300 import synth


def test_splitmix64_published_vector():
    # splitmix64 started from state 0: the first outputs are the well-known reference values
    z = synth.splitmix64(0, 3)
    assert [int(v) for v in z] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_weight_init_bounds_and_blob_roundtrip():
    spec = synth.spec_48()
    w = synth.init_weights(spec, 123, bn=True)
    for layer, a in enumerate(w.conv_w):
        fan_in = (1 if layer == 0 else 48) * 9
        assert np.abs(a).max() <= math.sqrt(6 / fan_in)
        assert np.abs(w.conv_b[layer]).max() <= 1 / math.sqrt(fan_in)
    blob = synth.pack_blob(spec, w)
    hdr, w2 = synth.unpack_blob(blob)
    assert hdr["L"] == 8 and hdr["C"] == 48 and hdr["has_bn"] == 1 and hdr["dil"] == list(spec.dilations)
    for a, b in zip(w.conv_w, w2.conv_w):
        np.testing.assert_array_equal(a.astype(np.float32), b)
    assert synth.init_weights(spec, 123, bn=True).conv_w[3][5, 7, 1, 2] == w.conv_w[3][5, 7, 1, 2]


def test_psf_mass_and_centre():
    em = synth.Emitters(frame=np.array([0], np.int32), x=np.array([20.3]), y=np.array([17.8]), z=np.array([0.0]),
                        photons=np.array([3000.0]), bg=np.array([0.0]))
    mu = synth.render_expected(em, 1, 40, 40, astig=False)
    assert abs(mu.sum() - 3000.0) < 3000.0 * 1e-5
    ii, jj = np.mgrid[0:40, 0:40]
    assert abs((mu[0] * jj).sum() / mu.sum() - 20.3) < 1e-6
    assert abs((mu[0] * ii).sum() / mu.sum() - 17.8) < 1e-6


def test_astigmatic_widths():
    sx, sy = synth.sigma_xy(np.array([-400.0, 0.0, 400.0]), astig=True)
    np.testing.assert_allclose(sx, 1.3 * np.sqrt(1 + (np.array([0.0, 400.0, 800.0]) / 500.0) ** 2))
    np.testing.assert_allclose(sy, sx[::-1])


def test_poisson_moments_and_adu():
    rng = np.random.default_rng(0)
    em = synth.Emitters(frame=np.zeros(0, np.int32), x=np.zeros(0), y=np.zeros(0), z=np.zeros(0),
                        photons=np.zeros(0), bg=np.array([100.0]))
    adu = synth.simulate(em, 1, 300, 300, synth.Camera(2.0, 100.0), False, rng).astype(np.float64)
    e = (adu - 100.0) / 2.0
    assert abs(e.mean() - 100.0) < 0.2
    assert abs(e.var() / 100.0 - 1.0) < 0.03


def test_scmos_maps_distribution():
    cam = synth.scmos_camera(np.random.default_rng(1), 512, 512)
    assert abs(cam.gain_map.mean() - 2.0) < 0.002 and abs(cam.gain_map.std() - 0.1) < 0.002
    assert abs(cam.offset_map.mean() - 100.0) < 0.05 and abs(cam.offset_map.std() - 5.0) < 0.05


def test_training_targets():
    rng = np.random.default_rng(2)
    frames, tgt, em, _ = synth.training_batch(rng, B=8, H=32, W=32)
    assert frames.shape == (8, 32, 32) and tgt.shape == (8, 5, 32, 32)
    m = tgt[:, 0] > 0.5
    assert m.sum() <= em.x.size
    assert np.all(np.abs(tgt[:, 1][m]) <= 0.5 + 1e-6) and np.all(np.abs(tgt[:, 2][m]) <= 0.5 + 1e-6)


def test_training_net_refuses_topologies_it_cannot_train():
    """The training kernels cover the plain stack with five heads and one input frame; other
    specs are refused when the trainable net is built, not trained wrongly."""
    import pytest

    from paper_2410_02314_gb300.train import DilatedLocNet

    plain = synth.NetSpec(in_ch=1, channels=16, dilations=(1, 2, 1))
    DilatedLocNet.from_blob(plain.to_json(), synth.pack_blob(plain, synth.init_weights(plain, 1)))
    for kw in (dict(dcd={"growth": 16, "blocks": [[2]]}), dict(unet=1), dict(n_heads=9), dict(in_ch=3)):
        spec = synth.NetSpec(**{**plain.__dict__, **kw})
        with pytest.raises(ValueError):
            DilatedLocNet.from_blob(spec.to_json(), synth.pack_blob(spec, synth.init_weights(spec, 1)))
