"""GPU parity of nets with the four uncertainty heads (Sec. 3.2: DECODE-style outputs with
the offset uncertainties) through the C ABI.

Maps (9 channels: p, dx, dy, zhat, Nhat, then softplus of the heads sx, sy, sz, sN) against
the oracle, as normalised max errors: channels 0-4 as raw heads (p as its logit), channels
5-8 as the softplus maps.  FP32 <= 1e-4; BF16 against the oracle's bf16 mode (max <= 2e-2,
RMS <= 2e-3) and float64 (<= 3e-2).  Records and their uncertainties are bit-exact against
the oracle's decode of the same GPU maps."""
import json

import numpy as np
import pytest
import torch

import oracle
import paper_2410_02314_gb300 as sml
from paper_2410_02314_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__

    __graft_entry__.build()
    torch.cuda.set_device(0)


def _nets():
    yield "plain48", synth.NetSpec(in_ch=1, channels=48, dilations=(1, 2, 4, 8, 4, 1), n_heads=9)
    yield "dcd32", synth.NetSpec(in_ch=1, channels=32, dilations=(1, 2, 1), n_heads=9,
                                 dcd={"growth": 16, "blocks": [[2, 4, 8]]})


def _maps(loc, frames, cam):
    T, H, W = frames.shape
    maps = torch.empty((T, 9, H, W), dtype=torch.float32, device="cuda")
    logits = torch.empty((T, H, W), dtype=torch.float32, device="cuda")
    gm = None if cam.gain_map is None else torch.from_numpy(cam.gain_map).cuda()
    om = None if cam.offset_map is None else torch.from_numpy(cam.offset_map).cuda()
    loc.forward_maps(torch.from_numpy(frames).cuda(), maps, logits, gain=cam.gain, offset=cam.offset, gain_map=gm,
                     offset_map=om)
    torch.cuda.synchronize()
    return maps.cpu().numpy(), logits.cpu().numpy()


def _heads_view(maps, logits):
    """GPU maps in float64 with channel 0 replaced by the p logit."""
    h = maps.astype(np.float64)
    h[:, 0] = logits
    return h


def _err(got, ref, k):
    return float(np.abs(got[:, k] - ref[:, k]).max() / max(np.abs(ref[:, k]).max(), 1e-6))


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
@pytest.mark.parametrize("which", ["plain48", "dcd32"])
def test_nine_head_maps_and_records_match_oracle(prec, which):
    spec = dict(_nets())[which]
    spec = synth.NetSpec(**{**spec.__dict__, "precision": prec})
    blob = synth.pack_blob(spec, synth.init_weights(spec, 23))
    js = json.dumps(dict(json.loads(spec.to_json()), chunk_px=2 * 37 * 150))
    rng = np.random.default_rng(61)
    T, H, W = 5, 37, 150
    cam = synth.scmos_camera(rng, H, W)
    em = synth.emitters_density(rng, T, H, W, 2.0, astig=True)
    frames = synth.simulate(em, T, H, W, cam, True, rng)
    loc = sml.Localizer(js, blob)
    assert loc.num_heads == 9
    maps, logits = _maps(loc, frames, cam)
    net = oracle.Net(js, blob)
    kw = dict(gain=cam.gain, offset=cam.offset, gain_map=cam.gain_map.astype(np.float64),
              offset_map=cam.offset_map.astype(np.float64))
    ref = oracle.forward(net, frames, **kw)
    # the uncertainty maps as softplus values
    got_sp = maps[:, 5:].astype(np.float64)
    ref_sp = oracle.softplus(ref[:, 5:])
    sp_err = float(np.abs(got_sp - ref_sp).max() / np.abs(ref_sp).max())
    got = _heads_view(maps, logits)
    if prec == "fp32":
        errs = [_err(got, ref, k) for k in range(5)]
        print(which, prec, "heads", np.round(errs, 7), "softplus maps", sp_err)
        assert max(errs) <= 1e-4 and sp_err <= 1e-4
    else:
        refq = oracle.forward(oracle.quantized(net, "bf16"), frames, quant="bf16", **kw)
        errs = [_err(got, refq, k) for k in range(5)]
        rms = [float(np.sqrt(np.mean((got[:, k] - refq[:, k]) ** 2)) / max(np.abs(refq[:, k]).max(), 1e-6))
               for k in range(5)]
        spq = oracle.softplus(refq[:, 5:])
        spq_err = float(np.abs(got_sp - spq).max() / np.abs(spq).max())
        print(which, prec, "heads vs quantized", np.round(errs, 5), "rms", np.round(rms, 6), "softplus maps", spq_err,
              "vs float64", sp_err)
        assert max(errs) <= 2e-2 and max(rms) <= 2e-3 and spq_err <= 2e-2 and sp_err <= 3e-2
    # records + uncertainties: exactly the oracle's decode of these GPU maps
    want, want_sig = oracle.decode(maps, 0.5, net.z_scale, net.ph_scale, with_sigma=True)
    recs, sig = loc.localize_sigma(frames, 0.5, **oracle_cam(cam))
    assert len(want) > 0
    assert recs.tobytes() == want.tobytes() and sig.tobytes() == want_sig.tobytes()
    only = loc.localize(frames, 0.5, **oracle_cam(cam))
    assert only.tobytes() == recs.tobytes()
    # device frames and device camera maps, same bytes
    dcam = dict(gain=cam.gain, offset=cam.offset, gain_map=torch.from_numpy(cam.gain_map).cuda(),
                offset_map=torch.from_numpy(cam.offset_map).cuda())
    recs_d, sig_d = loc.localize_sigma(torch.from_numpy(frames).cuda(), 0.5, **dcam)
    assert recs_d.tobytes() == recs.tobytes() and sig_d.tobytes() == sig.tobytes()


def oracle_cam(cam):
    return dict(gain=cam.gain, offset=cam.offset, gain_map=cam.gain_map, offset_map=cam.offset_map)


def test_uncertainty_call_on_a_five_head_net_is_unsupported():
    w = synth.workload_small(precision="bf16")
    loc = sml.Localizer(w.spec.to_json(), w.blob)
    assert loc.num_heads == 5
    with pytest.raises(sml.SmlError) as e:
        loc.localize_sigma(w.frames, 0.5)
    assert e.value.code == sml.SML_ERR_UNSUPPORTED
