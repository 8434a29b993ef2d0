"""GPU parity of FP8 e4m3 nets with dense connection dilated blocks (Sec. 3.2.1) and the U-Net
fine stage (Sec. 3.2) through the C ABI.

A dense layer reads the block input and every earlier output of its block, a U-Net up conv a
skip and the upsampled deeper features: channels of several layers, each stored as e4m3 with
the scale of the layer that wrote it.  The library folds each input channel's scale into the
weights before rounding them per output channel; the oracle's fp8 mode rounds at the same
points.  Maps are compared with that mode under the measured FP8 depth gates of
tests/gpu_gates.py (the deviation from float64, the cost of e4m3 itself, is printed); records
are bit-exact against the oracle's decode of the GPU maps; the library's calibration is
compared with the oracle's activation maxima."""
import json

import numpy as np
import pytest
import torch

import oracle
import paper_2410_02314_gb300 as sml
from gpu_gates import FP8_CALIBRATION_REL, fp8_dense_gate
from paper_2410_02314_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__

    __graft_entry__.build()
    torch.cuda.set_device(0)


def _spec(C, g, blocks, dil, levels=0, in_ch=1, nh=5):
    dcd = {"growth": g, "blocks": [list(b) for b in blocks]} if blocks else None
    return synth.NetSpec(in_ch=in_ch, channels=C, dilations=tuple(dil), precision="bf16", dcd=dcd, unet=levels,
                         n_heads=nh)


def _cam_kw(cam):
    return dict(gain=cam.gain, offset=cam.offset,
                gain_map=None if cam.gain_map is None else cam.gain_map.astype(np.float64),
                offset_map=None if cam.offset_map is None else cam.offset_map.astype(np.float64))


def _maps(js, blob, frames, cam, nh):
    loc = sml.Localizer(js, blob)
    T, H, W = frames.shape
    maps = torch.empty((T, nh, H, W), dtype=torch.float32, device="cuda")
    logits = torch.empty((T, H, W), dtype=torch.float32, device="cuda")
    gm = None if cam.gain_map is None else torch.from_numpy(cam.gain_map).cuda()
    om = None if cam.offset_map is None else torch.from_numpy(cam.offset_map).cuda()
    loc.forward_maps(torch.from_numpy(np.ascontiguousarray(frames)).cuda(), maps, logits, gain=cam.gain,
                     offset=cam.offset, gain_map=gm, offset_map=om)
    torch.cuda.synchronize()
    m = maps.cpu().numpy()
    got = m.astype(np.float64)
    got[:, 0] = logits.cpu().numpy()
    return loc, m, got


def _norm(got, ref, ks, fn):
    return [float(fn(np.abs(got[:, k] - ref[:, k])) / max(np.abs(ref[:, k]).max(), 1e-6)) for k in ks]


def _check(net, got, frames, cam, scales, label):
    kw = _cam_kw(cam)
    refq = oracle.forward(oracle.quantized(net, "fp8", scales), frames, quant="fp8", scales=scales, **kw)
    ref = oracle.forward(net, frames, **kw)
    ks = range(5)  # the position maps (what the gates were measured on)
    mx, rms = np.max, lambda d: np.sqrt(np.mean(d * d))
    e = {"q_max": max(_norm(got, refq, ks, mx)), "q_rms": max(_norm(got, refq, ks, rms)),
         "f64_max": max(_norm(got, ref, ks, mx)), "f64_rms": max(_norm(got, ref, ks, rms))}
    n_tc = net.L - 1
    print(label, "tensor-core layers", n_tc, {k: round(v, 5) for k, v in e.items()},
          {k: round(fp8_dense_gate(n_tc, k), 4) for k in ("q_max", "q_rms")})
    for k in ("q_max", "q_rms"):
        assert e[k] <= fp8_dense_gate(n_tc, k), (label, k, e[k])


CASES = [
    # C, growth, blocks, plain dilations (stem first), U-Net levels, in_ch, heads
    (32, 16, ((2, 4), (1, 8, 3)), (1, 2, 1), 0, 1, 5),
    (16, 32, ((3, 5),), (2, 1), 0, 3, 5),
    (48, 16, ((1, 2),), (1, 4, 1), 0, 1, 5),
    (32, 0, (), (1, 2, 1), 2, 1, 5),
    (16, 16, ((2, 4),), (1, 1), 1, 1, 9),
    (48, 0, (), (1, 4, 2, 1), 2, 1, 5),
]


@pytest.mark.parametrize("C,g,blocks,dil,levels,in_ch,nh", CASES)
def test_fp8_dense_and_unet_maps_match_oracle(C, g, blocks, dil, levels, in_ch, nh):
    """Ragged frames (W not a multiple of the 128-pixel tile, odd H), per-pixel camera maps,
    several chunks; dense growths, widths, U-Net levels, three-frame input and nine heads;
    FP8 with the oracle's activation scales for these frames."""
    rng = np.random.default_rng(7 + C + g + levels)
    spec = _spec(C, g, blocks, dil, levels, in_ch, nh)
    blob = synth.pack_blob(spec, synth.init_weights(spec, 13))
    net = oracle.Net(spec.to_json(), blob)
    T, H, W = 5, 37, 150
    cam = synth.scmos_camera(rng, H, W)
    em = synth.emitters_density(rng, T, H, W, 2.0, astig=True)
    frames = synth.simulate(em, T, H, W, cam, True, rng)
    scales = oracle.act_scales(net, frames, **_cam_kw(cam))
    js = json.dumps(dict(json.loads(spec.to_json()), precision="fp8", act_scales=scales, chunk_px=2 * H * W))
    loc, m, got = _maps(js, blob, frames, cam, nh)
    assert loc.last_launch_count == 3 * (net.L + 2 * levels)  # conv layers + pool/upsample steps per chunk
    _check(net, got, frames, cam, scales, f"C={C} g={g} blocks={blocks} unet={levels}")
    if nh == 5:  # the fused localize call returns the oracle's decode of these maps, bit for bit
        recs = loc.localize(frames, 0.5, gain=cam.gain, offset=cam.offset, gain_map=cam.gain_map,
                            offset_map=cam.offset_map)
        want = oracle.decode(m, 0.5, net.z_scale, net.ph_scale)
        assert recs.tobytes() == want.tobytes()


@pytest.mark.parametrize("which", ["dcd", "dilatedloc"])
def test_fp8_benchmark_nets_whole_frame(which):
    """The 22-layer dense-block benchmark net and the 26-layer full topology (dense blocks,
    two-level U-Net) on a whole 256x256 frame of the batched workload, FP8 with the scales of
    the library's own calibration (a bf16 pass over the frame), which stay within the
    measured bound of the oracle's float64 maxima; records bit-exact."""
    spec = synth.spec_dcd("bf16") if which == "dcd" else synth.spec_dilatedloc("bf16")
    w = synth.workload_batched(T=1, precision="bf16", seed=3)
    blob = synth.pack_blob(spec, synth.init_weights(spec, 21))
    net = oracle.Net(spec.to_json(), blob)
    d_frames = torch.from_numpy(w.frames).cuda()
    js = sml.calibrate_fp8(spec.to_json(), blob, d_frames, gain=w.cam.gain, offset=w.cam.offset)
    lib_scales = json.loads(js)["act_scales"]
    scales = oracle.act_scales(net, w.frames, w.cam.gain, w.cam.offset)
    dev = max(abs(a / b - 1.0) for a, b in zip(lib_scales[1:], scales[1:]))
    assert lib_scales[0] == 1.0 and dev <= FP8_CALIBRATION_REL, dev
    loc, m, got = _maps(js, blob, w.frames, w.cam, net.nh)
    _check(net, got, w.frames, w.cam, lib_scales, which)
    # random-init p maps sit low: a threshold at their 99.5th percentile keeps detections
    p_min = float(np.float32(np.quantile(m[:, 0], 0.995)))
    recs = loc.localize(d_frames, p_min, gain=w.cam.gain, offset=w.cam.offset)
    want = oracle.decode(m, p_min, net.z_scale, net.ph_scale, with_sigma=net.nh == 9)
    want = want[0] if net.nh == 9 else want
    assert len(want) > 0 and recs.tobytes() == want.tobytes()
