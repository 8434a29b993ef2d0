"""GPU parity of nets with the U-Net fine stage (Sec. 3.2; two upsampling stages, Sec. 4.2)
through the C ABI: 2x2 max pooling and nearest upsampling kernels between resolution
levels, convs on the half- and quarter-resolution buffers, the skip concatenation as an
offset store.  FP32 against float64 (<= 1e-4); BF16 against the oracle's bf16 mode (max and
RMS) and float64 (max) under the depth gate of tests/gpu_gates.py (the measured error grows
linearly with the number of tensor-core layers); records bit-exact against the oracle's
decode of the GPU maps."""
import json

import numpy as np
import pytest
import torch

import oracle
import paper_2410_02314_gb300 as sml
from gpu_gates import bf16_gate
from paper_2410_02314_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__

    __graft_entry__.build()
    torch.cuda.set_device(0)


def _maps(loc, frames, cam, nh):
    T, H, W = frames.shape
    maps = torch.empty((T, nh, H, W), dtype=torch.float32, device="cuda")
    logits = torch.empty((T, H, W), dtype=torch.float32, device="cuda")
    gm = None if cam.gain_map is None else torch.from_numpy(cam.gain_map).cuda()
    om = None if cam.offset_map is None else torch.from_numpy(cam.offset_map).cuda()
    loc.forward_maps(torch.from_numpy(frames).cuda(), maps, logits, gain=cam.gain, offset=cam.offset, gain_map=gm,
                     offset_map=om)
    torch.cuda.synchronize()
    m = maps.cpu().numpy()
    got = m.astype(np.float64)
    got[:, 0] = logits.cpu().numpy()
    return m, got


def gate(net, kind):
    """The BF16 depth gate for this net's tensor-core layers (all conv layers after the first)."""
    return bf16_gate(net.L - 1, kind)


def _err(got, ref, ks):
    return [float(np.abs(got[:, k] - ref[:, k]).max() / max(np.abs(ref[:, k]).max(), 1e-6)) for k in ks]


def _rms(got, ref, ks):
    return [float(np.sqrt(np.mean((got[:, k] - ref[:, k]) ** 2)) / max(np.abs(ref[:, k]).max(), 1e-6)) for k in ks]


CASES = [
    # prec, C, levels, dcd, plain dilations, heads, frame size
    ("fp32", 32, 1, None, (1, 2, 1), 5, (37, 150)),
    ("bf16", 32, 1, None, (1, 2, 1), 5, (37, 150)),
    ("fp32", 32, 2, None, (1, 4, 2, 1), 5, (37, 150)),
    ("bf16", 32, 2, None, (1, 4, 2, 1), 5, (37, 150)),
    ("bf16", 48, 2, None, (1, 2, 1), 5, (64, 131)),
    ("fp32", 16, 2, {"growth": 16, "blocks": [[2, 4]]}, (1, 1), 9, (29, 70)),
    ("bf16", 32, 2, {"growth": 16, "blocks": [[2, 4], [8]]}, (1, 2, 1), 9, (37, 150)),
    ("bf16", 32, 2, None, (1, 1), 5, (3, 5)),  # frames smaller than the pooling grid
]


@pytest.mark.parametrize("prec,C,levels,dcd,dil,nh,size", CASES)
def test_unet_maps_and_records_match_oracle(prec, C, levels, dcd, dil, nh, size):
    H, W = size
    spec = synth.NetSpec(in_ch=1, channels=C, dilations=dil, precision=prec, unet=levels, dcd=dcd, n_heads=nh)
    blob = synth.pack_blob(spec, synth.init_weights(spec, 31 + C + levels))
    T = 5
    js = json.dumps(dict(json.loads(spec.to_json()), chunk_px=2 * H * W))  # 3 chunks
    rng = np.random.default_rng(H * W + levels)
    cam = synth.scmos_camera(rng, H, W)
    em = synth.emitters_density(rng, T, H, W, 2.0, astig=True)
    frames = synth.simulate(em, T, H, W, cam, True, rng)
    loc = sml.Localizer(js, blob)
    maps, got = _maps(loc, frames, cam, nh)
    net = oracle.Net(js, blob)
    # launches per chunk: every conv layer, plus a pool and an upsample per level
    assert loc.last_launch_count == 3 * (net.L + 2 * levels)
    kw = dict(gain=cam.gain, offset=cam.offset, gain_map=cam.gain_map.astype(np.float64),
              offset_map=cam.offset_map.astype(np.float64))
    ref = oracle.forward(net, frames, **kw)
    e = _err(got, ref, range(5))
    if prec == "fp32":
        print(prec, C, levels, dcd is not None, "vs float64", np.round(e, 7))
        assert max(e) <= 1e-4
    else:
        refq = oracle.forward(oracle.quantized(net, "bf16"), frames, quant="bf16", **kw)
        eq, rq = _err(got, refq, range(5)), _rms(got, refq, range(5))
        print(prec, C, levels, dcd is not None, "vs quantized", np.round(eq, 5), "rms", np.round(rq, 6), "vs float64",
              np.round(e, 4))
        assert max(eq) <= gate(net, "q_max") and max(rq) <= gate(net, "q_rms") and max(e) <= gate(net, "f64_max")
    if nh == 9:
        want, want_sig = oracle.decode(maps, 0.5, net.z_scale, net.ph_scale, with_sigma=True)
        recs, sig = loc.localize_sigma(frames, 0.5, gain=cam.gain, offset=cam.offset, gain_map=cam.gain_map,
                                       offset_map=cam.offset_map)
        assert recs.tobytes() == want.tobytes() and sig.tobytes() == want_sig.tobytes()
    else:
        want = oracle.decode(maps, 0.5, net.z_scale, net.ph_scale)
        recs = loc.localize(frames, 0.5, gain=cam.gain, offset=cam.offset, gain_map=cam.gain_map,
                            offset_map=cam.offset_map)
        assert recs.tobytes() == want.tobytes()


def test_unet_chunking_is_bit_exact():
    spec = synth.NetSpec(in_ch=1, channels=32, dilations=(1, 2, 1), precision="bf16", unet=2)
    blob = synth.pack_blob(spec, synth.init_weights(spec, 3))
    T, H, W = 6, 50, 77
    frames = np.random.default_rng(2).integers(95, 900, (T, H, W)).astype(np.uint16)
    cam = synth.Camera(1.0, 100.0)
    one = _maps(sml.Localizer(spec.to_json(), blob), frames, cam, 5)[0]
    small = json.dumps(dict(json.loads(spec.to_json()), chunk_px=H * W))
    two = _maps(sml.Localizer(small, blob), frames, cam, 5)[0]
    assert np.array_equal(one, two)


def test_full_topology_full_size_sampled():
    """256 frames of 256x256 through the full-topology net (dense blocks, two-level U-Net, nine
    heads; BF16): sampled corner and interior blocks match the oracle's exact windowed forward
    (bf16 mode and float64), and records with their uncertainties are bit-exact against the
    decode of all 16.8 Mpixel of GPU maps."""
    w = synth.workload_dilatedloc()
    js = w.spec.to_json()
    loc = sml.Localizer(js, w.blob)
    maps, got = _maps(loc, w.frames, w.cam, 9)
    net = oracle.Net(js, w.blob)
    qnet = oracle.quantized(net, "bf16")
    worst = worst_q = 0.0
    for t, (i0, j0) in [(0, (0, 0)), (130, (117, 93)), (255, (232, 232))]:
        blk = got[t : t + 1, :, i0 : i0 + 24, j0 : j0 + 24]
        ref = oracle.forward_window(net, w.frames[t : t + 1], i0, i0 + 24, j0, j0 + 24)
        refq = oracle.forward_window(qnet, w.frames[t : t + 1], i0, i0 + 24, j0, j0 + 24, quant="bf16")
        worst = max(worst, max(_err(blk, ref, range(5))))
        worst_q = max(worst_q, max(_err(blk, refq, range(5))))
    print("full topology sampled worst", worst, "vs quantized", worst_q, "gates", gate(net, "f64_max"),
          gate(net, "q_max"))
    assert worst <= gate(net, "f64_max") and worst_q <= gate(net, "q_max")
    want, want_sig = oracle.decode(maps, 0.5, net.z_scale, net.ph_scale, with_sigma=True)
    recs, sig = loc.localize_sigma(w.frames, 0.5, capacity=4_000_000)
    assert recs.tobytes() == want.tobytes() and sig.tobytes() == want_sig.tobytes()


def test_full_topology_with_three_frame_input_across_chunk_edges():
    """Dense blocks + U-Net + nine heads with the three-frame input: chunks of two frames read
    their neighbours; maps equal the single-chunk run bit for bit and match the bf16 oracle."""
    spec = synth.NetSpec(in_ch=3, channels=16, dilations=(1, 1), precision="bf16", n_heads=9, unet=2,
                         dcd={"growth": 16, "blocks": [[2, 4]]})
    blob = synth.pack_blob(spec, synth.init_weights(spec, 41))
    T, H, W = 5, 40, 70
    rng = np.random.default_rng(43)
    frames = rng.integers(95, 900, (T, H, W)).astype(np.uint16)
    cam = synth.Camera(2.0, 100.0)
    one, got = _maps(sml.Localizer(spec.to_json(), blob), frames, cam, 9)
    small = json.dumps(dict(json.loads(spec.to_json()), chunk_px=2 * H * W))
    two, _ = _maps(sml.Localizer(small, blob), frames, cam, 9)
    assert np.array_equal(one, two)
    net = oracle.Net(spec.to_json(), blob)
    refq = oracle.forward(oracle.quantized(net, "bf16"), frames, gain=2.0, offset=100.0, quant="bf16")
    assert max(_err(got, refq, range(5))) <= gate(net, "q_max")


def test_stack_file_pipeline_on_the_full_topology(tmp_path):
    """The stack-file pipeline (reader thread, pinned ring, overlapped copies) runs any one-frame
    net: its records equal one sml_localize call on the same frames."""
    spec = synth.NetSpec(in_ch=1, channels=16, dilations=(1, 1), precision="bf16", n_heads=9, unet=2,
                         dcd={"growth": 16, "blocks": [[2, 4]]})
    blob = synth.pack_blob(spec, synth.init_weights(spec, 47))
    T, H, W = 37, 64, 96
    rng = np.random.default_rng(5)
    em = synth.emitters_density(rng, T, H, W, 2.0)
    frames = synth.simulate(em, T, H, W, synth.Camera(1.0, 100.0), False, rng)
    path = tmp_path / "stack.raw"
    frames.tofile(path)
    loc = sml.Localizer(spec.to_json(), blob)
    recs, _ = loc.localize_file(str(path), T, H, W, 0.5, batch=8)
    want = loc.localize(frames, 0.5)
    assert len(want) > 0 and recs.tobytes() == want.tobytes()
