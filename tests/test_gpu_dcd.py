"""GPU parity of nets with dense connection dilated blocks (Sec. 3.2.1) through the C ABI.

Dense layers read a channel range of the block's concatenation buffer and append their
outputs to it; transitions write the next block input into the other buffer.  The FP32 path
(SIMT) is compared with the float64 oracle (<= 1e-4, normalised max error per map); BF16
(tensor cores) with the oracle's bf16 mode, which rounds weights and every stored activation
where the library does, and with float64, under the depth gate of tests/gpu_gates.py (the
measured error grows linearly with the number of tensor-core layers)."""
import json

import numpy as np
import pytest
import torch

import oracle
import paper_2410_02314_gb300 as sml
from gpu_gates import bf16_gate
from paper_2410_02314_gb300 import synth

pytestmark = pytest.mark.gpu

TOL = {"fp32": 1e-4}


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__

    __graft_entry__.build()
    torch.cuda.set_device(0)


def _net(C, g, blocks, dil, prec, in_ch=1, seed=11):
    spec = synth.NetSpec(in_ch=in_ch, channels=C, dilations=tuple(dil), precision=prec,
                         dcd={"growth": g, "blocks": [list(b) for b in blocks]})
    return spec.to_json(), synth.pack_blob(spec, synth.init_weights(spec, seed))


def _maps(js, blob, frames, cam):
    loc = sml.Localizer(js, blob)
    T, H, W = frames.shape
    maps = torch.empty((T, 5, H, W), dtype=torch.float32, device="cuda")
    logits = torch.empty((T, H, W), dtype=torch.float32, device="cuda")
    gm = None if cam.gain_map is None else torch.from_numpy(cam.gain_map).cuda()
    om = None if cam.offset_map is None else torch.from_numpy(cam.offset_map).cuda()
    loc.forward_maps(torch.from_numpy(np.ascontiguousarray(frames)).cuda(), maps, logits, gain=cam.gain,
                     offset=cam.offset, gain_map=gm, offset_map=om)
    torch.cuda.synchronize()
    got = maps.cpu().numpy().astype(np.float64)
    got[:, 0] = logits.cpu().numpy()
    return loc, maps, got


def gate(net, kind):
    """The BF16 depth gate for this net's tensor-core layers (all conv layers after the first)."""
    return bf16_gate(net.L - 1, kind)


def _err(got, ref):
    return [float(np.abs(got[:, k] - ref[:, k]).max() / max(np.abs(ref[:, k]).max(), 1e-6)) for k in range(5)]


def _rms(got, ref):
    return [float(np.sqrt(np.mean((got[:, k] - ref[:, k]) ** 2)) / max(np.abs(ref[:, k]).max(), 1e-6)) for k in range(5)]


def _cam_kw(cam):
    return dict(gain=cam.gain, offset=cam.offset,
                gain_map=None if cam.gain_map is None else cam.gain_map.astype(np.float64),
                offset_map=None if cam.offset_map is None else cam.offset_map.astype(np.float64))


CASES = [
    # prec, C, growth, blocks, plain dilations (stem first), in_ch
    ("fp32", 32, 16, ((2, 4), (1, 8, 3)), (1, 2, 1), 1),
    ("bf16", 32, 16, ((2, 4), (1, 8, 3)), (1, 2, 1), 1),
    ("fp32", 16, 32, ((3, 5),), (2, 1), 3),
    ("bf16", 16, 32, ((3, 5),), (2, 1), 3),
    ("fp32", 48, 16, ((1, 2),), (1, 4, 1), 1),
    ("bf16", 48, 16, ((1, 2),), (1, 4, 1), 1),
    ("bf16", 32, 32, ((2,), (4,)), (1, 1), 1),
    ("bf16", 64, 16, ((2,), (7,)), (1, 1), 1),
]


@pytest.mark.parametrize("prec,C,g,blocks,dil,in_ch", CASES)
def test_dcd_maps_match_oracle(prec, C, g, blocks, dil, in_ch):
    """Ragged frames (W not a multiple of the 128-pixel tile, odd H), per-pixel camera maps,
    several chunks; every dense growth / width combination of the case list."""
    rng = np.random.default_rng(5 + C + g)
    js, blob = _net(C, g, blocks, dil, prec, in_ch)
    js = json.dumps(dict(json.loads(js), chunk_px=2 * 37 * 150))
    T, H, W = 5, 37, 150
    cam = synth.scmos_camera(rng, H, W)
    em = synth.emitters_density(rng, T, H, W, 2.0, astig=True)
    frames = synth.simulate(em, T, H, W, cam, True, rng)
    loc, maps, got = _maps(js, blob, frames, cam)
    net = oracle.Net(js, blob)
    assert loc.last_launch_count == net.L * 3  # one launch per conv layer and chunk (3 chunks of <= 2 frames)
    ref = oracle.forward(net, frames, **_cam_kw(cam))
    e = _err(got, ref)
    if prec == "fp32":
        print(prec, C, g, "vs float64", np.round(e, 7))
        assert max(e) <= TOL["fp32"]
        return
    refq = oracle.forward(oracle.quantized(net, "bf16"), frames, quant="bf16", **_cam_kw(cam))
    eq, rq = _err(got, refq), _rms(got, refq)
    print(prec, C, g, "vs quantized", np.round(eq, 5), "rms", np.round(rq, 6), "vs float64", np.round(e, 4))
    assert max(eq) <= gate(net, "q_max") and max(rq) <= gate(net, "q_rms") and max(e) <= gate(net, "f64_max")


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_dcd_chunking_and_localize_are_consistent(prec):
    """Maps do not depend on the chunk size (bit for bit); the fused localize call of host and
    of device frames returns exactly the oracle's decode of those maps; one chunk launches
    layer 1, every further conv layer and the three decode kernels."""
    rng = np.random.default_rng(19)
    js, blob = _net(32, 16, ((2, 4, 8),), (1, 1), prec)
    spec_layers = 1 + 3 + 1 + 1
    T, H, W = 6, 48, 200
    frames = rng.integers(95, 900, (T, H, W)).astype(np.uint16)
    cam = synth.Camera(2.0, 100.0)
    small = json.dumps(dict(json.loads(js), chunk_px=2 * H * W))
    _, m1, _ = _maps(js, blob, frames, cam)
    _, m2, _ = _maps(small, blob, frames, cam)
    assert torch.equal(m1, m2)
    loc = sml.Localizer(js, blob)
    host = loc.localize(frames, 0.5, gain=2.0, offset=100.0)
    assert loc.last_launch_count == spec_layers + 3
    dev = sml.Localizer(small, blob).localize(torch.from_numpy(frames).cuda(), 0.5, gain=2.0, offset=100.0)
    net = oracle.Net(js, blob)
    want = oracle.decode(m1.cpu().numpy(), 0.5, net.z_scale, net.ph_scale)
    assert len(want) > 0 and host.tobytes() == want.tobytes() == dev.tobytes()


def test_dcd_full_size_sampled():
    """256 frames of 256x256 through the 22-layer dense-block net (the dense-block benchmark
    workload, BF16): sampled corner and interior blocks match the oracle's exact windowed
    forward (bf16 mode and float64), and the decode of all 16.8 Mpixel is bit-exact."""
    w = synth.workload_dcd()
    js = w.spec.to_json()
    loc, maps, got = _maps(js, w.blob, w.frames, w.cam)
    net = oracle.Net(js, w.blob)
    qnet = oracle.quantized(net, "bf16")
    worst, worst_q = 0.0, 0.0
    for t, (i0, j0) in [(0, (0, 0)), (201, (116, 116)), (255, (232, 100))]:
        blk = got[t : t + 1, :, i0 : i0 + 24, j0 : j0 + 24]
        ref = oracle.forward_window(net, w.frames[t : t + 1], i0, i0 + 24, j0, j0 + 24)
        refq = oracle.forward_window(qnet, w.frames[t : t + 1], i0, i0 + 24, j0, j0 + 24, quant="bf16")
        worst = max(worst, max(_err(blk, ref)))
        worst_q = max(worst_q, max(_err(blk, refq)))
    print("dcd full-size sampled worst", worst, "vs quantized", worst_q, "gates", gate(net, "f64_max"),
          gate(net, "q_max"))
    assert worst <= gate(net, "f64_max") and worst_q <= gate(net, "q_max")
    recs = loc.localize(w.frames, 0.5, capacity=4_000_000)
    want = oracle.decode(maps.cpu().numpy(), 0.5, net.z_scale, net.ph_scale)
    assert recs.tobytes() == want.tobytes()
