"""GPU parity: the CUDA path through the C ABI against the CPU oracle.

Tolerances, as normalised max errors max|gpu - ref| / max|ref| per map (p compared as logits).
They follow from the arithmetic: FP32 sums of a few hundred products per layer over 8 layers
stay near 1e-6; BF16/FP8 differ from an oracle that rounds at the same points only where the
tensor core's FP32 accumulation and the oracle's FP64 one land on opposite sides of a rounding
boundary (one ulp of that element, attenuated downstream):
  * FP32 vs the float64 oracle: <= 1e-4;
  * BF16 / FP8 vs the oracle's quantized mode (activations and weights rounded at the same
    points as the tensor-core path, float64 elsewhere): max <= TOL_Q and RMS <= TOL_Q_RMS;
  * BF16 / FP8 vs the unquantized float64 oracle (the precision cost, stated per config):
    BF16 <= 3e-2; FP8 <= 0.4 max and <= 0.08 RMS;
  * decode: bit-exact (same bytes) when both sides decode the same float32 maps;
  * the fused localize call equals the decode of the maps the same network produced.
"""
import json

import numpy as np
import pytest
import torch

import oracle
import paper_2410_02314_gb300 as sml
from gpu_gates import FP8_FRAME, bf16_gate
from paper_2410_02314_gb300 import synth

pytestmark = pytest.mark.gpu

TOL = {"fp32": 1e-4, "bf16": 3e-2, "fp8": 0.4}
TOL_Q = {"bf16": 2e-2, "fp8": 1e-1}          # max vs the quantized oracle
TOL_Q_RMS = {"bf16": 2e-3, "fp8": 2e-2}      # RMS vs the quantized oracle
FP8_RMS = 0.08


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__

    __graft_entry__.build()
    torch.cuda.set_device(0)


def with_precision(w, prec, **extra):
    spec = synth.NetSpec(**{**w.spec.__dict__, "precision": prec})
    js = spec.to_json()
    if extra:
        import json

        d = json.loads(js)
        d.update(extra)
        js = json.dumps(d)
    return js


def gpu_maps(spec_json, blob, frames, cam):
    loc = sml.Localizer(spec_json, blob)
    fr = torch.from_numpy(np.ascontiguousarray(frames)).cuda()
    T, H, W = frames.shape
    maps = torch.empty((T, 5, H, W), dtype=torch.float32, device="cuda")
    logits = torch.empty((T, H, W), dtype=torch.float32, device="cuda")
    gm = None if cam.gain_map is None else torch.from_numpy(cam.gain_map).cuda()
    om = None if cam.offset_map is None else torch.from_numpy(cam.offset_map).cuda()
    loc.forward_maps(fr, maps, logits, gain=cam.gain, offset=cam.offset, gain_map=gm, offset_map=om)
    torch.cuda.synchronize()
    return loc, maps, logits


def map_errors(maps, logits, ref):
    got = maps.cpu().numpy().astype(np.float64)
    got[:, 0] = logits.cpu().numpy()
    return [float(np.abs(got[:, k] - ref[:, k]).max() / max(np.abs(ref[:, k]).max(), 1e-6)) for k in range(5)]


def map_rms(maps, logits, ref):
    got = maps.cpu().numpy().astype(np.float64)
    got[:, 0] = logits.cpu().numpy()
    return [float(np.sqrt(np.mean((got[:, k] - ref[:, k]) ** 2)) / max(np.abs(ref[:, k]).max(), 1e-6))
            for k in range(5)]


def check_quantized(prec, js, blob, frames, cam, maps, logits, scales=None, full=None, gates=None):
    """Tight check against the oracle's quantized mode, loose check against float64; gates
    (q_max, q_rms, f64_max, f64_rms) override the sampled-block gates (whole FP8 frames)."""
    net = oracle.Net(js, blob)
    kw = dict(gain=cam.gain, offset=cam.offset,
              gain_map=None if cam.gain_map is None else cam.gain_map.astype(np.float64),
              offset_map=None if cam.offset_map is None else cam.offset_map.astype(np.float64))
    refq = oracle.forward(oracle.quantized(net, prec), frames, quant=prec, scales=scales, **kw)
    eq = map_errors(maps, logits, refq)
    eq_rms = map_rms(maps, logits, refq)
    ref = full if full is not None else oracle.forward(net, frames, **kw)
    e = map_errors(maps, logits, ref)
    print(prec, "vs quantized oracle", np.round(eq, 5), "rms", np.round(eq_rms, 6), "vs float64", np.round(e, 4),
          "rms vs float64", np.round(map_rms(maps, logits, ref), 4))
    g = gates or {"q_max": TOL_Q[prec], "q_rms": TOL_Q_RMS[prec], "f64_max": TOL[prec], "f64_rms": FP8_RMS}
    assert max(eq) <= g["q_max"]
    assert max(eq_rms) <= g["q_rms"]
    assert max(e) <= g["f64_max"]
    if prec == "fp8":
        assert max(map_rms(maps, logits, ref)) <= g["f64_rms"]


def cam_kwargs(cam):
    return dict(gain=cam.gain, offset=cam.offset, gain_map=cam.gain_map, offset_map=cam.offset_map)


# ----------------------------------------------------------------------------- UMMA unit


def _bf16_bits(x):
    return torch.from_numpy(x.astype(np.float32)).to(torch.bfloat16)


def _tf32_values(x):
    """float32 values with 10 explicit mantissa bits (exactly representable in tf32)."""
    bits = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32) & np.uint32(0xFFFFE000)
    return bits.view(np.float32)


@pytest.mark.parametrize("kind,N,d_col", [("bf16", 48, 0), ("e4m3", 48, 0), ("bf16", 144, 48), ("bf16", 48, 336),
                                          ("e4m3", 144, 192), ("bf16", 96, 288), ("tf32", 48, 0), ("tf32", 64, 64)])
def test_umma_selftest_matches_matmul(kind, N, d_col):
    """One tcgen05 MMA chain: N = 48/96/144 accumulators at offset TMEM columns, as the
    sliding-window conv uses them; TF32 as the tensor-core layer 1 uses it."""
    rng = np.random.default_rng(0)
    K = 64
    a = rng.normal(0, 1, (128, K)).astype(np.float32)
    b = rng.normal(0, 1, (N, K)).astype(np.float32)
    if kind == "e4m3":
        at = torch.from_numpy(a).to(torch.float8_e4m3fn)
        bt = torch.from_numpy(b).to(torch.float8_e4m3fn)
        e, s = 16, 32
    elif kind == "tf32":
        at, bt = torch.from_numpy(_tf32_values(a)), torch.from_numpy(_tf32_values(b))
        e, s = 4, 8
    else:
        at, bt = _bf16_bits(a), _bf16_bits(b)
        e, s = 8, 16
    af, bf = at.float().numpy().astype(np.float64), bt.float().numpy().astype(np.float64)
    a_img = at.reshape(128, K // e, e).permute(1, 0, 2).contiguous()
    b_img = bt.reshape(N // 8, 8, K // s, s // e, e).permute(2, 0, 3, 1, 4).contiguous()
    da, db = a_img.view(torch.uint8).cuda(), b_img.view(torch.uint8).cuda()
    dd = torch.zeros((128, N), dtype=torch.float32, device="cuda")
    sml.sml_debug_umma(da, db, dd, N, K, kind=kind, d_col=d_col)
    ref = af @ bf.T
    got = dd.cpu().numpy()
    assert np.abs(got - ref).max() <= 1e-5 * np.abs(ref).max()


# ----------------------------------------------------------------------------- maps


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_small_workload_maps_match_oracle(prec):
    w = synth.workload_small()
    js = with_precision(w, prec)
    loc, maps, logits = gpu_maps(js, w.blob, w.frames, w.cam)
    if prec == "bf16":
        check_quantized(prec, js, w.blob, w.frames, w.cam, maps, logits)
        return
    ref = oracle.forward(oracle.Net(js, w.blob), w.frames, w.cam.gain, w.cam.offset)
    errs = map_errors(maps, logits, ref)
    print(prec, "normalised max map errors", errs)
    assert max(errs) <= TOL[prec]


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_ragged_frames_multi_chunk_and_scmos(prec):
    """W not a multiple of the 128-pixel tile, odd H, several chunks, per-pixel camera maps."""
    rng = np.random.default_rng(7)
    T, H, W = 5, 37, 150
    cam = synth.scmos_camera(rng, H, W)
    em = synth.emitters_density(rng, T, H, W, 2.0, astig=True)
    frames = synth.simulate(em, T, H, W, cam, True, rng)
    spec = synth.spec_48(prec)
    blob = synth.pack_blob(spec, synth.init_weights(spec, 17))
    js = with_precision(synth.Workload("r", frames, cam, em, spec, blob, True), prec, chunk_px=2 * H * W)
    loc, maps, logits = gpu_maps(js, blob, frames, cam)
    net = oracle.Net(js, blob)
    ref = oracle.forward(net, frames, cam.gain, cam.offset, cam.gain_map.astype(np.float64),
                         cam.offset_map.astype(np.float64))
    if prec == "bf16":
        check_quantized(prec, js, blob, frames, cam, maps, logits, full=ref)
    errs = map_errors(maps, logits, ref)
    print(prec, "ragged errors", errs)
    assert max(errs) <= TOL[prec]
    # fused path (host frames + host camera maps) decodes exactly the maps above
    recs = loc.localize(frames, 0.5, **cam_kwargs(cam))
    want = oracle.decode(maps.cpu().numpy(), 0.5, net.z_scale, net.ph_scale)
    assert recs.tobytes() == want.tobytes()


@pytest.mark.parametrize("stages", [1, 3, 17])
def test_tma_ring_depth_outside_range_is_rejected(stages):
    """The waiter/MMA handoff needs a ring of at least 4 stages; 1..3 and >16 are spec errors."""
    import json

    spec = synth.NetSpec(in_ch=1, channels=32, dilations=(1, 2, 1), precision="bf16")
    blob = synth.pack_blob(spec, synth.init_weights(spec, 5))
    js = json.dumps(dict(json.loads(spec.to_json()), tc_stages=stages))
    with pytest.raises(sml.SmlError) as e:
        sml.Localizer(js, blob)
    assert e.value.code == sml.SML_ERR_BAD_SPEC


@pytest.mark.parametrize("stages", [0, 4])
def test_dilation_larger_than_tile_margin(stages):
    """Dilations up to 64 (TMA box 256 pixels) and a frame narrower than the dilation, with
    the deepest and a shallow TMA ring."""
    import json

    rng = np.random.default_rng(8)
    spec = synth.NetSpec(in_ch=1, channels=32, dilations=(1, 64, 3, 17), precision="bf16")
    blob = synth.pack_blob(spec, synth.init_weights(spec, 5))
    frames = rng.integers(100, 600, (2, 90, 40)).astype(np.uint16)
    cam = synth.Camera(1.0, 100.0)
    js = json.dumps(dict(json.loads(spec.to_json()), tc_stages=stages))
    loc, maps, logits = gpu_maps(js, blob, frames, cam)
    check_quantized("bf16", js, blob, frames, cam, maps, logits)


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
@pytest.mark.parametrize("d1,in_ch", [(2, 1), (3, 3), (4, 1), (5, 3), (64, 1)])
def test_first_layer_dilation(prec, d1, in_ch):
    """The first layer at dilations below the block height (its input rows overlap and are
    staged once) and above it, on a frame with a ragged 128-pixel strip and a ragged row block,
    with per-pixel camera maps; single- and three-frame input."""
    rng = np.random.default_rng(11 + d1)
    spec = synth.NetSpec(in_ch=in_ch, channels=32, dilations=(d1, 1), precision=prec)
    blob = synth.pack_blob(spec, synth.init_weights(spec, 6))
    T, H, W = 3, 71, 150
    frames = rng.integers(90, 900, (T, H, W)).astype(np.uint16)
    cam = synth.Camera(1.0, 100.0, gain_map=rng.uniform(0.5, 2.0, (H, W)).astype(np.float32),
                       offset_map=rng.uniform(80.0, 120.0, (H, W)).astype(np.float32))
    js = spec.to_json()
    loc, maps, logits = gpu_maps(js, blob, frames, cam)
    if prec == "bf16":
        check_quantized("bf16", js, blob, frames, cam, maps, logits)
    else:
        net = oracle.Net(js, blob)
        ref = oracle.forward(net, frames, gain=cam.gain, offset=cam.offset, gain_map=cam.gain_map.astype(np.float64),
                             offset_map=cam.offset_map.astype(np.float64))
        assert max(map_errors(maps, logits, ref)) <= TOL["fp32"]
    loc.close()


# ----------------------------------------------------------------------------- decode


def test_decode_bit_exact_on_gpu_maps():
    w = synth.workload_small()
    js = w.spec.to_json()
    loc, maps, _ = gpu_maps(js, w.blob, w.frames, w.cam)
    T, _, H, W = maps.shape
    cap = T * H * W
    d_out = torch.empty(cap * 24, dtype=torch.uint8, device="cuda")
    d_n = torch.zeros(1, dtype=torch.int64, device="cuda")
    loc.decode_maps(maps, 0.5, d_out, d_n)
    torch.cuda.synchronize()
    n = int(d_n.item())
    got = sml.records_from_bytes(d_out, n)
    net = oracle.Net(js, w.blob)
    want = oracle.decode(maps.cpu().numpy(), 0.5, net.z_scale, net.ph_scale)
    assert n == len(want) and n > 0
    assert got.tobytes() == want.tobytes()


def test_decode_golden_cases_on_gpu():
    import json
    import os

    cases = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "decode_cases.json")))["cases"]
    for case in cases:
        spec = synth.NetSpec(in_ch=1, channels=16, dilations=(1, 1), z_scale=case["z_scale"],
                             ph_scale=case["ph_scale"])
        loc = sml.Localizer(spec.to_json(), synth.pack_blob(spec, synth.init_weights(spec, 1)))
        p = np.asarray(case["p"], dtype=np.float32)
        T, H, W = p.shape
        m = np.zeros((T, 5, H, W), dtype=np.float32)
        m[:, 0] = p
        m[:, 1], m[:, 2], m[:, 3], m[:, 4] = case["dx"], case["dy"], case["zhat"], case["nhat"]
        d_out = torch.empty(64 * 24, dtype=torch.uint8, device="cuda")
        d_n = torch.zeros(1, dtype=torch.int64, device="cuda")
        loc.decode_maps(torch.from_numpy(m).cuda(), case["p_min"], d_out, d_n)
        torch.cuda.synchronize()
        got = sml.records_from_bytes(d_out, int(d_n.item()))
        rows = [[int(r["frame"])] + [float(r[k]) for k in ("x", "y", "z", "photons", "p")] for r in got]
        want = [[int(e[0])] + [float(np.float32(v)) for v in e[1:]] for e in case["expected"]]
        assert rows == want, case["name"]


def test_empty_input_and_capacity_overflow():
    w = synth.workload_small()
    loc = sml.Localizer(w.spec.to_json(), w.blob)
    assert len(loc.localize(w.frames[:0], 0.5)) == 0
    full = loc.localize(w.frames, 0.5, gain=w.cam.gain, offset=w.cam.offset)
    assert len(full) > 2
    with pytest.raises(sml.SmlError) as e:
        loc.localize(w.frames, 0.5, gain=w.cam.gain, offset=w.cam.offset, capacity=len(full) - 1)
    assert e.value.code == sml.SML_ERR_CAPACITY and e.value.needed == len(full)
    exact = loc.localize(w.frames, 0.5, gain=w.cam.gain, offset=w.cam.offset, capacity=len(full))
    assert exact.tobytes() == full.tobytes()


def test_device_and_host_frames_agree_and_async_path():
    w = synth.workload_small(precision="bf16")
    js = with_precision(w, "bf16")
    loc = sml.Localizer(js, w.blob)
    host = loc.localize(w.frames, 0.5, gain=w.cam.gain, offset=w.cam.offset)
    dev = loc.localize(torch.from_numpy(w.frames).cuda(), 0.5, gain=w.cam.gain, offset=w.cam.offset)
    assert host.tobytes() == dev.tobytes()
    d_out = torch.empty(len(host) * 24 + 24, dtype=torch.uint8, device="cuda")
    d_n = torch.zeros(1, dtype=torch.int64, device="cuda")
    loc.localize_async(torch.from_numpy(w.frames).cuda(), 0.5, d_out, d_n, gain=w.cam.gain, offset=w.cam.offset)
    torch.cuda.synchronize()
    assert sml.records_from_bytes(d_out, int(d_n.item())).tobytes() == host.tobytes()


def test_result_independent_of_chunking_and_batch():
    """A frame's records are the same alone, inside a batch, and across chunk sizes."""
    w = synth.workload_batched(T=6, H=128, W=192, precision="bf16")
    a = sml.Localizer(with_precision(w, "bf16"), w.blob).localize(w.frames, 0.5)
    b = sml.Localizer(with_precision(w, "bf16", chunk_px=128 * 192), w.blob).localize(w.frames, 0.5)
    assert a.tobytes() == b.tobytes()
    alone = sml.Localizer(with_precision(w, "bf16"), w.blob).localize(w.frames[3:4], 0.5)
    sub = a[a["frame"] == 3].copy()
    sub["frame"] = 0
    assert alone.tobytes() == sub.tobytes()


# ----------------------------------------------------------------------------- full size


@pytest.mark.parametrize("prec", ["bf16", "fp32"])
def test_batched_256_full_size_sampled(prec):
    """256 frames of 256x256 with the 48-channel net (the benchmark workload): the maps of
    sampled interior and border blocks match the oracle's exact windowed forward, and the
    decode of all 16.8 Mpixel of GPU maps is bit-exact."""
    w = synth.workload_batched(precision=prec)
    js = with_precision(w, prec)
    loc, maps, logits = gpu_maps(js, w.blob, w.frames, w.cam)
    net = oracle.Net(js, w.blob)
    m = maps.cpu().numpy()
    lg = logits.cpu().numpy()
    worst, worst_q = 0.0, 0.0
    qnet = oracle.quantized(net, prec) if prec != "fp32" else None
    for t, (i0, j0) in [(0, (0, 0)), (77, (100, 120)), (255, (232, 232)), (130, (0, 200))]:
        got = m[t : t + 1, :, i0 : i0 + 24, j0 : j0 + 24].astype(np.float64)
        got[:, 0] = lg[t : t + 1, i0 : i0 + 24, j0 : j0 + 24]
        refs = [(oracle.forward_window(net, w.frames[t : t + 1], i0, i0 + 24, j0, j0 + 24), False)]
        if qnet is not None:
            refs.append((oracle.forward_window(qnet, w.frames[t : t + 1], i0, i0 + 24, j0, j0 + 24, quant=prec), True))
        for ref, is_q in refs:
            for k in range(5):
                e = np.abs(got[:, k] - ref[:, k]).max() / max(np.abs(ref[:, k]).max(), 1e-6)
                if is_q:
                    worst_q = max(worst_q, e)
                else:
                    worst = max(worst, e)
    print(prec, "full-size sampled worst normalised error", worst, "vs quantized oracle", worst_q)
    assert worst <= TOL[prec]
    if qnet is not None:
        assert worst_q <= TOL_Q[prec]
    recs = loc.localize(w.frames, 0.5, capacity=4_000_000)
    want = oracle.decode(m, 0.5, net.z_scale, net.ph_scale)
    assert recs.tobytes() == want.tobytes()


@pytest.mark.parametrize("prec", ["bf16", "fp32"])
def test_batched_256_full_frames(prec):
    """Whole frames 0, 127 and 255 of the benchmark batch (256 frames of 256x256, run as the
    bench runs it: one 16.8-Mpixel chunk), every pixel of all 5 maps, against the oracle's
    forward of those frames: float64 (FP32 <= 1e-4, BF16 <= 3e-2) and, for BF16, the bf16
    mode (max <= 2e-2, RMS <= 2e-3)."""
    w = synth.workload_batched(precision=prec)
    js = with_precision(w, prec)
    loc, maps, logits = gpu_maps(js, w.blob, w.frames, w.cam)
    sel = [0, 127, 255]
    m, lg = maps[sel], logits[sel]
    fr = np.ascontiguousarray(w.frames[sel])
    if prec == "fp32":
        e = map_errors(m, lg, oracle.forward(oracle.Net(js, w.blob), fr, w.cam.gain, w.cam.offset))
        print("fp32 full frames vs float64", np.round(e, 8))
        assert max(e) <= TOL["fp32"]
    else:
        check_quantized(prec, js, w.blob, fr, w.cam, m, lg)
    loc.close()


def test_deep_plain_stack_under_the_depth_gate():
    """A plain 48-channel stack of 29 layers (28 tensor-core layers, the version-2 blob), two
    ragged 96x200 frames: FP32 against float64 (<= 1e-4) and BF16 against the oracle's bf16 mode
    and float64 under the measured depth gate (tests/gpu_gates.py)."""
    dil = (1,) + tuple((2, 4, 8, 16, 8, 4, 1)[k % 7] for k in range(27)) + (1,)
    rng = np.random.default_rng(29)
    em = synth.emitters_density(rng, 2, 96, 200, 1.0)
    cam = synth.Camera(1.0, 100.0)
    frames = synth.simulate(em, 2, 96, 200, cam, False, rng)
    for prec in ("fp32", "bf16"):
        spec = synth.NetSpec(in_ch=1, channels=48, dilations=dil, precision=prec)
        assert spec.L == 29
        blob = synth.pack_blob(spec, synth.init_weights(spec, 7))
        loc, maps, logits = gpu_maps(spec.to_json(), blob, frames, cam)
        net = oracle.Net(spec.to_json(), blob)
        ref = oracle.forward(net, frames, cam.gain, cam.offset)
        e = map_errors(maps, logits, ref)
        if prec == "fp32":
            print("29-layer fp32 vs float64", np.round(e, 8))
            assert max(e) <= TOL["fp32"]
        else:
            refq = oracle.forward(oracle.quantized(net, "bf16"), frames, cam.gain, cam.offset, quant="bf16")
            eq, rq = map_errors(maps, logits, refq), map_rms(maps, logits, refq)
            print("29-layer bf16 vs float64", np.round(e, 4), "vs bf16 mode", np.round(eq, 4), "rms", np.round(rq, 5))
            assert max(e) <= bf16_gate(28, "f64_max") and max(eq) <= bf16_gate(28, "q_max")
            assert max(rq) <= bf16_gate(28, "q_rms")
        loc.close()


_F64_2048 = {}


@pytest.mark.parametrize("prec", ["bf16", "fp8"])
def test_large_fov_2048_whole_frame(prec):
    """One whole 2048x2048 sCMOS frame (per-pixel gain and offset maps, astigmatic emitters at
    2 per um^2), every pixel of all 5 maps, from a two-frame call in the large field-of-view
    configuration, against the oracle's forward of that frame: float64 and the quantized mode
    of the precision (BF16: max <= 2e-2, RMS <= 2e-3, float64 <= 3e-2; FP8 with the oracle's
    activation scales, the whole-frame gates of tests/gpu_gates.py measured on whole frames:
    max <= 0.2, RMS <= 2e-2, float64 <= 0.55 max and 0.1 RMS)."""
    w = synth.workload_large_fov(T=2, precision="bf16")
    net = oracle.Net(w.spec.to_json(), w.blob)
    gm, om = w.cam.gain_map.astype(np.float64), w.cam.offset_map.astype(np.float64)
    js, scales = w.spec.to_json(), None
    if prec == "fp8":
        scales = oracle.act_scales(net, w.frames[:1, 700:956, 900:1156], w.cam.gain, w.cam.offset,
                                   gm[700:956, 900:1156], om[700:956, 900:1156])
        js = json.dumps(dict(json.loads(js), precision="fp8", act_scales=scales))
    loc, maps, logits = gpu_maps(js, w.blob, w.frames, w.cam)
    fr = np.ascontiguousarray(w.frames[1:2])
    if "ref" not in _F64_2048:
        _F64_2048["ref"] = oracle.forward(net, fr, w.cam.gain, w.cam.offset, gm, om)
    check_quantized(prec, js, w.blob, fr, w.cam, maps[1:2], logits[1:2], scales=scales, full=_F64_2048["ref"],
                    gates=FP8_FRAME if prec == "fp8" else None)
    loc.close()


# ----------------------------------------------------------------------------- FP8


@pytest.mark.parametrize("which", ["small", "batched"])
def test_fp8_maps_within_gate(which):
    """FP8 e4m3 activations and weights (per-output-channel weight scales, per-layer activation
    scales from a bf16 calibration pass), FP32 accumulation, FP32 heads: maps within 1.5e-1."""
    if which == "small":
        w = synth.workload_small(precision="bf16")
    else:
        w = synth.workload_batched(T=6, H=256, W=256, precision="bf16")
    import json

    net = oracle.Net(w.spec.to_json(), w.blob)
    scales = oracle.act_scales(net, w.frames, w.cam.gain, w.cam.offset)  # inputs from the oracle side
    js8 = json.dumps(dict(json.loads(w.spec.to_json()), precision="fp8", act_scales=scales))
    loc, maps, logits = gpu_maps(js8, w.blob, w.frames, w.cam)
    check_quantized("fp8", js8, w.blob, w.frames, w.cam, maps, logits, scales=scales)
    recs = loc.localize(w.frames, 0.5, gain=w.cam.gain, offset=w.cam.offset)
    net = oracle.Net(js8, w.blob)
    assert recs.tobytes() == oracle.decode(maps.cpu().numpy(), 0.5, net.z_scale, net.ph_scale).tobytes()


@pytest.mark.parametrize("W", [256, 250, 255])
def test_fp8_pixel_pair_rows_equal_single_rows(W):
    """FP8 activations of even-width frames are loaded as 32-byte pixel pairs (one TMA row per
    two pixels); the same bytes land in shared memory as with 16-byte rows, so the maps are
    bit-identical.  Odd dilations (the last layer, d = 1) start the box one pixel early; odd
    widths keep the 16-byte rows."""
    w = synth.workload_batched(T=3, H=96, W=W, precision="bf16")
    net = oracle.Net(w.spec.to_json(), w.blob)
    scales = oracle.act_scales(net, w.frames, w.cam.gain, w.cam.offset)
    js = dict(json.loads(w.spec.to_json()), precision="fp8", act_scales=scales)
    _, m_pair, l_pair = gpu_maps(json.dumps(js), w.blob, w.frames, w.cam)
    _, m_row, l_row = gpu_maps(json.dumps(dict(js, fp8_pair_rows=0)), w.blob, w.frames, w.cam)
    assert torch.equal(m_pair, m_row) and torch.equal(l_pair, l_row)


def test_activation_amax_matches_oracle_activations():
    """The calibration maxima equal the maxima of the oracle's per-layer activations (FP32
    context, within the FP32 map tolerance)."""
    w = synth.workload_small()
    ctx = sml.sml_create(w.spec.to_json(), w.blob)
    amax = sml.sml_activation_amax(ctx, torch.from_numpy(w.frames).cuda(), gain=w.cam.gain, offset=w.cam.offset)
    sml.sml_destroy(ctx)
    net = oracle.Net(w.spec.to_json(), w.blob)
    x0 = oracle.ingest(w.frames, w.cam.gain, w.cam.offset, in_scale=net.in_scale)
    _, acts = oracle.forward_x(net, x0, acts=True)
    for l in range(1, net.L):
        ref = acts[:, l - 1].max()
        assert abs(amax[l] - ref) <= 1e-4 * ref, (l, amax[l], ref)


def test_calibrate_fp8_scales_follow_the_oracle_activations():
    """sml_calibrate_fp8 on an FP32 context: act_scales[0] = 1 and act_scales[l] = margin *
    amax[l] / 448 with amax[l] the oracle's largest activation entering layer l (within the
    FP32 map tolerance); calibrate_fp8 puts exactly those scales into the fp8 spec."""
    w = synth.workload_small()
    ctx = sml.sml_create(w.spec.to_json(), w.blob)
    d = torch.from_numpy(w.frames).cuda()
    for margin in (1.0, 1.25):
        sc = sml.sml_calibrate_fp8(ctx, d, margin, gain=w.cam.gain, offset=w.cam.offset)
        net = oracle.Net(w.spec.to_json(), w.blob)
        ref = oracle.act_scales(net, w.frames, w.cam.gain, w.cam.offset)
        assert sc[0] == 1.0
        for l in range(1, net.L):
            assert abs(sc[l] - margin * ref[l]) <= 1e-4 * margin * ref[l], (l, sc[l], ref[l])
    assert sml.sml_num_layers(ctx) == net.L
    with pytest.raises(sml.SmlError):
        sml.sml_calibrate_fp8(ctx, d, 0.0, gain=w.cam.gain, offset=w.cam.offset)
    sml.sml_destroy(ctx)
    js = json.loads(sml.calibrate_fp8(w.spec.to_json(), w.blob, d, 1.25, gain=w.cam.gain, offset=w.cam.offset))
    assert js["precision"] == "fp8" and len(js["act_scales"]) == net.L and js["act_scales"][0] == 1.0


@pytest.mark.parametrize("prec", ["bf16", "fp8"])
def test_large_fov_2048_sampled(prec):
    """Large field of view: 2048 x 2048 sCMOS frames (per-pixel gain and offset maps), 2 emitters
    per um^2 with the astigmatic PSF, processed as whole-frame layer passes (no halo tiles):
    sampled interior, edge and corner blocks against the oracle's windowed forward (quantized
    mode and float64), and a bit-exact decode of all pixels."""
    import json

    w = synth.workload_large_fov(T=2, precision="bf16")
    net = oracle.Net(w.spec.to_json(), w.blob)
    gm, om = w.cam.gain_map.astype(np.float64), w.cam.offset_map.astype(np.float64)
    scales = None
    js = w.spec.to_json()
    if prec == "fp8":
        scales = oracle.act_scales(net, w.frames[:1, 700:956, 900:1156], w.cam.gain, w.cam.offset,
                                   gm[700:956, 900:1156], om[700:956, 900:1156])
        js = json.dumps(dict(json.loads(js), precision="fp8", act_scales=scales))
    loc, maps, logits = gpu_maps(js, w.blob, w.frames, w.cam)
    m, lg = maps.cpu().numpy(), logits.cpu().numpy()
    qnet = oracle.quantized(net, prec)
    worst, worst_q = 0.0, 0.0
    for t, (i0, j0) in [(0, (0, 0)), (1, (1000, 1017)), (0, (2024, 1500)), (1, (300, 2024)), (1, (2024, 2024))]:
        got = m[t : t + 1, :, i0 : i0 + 24, j0 : j0 + 24].astype(np.float64)
        got[:, 0] = lg[t : t + 1, i0 : i0 + 24, j0 : j0 + 24]
        kw = dict(gain=w.cam.gain, offset=w.cam.offset, gain_map=gm, offset_map=om)
        ref = oracle.forward_window(net, w.frames[t : t + 1], i0, i0 + 24, j0, j0 + 24, **kw)
        refq = oracle.forward_window(qnet, w.frames[t : t + 1], i0, i0 + 24, j0, j0 + 24, quant=prec, scales=scales, **kw)
        for k in range(5):
            worst = max(worst, np.abs(got[:, k] - ref[:, k]).max() / max(np.abs(ref[:, k]).max(), 1e-6))
            worst_q = max(worst_q, np.abs(got[:, k] - refq[:, k]).max() / max(np.abs(refq[:, k]).max(), 1e-6))
    print(prec, "2048^2 sampled worst error vs float64", worst, "vs quantized oracle", worst_q)
    assert worst <= TOL[prec] and worst_q <= TOL_Q[prec]
    recs = loc.localize(w.frames, 0.5, gain=w.cam.gain, offset=w.cam.offset, gain_map=w.cam.gain_map,
                        offset_map=w.cam.offset_map, capacity=4_000_000)
    assert recs.tobytes() == oracle.decode(m, 0.5, net.z_scale, net.ph_scale).tobytes()


# ----------------------------------------------------------------------------- three-frame context


def _context_net(C, dil, prec, seed=31):
    spec = synth.NetSpec(in_ch=3, channels=C, dilations=tuple(dil), precision=prec)
    return spec.to_json(), synth.pack_blob(spec, synth.init_weights(spec, seed))


@pytest.mark.parametrize("prec,C", [("fp32", 16), ("fp32", 48), ("bf16", 32), ("bf16", 48)])
def test_three_frame_context_matches_oracle(prec, C):
    """in_ch = 3 (frames t-1, t, t+1 as the first layer's input channels, zero beyond the
    stack): parity with the oracle, with per-pixel camera maps and a ragged frame size."""
    rng = np.random.default_rng(41)
    js, blob = _context_net(C, (1, 2, 5, 1), prec)
    T, H, W = 5, 37, 150
    frames = rng.integers(95, 700, (T, H, W)).astype(np.uint16)
    cam = synth.Camera(1.0, 100.0, rng.normal(2.0, 0.1, (H, W)).astype(np.float32),
                       rng.normal(100.0, 5.0, (H, W)).astype(np.float32))
    _, maps, logits = gpu_maps(js, blob, frames, cam)
    if prec == "fp32":
        net = oracle.Net(js, blob)
        ref = oracle.forward(net, frames, gain=cam.gain, offset=cam.offset, gain_map=cam.gain_map.astype(np.float64),
                             offset_map=cam.offset_map.astype(np.float64))
        err = map_errors(maps, logits, ref)
        print("fp32 context", np.round(err, 7))
        assert max(err) <= TOL["fp32"]
    else:
        check_quantized(prec, js, blob, frames, cam, maps, logits)


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_three_frame_context_across_chunk_edges(prec):
    """Chunks of 2 frames split a 7-frame stack; each chunk's first layer reads the frames
    just outside it.  Maps and records equal the single-chunk run bit for bit, from device
    and from host frames."""
    import json

    rng = np.random.default_rng(43)
    js, blob = _context_net(32, (1, 4, 2), prec)
    T, H, W = 7, 40, 64
    frames = rng.integers(95, 900, (T, H, W)).astype(np.uint16)
    cam = synth.Camera(2.0, 100.0)
    small = json.dumps(dict(json.loads(js), chunk_px=2 * H * W))
    _, maps_one, logits_one = gpu_maps(js, blob, frames, cam)
    _, maps_two, logits_two = gpu_maps(small, blob, frames, cam)
    assert torch.equal(maps_one, maps_two) and torch.equal(logits_one, logits_two)
    one = sml.Localizer(js, blob).localize(frames, 0.5, gain=2.0, offset=100.0)
    loc2 = sml.Localizer(small, blob)
    host = loc2.localize(frames, 0.5, gain=2.0, offset=100.0)
    dev = loc2.localize(torch.from_numpy(frames).cuda(), 0.5, gain=2.0, offset=100.0)
    assert len(one) > 0 and one.tobytes() == host.tobytes() == dev.tobytes()


@pytest.mark.parametrize("in_ch", [1, 3])
def test_large_host_stacks_equal_device_frames(in_ch):
    """Host frames staged to the device per chunk give the device-frame records byte for
    byte: 150 frames of 256x256 as one chunk and as chunks of 64 frames (a short tail; with
    three-frame input each chunk also reads its neighbours' edge frames), from pageable and
    from pinned host memory."""
    import json

    rng = np.random.default_rng(47 + in_ch)
    spec = synth.NetSpec(in_ch=in_ch, channels=16, dilations=(1, 2, 1), precision="bf16")
    js = spec.to_json()
    blob = synth.pack_blob(spec, synth.init_weights(spec, 13))
    T, H, W = 150, 256, 256
    frames = rng.integers(95, 700, (T, H, W)).astype(np.uint16)
    kw = dict(gain=2.0, offset=100.0, capacity=T * H * W // 4)  # random-init net on noise: many maxima
    ref = sml.Localizer(js, blob).localize(torch.from_numpy(frames).cuda(), 0.5, **kw)
    assert len(ref) > 0
    pinned = torch.from_numpy(frames).pin_memory()
    for chunk_frames in (256, 64):
        loc = sml.Localizer(json.dumps(dict(json.loads(js), chunk_px=chunk_frames * H * W)), blob)
        assert loc.localize(frames, 0.5, **kw).tobytes() == ref.tobytes(), chunk_frames
        assert loc.localize(pinned, 0.5, **kw).tobytes() == ref.tobytes(), chunk_frames
        assert loc.localize(torch.from_numpy(frames).cuda(), 0.5, **kw).tobytes() == ref.tobytes(), chunk_frames
        loc.close()
