"""Measurement (GPU): FP8 e4m3 map error of nets with dense connection dilated blocks
(Sec. 3.2.1) and the U-Net fine stage (Sec. 3.2), over whole frames.

Each net runs in FP8 with the oracle's activation scales (one per stored layer output) and is
compared, every pixel of the five position maps, with the oracle's fp8 mode (weights folded with their input channels' scales and
rounded per output channel, every stored output rounded to e4m3 with its layer's scale, as
the library does) and with its float64 forward: normalised max, RMS and 99.99th percentile of
|gpu - ref| (p compared as logits), worst over the weight seeds.  Two workloads: two whole
256x256 frames of the batched workload through five nets (two of them the dense-block
benchmark net and the full topology), and five ragged 37x150 sCMOS astigmatic frames (2
emitters/um^2, per-pixel gain and offset maps) through the nets of the GPU parity cases.  The
library's own calibration (sml_calibrate_fp8 on a bf16 context) is compared with the oracle's
scales on the first workload.

    python tests/measure_fp8_dense_error.py [--out fp8_dense_error.json]
"""
from __future__ import annotations

import argparse
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def stats(got, ref):
    out = {}
    for name, fn in (("max", lambda d: d.max()), ("rms", lambda d: np.sqrt(np.mean(d * d))),
                     ("p9999", lambda d: np.quantile(d, 0.9999))):
        out[name] = max(float(fn(np.abs(got[:, k] - ref[:, k])) / max(np.abs(ref[:, k]).max(), 1e-6)) for k in range(5))
    return out


def nets():
    from paper_2410_02314_gb300 import synth

    small = {"growth": 16, "blocks": [[2, 4]]}
    two = {"growth": 16, "blocks": [[2, 4], [1, 8, 3]]}
    return [
        ("dcd 1 block", synth.NetSpec(in_ch=1, channels=32, dilations=(1, 2, 1), dcd=small), (1, 2, 3, 4)),
        ("dcd 2 blocks", synth.NetSpec(in_ch=1, channels=32, dilations=(1, 2, 1), dcd=two), (1, 2, 3, 4)),
        ("unet 2 levels", synth.NetSpec(in_ch=1, channels=32, dilations=(1, 2, 4, 1), unet=2), (1, 2, 3, 4)),
        ("dcd benchmark net", synth.spec_dcd("bf16"), (1, 2)),
        ("full topology", synth.spec_dilatedloc("bf16"), (1, 2)),
    ]


# the nets of the ragged-frame GPU parity cases: C, growth, blocks, dilations, levels, in_ch, heads
CASES = [
    (32, 16, ((2, 4), (1, 8, 3)), (1, 2, 1), 0, 1, 5),
    (16, 32, ((3, 5),), (2, 1), 0, 3, 5),
    (48, 16, ((1, 2),), (1, 4, 1), 0, 1, 5),
    (32, 0, (), (1, 2, 1), 2, 1, 5),
    (16, 16, ((2, 4),), (1, 1), 1, 1, 9),
    (48, 0, (), (1, 4, 2, 1), 2, 1, 5),
]


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default="")
    ap.add_argument("--workloads", default="ragged,batched", help="comma-separated subset of ragged,batched")
    args = ap.parse_args()
    which = set(args.workloads.split(","))

    import torch

    import __graft_entry__
    import oracle
    import paper_2410_02314_gb300 as sml
    from paper_2410_02314_gb300 import synth

    __graft_entry__.build()
    torch.cuda.set_device(0)
    w = synth.workload_batched(T=2, precision="bf16", seed=3)
    frames, cam = w.frames, w.cam
    d_frames = torch.from_numpy(frames).cuda()
    rows = []

    def maps_of(js, blob, frames, cam, nh):
        loc = sml.Localizer(js, blob)
        T, H, W = frames.shape
        maps = torch.empty((T, nh, H, W), dtype=torch.float32, device="cuda")
        logits = torch.empty((T, H, W), dtype=torch.float32, device="cuda")
        gm = None if cam.gain_map is None else torch.from_numpy(cam.gain_map).cuda()
        om = None if cam.offset_map is None else torch.from_numpy(cam.offset_map).cuda()
        loc.forward_maps(torch.from_numpy(frames).cuda(), maps, logits, gain=cam.gain, offset=cam.offset, gain_map=gm,
                         offset_map=om)
        torch.cuda.synchronize()
        got = maps.cpu().numpy().astype(np.float64)
        got[:, 0] = logits.cpu().numpy()
        loc.close()
        return got

    for C, g, blocks, dil, levels, in_ch, nh in (CASES if "ragged" in which else []):
        name = f"ragged sCMOS: C={C} growth={g} blocks={list(map(list, blocks))} unet={levels} in_ch={in_ch}"
        for seed in (1, 2, 3, 4):
            rng = np.random.default_rng(7 + C + g + levels + 1000 * seed)
            dcd = {"growth": g, "blocks": [list(b) for b in blocks]} if blocks else None
            spec = synth.NetSpec(in_ch=in_ch, channels=C, dilations=tuple(dil), precision="bf16", dcd=dcd,
                                 unet=levels, n_heads=nh)
            blob = synth.pack_blob(spec, synth.init_weights(spec, 100 + seed))
            net = oracle.Net(spec.to_json(), blob)
            T, H, W = 5, 37, 150
            cam = synth.scmos_camera(rng, H, W)
            em = synth.emitters_density(rng, T, H, W, 2.0, astig=True)
            frames = synth.simulate(em, T, H, W, cam, True, rng)
            kw = dict(gain=cam.gain, offset=cam.offset, gain_map=cam.gain_map.astype(np.float64),
                      offset_map=cam.offset_map.astype(np.float64))
            scales = oracle.act_scales(net, frames, **kw)
            js = json.dumps(dict(json.loads(spec.to_json()), precision="fp8", act_scales=scales, chunk_px=2 * H * W))
            got = maps_of(js, blob, frames, cam, nh)
            refq = oracle.forward(oracle.quantized(net, "fp8", scales), frames, quant="fp8", scales=scales, **kw)
            ref = oracle.forward(net, frames, **kw)
            r = {"net": name, "seed": seed, "n_tc": net.L - 1, "vs_q": stats(got, refq), "vs_f64": stats(got, ref),
                 "calibration_rel_dev": 0.0}
            print(json.dumps(r), flush=True)
            rows.append(r)

    for name, spec, seeds in (nets() if "batched" in which else []):
        for seed in seeds:
            spec.precision = "bf16"
            blob = synth.pack_blob(spec, synth.init_weights(spec, 100 + seed))
            net = oracle.Net(spec.to_json(), blob)
            scales = oracle.act_scales(net, frames, cam.gain, cam.offset)
            lib_scales = json.loads(sml.calibrate_fp8(spec.to_json(), blob, d_frames, gain=cam.gain,
                                                      offset=cam.offset))["act_scales"]
            cal = max(abs(a / b - 1.0) for a, b in zip(lib_scales[1:], scales[1:]))
            js = json.dumps(dict(json.loads(spec.to_json()), precision="fp8", act_scales=scales))
            loc = sml.Localizer(js, blob)
            nh = net.nh
            maps = torch.empty((2, nh, 256, 256), dtype=torch.float32, device="cuda")
            logits = torch.empty((2, 256, 256), dtype=torch.float32, device="cuda")
            loc.forward_maps(d_frames, maps, logits, gain=cam.gain, offset=cam.offset)
            torch.cuda.synchronize()
            got = maps.cpu().numpy().astype(np.float64)
            got[:, 0] = logits.cpu().numpy()
            kw = dict(gain=cam.gain, offset=cam.offset)
            refq = oracle.forward(oracle.quantized(net, "fp8", scales), frames, quant="fp8", scales=scales, **kw)
            ref = oracle.forward(net, frames, **kw)
            loc.close()
            r = {"net": name, "seed": seed, "n_tc": net.L - 1, "vs_q": stats(got, refq), "vs_f64": stats(got, ref),
                 "calibration_rel_dev": cal}
            print(json.dumps(r), flush=True)
            rows.append(r)
    summary = {}
    for name in dict.fromkeys(r["net"] for r in rows):
        rs = [r for r in rows if r["net"] == name]
        summary[name] = {"n_tc": rs[0]["n_tc"], **{f"{ref}_{k}": max(r[ref][k] for r in rs)
                                                   for ref in ("vs_q", "vs_f64") for k in ("max", "rms", "p9999")},
                         "calibration_rel_dev": max(r["calibration_rel_dev"] for r in rs)}
    print(json.dumps({"summary": summary}, indent=1), flush=True)
    if args.out:
        with open(args.out, "w") as f:
            json.dump({"rows": rows, "summary": summary}, f, indent=1)


if __name__ == "__main__":
    main()
