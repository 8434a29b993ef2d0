"""Measurement (GPU): FP8 e4m3 map error over whole frames.

The 48-channel 8-layer net (7 tensor-core layers, Sec. 3.2.1) in FP8 with the oracle's
per-layer activation scales, against the oracle's fp8 mode (e4m3 rounding of weights and
stored activations where the tensor-core path rounds them) and its float64 forward, every
pixel of every map: whole 256x256 frames of the batched workload (8 weight seeds, two frames
each) and whole 2048x2048 sCMOS frames of the large field-of-view workload (2 weight seeds,
one frame each).  Per comparison: the normalised max error max|gpu - ref| / max|ref|, the
normalised RMS error and the normalised 99.99th percentile of |gpu - ref| (p compared as
logits).

    python tests/measure_fp8_error.py [--out fp8_error.json]
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


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default="")
    ap.add_argument("--seeds256", default="1,2,3,4,5,6,7,8")
    ap.add_argument("--seeds2048", default="1,2")
    args = ap.parse_args()

    import torch

    import __graft_entry__
    import oracle
    import paper_2410_02314_gb300 as sml
    from paper_2410_02314_gb300 import synth

    __graft_entry__.build()
    torch.cuda.set_device(0)

    def run(spec, blob, frames, cam, sel, crop):
        net = oracle.Net(spec.to_json(), blob)
        gm = None if cam.gain_map is None else cam.gain_map.astype(np.float64)
        om = None if cam.offset_map is None else cam.offset_map.astype(np.float64)
        (i0, i1, j0, j1) = crop
        scales = oracle.act_scales(net, frames[:1, i0:i1, j0:j1], cam.gain, cam.offset,
                                   None if gm is None else gm[i0:i1, j0:j1], None if om is None else om[i0:i1, j0:j1])
        js = json.dumps(dict(json.loads(spec.to_json()), precision="fp8", act_scales=scales))
        loc = sml.Localizer(js, blob)
        T, H, W = frames.shape
        maps = torch.empty((T, 5, H, W), dtype=torch.float32, device="cuda")
        logits = torch.empty((T, H, W), dtype=torch.float32, device="cuda")
        dg = None if cam.gain_map is None else torch.from_numpy(cam.gain_map).cuda()
        do = None if cam.offset_map is None else torch.from_numpy(cam.offset_map).cuda()
        loc.forward_maps(torch.from_numpy(frames).cuda(), maps, logits, gain=cam.gain, offset=cam.offset, gain_map=dg,
                         offset_map=do)
        torch.cuda.synchronize()
        got = maps.cpu().numpy().astype(np.float64)
        got[:, 0] = logits.cpu().numpy()
        got = got[sel]
        fr = np.ascontiguousarray(frames[sel])
        kw = dict(gain=cam.gain, offset=cam.offset, gain_map=gm, offset_map=om)
        refq = oracle.forward(oracle.quantized(net, "fp8"), fr, quant="fp8", scales=scales, **kw)
        ref = oracle.forward(net, fr, **kw)
        loc.close()
        return {"vs_q": stats(got, refq), "vs_f64": stats(got, ref)}

    rows = []
    for seed in (int(x) for x in args.seeds256.split(",") if x):
        w = synth.workload_batched(T=2, precision="bf16", seed=seed)
        r = run(w.spec, w.blob, w.frames, w.cam, [0, 1], (0, 256, 0, 256))
        r.update(workload="batched 256x256", seed=seed, frames=2)
        print(json.dumps(r), flush=True)
        rows.append(r)
    for seed in (int(x) for x in args.seeds2048.split(",") if x):
        w = synth.workload_large_fov(T=2, precision="bf16", seed=seed)
        r = run(w.spec, w.blob, w.frames, w.cam, [1], (700, 956, 900, 1156))
        r.update(workload="large_fov 2048x2048", seed=seed, frames=1)
        print(json.dumps(r), flush=True)
        rows.append(r)
    summary = {}
    for wl in sorted({r["workload"] for r in rows}):
        rs = [r for r in rows if r["workload"] == wl]
        summary[wl] = {f"{ref}_{k}": max(r[ref][k] for r in rs) for ref in ("vs_q", "vs_f64") for k in ("max", "rms", "p9999")}
    print(json.dumps({"summary": summary}), flush=True)
    if args.out:
        with open(args.out, "w") as f:
            json.dump({"rows": rows, "summary": summary}, f, indent=1)


if __name__ == "__main__":
    main()
