"""Measurement (GPU): reduced-precision map error against network depth.

Plain 48-channel dilated stacks with n = 7, 14, 21 and 28 tensor-core layers (layer 0 is the
SIMT first layer; the tensor-core layers take the dilations 2, 4, 8, 16, 8, 4, 1 in turn and
the last one, d = 1, feeds the heads), four weight seeds each, Kaiming-uniform init (Sec.
3.2.1 dilated convolution, Sec. 3.2 heads).  For each net the library's maps on two 256x256
frames of the batched workload are compared, per map, with the oracle's float64 forward and
with its bf16 mode (weights and stored activations rounded where the tensor-core path rounds
them), as the normalised max error max|gpu - ref| / max|ref| and the normalised RMS error (p
compared as logits).  FP32 (SIMT) is compared with float64 as well.

    python tests/measure_depth_error.py [--out depth_error.json]

Prints one JSON line per (depth, seed) and a summary per depth; the depth gate of the GPU
parity tests (tests/gpu_gates.py) is set from this curve.
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

CYCLE = (2, 4, 8, 16, 8, 4, 1)


def dilations(n_tc):
    """Layer 0 (d = 1), then n_tc tensor-core layers: n_tc - 1 from CYCLE in turn, the last d = 1."""
    mid = [CYCLE[k % len(CYCLE)] for k in range(n_tc - 1)]
    return (1, *mid, 1)


def errors(got, ref):
    mx = [float(np.abs(got[:, k] - ref[:, k]).max() / max(np.abs(ref[:, k]).max(), 1e-6)) for k in range(5)]
    rms = [float(np.sqrt(np.mean((got[:, k] - ref[:, k]) ** 2)) / max(np.abs(ref[:, k]).max(), 1e-6))
           for k in range(5)]
    return mx, rms


def gpu_maps(js, blob, frames, cam):
    import torch

    import paper_2410_02314_gb300 as sml

    loc = sml.Localizer(js, blob)
    T, H, W = frames.shape
    maps = torch.empty((T, 5, H, W), dtype=torch.float32, device="cuda")
    logits = torch.empty((T, H, W), dtype=torch.float32, device="cuda")
    loc.forward_maps(torch.from_numpy(frames).cuda(), maps, logits, gain=cam.gain, offset=cam.offset)
    torch.cuda.synchronize()
    got = maps.cpu().numpy().astype(np.float64)
    got[:, 0] = logits.cpu().numpy()
    loc.close()
    return got


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--depths", default="7,14,21,28")
    ap.add_argument("--seeds", default="1,2,3,4")
    ap.add_argument("--frames", type=int, default=2)
    ap.add_argument("--out", default="")
    args = ap.parse_args()

    import torch

    import __graft_entry__
    import oracle
    from paper_2410_02314_gb300 import synth

    __graft_entry__.build()
    torch.cuda.set_device(0)
    w = synth.workload_batched(T=args.frames, H=256, W=256, precision="bf16", seed=3)
    rows = []
    for n_tc in (int(x) for x in args.depths.split(",")):
        dil = dilations(n_tc)
        for seed in (int(x) for x in args.seeds.split(",")):
            t0 = time.time()
            res = {"n_tc": n_tc, "seed": seed, "dilations": list(dil)}
            for prec in ("bf16", "fp32"):
                spec = synth.NetSpec(in_ch=1, channels=48, dilations=dil, precision=prec)
                blob = synth.pack_blob(spec, synth.init_weights(spec, 1000 + seed))
                if prec == "bf16":
                    net = oracle.Net(spec.to_json(), blob)
                    ref = oracle.forward(net, w.frames, w.cam.gain, w.cam.offset)
                    refq = oracle.forward(oracle.quantized(net, "bf16"), w.frames, w.cam.gain, w.cam.offset,
                                          quant="bf16")
                got = gpu_maps(spec.to_json(), blob, w.frames, w.cam)
                mx, rms = errors(got, ref)
                res[f"{prec}_vs_f64_max"], res[f"{prec}_vs_f64_rms"] = max(mx), max(rms)
                if prec == "bf16":
                    mxq, rmsq = errors(got, refq)
                    res["bf16_vs_q_max"], res["bf16_vs_q_rms"] = max(mxq), max(rmsq)
                    res["bf16_vs_f64_max_per_map"] = mx
            res["seconds"] = time.time() - t0
            print(json.dumps(res), flush=True)
            rows.append(res)
    summary = {}
    for n_tc in sorted({r["n_tc"] for r in rows}):
        rs = [r for r in rows if r["n_tc"] == n_tc]
        summary[n_tc] = {k: {"max": max(r[k] for r in rs), "mean": float(np.mean([r[k] for r in rs]))}
                         for k in ("bf16_vs_f64_max", "bf16_vs_f64_rms", "bf16_vs_q_max", "bf16_vs_q_rms",
                                   "fp32_vs_f64_max")}
    print(json.dumps({"summary": summary}), flush=True)
    if args.out:
        with open(args.out, "w") as f:
            json.dump({"rows": rows, "summary": summary}, f, indent=1)


if __name__ == "__main__":
    main()
