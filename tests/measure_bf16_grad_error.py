"""Measurement (GPU): gradient error of BF16 training against the oracle's float64 gradient.

Nets: (C=16, 3 layers, 3 patches of 20x24), (C=32, dilations 1,2,4,8,4,1, 4 patches of
48x48), (C=48, dilations 1,2,4,8,16,8,4,1, 4 patches of 64x64), 6 weight seeds each, batches
of simulated astigmatic patches (up to 6 emitters).  The loss and the gradient of every
parameter from the library's BF16 path (tensor-core forward, input and weight gradients,
bf16 activations and activation gradients) against oracle.loss_grad; per parameter group
(conv weights, conv biases, head weights, head biases): the normalised max error
max|g - g_ref| / max|g_ref|, the relative L2 error |g - g_ref| / |g_ref| and the cosine.

    python tests/measure_bf16_grad_error.py [--out bf16_grad_error.json]
"""
from __future__ import annotations

import argparse
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

NETS = [(16, (1, 2, 4), 3, 20, 24), (32, (1, 2, 4, 8, 4, 1), 4, 48, 48), (48, (1, 2, 4, 8, 16, 8, 4, 1), 4, 64, 64)]
GROUPS = ("conv_w", "conv_b", "head_w", "head_b")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--seeds", default="1,2,3,4,5,6")
    ap.add_argument("--out", default="")
    args = ap.parse_args()

    import torch

    import __graft_entry__
    import oracle
    from paper_2410_02314_gb300 import synth
    from paper_2410_02314_gb300.train import DilatedLocNet

    __graft_entry__.build()
    torch.cuda.set_device(0)
    rows = []
    for C, dil, B, H, W in NETS:
        for seed in (int(x) for x in args.seeds.split(",")):
            spec = synth.NetSpec(in_ch=1, channels=C, dilations=dil)
            blob = synth.pack_blob(spec, synth.init_weights(spec, 100 + seed))
            frames, tgt, _, _ = synth.training_batch(np.random.default_rng(seed), B=B, H=H, W=W, max_emitters=6)
            onet = oracle.Net(spec.to_json(), blob)
            x0 = oracle.ingest(frames, 1.0, 100.0, in_scale=onet.in_scale)
            val, gw, gb, ghw, ghb, _ = oracle.loss_grad(onet, x0, tgt)
            net = DilatedLocNet.from_blob(spec.to_json(), blob, precision="bf16").cuda()
            loss = net.loss(torch.from_numpy(frames).cuda(), torch.from_numpy(tgt).cuda())
            loss.backward()
            got = [np.concatenate([p.grad.double().cpu().numpy().ravel() for p in net.w]),
                   np.concatenate([p.grad.double().cpu().numpy().ravel() for p in net.b]),
                   net.hw.grad.double().cpu().numpy().ravel(), net.hb.grad.double().cpu().numpy().ravel()]
            r = {"C": C, "L": len(dil), "seed": seed, "loss_rel": abs(float(loss.item()) - val) / abs(val),
                 "device_error": net.device_error()}
            for name, a, ref in zip(GROUPS, got, (gw, gb, ghw, ghb)):
                r[name] = {"max": float(np.abs(a - ref).max() / max(np.abs(ref).max(), 1e-30)),
                           "l2": float(np.linalg.norm(a - ref) / max(np.linalg.norm(ref), 1e-30)),
                           "cos": float(a @ ref / max(np.linalg.norm(a) * np.linalg.norm(ref), 1e-30))}
            print(json.dumps(r), flush=True)
            rows.append(r)
    summary = {}
    for C, dil, *_ in NETS:
        rs = [r for r in rows if r["C"] == C]
        summary[f"C{C}_L{len(dil)}"] = {
            "loss_rel": max(r["loss_rel"] for r in rs),
            **{f"{g}_{k}": (min if k == "cos" else max)(r[g][k] for r in rs) for g in GROUPS for k in ("max", "l2", "cos")}}
    print(json.dumps({"summary": summary}), flush=True)
    if args.out:
        with open(args.out, "w") as f:
            json.dump({"rows": rows, "summary": summary}, f, indent=1)


if __name__ == "__main__":
    main()
