"""GPU training kernels (forward + hand-written backward behind torch.autograd.Function)
against the CPU oracle's exact float64 gradient, which is itself pinned to central finite
differences (tests/test_oracle_grad.py)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2410_02314_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__

    __graft_entry__.build()
    torch.cuda.set_device(0)


@pytest.mark.parametrize("C,dil,B,H,W", [(16, (1, 2, 4), 3, 20, 24), (48, (1, 2, 4, 8, 16, 8, 4, 1), 2, 40, 36)])
def test_gradients_match_oracle(C, dil, B, H, W):
    from paper_2410_02314_gb300.train import DilatedLocNet

    spec = synth.NetSpec(in_ch=1, channels=C, dilations=dil)
    blob = synth.pack_blob(spec, synth.init_weights(spec, 3))
    net = DilatedLocNet.from_blob(spec.to_json(), blob).cuda()
    rng = np.random.default_rng(1)
    frames, tgt, _, _ = synth.training_batch(rng, B=B, H=H, W=W, max_emitters=4)
    loss = net.loss(torch.from_numpy(frames).cuda(), torch.from_numpy(tgt).cuda())
    loss.backward()
    onet = oracle.Net(spec.to_json(), blob)
    x0 = oracle.ingest(frames, 1.0, 100.0, in_scale=onet.in_scale)
    val, gw, gb, ghw, ghb, _ = oracle.loss_grad(onet, x0, tgt)
    assert abs(loss.item() - val) <= 1e-5 * abs(val)
    got_w = np.concatenate([p.grad.detach().cpu().numpy().ravel() for p in net.w])
    got_b = np.concatenate([p.grad.detach().cpu().numpy().ravel() for p in net.b])
    for got, ref, name in [(got_w, gw, "conv_w"), (got_b, gb, "conv_b"),
                           (net.hw.grad.cpu().numpy().ravel(), ghw, "head_w"),
                           (net.hb.grad.cpu().numpy().ravel(), ghb, "head_b")]:
        err = np.abs(got - ref).max() / max(np.abs(ref).max(), 1e-12)
        print(name, "normalised max gradient error", err)
        assert err <= 1e-4, name


def test_training_reduces_loss():
    from paper_2410_02314_gb300.train import DilatedLocNet, train

    spec = synth.NetSpec(in_ch=1, channels=32, dilations=(1, 2, 4, 8, 4, 1))
    net = DilatedLocNet(spec, synth.init_weights(spec, 11)).cuda()
    hist = train(net, steps=150, batch=64, patch=48, lr=1e-3, pool=4, log_every=10)
    print("loss history", hist)
    first = np.mean([l for _, l in hist[:2]])
    last = np.mean([l for _, l in hist[-2:]])
    assert last < 0.7 * first


def _evaluate(loc, rng, n_frames, lo, hi):
    from oracle import mle

    frames, _, em, cam = synth.training_batch(rng, B=n_frames, H=64, W=64, min_emitters=lo, max_emitters=hi)
    truth = [np.c_[em.x[em.frame == t], em.y[em.frame == t], em.z[em.frame == t], em.photons[em.frame == t]]
             for t in range(n_frames)]
    best = None
    for p_min in (0.01, 0.03, 0.1, 0.2, 0.3, 0.5):
        recs = loc.localize(frames, p_min)
        pred = [np.c_[recs["x"][recs["frame"] == t], recs["y"][recs["frame"] == t], recs["z"][recs["frame"] == t],
                      recs["photons"][recs["frame"] == t]].astype(np.float64) for t in range(n_frames)]
        s = mle.score(pred, truth)
        if best is None or s["jaccard"] > best[1]["jaccard"]:
            best = (p_min, s)
    electrons = (frames.astype(np.float64) - cam.offset) / cam.gain
    base = None
    for thr in (20.0, 40.0, 80.0):
        pred_m = [mle.detect_and_fit(electrons[t], float(em.bg[t]), thr) for t in range(n_frames)]
        s = mle.score(pred_m, truth)
        if base is None or s["jaccard"] > base[1]["jaccard"]:
            base = (thr, s)
    return best, base


def _record_jaccard(got, ref, n_frames, radius_px=0.5):
    """Jaccard index of two record arrays, matched per frame within radius_px laterally."""
    from paper_2410_02314_gb300 import evaluate

    tp = fp = fn = 0
    for t in range(n_frames):
        a = np.c_[got["x"][got["frame"] == t], got["y"][got["frame"] == t]].astype(np.float64)
        b = np.c_[ref["x"][ref["frame"] == t], ref["y"][ref["frame"] == t]].astype(np.float64)
        pairs = evaluate.match(a, b, radius_px)
        tp += len(pairs)
        fp += len(a) - len(pairs)
        fn += len(b) - len(pairs)
    return tp / max(1, tp + fp + fn)


def _reduced_precision_vs_float64(js_bf16, blob, frames, p_min, thresholds=(0.03, 0.1, 0.3, 0.5)):
    """Record-level and map-level cost of BF16 and FP8 inference on a trained net: records of
    the GPU paths against the float64 oracle's records (matched within 0.5 px) at p_min, and
    the normalised max and 99.9th-percentile map errors (p compared as logits).  Returns
    {prec: {threshold: Jaccard}} over `thresholds`."""
    import paper_2410_02314_gb300 as sml

    onet = oracle.Net(js_bf16, blob)
    heads = oracle.forward(onet, frames)
    refs = {th: oracle.decode(oracle.maps_f32(heads), th, onet.z_scale, onet.ph_scale) for th in thresholds}
    T, H, W = frames.shape
    d_frames = torch.from_numpy(frames).cuda()
    js_fp8 = sml.calibrate_fp8(js_bf16, blob, d_frames[: max(1, T // 2)])
    out = {}
    for prec, js in (("bf16", js_bf16), ("fp8", js_fp8)):
        loc = sml.Localizer(js, blob)
        maps = torch.empty((T, 5, H, W), dtype=torch.float32, device="cuda")
        logits = torch.empty((T, H, W), dtype=torch.float32, device="cuda")
        loc.forward_maps(d_frames, maps, logits)
        got = maps.cpu().numpy().astype(np.float64)
        got[:, 0] = logits.cpu().numpy()
        err = np.abs(got - heads)
        scale = np.maximum(np.abs(heads).max(axis=(0, 2, 3)), 1e-6)
        out[prec] = {th: _record_jaccard(loc.localize(frames, th), refs[th], T) for th in thresholds}
        print(prec, "vs float64 on the trained net: records", {th: len(r) for th, r in refs.items()}, "Jaccard",
              {th: round(j, 4) for th, j in out[prec].items()},
              "| map max", np.round([err[:, k].max() / scale[k] for k in range(5)], 4),
              "p99.9", np.round([np.percentile(err[:, k], 99.9) / scale[k] for k in range(5)], 4))
        loc.close()
    assert all(len(r) > 0 for r in refs.values())
    return out


def test_trained_net_vs_mle_baseline():
    """What the learned part gains: a net trained on the simulator with the library's own
    forward/backward kernels, then run through the inference path (BF16), against the method
    without a network (smoothed local maxima + Gaussian MLE, oracle/mle.py) on held-out
    astigmatic 64x64 frames at a low density (0-10 emitters, ~0.1/um^2) and at the batched
    workload's density (20-40 emitters, ~0.5-1/um^2).  Reported: Jaccard, lateral and axial
    RMSE (250 nm matching radius), each method at its best threshold."""
    import paper_2410_02314_gb300 as sml
    from paper_2410_02314_gb300.train import DilatedLocNet, train

    spec = synth.NetSpec(in_ch=1, channels=48, dilations=(1, 2, 4, 8, 16, 8, 4, 1))
    net = DilatedLocNet(spec, synth.init_weights(spec, 11)).cuda()
    hist = train(net, steps=1500, batch=64, patch=64, lr=1e-3, pool=24, log_every=250, seed=5, max_emitters=40)
    print("training loss", hist)
    js, blob = net.to_blob("bf16")
    loc = sml.Localizer(js, blob)
    rng = np.random.default_rng(1234)  # held-out frames, same simulator
    results = {}
    for name, lo, hi in (("low density", 0, 10), ("high density", 20, 40)):
        best, base = _evaluate(loc, rng, 32, lo, hi)
        results[name] = (best, base)
        print(name, "| trained net (p_min=%s)" % best[0], best[1], "| local max + MLE (thr=%s)" % base[0], base[1])
    assert hist[-1][1] < 0.5 * hist[0][1]
    # reduced precision against float64 on the trained net (p maps are bimodal here, unlike
    # those of randomly initialised nets): held-out high-density frames
    held, _, _, _ = synth.training_batch(np.random.default_rng(99), B=24, H=64, W=64, min_emitters=20, max_emitters=40)
    jac = _reduced_precision_vs_float64(js, blob, held, results["high density"][0][0])
    print("record Jaccard vs float64", jac)
    # gates from the first measurement on this net (thresholds with >= 100 float64 records;
    # its p rarely exceeds 0.5 at this density): BF16 0.990-0.995, FP8 e4m3 0.86-0.89
    for th in (0.03, 0.1, 0.3):
        assert jac["bf16"][th] >= 0.985 and jac["fp8"][th] >= 0.80, (th, jac)
    net_hi, mle_hi = results["high density"][0][1], results["high density"][1][1]
    assert net_hi["jaccard"] > mle_hi["jaccard"], "the trained net should detect overlapping emitters better"

    # single-emitter precision along z against the CRLB (Sec. 4.1.1), net and MLE on the same
    # frames (3000 photons, background 100, 64x64 frames, 9 axial positions)
    from oracle import mle
    from paper_2410_02314_gb300 import evaluate

    p_low = results["low density"][0][0]

    def fit_mle(frames):
        rows = []
        for t in range(frames.shape[0]):
            e = frames[t].astype(np.float64) - 100.0
            for r in mle.detect_and_fit(e, 100.0, 40.0, win=7):
                rows.append((t, r[0], r[1], r[2]))
        out = np.zeros(len(rows), dtype=[("frame", "<i4"), ("x", "<f4"), ("y", "<f4"), ("z", "<f4")])
        for k, r in enumerate(rows):
            out[k] = r
        return out

    zs = np.linspace(-600.0, 600.0, 9)
    kw = dict(n_per_z=48, photons=3000.0, bg=100.0, size=64, seed=7)
    net_rows = evaluate.precision_vs_z(lambda f: loc.localize(f, p_low), zs, **kw)
    mle_rows = evaluate.precision_vs_z(fit_mle, zs, **kw)
    print("z nm | net: det, rmse x/y/z nm | MLE: det, rmse x/y/z nm | sqrt CRLB x/y/z nm")
    for a, b in zip(net_rows, mle_rows):
        print("%5.0f | %.2f %5.1f %5.1f %6.1f | %.2f %5.1f %5.1f %6.1f | %4.1f %4.1f %5.1f" % (
            a["z_nm"], a["detected"], a["rmse_x_nm"], a["rmse_y_nm"], a["rmse_z_nm"], b["detected"], b["rmse_x_nm"],
            b["rmse_y_nm"], b["rmse_z_nm"], a["crlb_x_nm"], a["crlb_y_nm"], a["crlb_z_nm"]))
    assert min(r["detected"] for r in net_rows) > 0.8
    # the MLE is an efficient estimator: within a factor 2 of sqrt(CRLB) laterally
    assert all(r["rmse_x_nm"] < 2.0 * r["crlb_x_nm"] for r in mle_rows if r["detected"] > 0.5)
