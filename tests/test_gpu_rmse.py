"""Localization cost of each precision against the FP64 oracle, per benchmark configuration:
the GPU records and the oracle's records (its float64 forward, then the float32 decode) are
matched per frame within 0.5 px; reported are the Jaccard index of the two record sets and,
over matched pairs, the lateral and axial RMSE (nm, 100 nm pixels) and the photon-count
relative RMSE.  The nets are random-init, so these measure the arithmetic, not localization
quality.  Gates are a few times the values measured on a GB300 (printed by the test)."""
import math

import numpy as np
import pytest
import torch

import oracle
import paper_2410_02314_gb300 as sml
from paper_2410_02314_gb300 import evaluate, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__

    __graft_entry__.build()
    torch.cuda.set_device(0)


def _compare(got, ref, T):
    tp = fp = fn = 0
    dl2, dz2, dn2 = [], [], []
    for t in range(T):
        a, b = got[got["frame"] == t], ref[ref["frame"] == t]
        pairs = evaluate.match(np.c_[a["x"], a["y"]], np.c_[b["x"], b["y"]], 0.5)
        tp += len(pairs)
        fp += len(a) - len(pairs)
        fn += len(b) - len(pairs)
        for i, j in pairs:
            dl2.append((100.0 * (float(a["x"][i]) - float(b["x"][j]))) ** 2 + (100.0 * (float(a["y"][i]) - float(b["y"][j]))) ** 2)
            dz2.append((float(a["z"][i]) - float(b["z"][j])) ** 2)
            dn2.append(((float(a["photons"][i]) - float(b["photons"][j])) / max(abs(float(b["photons"][j])), 1.0)) ** 2)
    r = lambda v: math.sqrt(float(np.mean(v))) if v else float("nan")
    return {"records": len(ref), "jaccard": tp / max(1, tp + fp + fn), "rmse_lateral_nm": r(dl2), "rmse_axial_nm": r(dz2),
            "rmse_photons_rel": r(dn2)}


def _oracle_records(js, blob, frames, cam, p_min):
    net = oracle.Net(js, blob)
    kw = dict(gain=cam.gain, offset=cam.offset,
              gain_map=None if cam.gain_map is None else cam.gain_map.astype(np.float64),
              offset_map=None if cam.offset_map is None else cam.offset_map.astype(np.float64))
    return oracle.decode(oracle.maps_f32(oracle.forward(net, frames, **kw)), p_min, net.z_scale, net.ph_scale)


def _gpu_records(js, blob, frames, cam, p_min):
    loc = sml.Localizer(js, blob)
    recs = loc.localize(frames, p_min, gain=cam.gain, offset=cam.offset, gain_map=cam.gain_map, offset_map=cam.offset_map)
    loc.close()
    return recs


# (config, precision): gates (max lateral RMSE nm, min Jaccard), a few times the values measured
# on a GB300: small FP32 0.0 nm / 1.0, BF16 0.07 / 0.968; batched FP32 0.0002 / 1.0, BF16
# 0.19 / 0.929; large-FOV crop BF16 0.31 / 0.893.  FP8 records are gated on the trained net
# only (tests/test_gpu_train.py): random-init p maps hover at the threshold, so the record
# Jaccard of FP8 against float64 here (0.25-0.36 measured) says nothing a gate could hold
# to; FP8's maps are gated against the oracle in tests/test_gpu_parity.py.
CASES = {
    ("small_64", "fp32"): (0.01, 0.999),
    ("small_64", "bf16"): (0.5, 0.9),
    ("batched_256", "fp32"): (0.01, 0.999),
    ("batched_256", "bf16"): (1.0, 0.85),
    ("large_fov_512", "bf16"): (1.5, 0.8),
}


def _workload(name, prec):
    if name == "small_64":
        w = synth.workload_small(precision="bf16" if prec == "fp8" else prec)
        return w.spec, w.blob, w.frames, w.cam
    if name == "batched_256":
        w = synth.workload_batched(T=4, precision="bf16" if prec == "fp8" else prec)
        return w.spec, w.blob, w.frames, w.cam
    w = synth.workload_large_fov(T=2, H=512, W=512, precision="bf16")
    return w.spec, w.blob, w.frames, w.cam


@pytest.mark.parametrize("name,prec", list(CASES))
def test_localization_rmse_against_the_fp64_oracle(name, prec):
    spec, blob, frames, cam = _workload(name, prec)
    js = synth.NetSpec(**{**spec.__dict__, "precision": "bf16" if prec == "fp8" else prec}).to_json()
    if prec == "fp8":
        gm = None if cam.gain_map is None else torch.from_numpy(cam.gain_map).cuda()
        om = None if cam.offset_map is None else torch.from_numpy(cam.offset_map).cuda()
        js = sml.calibrate_fp8(js, blob, torch.from_numpy(frames).cuda(), gain=cam.gain, offset=cam.offset, gain_map=gm,
                               offset_map=om)
    ref = _oracle_records(js, blob, frames, cam, 0.5)
    got = _gpu_records(js, blob, frames, cam, 0.5)
    s = _compare(got, ref, frames.shape[0])
    print(name, prec, {k: round(v, 4) if isinstance(v, float) else v for k, v in s.items()})
    max_rmse, min_jac = CASES[(name, prec)]
    assert s["records"] > 0 and s["rmse_lateral_nm"] <= max_rmse and s["jaccard"] >= min_jac
