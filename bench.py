"""Benchmark: localization throughput of the dilated-conv localization path on one GB300.

Workload (the batched-inference configuration): 256 frames of 256x256 uint16, 1 emitter per
um^2 at 100 nm pixels, sigma 1.3 px, photons LogNormal(ln 3000, 0.5), background U(50,200);
48-channel 8-layer dilated net (dilations 1,2,4,8,16,8,4,1), random-init weights from a seed.
One step = the whole path (camera transform, 8 conv layers, heads, decode into records) over
the 256-frame batch.  `value` is frames/s with inputs resident in HBM; `e2e` is the same
metric through the synchronous C-ABI call with host buffers (H2D of the frames and D2H of
the records inside the timed region).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision bf16|fp32|fp8] [--impl reference]

With N > 1 (launched by torchrun) every rank processes its own batch: replicas with no
collective on the data path ("weak" scaling); rank 0 prints the max-over-ranks timing.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

T_FRAMES, H, W = 256, 256, 256
P_MIN = 0.5
FALLBACK_PEAKS = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return dict(FALLBACK_PEAKS), "fallback"


def conv_flops_per_px(C):
    return 2 * 9 * C * C


def conv_class_work(spec, px, elem_bytes):
    """Algorithmic FLOPs and HBM bytes of one chunk's conv-class launches (every conv layer but
    the first and the last, and the U-Net's pool and upsample launches) over px full-resolution
    pixels, and the number of those launches.  A conv reads its ci input channels and writes
    its co outputs once per pixel of its level (px / 4^level); a pool or upsample reads and
    writes C channels at the two levels it joins."""
    lay = spec.layers()
    C, U = spec.channels, spec.unet
    feat = lay[1 : len(lay) - 1 - 2 * U]
    flops = sum(18 * ci * co for ci, co, _ in feat) * px
    nbytes = sum(ci + co for ci, co, _ in feat) * px * elem_bytes
    launches = len(feat)
    for lv in range(1, U + 1):
        lo, hi = px / 4 ** lv, px / 4 ** (lv - 1)
        flops += 18 * C * C * lo + 18 * 2 * C * C * hi  # down conv at lv, up conv at lv - 1
        nbytes += ((C + C) * lo + (2 * C + C) * hi + 2 * C * (lo + hi)) * elem_bytes  # convs, pool, upsample
        launches += 4
    return flops, nbytes, launches


def measure_peaks(dev, n=8192, reps=5):
    """Dense peaks measured here, next to the measured BF16 and copy figures: FP8 e4m3
    through torch._scaled_mm (cuBLASLt, 2 n^3 FLOP per call) and FP32 through torch.matmul
    with TF32 off (cuBLAS SGEMM on the FMA pipes), best of `reps` calls (burst), CUDA events."""
    import torch

    def best(fn, flops):
        for _ in range(2):
            fn()
        torch.cuda.synchronize()
        t = []
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            fn()
            b.record()
            torch.cuda.synchronize()
            t.append(a.elapsed_time(b) / 1000.0)
        return flops / min(t) / 1e12

    out = {"how": f"best of {reps} calls, {n}^3: fp8 torch._scaled_mm (e4m3 x e4m3 -> bf16), fp32 torch.matmul "
                  f"with TF32 off (SGEMM)"}
    x = torch.randn(n, n, device=dev, dtype=torch.bfloat16)
    y = torch.randn(n, n, device=dev, dtype=torch.bfloat16)
    try:
        a8 = x.to(torch.float8_e4m3fn)
        b8 = y.to(torch.float8_e4m3fn).t().contiguous().t()
        one = torch.ones((), device=dev)
        out["fp8_tflops"] = best(lambda: torch._scaled_mm(a8, b8, scale_a=one, scale_b=one, out_dtype=torch.bfloat16),
                                 2 * n ** 3)
        del a8, b8
    except Exception as e:  # recorded, and the FP8 roofline then says which peak it used
        out["fp8_error"] = repr(e)[:200]
    tf32 = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = False
    try:
        xf, yf = x.float(), y.float()
        out["fp32_tflops"] = best(lambda: torch.matmul(xf, yf), 2 * n ** 3)
        del xf, yf
    finally:
        torch.backends.cuda.matmul.allow_tf32 = tf32
    del x, y
    torch.cuda.empty_cache()
    return out


def conv_roofline(spec, precision, px_per_launch, conv_ms, conv_n, pk, live, traffic):
    """Roofline of the dominant kernel, the middle-layer conv (k_dconv_tc; k_dconv_f32 in FP32).
    It is a dense contraction, so the tensor pipe bounds it (the ALU pipes for the FP32 SIMT
    path): achieved = the layer's FLOPs per launch (2 x 9 x Cin x Cout per pixel x the
    launch's pixels) / the mean launch time (CUDA events on the launching stream); peak = the
    burst dense peak of the launch's operand type: BF16 the measured cuBLAS figure,
    FP8 and FP32 measured here (measure_peaks).  The HBM side is reported beside it: the
    layer's activation bytes (Cin + Cout per pixel, read once and written once) over the
    launch time against the measured copy bandwidth, and the DRAM bytes ncu counted."""
    elem = {"bf16": 2, "fp8": 1, "fp32": 4}[precision]
    fl, nb, n_launch = conv_class_work(spec, px_per_launch, elem)
    flops_launch, bytes_launch = fl / n_launch, nb / n_launch
    avg_s = conv_ms / max(conv_n, 1) / 1000.0
    achieved = flops_launch / avg_s / 1e12
    if precision == "bf16":
        peak, peak_kind = pk["bf16_tflops"], f"bf16 dense burst, cuBLAS ({'measured' if 'when' in pk else 'fallback'})"
    elif precision == "fp8" and live.get("fp8_tflops"):
        peak, peak_kind = live["fp8_tflops"], "fp8 e4m3 dense burst, measured here (torch._scaled_mm)"
    elif precision == "fp8":
        peak, peak_kind = 2.0 * pk["bf16_tflops"], "fp8 = 2 x measured bf16 burst (nominal 4.5/2.25 ratio)"
    else:
        peak, peak_kind = live.get("fp32_tflops", 80.5), "fp32 FMA, measured here (SGEMM)"
    kernel = "k_dconv_tc (middle layers)" if precision != "fp32" else "k_dconv_f32 (middle layers)"
    hbm = {"bytes_per_launch": bytes_launch, "gbs": bytes_launch / avg_s / 1e9, "peak_gbs": pk["hbm_gbs"],
           "frac": bytes_launch / avg_s / 1e9 / pk["hbm_gbs"],
           "note": "the layer's own activation bytes (input and output once each); the method's algorithmic bytes "
                   "are the frames in and the records out (about 2.5 B/px for the whole path)"}
    if traffic is not None:
        hbm.update({"dram_gbs": traffic / avg_s / 1e9, "dram_frac": traffic / avg_s / 1e9 / pk["hbm_gbs"]})
    return {"bound": "tensor" if precision != "fp32" else "alu", "achieved": achieved, "peak": peak,
            "unit": "TFLOP/s", "frac": achieved / peak, "traffic": traffic, "kernel": kernel, "peak_kind": peak_kind,
            "flops_per_launch": flops_launch, "px_per_launch": px_per_launch, "launches": conv_n,
            "avg_launch_ms": avg_s * 1000, "hbm": hbm}


def algorithmic_flops_per_px(spec):
    C, L = spec.channels, spec.L
    return 2 * (9 * C + (L - 1) * 9 * C * C + 5 * C)


CLOCK_REASONS = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")


def _smi_time(text):
    """nvidia-smi's timestamp field (local time, e.g. 2026/12/04 01:53:02.123) as a datetime,
    or None if it does not parse."""
    import datetime

    for fmt in ("%Y/%m/%d %H:%M:%S.%f", "%Y/%m/%d %H:%M:%S"):
        try:
            return datetime.datetime.strptime(text.strip(), fmt)
        except ValueError:
            pass
    return None


def parse_clock_samples(lines, begin=None, end=None):
    """Summary of nvidia-smi samples (timestamp, index, clocks.sm, clocks.max.sm, power.draw,
    active reasons, then the four reasons of CLOCK_REASONS).  With begin/end (local
    datetimes of the timed region) only the samples taken inside it count; if none does (a
    region shorter than the sampling period) or the timestamps do not parse, all samples
    count and "window" says so."""
    rows = []
    for line in lines:
        parts = [x.strip() for x in line.split(",")]
        if len(parts) < 10:
            continue
        try:
            sm, mx = float(parts[2]), float(parts[3])
        except ValueError:
            continue
        active = [n for n, v in zip(CLOCK_REASONS, parts[6:10]) if v.lower().startswith("active")]
        rows.append((_smi_time(parts[0]), sm, mx, active))
    if not rows:
        return None
    inside = [r for r in rows if begin is not None and r[0] is not None and begin <= r[0] <= end]
    use, window = (inside, "timed region") if inside else (rows, "around the timed region")
    return {"sm_mhz": statistics.median(r[1] for r in use), "sm_max_mhz": max(r[2] for r in use),
            "samples": len(use), "window": window,
            "reasons": sorted({n for r in use for n in r[3]})}


class ClockSampler:
    """nvidia-smi clock and throttle-reason samples (every 50 ms) around the timed region; the
    summary keeps the samples stamped inside it."""

    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.begin = self.end = None
        import tempfile

        self.path = os.path.join(tempfile.gettempdir(), f"sml_bench_clocks_gpu{index}_{os.getpid()}.csv")

    def start(self):
        """Start sampling and wait (at most 3 s) until the first sample is written."""
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "50"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
            return
        t0 = time.time()
        while time.time() - t0 < 3.0 and self.proc.poll() is None:
            if os.path.getsize(self.path) > 0:
                break
            time.sleep(0.02)

    def mark_begin(self):
        import datetime

        self.begin = datetime.datetime.now()

    def mark_end(self):
        import datetime

        self.end = datetime.datetime.now()

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.1)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        with open(self.path) as f:
            return parse_clock_samples(f.readlines(), self.begin, self.end)


def kernel_source_hash():
    """sha256[:16] of the conv kernel's sources (k_tc.cu and the inline-PTX helpers it includes)."""
    h = hashlib.sha256()
    for name in ("k_tc.cu", "tc_ptx.cuh"):
        with open(os.path.join(ROOT, "paper_2410_02314_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def profiled_traffic(precision, workload="batched256"):
    """DRAM bytes per launch of the middle-layer conv kernel from the committed ncu summary,
    valid only if the kernel source hash recorded there matches the current source."""
    p = os.path.join(ROOT, "profiles", f"dconv_tc_{precision}_{workload}.md")
    if not os.path.exists(p):
        return None
    text = open(p).read()
    m_hash = re.search(r"conv kernel sources sha256\[:16\]:\s*([0-9a-f]{16})", text)
    m_bytes = re.search(r"dram bytes per full launch:\s*([0-9.e+]+)", text)
    if not m_hash or not m_bytes or m_hash.group(1) != kernel_source_hash():
        return None
    return float(m_bytes.group(1))


def cpu_baseline(w, budget_s=12.0):
    """The oracle as it stands (forward + decode) on whole frames of the workload, on the host
    cores; as many frames as fit the time budget (at least one)."""
    import oracle

    net = oracle.Net(w.spec.to_json(), w.blob)
    done, t0 = 0, time.perf_counter()
    while True:
        f = w.frames[done : done + 1]
        oracle.localize(net, f, P_MIN, w.cam.gain, w.cam.offset)
        done += 1
        el = time.perf_counter() - t0
        if el > budget_s or done >= 16:
            break
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return {"value": done / el, "unit": "frames/s", "cores": cores, "kind": "oracle",
            "sample": f"{done} of the {w.frames.shape[0]} frames ({w.frames.shape[1]}x{w.frames.shape[2]}), "
                      f"float64 forward + float32 decode, {el:.1f} s"}


def serving_pool(dev, seed=6):
    """Distinct sCMOS astigmatic frames for the serving stream, simulated on the device by the
    library's frame simulator (2 emitters/um^2, per-pixel gain/offset maps) and kept in pinned
    host memory: 2T frames per request size (T = 100, 50, 20 for 512^2, 1024^2, 2048^2)."""
    import numpy as np
    import torch

    import paper_2410_02314_gb300 as sml
    from paper_2410_02314_gb300 import synth

    rng = np.random.default_rng(seed)
    pool = {}
    for T, S in ((100, 512), (50, 1024), (20, 2048)):
        cam = synth.scmos_camera(rng, S, S)
        d_gain, d_off = torch.from_numpy(cam.gain_map).to(dev), torch.from_numpy(cam.offset_map).to(dev)
        em = synth.emitters_density(rng, 2 * T, S, S, 2.0, astig=True)
        d_adu = sml.sml_sim_frames(em, 2 * T, S, S, astig=True, gain_map=d_gain, offset_map=d_off, seed=seed + S)
        torch.cuda.synchronize()
        host = d_adu.cpu().pin_memory()  # int16 tensor holding the uint16 ADU bits
        pool[S] = (T, host, cam, d_gain, d_off)
        del d_adu
    torch.cuda.empty_cache()
    return pool


def serving_run(spec_json, blob, dev, capacity_px_per_s, pool, load=0.8, n_requests=200, slots=3):
    """Mixed stacks 100x512^2, 50x1024^2, 20x2048^2 uint16 (3:2:1), Poisson arrivals at
    `load` x the measured pixel capacity; continuous batching over `slots` contexts whose
    workspaces for the three sizes are created before the timed stream.  Each request's
    frames are a window of T consecutive frames at a random start in its size's pool of 2T
    distinct simulated frames.  The HBM budget is the device's free memory at the start plus
    what the slots hold, minus a 4 GiB reserve."""
    import numpy as np
    import torch

    from paper_2410_02314_gb300 import serve

    rng = np.random.default_rng(int(load * 1000))
    kinds = rng.choice([512, 1024, 2048], size=n_requests, p=[0.5, 1 / 3, 1 / 6])
    mean_px = np.mean([pool[int(k)][0] * int(k) * int(k) for k in kinds])
    rate = load * capacity_px_per_s / mean_px
    arrivals = serve.poisson_arrivals(n_requests, rate, rng)
    reqs = []
    for k, (kind, t) in enumerate(zip(kinds, arrivals)):
        T, host, cam, d_gain, d_off = pool[int(kind)]
        o = int(rng.integers(0, T + 1))
        reqs.append(serve.Request(rid=k, frames=host[o : o + T], arrival=float(t), gain=cam.gain, offset=cam.offset,
                                  gain_map=d_gain, offset_map=d_off))
    ex = serve.GpuExecutor(spec_json, blob, slots=slots, device=dev.index or 0)
    ex.warm([(100, 512, 512), (50, 1024, 1024), (20, 2048, 2048)], max_request=(20, 2048, 2048))
    sch = serve.Scheduler(ex, reserve=4 << 30)
    rep = serve.report(sch.run(reqs))
    rep.update({"load": load, "arrival_rate_per_s": rate, "slots": slots, "max_queue": sch.max_queue,
                "hbm_budget_bytes": sch.budget, "resident_bytes": ex.resident_bytes(),
                "peak_accounted_bytes": sch.peak_in_use,
                "mix": "100x512^2 : 50x1024^2 : 20x2048^2 = 3:2:1, sCMOS astigmatic, distinct frames per request"})
    for loc in ex.locs:
        loc.close()
    return rep


LFOV_FRAMES, LFOV_HW = 1000, 2048


def large_fov_frames(dev, frames=LFOV_FRAMES, sim_batch=16, seed=4):
    """The large field-of-view stack: `frames` distinct 2048x2048 sCMOS frames (per-pixel gain
    N(2,0.1) and offset N(100,5) maps resident on the device, 2 emitters/um^2, astigmatic PSF
    with z ~ U(-600,600) nm, Poisson noise), simulated on the device by the library's frame
    simulator in batches of `sim_batch` frames.  Returns (device int16 [T,H,W] holding the
    uint16 ADU bits, camera, device gain map, device offset map, emitters per frame,
    simulated frames/s)."""
    import numpy as np
    import torch

    import paper_2410_02314_gb300 as sml
    from paper_2410_02314_gb300 import synth

    H = W = LFOV_HW
    rng = np.random.default_rng(seed)
    cam = synth.scmos_camera(rng, H, W)
    d_gain, d_off = torch.from_numpy(cam.gain_map).to(dev), torch.from_numpy(cam.offset_map).to(dev)
    d_frames = torch.empty((frames, H, W), dtype=torch.int16, device=dev)
    n_em = 0
    t_sim = time.perf_counter()
    for c in range(0, frames, sim_batch):
        nb = min(sim_batch, frames - c)
        em = synth.emitters_density(rng, nb, H, W, 2.0, astig=True)
        n_em += em.x.size
        sml.sml_sim_frames(em, nb, H, W, astig=True, gain_map=d_gain, offset_map=d_off, seed=seed, frame0=c,
                           d_adu=d_frames[c : c + nb])
    torch.cuda.synchronize()
    return d_frames, cam, d_gain, d_off, n_em / frames, frames / (time.perf_counter() - t_sim)


def large_fov_cpu_baseline(net, frame, cam, budget_s=10.0, block=256):
    """The oracle (float64 forward + float32 decode) on blocks of `block` x `block` pixels of
    one 2048x2048 frame, each computed with its receptive-field halo (forward_window), as
    many as fit the time budget; frames/s extrapolated per pixel to whole frames."""
    import numpy as np

    import oracle

    H, W = frame.shape
    done_px, nblk, t0 = 0, 0, time.perf_counter()
    rng = np.random.default_rng(0)
    while True:
        i0, j0 = (int(v) * block for v in rng.integers(0, H // block, 2))
        hd = oracle.forward_window(net, frame[None], i0, i0 + block, j0, j0 + block, cam.gain, cam.offset,
                                   cam.gain_map.astype(np.float64), cam.offset_map.astype(np.float64))
        oracle.decode(oracle.maps_f32(hd), P_MIN, net.z_scale, net.ph_scale)
        done_px += block * block
        nblk += 1
        el = time.perf_counter() - t0
        if el > budget_s:
            break
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return {"value": done_px / el / (H * W), "unit": "frames/s", "cores": cores, "kind": "oracle",
            "sample": f"{nblk} blocks of {block}x{block} px of one {H}x{W} frame (each with its {net.R}-px receptive "
                      f"halo), float64 forward + float32 decode, {el:.1f} s; extrapolated per pixel to whole frames"}


def large_fov_line(dev, stream, flush, prec, lf, steps, warmup, pk, live, with_e2e=True, with_cpu=True):
    """The large field-of-view configuration as a bench line: the 1000-frame 2048x2048 stack
    (resident in HBM) through the 48-channel 8-layer net in `prec` (bf16 or fp8), one step =
    one sml_localize_async call over all frames (the library runs chunks of 4 frames);
    L2 flushed between steps.  Adds the middle-layer conv roofline, the end-to-end rate
    through sml_localize with pinned host frames and records, the oracle's extrapolated
    rate and the clocks."""
    import torch

    import oracle
    import paper_2410_02314_gb300 as sml
    from paper_2410_02314_gb300 import synth

    d_frames, cam, d_gain, d_off, em_per_frame, sim_fps = lf
    T, H, W = (int(x) for x in d_frames.shape)
    spec = synth.spec_48("bf16")
    blob = synth.pack_blob(spec, synth.init_weights(spec, 1004))
    camk = {"gain": cam.gain, "offset": cam.offset, "gain_map": d_gain, "offset_map": d_off}
    js = spec.to_json()
    if prec == "fp8":  # activation scales from a bf16 calibration pass over the first 4 frames
        js = sml.calibrate_fp8(js, blob, d_frames[:4], **camk)
    loc = sml.Localizer(js, blob)
    cap = T * 300000  # random-init nets detect about 170-230 k local maxima per frame
    d_out = torch.empty(cap * 24, dtype=torch.uint8, device=dev)
    d_n = torch.zeros(1, dtype=torch.int64, device=dev)
    for _ in range(max(1, warmup)):
        loc.localize_async(d_frames, P_MIN, d_out, d_n, stream=stream, **camk)
    torch.cuda.synchronize()
    launches = loc.last_launch_count
    clk = ClockSampler(dev.index or 0)
    clk.start()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    sml.sml_profile_enable(loc.ctx, True)
    clk.mark_begin()
    for a, b in ev:
        flush.zero_()
        a.record(stream)
        loc.localize_async(d_frames, P_MIN, d_out, d_n, stream=stream, **camk)
        b.record(stream)
    torch.cuda.synchronize()
    clk.mark_end()
    clocks = clk.stop()
    sml.sml_profile_enable(loc.ctx, False)
    ms = statistics.mean(a.elapsed_time(b) for a, b in ev)
    conv_ms, conv_n = sml.sml_profile_read(loc.ctx, sml.SML_KERNEL_CONV)
    n_rec = int(d_n.item())
    px_per_launch = 4 * H * W
    res = {"metric": "frames/s", "value": T / (ms / 1000), "unit": "frames/s", "steps": steps, "warmup": warmup,
           "ms_per_step": ms, "dtype": prec,
           "config": {"workload": f"large_fov_{T}x{H}x{W}_scmos_astig_48ch_8layer", "frames_per_step": T,
                      "frames": f"{T} distinct frames simulated on the device (astigmatic, 2 emitters/um^2, "
                                f"per-pixel gain/offset maps), {em_per_frame:.0f} emitters per frame",
                      "chunk": "4 frames (16,777,216 px) per launch", "l2": "flushed between steps (512 MB write)"},
           "mpix_per_s": T * H * W / (ms / 1000) / 1e6, "records_per_frame": n_rec / T,
           "gpu_launches": launches * steps, "simulated_frames_per_s": sim_fps,
           "roofline": conv_roofline(spec, prec, px_per_launch, conv_ms, conv_n, pk, live,
                                     profiled_traffic(prec, "large_fov")),
           "clocks": clocks}
    if with_e2e:
        host_frames = d_frames.cpu().pin_memory()
        host_out = torch.empty(cap * 24, dtype=torch.uint8).pin_memory()
        e2e_t = []
        for k in range(3):
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            recs = sml.sml_localize(loc.ctx, host_frames, P_MIN, out=host_out, **camk)
            if k:
                e2e_t.append(time.perf_counter() - t0)
        e2e_s = statistics.mean(e2e_t)
        res["e2e"] = {"value": T / e2e_s, "unit": "frames/s", "h2d_bytes_per_step": int(host_frames.numel() * 2),
                      "d2h_bytes_per_step": int(recs.numel() + 8), "steps": len(e2e_t)}
        del host_frames, host_out
    if with_cpu:
        net = oracle.Net(js, blob)
        frame0 = d_frames[0].cpu().numpy().view("uint16")
        res["cpu_baseline"] = large_fov_cpu_baseline(net, frame0, cam)
    loc.close()
    return res


def small_latency_run(dev, stream, calls=50):
    """The small configuration (4 frames of 64x64, 32-channel 6-layer FP32 net): device time
    per call and launches per call (latency-bound: no roofline)."""
    import torch

    import paper_2410_02314_gb300 as sml
    from paper_2410_02314_gb300 import synth

    w = synth.workload_small(precision="fp32")
    loc = sml.Localizer(w.spec.to_json(), w.blob)
    d_frames = torch.from_numpy(w.frames).to(dev)
    d_out = torch.empty(4 * 64 * 64 * 24, dtype=torch.uint8, device=dev)
    d_n = torch.zeros(1, dtype=torch.int64, device=dev)
    for _ in range(5):
        loc.localize_async(d_frames, P_MIN, d_out, d_n, stream=stream, gain=w.cam.gain, offset=w.cam.offset)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(calls)]
    for a, b in ev:
        a.record(stream)
        loc.localize_async(d_frames, P_MIN, d_out, d_n, stream=stream, gain=w.cam.gain, offset=w.cam.offset)
        b.record(stream)
    torch.cuda.synchronize()
    us = statistics.median(a.elapsed_time(b) for a, b in ev) * 1000
    res = {"workload": "4 x 64x64 frames, 32-channel 6-layer net, FP32", "us_per_call": us,
           "launches_per_call": loc.last_launch_count, "records_per_call": int(d_n.item())}
    loc.close()
    return res


def training_run(dev, steps=20, warmup=3, fp32=True):
    """The training configuration: the 48-channel 8-layer net on batches of 256 astigmatic
    64x64 patches (0-10 emitters each), Adam on FP32 master weights; one step = forward, loss,
    backward and the optimizer update.  BF16 (tensor-core forward, input gradient and weight
    gradient) and FP32 (SIMT) on the same device-simulated batches (a fresh batch per step,
    simulated before the timed region).  Device time per step with CUDA events."""
    import numpy as np
    import torch

    from paper_2410_02314_gb300 import synth
    from paper_2410_02314_gb300.train import DilatedLocNet, device_batch

    spec = synth.spec_48("fp32")
    rng = np.random.default_rng(5)
    batches = [device_batch(rng, 256, 64, 64, max_emitters=10, frame0=k * 256) for k in range(warmup + steps)]
    res = {"workload": "256 patches of 64x64 per step (astigmatic, 0-10 emitters), 48-channel 8-layer net, Adam",
           "batches": "simulated on the device before the timed region, one per step"}
    for prec in ("bf16", "fp32") if fp32 else ("bf16",):
        net = DilatedLocNet(spec, synth.init_weights(spec, 11), precision=prec).to(dev)
        opt = torch.optim.Adam(net.parameters(), lr=1e-3)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for k, (frames, tgt) in enumerate(batches):
            a = b = None
            if k >= warmup:
                a, b = ev[k - warmup]
                a.record()
            opt.zero_grad(set_to_none=True)
            loss = net.loss(frames, tgt)
            loss.backward()
            opt.step()
            if b is not None:
                b.record()
        torch.cuda.synchronize()
        ms = statistics.mean(x.elapsed_time(y) for x, y in ev)
        res[f"{prec}_steps_per_s"] = 1000.0 / ms
        res[f"{prec}_ms_per_step"] = ms
        res[f"{prec}_final_loss"] = float(loss.item())
        if prec == "bf16":
            res["bf16_device_error"] = net.device_error()
    if fp32:
        res["bf16_speedup_vs_fp32"] = res["bf16_steps_per_s"] / res["fp32_steps_per_s"]
    # the BF16 step captured once in a CUDA graph and replayed (one host launch per step)
    try:
        from paper_2410_02314_gb300.train import GraphedStep

        net = DilatedLocNet(spec, synth.init_weights(spec, 11), precision="bf16").to(dev)
        gstep = GraphedStep(net, (256, 64, 64), lr=1e-3)
        for frames, tgt in batches[:warmup]:
            gstep(frames, tgt)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for (frames, tgt), (a, b) in zip(batches[warmup:], ev):
            a.record()
            loss = gstep(frames, tgt)
            b.record()
        torch.cuda.synchronize()
        ms = statistics.mean(x.elapsed_time(y) for x, y in ev)
        res.update({"bf16_graph_steps_per_s": 1000.0 / ms, "bf16_graph_ms_per_step": ms,
                    "bf16_graph_final_loss": float(loss.item()), "bf16_graph_device_error": net.device_error()})
    except Exception as e:  # reported, not hidden: the eager numbers above stand
        res["bf16_graph_error"] = repr(e)[:300]
    return res


TOPOLOGIES = {
    "dcd": ("dcd_{T}x{H}x{W}_32ch_g16_4x4dense_22layer", "workload_dcd"),
    "dilatedloc": ("dilatedloc_{T}x{H}x{W}_32ch_g16_4x4dense_unet2_9heads_26layer", "workload_dilatedloc"),
}


def topology_run(dev, stream, flush, which, reps=5):
    """The paper's topology beyond the plain stack: the 256 frames of 256x256 of the main
    workload through the 22-layer dense-block net ("dcd": 32 channels, growth 16, four blocks
    of dilations 2, 4, 8, 16 with transitions; Sec. 3.2.1) or the full topology ("dilatedloc":
    those blocks, a two-level U-Net and the nine heads with uncertainties; Sec. 3.2), BF16, FP8
    (scales from the library's calibration over the first 16 frames) and FP32.  The conv-class kernels (dense layers, transitions, U-Net convs, pools and upsamples)
    are timed with the library's event pairs; their algorithmic HBM bytes are one read of
    every input channel and one write of every output channel per pixel of their level."""
    import torch

    import paper_2410_02314_gb300 as sml
    from paper_2410_02314_gb300 import synth

    name, maker = TOPOLOGIES[which]
    res = {"workload": name.format(T=T_FRAMES, H=H, W=W), "l2": "flushed between calls"}
    pk, pk_kind = peaks()
    for prec in ("bf16", "fp8", "fp32"):
        w = getattr(synth, maker)(T=T_FRAMES, H=H, W=W, precision="bf16" if prec == "fp8" else prec)
        d_frames = torch.from_numpy(w.frames).to(dev)
        js = w.spec.to_json()
        if prec == "fp8":
            js = sml.calibrate_fp8(js, w.blob, d_frames[:16], gain=w.cam.gain, offset=w.cam.offset)
        loc = sml.Localizer(js, w.blob)
        d_out = torch.empty(T_FRAMES * H * W // 4 * 24, dtype=torch.uint8, device=dev)
        d_n = torch.zeros(1, dtype=torch.int64, device=dev)
        for _ in range(3):
            loc.localize_async(d_frames, P_MIN, d_out, d_n, stream=stream)
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
        sml.sml_profile_enable(loc.ctx, True)
        for a, b in ev:
            flush.zero_()
            a.record(stream)
            loc.localize_async(d_frames, P_MIN, d_out, d_n, stream=stream)
            b.record(stream)
        torch.cuda.synchronize()
        sml.sml_profile_enable(loc.ctx, False)
        ms = statistics.mean(a.elapsed_time(b) for a, b in ev)
        conv_ms, conv_n = sml.sml_profile_read(loc.ctx, sml.SML_KERNEL_CONV)
        res[f"{prec}_frames_per_s"] = T_FRAMES / (ms / 1000)
        res[f"{prec}_launches_per_call"] = loc.last_launch_count
        if prec == "bf16":
            flops, nbytes, _ = conv_class_work(w.spec, T_FRAMES * H * W, 2)
            conv_s = conv_ms / reps / 1000.0
            res.update({"bf16_conv_ms_per_call": conv_ms / reps, "bf16_records_per_call": int(d_n.item()),
                        "conv_algorithmic_bytes_per_call": nbytes, "conv_hbm_gbs": nbytes / conv_s / 1e9,
                        "conv_hbm_frac": nbytes / conv_s / 1e9 / pk["hbm_gbs"],
                        "conv_tflops": flops / conv_s / 1e12, "peak_kind": pk_kind})
        elif prec == "fp8":
            _, nbytes8, _ = conv_class_work(w.spec, T_FRAMES * H * W, 1)
            conv_s = conv_ms / reps / 1000.0
            res.update({"fp8_conv_ms_per_call": conv_ms / reps, "fp8_records_per_call": int(d_n.item()),
                        "fp8_conv_algorithmic_bytes_per_call": nbytes8, "fp8_conv_hbm_gbs": nbytes8 / conv_s / 1e9})
        loc.close()
    return res


def file_pipeline_run(spec_json, blob, frames, cam, batch=256, repeat=4):
    """Stack-file pipeline (reader thread -> pinned buffers -> H2D -> localize -> D2H records,
    overlapped): the batch's frames written `repeat` times to one raw file in a temporary
    directory (so the reads come from the page cache, not the disk), localized in batches."""
    import tempfile

    import numpy as np

    import paper_2410_02314_gb300 as sml

    T, H, W = frames.shape
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "stack.raw")
        with open(path, "wb") as f:
            for _ in range(repeat):
                f.write(np.ascontiguousarray(frames, dtype="<u2").tobytes())
        loc = sml.Localizer(spec_json, blob)
        loc.localize_file(path, T, H, W, P_MIN, batch=batch, gain=cam.gain, offset=cam.offset)  # warm-up
        recs, st = loc.localize_file(path, T * repeat, H, W, P_MIN, batch=batch, gain=cam.gain, offset=cam.offset)
        loc.close()
    return {"workload": f"{T * repeat} frames of {H}x{W} from a raw stack file (page cache), batches of {batch}",
            "frames_per_s": st["frames"] / st["wall_seconds"], "read_mb_per_s": st["bytes_read"] / st["read_seconds"] / 1e6,
            "wall_s": st["wall_seconds"], "records": int(len(recs))}


def run_reference(args):
    """Reference arm: the CPU oracle, timed on bounded samples of the same workload."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from paper_2410_02314_gb300 import synth
    import oracle

    w = synth.workload_batched(T=T_FRAMES, H=H, W=W, precision=args.precision)
    net = oracle.Net(w.spec.to_json(), w.blob)
    frames_per_step = 1
    for k in range(args.warmup):
        oracle.localize(net, w.frames[k % T_FRAMES : k % T_FRAMES + 1], P_MIN)
    times = []
    for k in range(args.steps):
        t0 = time.perf_counter()
        oracle.localize(net, w.frames[k % T_FRAMES : k % T_FRAMES + 1], P_MIN)
        times.append(time.perf_counter() - t0)
    ms = 1000 * statistics.mean(times)
    val = frames_per_step / (ms / 1000)
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    line = {"impl": "reference", "metric": "frames/s", "value": val, "unit": "frames/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"batched_{T_FRAMES}x{H}x{W}_48ch_8layer", "frames_per_step": frames_per_step,
                       "note": "CPU oracle, one whole frame per step"},
            "cpu_baseline": {"value": val, "unit": "frames/s", "cores": cores, "kind": "oracle",
                             "sample": f"{frames_per_step} frame per step, {args.steps} steps"},
            "e2e": {"value": val, "unit": "frames/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    global T_FRAMES
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--precision", default="bf16", choices=["bf16", "fp32", "fp8"])
    ap.add_argument("--frames", type=int, default=T_FRAMES,
                    help="frames per step (default 256; smaller stacks for profiler captures)")
    ap.add_argument("--workload", default="batched", choices=["batched", "dcd", "dilatedloc", "large_fov", "training"],
                    help="batched: the 48-channel 8-layer net; dcd: the 22-layer dense-block net; dilatedloc: the "
                         "full topology (dense blocks, U-Net, uncertainty heads); "
                         "large_fov: 1000 distinct 2048x2048 sCMOS frames, bf16 or fp8, one GPU; training: "
                         "BF16 and FP32 training steps (256 patches of 64x64), one GPU")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--chunk-px", type=int, default=0)
    ap.add_argument("--tc-stages", type=int, default=0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp32", action="store_true")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--no-extra", action="store_true", help="skip the large-FOV and small-config measurements")
    ap.add_argument("--no-peaks", action="store_true",
                    help="skip the FP8/FP32 peak measurement (profiler captures: its GEMMs would join the launch list)")
    args = ap.parse_args()
    T_FRAMES = args.frames
    if args.impl == "reference":
        run_reference(args)
        return

    import numpy as np
    import torch

    import __graft_entry__
    import paper_2410_02314_gb300 as sml
    from paper_2410_02314_gb300 import replicas, synth

    ri = replicas.rank_info()
    rank, world, local = ri.rank, ri.world, ri.local
    if rank == 0:
        __graft_entry__.build()
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", init_method="env://")
        dist.barrier()
        __graft_entry__.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    if args.workload == "training":
        if world > 1:
            raise SystemExit("the training line runs on one GPU")
        tr = training_run(dev, steps=args.steps, warmup=max(3, args.warmup), fp32=not args.no_fp32)
        line = {"metric": "training steps/s", "value": tr["bf16_steps_per_s"], "unit": "steps/s", "n_gpus": 1,
                "steps": args.steps, "warmup": max(3, args.warmup), "ms_per_step": tr["bf16_ms_per_step"],
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
                "config": {"workload": "training_256x64x64_48ch_8layer", "parallelism": "replicas1"}, "training": tr}
        print(json.dumps(line), flush=True)
        return
    if args.workload == "large_fov":
        if world > 1 or args.precision == "fp32":
            raise SystemExit("the large field-of-view line runs on one GPU in bf16 or fp8")
        flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device=dev)  # > L2 (129 MB)
        lf = large_fov_frames(dev)
        live = measure_peaks(dev)
        line = large_fov_line(dev, torch.cuda.current_stream(), flush, args.precision, lf, args.steps, args.warmup,
                              peaks()[0], live, with_cpu=not args.no_cpu_baseline)
        line.update({"n_gpus": 1, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                     "data": "synthetic", "peaks_measured": live})
        line["config"]["parallelism"] = "replicas1"
        print(json.dumps(line), flush=True)
        return

    def workload(prec, d_frames=None):
        make = {"batched": synth.workload_batched, "dcd": synth.workload_dcd,
                "dilatedloc": synth.workload_dilatedloc}[args.workload]
        w = make(T=T_FRAMES, H=H, W=W, precision="bf16" if prec == "fp8" else prec, seed=replicas.frame_seed(3, rank))
        spec = json.loads(w.spec.to_json())
        if args.chunk_px:
            spec["chunk_px"] = args.chunk_px
        if args.tc_stages:
            spec["tc_stages"] = args.tc_stages
        js = json.dumps(spec)
        if prec == "fp8":  # per-layer activation scales from a bf16 pass over the first 16 frames
            if d_frames is None:
                d_frames = torch.from_numpy(w.frames).to(dev)
            js = sml.calibrate_fp8(js, w.blob, d_frames[:16], gain=w.cam.gain, offset=w.cam.offset)
        return w, js

    w, spec_json = workload(args.precision)
    loc = sml.Localizer(spec_json, w.blob)
    d_frames = torch.from_numpy(w.frames).to(dev)
    cap = T_FRAMES * H * W // 4
    d_out = torch.empty(cap * 24, dtype=torch.uint8, device=dev)
    d_n = torch.zeros(1, dtype=torch.int64, device=dev)
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device=dev)  # > L2 (129 MB)
    stream = torch.cuda.current_stream()

    def step():
        loc.localize_async(d_frames, P_MIN, d_out, d_n, stream=stream)

    def timed(steps, profile=False):
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        if profile:
            sml.sml_profile_enable(loc.ctx, True)
        for a, b in evs:
            flush.zero_()  # L2 flushed between steps, outside the timed events
            a.record(stream)
            step()
            b.record(stream)
        torch.cuda.synchronize()
        if profile:
            sml.sml_profile_enable(loc.ctx, False)
        return [a.elapsed_time(b) for a, b in evs]

    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()
    launches_per_step = loc.last_launch_count
    n_rec = int(d_n.item())

    clk = ClockSampler(local)
    clk.start()

    def timed_marked():
        clk.mark_begin()
        out = timed(args.steps, profile=True)  # ends with a device synchronise
        clk.mark_end()
        return out

    times = replicas.timed_region(timed_marked, dist, torch.cuda.synchronize)
    clocks = clk.stop()
    ms = replicas.max_over_ranks(statistics.mean(times), dist, dev)
    value = replicas.whole_job_rate(T_FRAMES, ms / 1000.0, world)

    live_peaks = {} if args.no_peaks else measure_peaks(dev)  # FP8 and FP32 dense peaks, after the timed region
    # dominant kernel: the middle-layer tensor-core (or FP32) conv, timed on its stream
    conv_ms, conv_n = sml.sml_profile_read(loc.ctx, sml.SML_KERNEL_CONV)
    heads_ms, heads_n = sml.sml_profile_read(loc.ctx, sml.SML_KERNEL_CONV_HEADS)
    l1_ms, l1_n = sml.sml_profile_read(loc.ctx, sml.SML_KERNEL_LAYER1)
    dec_ms, dec_n = sml.sml_profile_read(loc.ctx, sml.SML_KERNEL_DECODE)
    chunk_px = json.loads(spec_json).get("chunk_px", 1 << 24)
    frames_per_chunk = max(1, chunk_px // (H * W))
    px_per_launch = min(frames_per_chunk, T_FRAMES) * H * W
    pk, pk_kind = peaks()
    # the committed ncu figures are for full launches of 256 frames of 256x256 (16,777,216 px)
    traffic = (profiled_traffic(args.precision, {"batched": "batched256", "dcd": "dcd256"}.get(args.workload, ""))
               if px_per_launch == 256 * 256 * 256 else None)
    roofline = conv_roofline(w.spec, args.precision, px_per_launch, conv_ms, conv_n, pk, live_peaks, traffic)
    breakdown = {"layer1_ms": l1_ms / args.steps, "conv_ms": conv_ms / args.steps,
                 "conv_heads_ms": heads_ms / args.steps, "decode_ms": dec_ms / args.steps}

    # end to end through the synchronous C-ABI call with host buffers
    host_frames = torch.from_numpy(w.frames).pin_memory()
    host_out = torch.empty(cap * 24, dtype=torch.uint8).pin_memory()
    def e2e_run():
        out = []
        for k in range(args.warmup + args.steps):
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            r = sml.sml_localize(loc.ctx, host_frames, P_MIN, gain=w.cam.gain, offset=w.cam.offset, out=host_out)
            el = time.perf_counter() - t0
            if k >= args.warmup:
                out.append(el)
        return out, r

    e2e_times, recs = replicas.timed_region(e2e_run, dist, torch.cuda.synchronize)
    e2e_s = replicas.max_over_ranks(statistics.mean(e2e_times), dist, dev)
    e2e = {"value": replicas.whole_job_rate(T_FRAMES, e2e_s, world), "unit": "frames/s", "h2d_bytes_per_step": int(w.frames.nbytes),
           "d2h_bytes_per_step": int(recs.numel() + 8)}

    extra = {}
    others = [] if args.no_fp32 else [p for p in ("fp32", "bf16", "fp8") if p != args.precision]
    for prec in others:  # the same batch at the other precisions, same timing method
        wo, jso = workload(prec, d_frames)
        loco = sml.Localizer(jso, wo.blob)
        for _ in range(2):
            loco.localize_async(d_frames, P_MIN, d_out, d_n, stream=stream)
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(5)]
        for a, b in ev:
            flush.zero_()
            a.record(stream)
            loco.localize_async(d_frames, P_MIN, d_out, d_n, stream=stream)
            b.record(stream)
        torch.cuda.synchronize()
        mso = statistics.mean(a.elapsed_time(b) for a, b in ev)
        extra[f"{prec}_frames_per_s"] = world * T_FRAMES / (mso / 1000)
        loco.close()
    if "fp32_frames_per_s" in extra:
        extra["speedup_vs_fp32"] = value / extra["fp32_frames_per_s"]

    serving = None
    if not args.no_serve and world == 1:  # arrival rates at 0.5, 0.8 and 0.95 of the measured capacity
        pool = serving_pool(dev)
        serving = [serving_run(spec_json, w.blob, dev, value * H * W, pool, load=ld) for ld in (0.5, 0.8, 0.95)]
        del pool
    large_fov = small = file_pipe = dcd = training = None
    if not args.no_extra and world == 1:
        training = training_run(dev)
        lf = large_fov_frames(dev)
        large_fov = {p: large_fov_line(dev, stream, flush, p, lf, 3, 1, pk, live_peaks, with_cpu=(p == "bf16"))
                     for p in ("bf16", "fp8")}
        del lf
        torch.cuda.empty_cache()
        small = small_latency_run(dev, stream)
        file_pipe = file_pipeline_run(spec_json, w.blob, w.frames, w.cam)
        dcd = ({k: topology_run(dev, stream, flush, k) for k in TOPOLOGIES} if args.workload == "batched" else None)

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    cpu = None
    if not args.no_cpu_baseline and world == 1:
        cpu = cpu_baseline(w)
    line = {
        "metric": "frames/s",
        "value": value,
        "unit": "frames/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": args.precision,
        "data": "synthetic",
        "config": {"workload": f"batched_{T_FRAMES}x{H}x{W}_48ch_8layer" if args.workload == "batched"
                   else TOPOLOGIES[args.workload][0].format(T=T_FRAMES, H=H, W=W), "frames_per_step": T_FRAMES,
                   "precision": args.precision, "chunk_px": chunk_px, "tc_stages": args.tc_stages or "max",
                   "l2": "flushed between steps (512 MB write)",
                   "parallelism": f"replicas{world}"},
        "mpix_per_s": value * H * W / 1e6,
        "records_per_step": n_rec,
        "gpu_launches": launches_per_step * args.steps,
        "e2e": e2e,
        "roofline": roofline,
        "peaks_measured": live_peaks,
        "kernel_ms_per_step": breakdown,
        "cpu_baseline": cpu,
        "clocks": clocks,
        "serving": serving,
        "large_fov": large_fov,
        "small_latency": small,
        "file_pipeline": file_pipe,
        "topologies": dcd,
        "training": training,
        **extra,
    }
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
