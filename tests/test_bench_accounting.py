"""The work accounting behind bench.py's roofline figures, against per-pixel counts made by
hand from each net's layer plan (a 3x3 conv from ci to co channels is 2*9*ci*co FLOP per
pixel of its level and reads ci, writes co channels there)."""
import importlib.util
import os

import pytest

from paper_2410_02314_gb300 import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_module", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


PX = 256 * 256 * 256  # one chunk of the batched workload


def test_plain_48_channel_net(bench):
    # middle layers 2..7 of the 8-layer net: 6 convs 48 -> 48
    flops, nbytes, launches = bench.conv_class_work(synth.spec_48(), PX, 2)
    assert launches == 6
    assert flops == 6 * 41472 * PX  # 2*9*48*48
    assert nbytes == 6 * 192 * PX  # (48 + 48) channels x 2 bytes
    assert bench.conv_class_work(synth.spec_48(), PX, 1)[1] == 6 * 96 * PX  # e4m3
    # whole step: layer 1 (1 -> 48), 7 convs 48 -> 48, heads 48 -> 5
    assert bench.algorithmic_flops_per_px(synth.spec_48()) == 291648


def test_dense_block_net(bench):
    # per block: dense layers 32/48/64/80 -> 16 and a transition 96 -> 32; four blocks
    flops, nbytes, launches = bench.conv_class_work(synth.spec_dcd(), PX, 2)
    assert launches == 20
    assert flops == 4 * (18 * 16 * (32 + 48 + 64 + 80) + 18 * 96 * 32) * PX  # 479 232 per px
    assert nbytes == 4 * ((48 + 64 + 80 + 96) + (96 + 32)) * 2 * PX  # 3 328 B per px
    assert nbytes == 55834574848
    # e4m3 activations: one byte per channel, the same FLOPs
    f8, b8, l8 = bench.conv_class_work(synth.spec_dcd(), PX, 1)
    assert (f8, b8, l8) == (flops, nbytes // 2, launches)


def test_full_topology_adds_the_unet_stage(bench):
    # level 1 (px/4): down conv 32 -> 32; at full resolution: up conv 64 -> 32; pool reads 32
    # at full and writes 32 at px/4, upsample the reverse.  Level 2 likewise at px/16 and px/4.
    _, dcd_bytes, dcd_launches = bench.conv_class_work(synth.spec_dcd(), PX, 2)
    flops, nbytes, launches = bench.conv_class_work(synth.spec_dilatedloc(), PX, 2)
    assert launches == dcd_launches + 8
    lv1 = 64 / 4 + 96 + 64 * (1 / 4 + 1)
    lv2 = 64 / 16 + 96 / 4 + 64 * (1 / 16 + 1 / 4)
    assert lv1 + lv2 == 240
    assert nbytes == dcd_bytes + 240 * 2 * PX  # 3 808 B per px
    unet_flops = 18 * 32 * 32 * (1 / 4 + 1 / 16) + 18 * 64 * 32 * (1 + 1 / 4)
    dcd_flops = bench.conv_class_work(synth.spec_dcd(), PX, 2)[0]
    assert flops == pytest.approx(dcd_flops + unet_flops * PX, rel=1e-12)


def test_conv_roofline_is_the_tensor_pipe(bench):
    """The conv's roofline is the tensor pipe (a dense contraction; the ALU pipes in FP32):
    achieved = 41 472 FLOP per pixel x the launch's pixels / the mean launch time, against the
    burst peak of the launch's operand type; the HBM figures ride along."""
    pk = {"hbm_gbs": 6787.9, "bf16_tflops": 1936.3, "bf16_tflops_sustained": 1724.3, "when": "x"}
    live = {"fp8_tflops": 3510.0, "fp32_tflops": 69.5}
    # 120 launches summing 74.82 ms: 0.6235 ms each
    r = bench.conv_roofline(synth.spec_48(), "bf16", PX, 74.82, 120, pk, live, 3.33e9)
    assert r["bound"] == "tensor" and r["unit"] == "TFLOP/s" and r["peak"] == 1936.3
    assert r["achieved"] == pytest.approx(41472 * PX / 0.6235e-3 / 1e12, rel=1e-9)
    assert r["frac"] == pytest.approx(r["achieved"] / 1936.3, rel=1e-12)
    assert 0.57 < r["frac"] < 0.60  # 1 116 TFLOP/s
    assert r["hbm"]["bytes_per_launch"] == 192 * PX
    assert r["hbm"]["dram_gbs"] == pytest.approx(3.33e9 / 0.6235e-3 / 1e9, rel=1e-9)
    r8 = bench.conv_roofline(synth.spec_48(), "fp8", PX, 60.0, 120, pk, live, None)
    assert r8["bound"] == "tensor" and r8["peak"] == 3510.0 and r8["hbm"]["bytes_per_launch"] == 96 * PX
    r8b = bench.conv_roofline(synth.spec_48(), "fp8", PX, 60.0, 120, pk, {}, None)
    assert r8b["peak"] == 2 * 1936.3  # no FP8 measurement: the nominal ratio, stated
    r32 = bench.conv_roofline(synth.spec_48(), "fp32", PX, 600.0, 6, pk, live, None)
    assert r32["bound"] == "alu" and r32["peak"] == 69.5


def _smi_line(ts, sm, reasons=("Not Active",) * 4):
    # timestamp, index, clocks.sm, clocks.max.sm, power.draw, active mask, four reasons
    return ", ".join([ts, "0", str(sm), "2070", "900.5", "0x0000000000000000", *reasons])


def test_clock_samples_inside_the_timed_region(bench):
    import datetime

    lines = [_smi_line("2026/12/04 01:53:02.000", 1400),  # idle, before the region
             _smi_line("2026/12/04 01:53:02.150", 2070),
             _smi_line("2026/12/04 01:53:02.200", 2070, ("Not Active", "Not Active", "Not Active", "Active")),
             _smi_line("2026/12/04 01:53:02.250", 2055),
             _smi_line("2026/12/04 01:53:02.400", 1100)]  # after the region
    t = lambda s: datetime.datetime(2026, 12, 4, 1, 53, 2, int(s * 1e6))
    got = bench.parse_clock_samples(lines, t(0.1), t(0.3))
    assert got == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "samples": 3, "window": "timed region",
                   "reasons": ["sw_power_cap"]}


def test_clock_samples_fall_back_to_all_when_none_is_inside(bench):
    import datetime

    lines = [_smi_line("2026/12/04 01:53:02.000", 2070), "garbage", _smi_line("not a time", 2070,
                                                                               ("Active",) + ("Not Active",) * 3)]
    t = lambda s: datetime.datetime(2026, 12, 4, 1, 53, 2, int(s * 1e6))
    got = bench.parse_clock_samples(lines, t(0.5), t(0.6))
    assert got["samples"] == 2 and got["window"] == "around the timed region"
    assert got["reasons"] == ["hw_slowdown"]
    assert bench.parse_clock_samples([], None, None) is None


def test_clock_sampler_with_a_stand_in_nvidia_smi(bench, tmp_path, monkeypatch):
    """The sampler's process handling end to end, with a shell script in place of nvidia-smi
    that prints one timestamped sample every 50 ms: it starts before the region, the region's
    samples are kept, and stop() ends the sampling process."""
    import time

    fake = tmp_path / "nvidia-smi"
    fake.write_text("#!/bin/sh\nwhile true; do\n"
                    "  echo \"$(date +'%Y/%m/%d %H:%M:%S.%3N'), 0, 2070, 2070, 850.0, 0x0, Not Active, Not Active, "
                    "Not Active, Not Active\"\n  sleep 0.05\ndone\n")
    fake.chmod(0o755)
    monkeypatch.setenv("PATH", f"{tmp_path}:{os.environ['PATH']}")
    clk = bench.ClockSampler(0)
    clk.start()
    assert clk.proc is not None and os.path.getsize(clk.path) > 0  # sampling is live before the region
    clk.mark_begin()
    time.sleep(0.4)
    clk.mark_end()
    got = clk.stop()
    assert clk.proc.poll() is not None
    assert got["window"] == "timed region" and 3 <= got["samples"] <= 12
    assert got["sm_mhz"] == 2070.0 and got["reasons"] == []
