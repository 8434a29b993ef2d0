"""BF16 map tolerance against network depth, set from a measurement.

tests/measure_depth_error.py measured, on a GB300, the normalised map error of plain
48-channel dilated stacks with n = 7, 14, 21 and 28 tensor-core layers (12 weight seeds each,
two 256x256 frames of the batched workload), against the oracle's float64 forward and its
bf16 mode.  Worst seed per depth:

    n     vs float64 (max)   vs bf16 mode (max)   vs bf16 mode (RMS)
    7     0.0199             0.0119               0.0018
    14    0.0439             0.0356               0.0070
    21    0.0621             0.0483               0.0091
    28    0.0817             0.0785               0.0138

The error grows about linearly with n, not as sqrt(n): each layer adds its own rounding
(bf16 stores, and rounding-boundary flips against the bf16 mode), and the following layers
carry the earlier errors forward with gain near 1.  A least-squares line through the origin
on the worst seeds gives the slopes below (per tensor-core layer); the gate is 1.5 x the
line, and never below the gates of the 7-layer benchmark net (whose tests keep them).
FP32 (SIMT) stays within 1.1e-5 at every depth measured: its gate is 1e-4 at any depth."""

SLOPE = {"f64_max": 0.002956, "q_max": 0.002581, "q_rms": 0.000468}
BASE = {"f64_max": 3e-2, "q_max": 2e-2, "q_rms": 2e-3}
MARGIN = 1.5


def bf16_gate(n_tc: int, kind: str) -> float:
    """Gate on the normalised map error of a BF16 net with n_tc tensor-core layers: kind
    "f64_max" (max vs float64), "q_max" / "q_rms" (max / RMS vs the oracle's bf16 mode)."""
    return max(BASE[kind], MARGIN * SLOPE[kind] * n_tc)


# FP8 e4m3 over whole frames.  tests/measure_fp8_error.py measured, on a GB300, the 48-channel
# 8-layer net in FP8 (the oracle's activation scales) on whole frames: 256x256 frames of the
# batched workload (8 weight seeds, two frames each) and 2048x2048 sCMOS frames of the large
# field-of-view workload (2 weight seeds), every pixel of every map.  Worst over all frames:
#   vs the oracle's fp8 mode:  max 0.133, RMS 0.0082, 99.99th percentile 0.088
#   vs float64:                max 0.364, RMS 0.068,  99.99th percentile 0.286
# The FP8 gates of the sampled-block tests (max 0.1 vs the fp8 mode, 0.4 vs float64) were set
# on a few thousand sampled pixels; the maximum over the 65 536 to 4 194 304 pixels of a whole
# frame reaches further into the tail of the rounding-flip distribution (one e4m3 ulp is
# 6-12 % of a value), so whole-frame comparisons take these gates, 1.5 x the measured worst
# (RMS vs the fp8 mode keeps its 0.02, 2.4 x the measured worst).
FP8_FRAME = {"q_max": 0.2, "q_rms": 0.02, "f64_max": 0.55, "f64_rms": 0.1}
