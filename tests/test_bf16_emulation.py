"""The BF16 training emulation (tests/bf16_emulation.py) is pinned to the oracle: without its
bf16 roundings it must give the oracle's exact float64 loss and gradient (which are pinned to
central finite differences, tests/test_oracle_grad.py), so a dropped term, a wrong tap mirror
or a misplaced mask in its backward would show here, on the CPU."""
import numpy as np
import pytest

import oracle
from bf16_emulation import bf16_emulation
from paper_2410_02314_gb300 import synth


@pytest.mark.parametrize("C,dil,B,H,W", [(16, (1, 2, 4), 2, 14, 17), (16, (3, 1, 2, 1), 2, 12, 20)])
def test_emulation_without_rounding_is_the_exact_gradient(C, dil, B, H, W):
    spec = synth.NetSpec(in_ch=1, channels=C, dilations=dil)
    blob = synth.pack_blob(spec, synth.init_weights(spec, 5))
    wts = synth.blob_f32_weights(blob, spec)
    frames, tgt, _, _ = synth.training_batch(np.random.default_rng(2), B=B, H=H, W=W, max_emitters=4)
    onet = oracle.Net(spec.to_json(), blob)
    x0 = oracle.ingest(frames, 1.0, 100.0, in_scale=onet.in_scale)
    val, gw, gb, ghw, ghb, _ = oracle.loss_grad(onet, x0, tgt)
    val_e, g = bf16_emulation(frames, tgt, spec, wts, rounding=False)
    assert abs(val_e - val) <= 1e-6 * abs(val)  # the float32 input transform is the only difference
    for a, r in zip(g, (gw, gb, ghw, ghb)):
        assert np.abs(a - r).max() <= 1e-6 * np.abs(r).max()
    # with the roundings the emulation stays close to, but not equal to, the exact gradient
    val_q, gq = bf16_emulation(frames, tgt, spec, wts)
    assert 0 < abs(val_q - val) <= 1e-2 * abs(val)
    assert any(np.abs(a - r).max() > 0 for a, r in zip(gq, (gw, gb, ghw, ghb)))
