"""Pins for the oracle's training loss and gradient.

* The loss equals PyTorch's binary_cross_entropy_with_logits (mean) plus a masked squared
  error computed with plain numpy, on the oracle's own heads.
* Every gradient entry that is checked matches a central finite difference of the oracle's
  float64 forward + loss (relative error below 1e-6).
"""
import numpy as np
import torch
import torch.nn.functional as F

import oracle
from paper_2410_02314_gb300 import synth


def tiny_problem(seed=3, B=2, H=9, W=10, C=3, dil=(1, 2, 3)):
    spec = synth.NetSpec(in_ch=1, channels=C, dilations=dil)
    blob = synth.pack_blob(spec, synth.init_weights(spec, seed))
    net = oracle.Net(spec.to_json(), blob)
    rng = np.random.default_rng(seed)
    x0 = rng.normal(0.3, 0.5, (B, 1, H, W))
    y = np.zeros((B, 5, H, W))
    mask = rng.random((B, H, W)) < 0.15
    y[:, 0] = mask
    y[:, 1:] = rng.normal(0.0, 0.5, (B, 4, H, W)) * mask[:, None]
    return net, x0, y


def test_loss_matches_torch_bce_plus_masked_l2():
    net, x0, y = tiny_problem()
    h = oracle.forward_x(net, x0)
    val, _ = oracle.loss(h, y)
    bce = F.binary_cross_entropy_with_logits(torch.from_numpy(h[:, 0]), torch.from_numpy(y[:, 0])).item()
    m = y[:, 0] > 0.5
    l2 = sum(((h[:, k] - y[:, k]) ** 2)[m].sum() for k in range(1, 5)) / max(1, m.sum())
    assert abs(val - (bce + l2)) <= 1e-12 * abs(bce + l2)


def _set(net, which, idx, v):
    getattr(net, which)[idx] = v


def test_gradient_matches_central_differences():
    net, x0, y = tiny_problem()
    val, gw, gb, ghw, ghb, _ = oracle.loss_grad(net, x0, y)
    rng = np.random.default_rng(9)
    checks = [("conv_w", gw), ("conv_b", gb), ("head_w", ghw), ("head_b", ghb)]
    eps = 1e-6
    for name, g in checks:
        arr = getattr(net, name)
        idxs = rng.choice(arr.size, size=min(arr.size, 12), replace=False)
        for k in idxs:
            old = arr[k]
            arr[k] = old + eps
            lp = oracle.loss(oracle.forward_x(net, x0), y)[0]
            arr[k] = old - eps
            lm = oracle.loss(oracle.forward_x(net, x0), y)[0]
            arr[k] = old
            fd = (lp - lm) / (2 * eps)
            assert abs(fd - g[k]) <= 1e-6 * max(abs(fd), 1e-3), (name, k, fd, g[k])


def test_loss_of_targets_without_emitters():
    """With no target pixels the L2 term vanishes and the loss is the mean BCE."""
    net, x0, y = tiny_problem()
    y[:] = 0.0
    h = oracle.forward_x(net, x0)
    val, dh = oracle.loss(h, y)
    p = 1.0 / (1.0 + np.exp(-h[:, 0]))
    assert abs(val - np.mean(-np.log1p(-p))) < 1e-12
    assert np.all(dh[:, 1:] == 0.0)
