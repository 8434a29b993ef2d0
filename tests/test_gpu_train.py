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
