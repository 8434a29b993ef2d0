"""BF16 training on the tensor cores (include/sml_train.h, BF16 section).

Per kernel, against float64 PyTorch of the same bf16 inputs: the forward conv, the input
gradient (transposed conv with the lower layer's ReLU mask) and the weight/bias gradient
contraction (tcgen05 with MN-major operands).  Whole network: the loss and every gradient
against the oracle's exact float64 gradient (itself pinned to central finite differences,
tests/test_oracle_grad.py), and a net trained in BF16 on fresh device-simulated batches of
the training configuration (256 patches of 64x64, 48-channel 8-layer net) against the method
without a network."""
import time

import numpy as np
import pytest
import torch
import torch.nn.functional as F

import oracle
from bf16_emulation import bf16_emulation
from paper_2410_02314_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__

    __graft_entry__.build()
    torch.cuda.set_device(0)


def to_rp(x):
    """NCHW float -> row-planar bf16 [B][H][C/16][W][16] (CUDA)."""
    B, C, H, W = x.shape
    return x.reshape(B, C // 16, 16, H, W).permute(0, 3, 1, 4, 2).contiguous().to(torch.bfloat16).cuda()


def from_rp(a):
    """Row-planar [B][H][G][W][16] -> NCHW float64 (CPU)."""
    B, H, G, W, _ = a.shape
    return a.permute(0, 2, 4, 1, 3).reshape(B, 16 * G, H, W).double().cpu()


def bf16(x):
    return x.to(torch.bfloat16).double()


@pytest.mark.parametrize("C,d,B,H,W", [(48, 1, 2, 20, 40), (48, 4, 3, 33, 150), (32, 16, 2, 40, 130), (16, 2, 1, 9, 17)])
def test_bf16_conv_kernels_match_float64(C, d, B, H, W):
    """Forward, input gradient and weight gradient of one C -> C layer (dilation d, ragged
    frames wider than one 128-pixel strip) against float64 PyTorch on the same bf16 values:
    the outputs differ only by FP32 accumulation and the final bf16 rounding (1 ulp)."""
    from paper_2410_02314_gb300 import train as T

    g = torch.Generator().manual_seed(C + d)
    x = torch.relu(torch.randn(B, C, H, W, generator=g, dtype=torch.float64))
    w = (torch.rand(C, C, 3, 3, generator=g, dtype=torch.float64) - 0.5) * 2 * (6.0 / (9 * C)) ** 0.5
    b = (torch.rand(C, generator=g, dtype=torch.float64) - 0.5) * 0.2
    dz = torch.randn(B, C, H, W, generator=g, dtype=torch.float64) * (torch.rand(B, C, H, W, generator=g) > 0.4)
    xq, wq, dzq = bf16(x), bf16(w), bf16(dz)
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    fwd, dg = T.sml_train_bf16_pack(w.float().cuda().contiguous())
    # forward
    y = from_rp(T.sml_train_bf16_conv_fwd(to_rp(x), fwd, b.float().cuda(), d, err))
    ref = torch.relu(F.conv2d(xq, wq, b.float().double(), padding=d, dilation=d))
    assert (y - ref).abs().max().item() <= 2 ** -8 * ref.abs().max().item() + 1e-6
    # input gradient of the layer below: conv_transpose of dz, masked by x > 0
    dzin = from_rp(T.sml_train_bf16_conv_dgrad(to_rp(dz), to_rp(x), dg, d, err))
    ref_in = F.conv_transpose2d(dzq, wq, padding=d, dilation=d) * (xq > 0)
    assert (dzin - ref_in).abs().max().item() <= 2 ** -8 * ref_in.abs().max().item() + 1e-6
    # weight and bias gradient
    dw, db = T.sml_train_bf16_conv_wgrad(to_rp(x), to_rp(dz), d, err)
    xr = xq.clone().requires_grad_(True)
    wr = wq.clone().requires_grad_(True)
    br = torch.zeros(C, dtype=torch.float64, requires_grad=True)
    (F.conv2d(xr, wr, br, padding=d, dilation=d) * dzq).sum().backward()
    e_w = (dw.double().cpu() - wr.grad).abs().max().item() / wr.grad.abs().max().item()
    e_b = (db.double().cpu() - br.grad).abs().max().item() / br.grad.abs().max().item()
    print(C, d, "wgrad rel err", e_w, "bias", e_b)
    assert e_w <= 1e-5 and e_b <= 1e-5
    torch.cuda.synchronize()
    assert int(err.item()) == 0


@pytest.mark.parametrize("C,d,B,H,W", [(48, 1, 3, 21, 37), (48, 8, 2, 64, 150), (32, 3, 5, 13, 70), (16, 2, 1, 9, 17)])
def test_bf16_first_layer_grad_and_heads_match_float64(C, d, B, H, W):
    """The first layer's weight and bias gradient (FP32 input, bf16 pre-activation gradient)
    and the fused heads + loss + head gradients on bf16 activations, against float64 PyTorch
    of the same values.  Pixel counts and row counts are ragged (no multiple of a block's
    pixel or row step), so the kernels' partial tails are exercised."""
    from paper_2410_02314_gb300 import train as T

    g = torch.Generator().manual_seed(7 * C + d)
    # first layer: dw[c][tap] = sum_p dz0[p][c] x0[p + off(tap)], db[c] = sum_p dz0[p][c]
    x0 = torch.randn(B, H, W, generator=g, dtype=torch.float64).float()
    dz0 = torch.randn(B, C, H, W, generator=g, dtype=torch.float64) * (torch.rand(B, C, H, W, generator=g) > 0.5)
    dz0q = bf16(dz0)
    dw, db = T.sml_train_bf16_l0_wgrad(x0.cuda(), to_rp(dz0), d)
    wr = torch.zeros(C, 1, 3, 3, dtype=torch.float64, requires_grad=True)
    br = torch.zeros(C, dtype=torch.float64, requires_grad=True)
    (F.conv2d(x0.double().unsqueeze(1), wr, br, padding=d, dilation=d) * dz0q).sum().backward()
    e_w = (dw.double().cpu() - wr.grad).abs().max().item() / wr.grad.abs().max().item()
    e_b = (db.double().cpu() - br.grad).abs().max().item() / br.grad.abs().max().item()
    print(C, d, "first-layer wgrad rel err", e_w, "bias", e_b)
    assert e_w <= 1e-5 and e_b <= 1e-5
    # heads + loss: BCE on the logit head (mean over pixels) + L2 on the other four heads over
    # target pixels (divided by their count), gradients of 0.75 x loss
    a = torch.relu(torch.randn(B, C, H, W, generator=g, dtype=torch.float64))
    hw = ((torch.rand(5, C, generator=g, dtype=torch.float64) - 0.5) * 0.5).float()
    hb = ((torch.rand(5, generator=g, dtype=torch.float64) - 0.5) * 0.5).float()
    tgt = torch.randn(B, 5, H, W, generator=g, dtype=torch.float64).float()
    tgt[:, 0] = (torch.rand(B, H, W, generator=g) < 0.1).float()
    gs = torch.tensor([0.75], device="cuda")
    h, loss, dz, dhw, dhb = T.sml_train_bf16_heads_loss(to_rp(a), tgt.cuda(), hw.cuda(), hb.cuda(), grad_scale=gs)
    aq = bf16(a).requires_grad_(True)
    hwr = hw.double().requires_grad_(True)
    hbr = hb.double().requires_grad_(True)
    hh = torch.einsum("kc,bchw->bkhw", hwr, aq) + hbr[None, :, None, None]
    t64 = tgt.double()
    m = t64[:, 0] > 0.5
    lref = F.binary_cross_entropy_with_logits(hh[:, 0], t64[:, 0], reduction="sum") / (B * H * W) + \
        ((hh[:, 1:] - t64[:, 1:]) ** 2 * m[:, None]).sum() / max(1, int(m.sum()))
    (0.75 * lref).backward()
    e_h = (h.double().cpu() - hh.detach()).abs().max().item() / hh.detach().abs().max().item()
    e_l = abs(loss.item() - lref.item()) / abs(lref.item())
    ref_dz = aq.grad * (aq.detach() > 0)
    e_dz = (from_rp(dz) - ref_dz).abs().max().item() / ref_dz.abs().max().item()
    e_hw = (dhw.double().cpu() - hwr.grad).abs().max().item() / hwr.grad.abs().max().item()
    e_hb = (dhb.double().cpu() - hbr.grad).abs().max().item() / hbr.grad.abs().max().item()
    print(C, "heads rel err: h", e_h, "loss", e_l, "dz", e_dz, "dhw", e_hw, "dhb", e_hb)
    assert e_h <= 1e-5 and e_l <= 1e-5 and e_hw <= 1e-5 and e_hb <= 1e-5
    assert e_dz <= 2 ** -8  # one bf16 rounding of the FP32 gradient


def _loss_and_grads(net, frames, tgt):
    for p in net.parameters():
        p.grad = None
    loss = net.loss(torch.from_numpy(frames).cuda(), torch.from_numpy(tgt).cuda())
    loss.backward()
    g = [p.grad.detach().double().cpu().numpy().ravel() for p in net.w] + \
        [p.grad.detach().double().cpu().numpy().ravel() for p in net.b] + \
        [net.hw.grad.double().cpu().numpy().ravel(), net.hb.grad.double().cpu().numpy().ravel()]
    return float(loss.item()), g


def _groups(net, L):
    g = [np.concatenate([p.grad.detach().double().cpu().numpy().ravel() for p in net.w]),
         np.concatenate([p.grad.detach().double().cpu().numpy().ravel() for p in net.b]),
         net.hw.grad.double().cpu().numpy().ravel(), net.hb.grad.double().cpu().numpy().ravel()]
    return g


def _cmp(got, ref):
    rel = [float(np.abs(a - r).max() / max(np.abs(r).max(), 1e-30)) for a, r in zip(got, ref)]
    cos = [float(a @ r / max(np.linalg.norm(a) * np.linalg.norm(r), 1e-30)) for a, r in zip(got, ref)]
    return rel, cos


# Gates of the BF16 path against the float64 oracle, from tests/measure_bf16_grad_error.py on a
# GB300 (18 nets: C = 16, 32, 48 with 3, 6, 8 layers, 6 weight seeds each): worst loss error
# 9.0e-4; conv weight and bias gradients worst normalised max error 0.177, worst cosine 0.985;
# head gradients worst 0.0061.  The spread comes from the bf16 forward itself: ReLU masks of
# near-zero pre-activations differ from float64 and route the gradient differently (some seeds
# agree to 0.3 %, others to 17 %).  Gates: 1.5 x the worst (cosine: 1.5 x its distance to 1).
F64_LOSS, F64_CONV_MAX, F64_CONV_COS, F64_HEAD_MAX = 1.4e-3, 0.27, 0.978, 0.01


@pytest.mark.parametrize("C,dil,B,H,W", [(16, (1, 2, 4), 3, 20, 24), (48, (1, 2, 4, 8, 16, 8, 4, 1), 4, 64, 64)])
def test_bf16_gradients_match_oracle_and_emulation(C, dil, B, H, W):
    """The whole network in BF16 (forward, heads + loss, backward): against the oracle's
    float64 loss and gradient (itself pinned to finite differences) under the measured gates
    above, and against a float64 emulation of the same bf16 roundings, which isolates the
    kernels from the bf16 numerics; the FP32 SIMT path on the same batch is checked too."""
    from paper_2410_02314_gb300.train import DilatedLocNet

    spec = synth.NetSpec(in_ch=1, channels=C, dilations=dil)
    wts = synth.init_weights(spec, 3)
    blob = synth.pack_blob(spec, wts)
    wts = synth.blob_f32_weights(blob, spec)
    rng = np.random.default_rng(1)
    frames, tgt, _, _ = synth.training_batch(rng, B=B, H=H, W=W, max_emitters=6)
    onet = oracle.Net(spec.to_json(), blob)
    x0 = oracle.ingest(frames, 1.0, 100.0, in_scale=onet.in_scale)
    val, gw, gb, ghw, ghb, _ = oracle.loss_grad(onet, x0, tgt)
    ref64 = [gw, gb, ghw, ghb]
    val_e, ref_e = bf16_emulation(frames, tgt, spec, wts)
    res = {}
    for prec in ("bf16", "fp32"):
        net = DilatedLocNet.from_blob(spec.to_json(), blob, precision=prec).cuda()
        for p in net.parameters():
            p.grad = None
        loss = net.loss(torch.from_numpy(frames).cuda(), torch.from_numpy(tgt).cuda())
        loss.backward()
        got = _groups(net, len(dil))
        res[prec] = (float(loss.item()), got)
        rel, cos = _cmp(got, ref64)
        print(prec, C, len(dil), "vs float64: loss", abs(loss.item() - val) / abs(val), "grad max (w, b, hw, hb)",
              np.round(rel, 5), "cos", np.round(cos, 6))
        if prec == "bf16":
            assert not net.device_error()
            rel_e, cos_e = _cmp(got, ref_e)
            print("bf16 vs bf16 emulation: loss", abs(loss.item() - val_e) / abs(val_e), "grad max", np.round(rel_e, 5),
                  "cos", np.round(cos_e, 7))
            assert abs(loss.item() - val) <= F64_LOSS * abs(val)
            assert max(rel[:2]) <= F64_CONV_MAX and min(cos[:2]) >= F64_CONV_COS and max(rel[2:]) <= F64_HEAD_MAX
            res["emulation"] = (abs(loss.item() - val_e) / abs(val_e), rel_e, cos_e)
        else:
            assert abs(loss.item() - val) <= 1e-5 * abs(val) and max(rel) <= 1e-4
    loss_e, rel_e, cos_e = res["emulation"]
    assert loss_e <= 1e-4 and max(rel_e) <= 0.05 and min(cos_e) >= 0.999


def test_bf16_training_on_device_batches_beats_mle():
    """Training configuration: the 48-channel 8-layer net, BF16 forward and backward with FP32
    masters (Adam), fresh batches of 256 astigmatic 64x64 patches per step from the device
    simulator.  The trained net (BF16 inference) against local maxima + Gaussian MLE on held-out
    frames at high density; steps per second of BF16 and FP32 training on the same batches."""
    import paper_2410_02314_gb300 as sml
    from paper_2410_02314_gb300.train import DilatedLocNet, device_batch, train

    from test_gpu_train import _evaluate

    spec = synth.NetSpec(in_ch=1, channels=48, dilations=(1, 2, 4, 8, 16, 8, 4, 1))
    # throughput: 20 steps each on the same device batch
    rates = {}
    for prec in ("bf16", "fp32"):
        net = DilatedLocNet(spec, synth.init_weights(spec, 11), precision=prec).cuda()
        opt = torch.optim.Adam(net.parameters(), lr=1e-3)
        frames, tgt = device_batch(np.random.default_rng(0), 256, 64, 64, max_emitters=10)
        for k in range(23):
            if k == 3:
                torch.cuda.synchronize()
                t0 = time.perf_counter()
            opt.zero_grad(set_to_none=True)
            net.loss(frames, tgt).backward()
            opt.step()
        torch.cuda.synchronize()
        rates[prec] = 20 / (time.perf_counter() - t0)
    print("training steps/s (256 x 64x64 patches, 48-ch 8-layer):", rates)
    net = DilatedLocNet(spec, synth.init_weights(spec, 11), precision="bf16").cuda()
    hist = train(net, steps=1500, batch=256, patch=64, lr=1e-3, log_every=250, seed=5, max_emitters=40, fresh=True)
    print("bf16 training loss", hist)
    assert hist[-1][1] < 0.5 * hist[0][1]
    js, blob = net.to_blob("bf16")
    loc = sml.Localizer(js, blob)
    best, base = _evaluate(loc, np.random.default_rng(1234), 32, 20, 40)
    print("high density | bf16-trained net (p_min=%s)" % best[0], best[1], "| local max + MLE (thr=%s)" % base[0], base[1])
    assert best[1]["jaccard"] > base[1]["jaccard"]
    assert rates["bf16"] > rates["fp32"]


def test_graphed_training_step_matches_eager():
    """The BF16 training step captured in a CUDA graph (GraphedStep) replays the eager steps on
    the same batches: with the same optimizer arithmetic (Adam with its state on the device,
    as the graph needs it) the losses and parameters after five steps are the same."""
    from paper_2410_02314_gb300.train import DilatedLocNet, GraphedStep, device_batch

    spec = synth.NetSpec(in_ch=1, channels=32, dilations=(1, 2, 4, 1))
    rng = np.random.default_rng(3)
    batches = [device_batch(rng, 16, 48, 48, max_emitters=6, frame0=16 * k) for k in range(5)]
    eager = DilatedLocNet(spec, synth.init_weights(spec, 5), precision="bf16").cuda()
    opt = torch.optim.Adam(eager.parameters(), lr=1e-3, capturable=True)
    losses_e = []
    for frames, tgt in batches:
        opt.zero_grad(set_to_none=True)
        loss = eager.loss(frames, tgt)
        loss.backward()
        opt.step()
        losses_e.append(float(loss.item()))
    graphed = DilatedLocNet(spec, synth.init_weights(spec, 5), precision="bf16").cuda()
    step = GraphedStep(graphed, (16, 48, 48), lr=1e-3)
    losses_g = [float(step(frames, tgt).item()) for frames, tgt in batches]
    print("eager", losses_e, "graphed", losses_g)
    assert np.allclose(losses_g, losses_e, rtol=1e-6, atol=0)
    for a, b in zip(eager.parameters(), graphed.parameters()):
        assert torch.allclose(a, b, rtol=1e-6, atol=1e-9)
    assert not graphed.device_error()
