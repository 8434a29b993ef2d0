"""Training the dilated-conv localization network on simulated frames, on the GPU.

Every forward and backward step runs in the library's hand-written kernels
(include/sml_train.h) behind ``torch.autograd.Function``s; PyTorch holds the FP32 master
weights, allocates memory and runs the Adam update.  The loss is the binary cross-entropy on
the detection probability (Sec. 3.3) plus a masked L2 on the offset, z and photon heads.

    net = DilatedLocNet.from_blob(spec_json, blob).cuda()
    loss = net.loss(frames_u16_cuda, targets_cuda)   # scalar tensor, differentiable
    blob = net.to_blob()                             # trained weights for sml_create
"""
from __future__ import annotations

import ctypes
import json
import math
import struct

import numpy as np
import torch

from . import SmlError, lib
from . import synth

_P = ctypes.c_void_p
_I = ctypes.c_int
_F = ctypes.c_float
_S = ctypes.c_size_t
_bound = False


def _bind():
    global _bound
    if _bound:
        return lib()
    L = lib()
    L.sml_train_ingest.argtypes = [_P, ctypes.c_longlong, _F, _F, _F, _P, _P]
    L.sml_train_conv_fwd.argtypes = [_P, _I, _I, _I, _I, _I, _I, _P, _P, _P, _P]
    L.sml_train_conv_bwd_work_bytes.argtypes = [_I, _I, _I, _I, _I]
    L.sml_train_conv_bwd_work_bytes.restype = _S
    L.sml_train_conv_bwd.argtypes = [_P, _P, _P, _I, _I, _I, _I, _I, _I, _P, _P, _P, _P, _P, _S, _P]
    L.sml_train_heads_work_bytes.argtypes = [_I, _I, _I, _I]
    L.sml_train_heads_work_bytes.restype = _S
    L.sml_train_heads_loss.argtypes = [_P, _P, _I, _I, _I, _I, _P, _P, _P, _P, _P, _P, _P, _P, _P, _S, _P]
    for n in ("sml_train_ingest", "sml_train_conv_fwd", "sml_train_conv_bwd", "sml_train_heads_loss"):
        getattr(L, n).restype = _I
    _bound = True
    return L


def _p(t):
    return None if t is None else t.data_ptr()


def _stream():
    return torch.cuda.current_stream().cuda_stream


def _ok(code):
    if code != 0:
        raise SmlError(code, "training kernel call failed (bad sizes or CUDA error)")


# ----------------------------------------------------------------------------- C names


def sml_train_ingest(frames, gain, offset, in_scale):
    L = _bind()
    x0 = torch.empty(frames.shape, dtype=torch.float32, device=frames.device)
    _ok(L.sml_train_ingest(_p(frames), frames.numel(), gain, offset, in_scale, _p(x0), _stream()))
    return x0


def sml_train_conv_fwd(x, w, b, d):
    L = _bind()
    B, H, W, cin = x.shape
    cout = w.shape[0]
    y = torch.empty((B, H, W, cout), dtype=torch.float32, device=x.device)
    _ok(L.sml_train_conv_fwd(_p(x), B, H, W, cin, cout, d, _p(w), _p(b), _p(y), _stream()))
    return y


def sml_train_conv_bwd(x, y, dy, w, d, need_dx=True):
    L = _bind()
    B, H, W, cin = x.shape
    cout = w.shape[0]
    nbytes = L.sml_train_conv_bwd_work_bytes(B, H, W, cin, cout)
    work = torch.empty(nbytes, dtype=torch.uint8, device=x.device)
    dx = torch.empty_like(x) if need_dx else None
    dw = torch.empty_like(w)
    db = torch.empty(cout, dtype=torch.float32, device=x.device)
    _ok(L.sml_train_conv_bwd(_p(x), _p(y), _p(dy), B, H, W, cin, cout, d, _p(w), _p(dx), _p(dw), _p(db), _p(work),
                             nbytes, _stream()))
    return dx, dw, db


def sml_train_heads_loss(a, tgt, hw, hb, grad_scale=None):
    L = _bind()
    B, H, W, C = a.shape
    nbytes = L.sml_train_heads_work_bytes(B, H, W, C)
    work = torch.empty(nbytes, dtype=torch.uint8, device=a.device)
    h = torch.empty((B, 5, H, W), dtype=torch.float32, device=a.device)
    loss = torch.empty(1, dtype=torch.float32, device=a.device)
    da = dhw = dhb = None
    if grad_scale is not None:
        da = torch.empty_like(a)
        dhw = torch.empty_like(hw)
        dhb = torch.empty_like(hb)
    _ok(L.sml_train_heads_loss(_p(a), _p(tgt), B, H, W, C, _p(hw), _p(hb), _p(h), _p(loss), _p(grad_scale), _p(da),
                               _p(dhw), _p(dhb), _p(work), nbytes, _stream()))
    return h, loss, da, dhw, dhb


# ----------------------------------------------------------------------------- autograd


class ConvReLU(torch.autograd.Function):
    """y = ReLU(b + dilated 3x3 conv of x); NHWC activations, forward and backward in CUDA."""

    @staticmethod
    def forward(ctx, x, w, b, d):
        y = sml_train_conv_fwd(x.contiguous(), w.contiguous(), b.contiguous(), d)
        ctx.save_for_backward(x, w, y)
        ctx.d = d
        return y

    @staticmethod
    def backward(ctx, dy):
        x, w, y = ctx.saved_tensors
        need_dx = ctx.needs_input_grad[0] and x.shape[-1] > 1
        dx, dw, db = sml_train_conv_bwd(x, y, dy.contiguous(), w, ctx.d, need_dx=need_dx)
        return dx, dw, db, None


class HeadsLoss(torch.autograd.Function):
    """Heads + loss (BCE on p, masked L2 on the rest); returns (loss, heads)."""

    @staticmethod
    def forward(ctx, a, hw, hb, tgt):
        h, loss, _, _, _ = sml_train_heads_loss(a.contiguous(), tgt.contiguous(), hw.contiguous(), hb.contiguous())
        ctx.save_for_backward(a, hw, hb, tgt)
        ctx.mark_non_differentiable(h)
        return loss[0], h

    @staticmethod
    def backward(ctx, gl, gh):
        a, hw, hb, tgt = ctx.saved_tensors
        gs = gl.reshape(1).to(torch.float32).contiguous()
        _, _, da, dhw, dhb = sml_train_heads_loss(a, tgt, hw, hb, grad_scale=gs)
        return da, dhw, dhb, None


class DilatedLocNet(torch.nn.Module):
    """The plain dilated stack with 1x1 heads; FP32 master weights in PyTorch layout."""

    def __init__(self, spec: synth.NetSpec, weights: synth.Weights):
        super().__init__()
        if weights.bn is not None:
            raise ValueError("train a net without BatchNorm (fold it first)")
        if spec.dcd or spec.unet or spec.n_heads != synth.N_HEADS or spec.in_ch != 1:
            raise ValueError("training covers the plain dilated stack with the five position heads and one input "
                             "frame (no dense blocks, U-Net, uncertainty heads or three-frame input)")
        self.spec = spec
        self.w = torch.nn.ParameterList([torch.nn.Parameter(torch.tensor(a, dtype=torch.float32)) for a in weights.conv_w])
        self.b = torch.nn.ParameterList([torch.nn.Parameter(torch.tensor(a, dtype=torch.float32)) for a in weights.conv_b])
        self.hw = torch.nn.Parameter(torch.tensor(weights.head_w, dtype=torch.float32))
        self.hb = torch.nn.Parameter(torch.tensor(weights.head_b, dtype=torch.float32))

    @classmethod
    def from_blob(cls, spec_json: str, blob: bytes):
        s = json.loads(spec_json)
        spec = synth.NetSpec(in_ch=s.get("in_ch", 1), channels=s["channels"], dilations=tuple(s["dilations"]),
                             precision=s.get("precision", "fp32"), in_scale=s.get("in_scale", 1e-3),
                             z_scale=s.get("z_scale", 1000.0), ph_scale=s.get("ph_scale", 10000.0),
                             dcd=s.get("dcd"), unet=int((s.get("unet") or {}).get("levels", 0)),
                             n_heads=len(s.get("heads", synth.HEAD_NAMES[: synth.N_HEADS])))
        return cls(spec, synth.unpack_blob(blob, spec)[1])

    def features(self, frames, gain=1.0, offset=100.0):
        x = sml_train_ingest(frames.contiguous(), gain, offset, self.spec.in_scale).unsqueeze(-1)
        for w, b, d in zip(self.w, self.b, self.spec.dilations):
            x = ConvReLU.apply(x, w, b, d)
        return x

    def loss(self, frames, targets, gain=1.0, offset=100.0):
        a = self.features(frames, gain, offset)
        loss, _ = HeadsLoss.apply(a, self.hw, self.hb, targets)
        return loss

    def to_blob(self, precision="bf16") -> tuple[str, bytes]:
        w = synth.Weights([p.detach().cpu().double().numpy() for p in self.w],
                          [p.detach().cpu().double().numpy() for p in self.b], None, 0.0,
                          self.hw.detach().cpu().double().numpy(), self.hb.detach().cpu().double().numpy())
        spec = synth.NetSpec(**{**self.spec.__dict__, "precision": precision})
        return spec.to_json(), synth.pack_blob(spec, w)


def train(net: DilatedLocNet, steps: int, batch: int = 256, patch: int = 64, lr: float = 1e-3, seed: int = 5,
          pool: int = 16, log_every: int = 50, device="cuda", max_emitters: int = 10):
    """Adam on simulated astigmatic patches (0..max_emitters emitters each).  A pool of
    simulated batches is generated once and cycled; returns the loss history."""
    rng = np.random.default_rng(seed)
    data = []
    for _ in range(pool):
        f, t, _, cam = synth.training_batch(rng, B=batch, H=patch, W=patch, z_scale=net.spec.z_scale,
                                            ph_scale=net.spec.ph_scale, max_emitters=max_emitters)
        data.append((torch.from_numpy(f).to(device), torch.from_numpy(t).to(device)))
    opt = torch.optim.Adam(net.parameters(), lr=lr)
    hist = []
    for step in range(steps):
        frames, tgt = data[step % pool]
        opt.zero_grad(set_to_none=True)
        loss = net.loss(frames, tgt, 1.0, 100.0)
        loss.backward()
        opt.step()
        if step % log_every == 0 or step == steps - 1:
            hist.append((step, float(loss.item())))
    return hist
