"""Training the dilated-conv localization network on simulated frames, on the GPU.

Every forward and backward step runs in the library's hand-written kernels
(include/sml_train.h) behind ``torch.autograd.Function``s; PyTorch holds the FP32 master
weights, allocates memory and runs the Adam update.  The loss is the binary cross-entropy on
the detection probability (Sec. 3.3) plus a masked L2 on the offset, z and photon heads.

Two precisions: "fp32" (SIMT FMA kernels, NHWC float activations, one Function per layer) and
"bf16" (the tensor-core conv of the inference path for the forward and the input gradient,
a tcgen05 weight-gradient contraction, bf16 row-planar activations and activation gradients,
FP32 accumulation and FP32 master weights; one Function for the whole network).

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


# ----------------------------------------------------------------------------- BF16 (tensor cores)

_bf16_bound = False


def _bind_bf16():
    global _bf16_bound
    L = _bind()
    if _bf16_bound:
        return L
    L.sml_train_bf16_bimg_bytes.argtypes = [_I]
    L.sml_train_bf16_bimg_bytes.restype = _S
    L.sml_train_bf16_pack.argtypes = [_P, _I, _P, _P, _P]
    L.sml_train_bf16_layer0.argtypes = [_P, _I, _I, _I, _F, _F, _F, _P, _P, _I, _I, _P, _P]
    L.sml_train_bf16_conv_fwd.argtypes = [_P, _I, _I, _I, _I, _I, _P, _P, _P, _P, _P]
    L.sml_train_bf16_conv_dgrad.argtypes = [_P, _P, _I, _I, _I, _I, _I, _P, _P, _P, _P]
    L.sml_train_bf16_wgrad_work_bytes.argtypes = [_I]
    L.sml_train_bf16_wgrad_work_bytes.restype = _S
    L.sml_train_bf16_conv_wgrad.argtypes = [_P, _P, _I, _I, _I, _I, _I, _P, _P, _P, _S, _P, _P]
    L.sml_train_bf16_heads_loss.argtypes = [_P, _P, _I, _I, _I, _I, _P, _P, _P, _P, _P, _P, _P, _P, _P, _S, _P]
    L.sml_train_bf16_l0_wgrad.argtypes = [_P, _P, _I, _I, _I, _I, _I, _P, _P, _P, _S, _P]
    for n in ("sml_train_bf16_pack", "sml_train_bf16_layer0", "sml_train_bf16_conv_fwd", "sml_train_bf16_conv_dgrad",
              "sml_train_bf16_conv_wgrad", "sml_train_bf16_heads_loss", "sml_train_bf16_l0_wgrad"):
        getattr(L, n).restype = _I
    _bf16_bound = True
    return L


def rp_empty(B, H, W, C, device):
    """A row-planar bf16 activation tensor [B][H][C/16][W][16]."""
    return torch.empty((B, H, C // 16, W, 16), dtype=torch.bfloat16, device=device)


def rp_to_nhwc(a):
    """Row-planar [B][H][G][W][16] -> NHWC [B][H][W][16 G] (a copy, for tests)."""
    B, H, G, W, _ = a.shape
    return a.permute(0, 1, 3, 2, 4).reshape(B, H, W, 16 * G)


def sml_train_bf16_pack(w):
    L = _bind_bf16()
    C = int(w.shape[0])
    nb = L.sml_train_bf16_bimg_bytes(C)
    fwd = torch.empty(nb, dtype=torch.uint8, device=w.device)
    dg = torch.empty(nb, dtype=torch.uint8, device=w.device)
    _ok(L.sml_train_bf16_pack(_p(w), C, _p(fwd), _p(dg), _stream()))
    return fwd, dg


def sml_train_bf16_layer0(frames, w0, b0, d, gain, offset, in_scale):
    L = _bind_bf16()
    B, H, W = frames.shape
    C = int(w0.shape[0])
    a0 = rp_empty(B, H, W, C, frames.device)
    w0, b0 = w0.detach().contiguous(), b0.detach().contiguous()
    _ok(L.sml_train_bf16_layer0(_p(frames), B, H, W, gain, offset, in_scale, _p(w0), _p(b0), C, d, _p(a0), _stream()))
    return a0


def sml_train_bf16_conv_fwd(x, bimg_fwd, b, d, err):
    L = _bind_bf16()
    B, H, G, W, _ = x.shape
    y = torch.empty_like(x)
    _ok(L.sml_train_bf16_conv_fwd(_p(x), B, H, W, 16 * G, d, _p(bimg_fwd), _p(b), _p(y), _p(err), _stream()))
    return y


def sml_train_bf16_conv_dgrad(dz, x, bimg_dgrad, d, err):
    L = _bind_bf16()
    B, H, G, W, _ = dz.shape
    dz_in = torch.empty_like(dz)
    _ok(L.sml_train_bf16_conv_dgrad(_p(dz), _p(x), B, H, W, 16 * G, d, _p(bimg_dgrad), _p(dz_in), _p(err), _stream()))
    return dz_in


def sml_train_bf16_conv_wgrad(x, dz, d, err):
    L = _bind_bf16()
    B, H, G, W, _ = x.shape
    C = 16 * G
    nbytes = L.sml_train_bf16_wgrad_work_bytes(C)
    work = torch.empty(nbytes, dtype=torch.uint8, device=x.device)
    dw = torch.empty((C, C, 3, 3), dtype=torch.float32, device=x.device)
    db = torch.empty(C, dtype=torch.float32, device=x.device)
    _ok(L.sml_train_bf16_conv_wgrad(_p(x), _p(dz), B, H, W, C, d, _p(dw), _p(db), _p(work), nbytes, _p(err), _stream()))
    return dw, db


def sml_train_bf16_heads_loss(a, tgt, hw, hb, grad_scale=None):
    L = _bind_bf16()
    B, H, G, W, _ = a.shape
    C = 16 * G
    nbytes = L.sml_train_heads_work_bytes(B, H, W, C)
    work = torch.empty(nbytes, dtype=torch.uint8, device=a.device)
    h = torch.empty((B, 5, H, W), dtype=torch.float32, device=a.device)
    loss = torch.empty(1, dtype=torch.float32, device=a.device)
    dz = dhw = dhb = None
    if grad_scale is not None:
        dz = torch.empty_like(a)
        dhw = torch.empty_like(hw)
        dhb = torch.empty_like(hb)
    _ok(L.sml_train_bf16_heads_loss(_p(a), _p(tgt), B, H, W, C, _p(hw), _p(hb), _p(h), _p(loss), _p(grad_scale),
                                    _p(dz), _p(dhw), _p(dhb), _p(work), nbytes, _stream()))
    return h, loss, dz, dhw, dhb


def sml_train_bf16_l0_wgrad(x0, dz0, d):
    L = _bind_bf16()
    B, H, G, W, _ = dz0.shape
    C = 16 * G
    nbytes = L.sml_train_conv_bwd_work_bytes(B, H, W, 1, C)
    work = torch.empty(nbytes, dtype=torch.uint8, device=dz0.device)
    dw = torch.empty((C, 1, 3, 3), dtype=torch.float32, device=dz0.device)
    db = torch.empty(C, dtype=torch.float32, device=dz0.device)
    _ok(L.sml_train_bf16_l0_wgrad(_p(x0), _p(dz0), B, H, W, C, d, _p(dw), _p(db), _p(work), nbytes, _stream()))
    return dw, db


class DilatedStackBF16(torch.autograd.Function):
    """The whole dilated stack, heads and loss in BF16 on the tensor cores:
    forward(frames, targets, meta, *params) -> loss, params = (w_0..w_{L-1}, b_0..b_{L-1}, hw, hb)
    as FP32 masters.  meta = (dilations, gain, offset, in_scale, err) with err a device int32
    that the tensor-core kernels set if a bounded wait gave up.  The activations of every layer
    stay saved (bf16 row-planar) for the backward sweep, which returns FP32 gradients of every
    parameter."""

    @staticmethod
    def forward(ctx, frames, tgt, meta, *params):
        dil, gain, offset, in_scale, err = meta
        L = len(dil)
        ws, bs, hw, hb = params[:L], params[L : 2 * L], params[2 * L], params[2 * L + 1]
        packs = [None] + [sml_train_bf16_pack(ws[l].detach().contiguous()) for l in range(1, L)]
        acts = [sml_train_bf16_layer0(frames, ws[0], bs[0], dil[0], gain, offset, in_scale)]
        for l in range(1, L):
            acts.append(sml_train_bf16_conv_fwd(acts[-1], packs[l][0], bs[l].detach().contiguous(), dil[l], err))
        _, loss, _, _, _ = sml_train_bf16_heads_loss(acts[-1], tgt, hw.detach().contiguous(), hb.detach().contiguous())
        x0 = sml_train_ingest(frames, gain, offset, in_scale)
        ctx.save_for_backward(x0, tgt, hw, hb, *acts)
        ctx.packs, ctx.dil, ctx.err = packs, dil, err
        return loss[0]

    @staticmethod
    def backward(ctx, gl):
        x0, tgt, hw, hb, *acts = ctx.saved_tensors
        dil, packs, err = ctx.dil, ctx.packs, ctx.err
        L = len(dil)
        gs = gl.reshape(1).to(torch.float32).contiguous()
        _, _, dz, dhw, dhb = sml_train_bf16_heads_loss(acts[-1], tgt, hw.detach().contiguous(), hb.detach().contiguous(),
                                                       grad_scale=gs)
        dws, dbs = [None] * L, [None] * L
        for l in range(L - 1, 0, -1):
            dws[l], dbs[l] = sml_train_bf16_conv_wgrad(acts[l - 1], dz, dil[l], err)
            dz = sml_train_bf16_conv_dgrad(dz, acts[l - 1], packs[l][1], dil[l], err)
        dws[0], dbs[0] = sml_train_bf16_l0_wgrad(x0, dz, dil[0])
        return (None, None, None, *dws, *dbs, dhw, dhb)


class DilatedLocNet(torch.nn.Module):
    """The plain dilated stack with 1x1 heads; FP32 master weights in PyTorch layout."""

    def __init__(self, spec: synth.NetSpec, weights: synth.Weights, precision: str = "fp32"):
        super().__init__()
        if precision not in ("fp32", "bf16"):
            raise ValueError("training precision is fp32 or bf16")
        if precision == "bf16" and spec.channels not in (16, 32, 48):
            raise ValueError("bf16 training takes 16, 32 or 48 channels")
        self.precision = precision
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
    def from_blob(cls, spec_json: str, blob: bytes, precision: str = "fp32"):
        s = json.loads(spec_json)
        spec = synth.NetSpec(in_ch=s.get("in_ch", 1), channels=s["channels"], dilations=tuple(s["dilations"]),
                             precision=s.get("precision", "fp32"), in_scale=s.get("in_scale", 1e-3),
                             z_scale=s.get("z_scale", 1000.0), ph_scale=s.get("ph_scale", 10000.0),
                             dcd=s.get("dcd"), unet=int((s.get("unet") or {}).get("levels", 0)),
                             n_heads=len(s.get("heads", synth.HEAD_NAMES[: synth.N_HEADS])))
        return cls(spec, synth.unpack_blob(blob, spec)[1], precision)

    def features(self, frames, gain=1.0, offset=100.0):
        x = sml_train_ingest(frames.contiguous(), gain, offset, self.spec.in_scale).unsqueeze(-1)
        for w, b, d in zip(self.w, self.b, self.spec.dilations):
            x = ConvReLU.apply(x, w, b, d)
        return x

    def loss(self, frames, targets, gain=1.0, offset=100.0):
        if self.precision == "bf16":
            if getattr(self, "_err", None) is None or self._err.device != frames.device:
                self._err = torch.zeros(1, dtype=torch.int32, device=frames.device)
            meta = (tuple(int(d) for d in self.spec.dilations), float(gain), float(offset), float(self.spec.in_scale),
                    self._err)
            return DilatedStackBF16.apply(frames.contiguous(), targets.contiguous(), meta, *self.w, *self.b, self.hw,
                                          self.hb)
        a = self.features(frames, gain, offset)
        loss, _ = HeadsLoss.apply(a, self.hw, self.hb, targets)
        return loss

    def device_error(self) -> bool:
        """Whether a tensor-core kernel of the BF16 path gave up on a bounded wait since the
        last call (synchronises; clears the flag)."""
        err = getattr(self, "_err", None)
        if err is None:
            return False
        v = int(err.item())
        err.zero_()
        return v != 0

    def to_blob(self, precision="bf16") -> tuple[str, bytes]:
        w = synth.Weights([p.detach().cpu().double().numpy() for p in self.w],
                          [p.detach().cpu().double().numpy() for p in self.b], None, 0.0,
                          self.hw.detach().cpu().double().numpy(), self.hb.detach().cpu().double().numpy())
        spec = synth.NetSpec(**{**self.spec.__dict__, "precision": precision})
        return spec.to_json(), synth.pack_blob(spec, w)


class GraphedStep:
    """One training step (forward, loss, backward, Adam update) captured once in a CUDA graph
    and replayed: the host then issues one launch per step instead of the ~100 kernel launches
    and library calls of the step, whose host-side cost otherwise exceeds their device time
    at the training batch size.  The batch is copied into the graph's static input tensors
    before each replay; the optimizer runs with capturable state on the device.

        step = GraphedStep(net, frames_shape, lr=1e-3)
        loss = step(frames, targets)   # a device scalar (no synchronisation)
    """

    def __init__(self, net: "DilatedLocNet", frames_shape, lr: float = 1e-3, warmup: int = 2, gain=1.0,
                 offset=100.0):
        dev = net.hw.device
        B, H, W = frames_shape
        self.net = net
        self.frames = torch.zeros((B, H, W), dtype=torch.int16, device=dev)
        self.tgt = torch.zeros((B, 5, H, W), dtype=torch.float32, device=dev)
        self.opt = torch.optim.Adam(net.parameters(), lr=lr, capturable=True)
        if net.precision == "bf16" and getattr(net, "_err", None) is None:
            net._err = torch.zeros(1, dtype=torch.int32, device=dev)
        saved = [p.detach().clone() for p in net.parameters()]
        side = torch.cuda.Stream(device=dev)
        side.wait_stream(torch.cuda.current_stream(dev))
        with torch.cuda.stream(side):  # warm-up outside the graph (allocator, optimizer state)
            for _ in range(max(1, warmup)):
                self.opt.zero_grad(set_to_none=True)
                net.loss(self.frames, self.tgt, gain, offset).backward()
                self.opt.step()
        torch.cuda.current_stream(dev).wait_stream(side)
        # the warm-up steps must not count: parameters and optimizer state back to the start,
        # in place (the graph captures these tensors' addresses)
        with torch.no_grad():
            for p, v in zip(net.parameters(), saved):
                p.copy_(v)
            for st in self.opt.state.values():
                for v in st.values():
                    if torch.is_tensor(v):
                        v.zero_()
        self.graph = torch.cuda.CUDAGraph()
        self.opt.zero_grad(set_to_none=True)
        with torch.cuda.graph(self.graph):
            self.loss = net.loss(self.frames, self.tgt, gain, offset)
            self.loss.backward()
            self.opt.step()

    def __call__(self, frames, tgt):
        self.frames.copy_(frames.view(torch.int16), non_blocking=True)
        self.tgt.copy_(tgt, non_blocking=True)
        self.graph.replay()
        return self.loss


def device_batch(rng, B, H, W, max_emitters=10, min_emitters=0, z_scale=1000.0, ph_scale=10000.0, seed=5, frame0=0,
                 device="cuda"):
    """A fresh batch of training patches: emitters drawn on the host, frames rendered on the
    device by the library's simulator (astigmatic PSF, Poisson noise, gain 1, offset 100;
    include/sml_sim.h), targets written on the device from their nonzero entries."""
    from . import sml_sim_frames

    em = synth.training_emitters(rng, B, H, W, max_emitters, True, min_emitters)
    frames = sml_sim_frames(em, B, H, W, astig=True, gain=1.0, offset=100.0, seed=seed, frame0=frame0)
    idx, val = synth.training_target_entries(em, H, W, z_scale, ph_scale)
    tgt = torch.zeros((B, 5, H, W), dtype=torch.float32, device=device)
    tgt.view(-1)[torch.from_numpy(idx).to(device)] = torch.from_numpy(val).to(device)
    return frames.view(torch.int16), tgt


def train(net: DilatedLocNet, steps: int, batch: int = 256, patch: int = 64, lr: float = 1e-3, seed: int = 5,
          pool: int = 16, log_every: int = 50, device="cuda", max_emitters: int = 10, fresh: bool = False):
    """Adam on simulated astigmatic patches (0..max_emitters emitters each).  fresh = False: a
    pool of `pool` host-simulated batches generated once and cycled; fresh = True: a new batch
    every step from the device simulator (device_batch).  Returns the loss history."""
    rng = np.random.default_rng(seed)
    data = []
    if not fresh:
        for _ in range(pool):
            f, t, _, cam = synth.training_batch(rng, B=batch, H=patch, W=patch, z_scale=net.spec.z_scale,
                                                ph_scale=net.spec.ph_scale, max_emitters=max_emitters)
            data.append((torch.from_numpy(f).to(device), torch.from_numpy(t).to(device)))
    opt = torch.optim.Adam(net.parameters(), lr=lr)
    hist = []
    for step in range(steps):
        if fresh:
            frames, tgt = device_batch(rng, batch, patch, patch, max_emitters, 0, net.spec.z_scale, net.spec.ph_scale,
                                       seed=seed, frame0=step * batch, device=device)
        else:
            frames, tgt = data[step % pool]
        opt.zero_grad(set_to_none=True)
        loss = net.loss(frames, tgt, 1.0, 100.0)
        loss.backward()
        opt.step()
        if step % log_every == 0 or step == steps - 1:
            hist.append((step, float(loss.item())))
            if net.precision == "bf16" and net.device_error():
                raise SmlError(-5, "a tensor-core training kernel gave up on a bounded wait")
    return hist
