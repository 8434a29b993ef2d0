"""CPU oracle for the localization path -- TEST INFRASTRUCTURE ONLY.

Only tests/, ``__graft_entry__.smoke()`` and bench.py's CPU-baseline leg may import this
package.  The product library never calls it and shares no code with it: the oracle has
its own net-spec and weight-blob parser (below), its own C implementation
(``sml_oracle.c``) and its own record type.

What it computes (each function cites the passage it follows):
  * ``forward``        -- float64 forward of the plain dilated 3x3 stack (Sec. 3.2.1) with
                          DECODE-style per-pixel heads (Sec. 3.2); one input frame, or three
                          consecutive frames as channels (``context_input``);
  * ``maps_f32``       -- per-pixel maps handed to the decode: p = sigmoid(logit), dx, dy,
                          zhat, Nhat, rounded once to float32;
  * ``decode``         -- float32 decode of maps into (frame, x, y, z, photons, p) records
                          (post-processing on the device, Sec. 2.2 and Sec. 4.2.1);
  * ``localize``       -- forward, maps, decode;
  * ``forward_window`` -- exact heads of an interior block of a large frame from a crop
                          that covers the receptive field (for sampled parity checks);
  * ``loss_grad``      -- BCE (Sec. 3.3) + masked L2 training loss and its gradient.
Pins for each of these live in tests/test_oracle_*.py.
"""
from __future__ import annotations

import ctypes
import json
import os
import struct
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIBDIR = os.path.join(_HERE, "_lib")
_LIB = os.path.join(_LIBDIR, "liboracle.so")
_SRC = os.path.join(_HERE, "sml_oracle.c")
_lock = threading.Lock()
_lib = None

NH = 5  # position heads: logit p, dx, dy, zhat, Nhat
NH_SIGMA = 9  # with the uncertainty heads sx, sy, sz, sN (Sec. 3.2)
RECORD_DTYPE = np.dtype(
    [("frame", "<i4"), ("x", "<f4"), ("y", "<f4"), ("z", "<f4"), ("photons", "<f4"), ("p", "<f4")]
)
SIGMA_DTYPE = np.dtype([("sigma_x", "<f4"), ("sigma_y", "<f4"), ("sigma_z", "<f4"), ("sigma_photons", "<f4")])


def build(force: bool = False) -> str:
    """Compile sml_oracle.c with gcc (float64 forward, float32 decode without FMA contraction)."""
    os.makedirs(_LIBDIR, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
               "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            P = ctypes.c_void_p
            I = ctypes.c_int
            D = ctypes.c_double
            F = ctypes.c_float
            lib.orc_forward_x.argtypes = [P, I, I, I, I, I, I, P, P, P, P, D, P, P, P, P]
            lib.orc_forward_x.restype = None
            lib.orc_forward_xq.argtypes = [P, I, I, I, I, I, I, P, P, P, P, D, P, P, P, P, I, P]
            lib.orc_forward_xq.restype = None
            lib.orc_forward_xqh.argtypes = [P, I, I, I, I, I, I, P, P, P, P, D, I, P, P, P, P, I, P]
            lib.orc_forward_xqh.restype = None
            lib.orc_decode_h.argtypes = [P, I, I, I, I, F, F, F, P, P, ctypes.c_long]
            lib.orc_decode_h.restype = ctypes.c_long
            lib.orc_softplus.argtypes = [P, ctypes.c_size_t, P]
            lib.orc_softplus.restype = None
            lib.orc_conv.argtypes = [P, I, I, I, P, P, I, I, P]
            lib.orc_conv.restype = None
            lib.orc_round_array.argtypes = [P, ctypes.c_size_t, I]
            lib.orc_round_array.restype = None
            lib.orc_ingest.argtypes = [P, I, I, I, P, P, D, D, D, P]
            lib.orc_ingest.restype = None
            lib.orc_decode.argtypes = [P, I, I, I, F, F, F, P, ctypes.c_long]
            lib.orc_decode.restype = ctypes.c_long
            lib.orc_loss.argtypes = [P, P, I, I, I, P]
            lib.orc_loss.restype = D
            lib.orc_loss_grad.argtypes = [P, P, I, I, I, I, I, I, P, P, P, P, P, P, P, P, P, P]
            lib.orc_loss_grad.restype = D
            _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


# ----------------------------------------------------------------------------- parsing


class Net:
    """Network description parsed from a JSON net spec and an SMLW weight blob.

    Plain stacks: L conv layers of C channels with the spec's dilations (version-1 blobs up to
    16 layers, version 2 with reserved = 0 for 17 to 32).
    Nets with dense connection dilated blocks (spec key "dcd", version-2 blobs; Sec. 3.2.1):
    a stem conv (dilations[0], in_ch -> C); per block, dense layers whose input is the block
    input and every earlier output of the block concatenated (C + j*growth channels, growth
    outputs, the block's dilations) and a transition conv (d = 1, C + k*growth -> C); then the
    plain C -> C layers dilations[1:].
    A U-Net fine stage (spec key "unet": {"levels": L}, L in 1..2; Sec. 3.2, version-2 blobs)
    sits right before the last conv layer: per level down a 2x2 max pool (ceil) and a 3x3
    conv C -> C ("down"), per level up a nearest 2x upsample concatenated after that level's
    skip features and a 3x3 conv 2C -> C ("up").  ``layers`` lists (cin, cout, dilation,
    kind) of every conv layer in execution order."""

    def __init__(self, spec_json: str, blob: bytes):
        s = json.loads(spec_json)
        self.in_ch = int(s.get("in_ch", 1))
        self.C = int(s["channels"])
        self.plain_dil = [int(d) for d in s["dilations"]]
        self.in_scale = float(s.get("in_scale", 1e-3))
        self.z_scale = float(s.get("z_scale", 1000.0))
        self.ph_scale = float(s.get("ph_scale", 10000.0))
        # heads: the 5 position heads, or those and the 4 uncertainty heads (Sec. 3.2)
        self.nh = len(s.get("heads", ["p", "dx", "dy", "z", "N"]))
        if self.nh not in (NH, NH_SIGMA):
            raise ValueError("heads must list 5 or 9 outputs")
        C = self.C
        dcd = s.get("dcd")
        if dcd:
            self.growth = int(dcd["growth"])
            self.layers = [(self.in_ch, C, self.plain_dil[0], "stem")]
            for block in dcd["blocks"]:
                for j, d in enumerate(block):
                    self.layers.append((C + j * self.growth, self.growth, int(d), "dense"))
                self.layers.append((C + len(block) * self.growth, C, 1, "transition"))
            self.layers += [(C, C, d, "plain") for d in self.plain_dil[1:]]
            fmt, version = "<8s7I32i", 2
        else:
            self.growth = 0
            self.layers = [(self.in_ch if l == 0 else C, C, d, "plain") for l, d in enumerate(self.plain_dil)]
            # plain stacks beyond 16 layers carry their 17..32 dilations in the version-2 header
            fmt, version = ("<8s7I16i", 1) if len(self.layers) <= 16 else ("<8s7I32i", 2)
        unet = s.get("unet")
        self.unet = int(unet["levels"]) if unet else 0
        if self.unet:
            if self.unet not in (1, 2) or len(self.layers) < 2:
                raise ValueError("unet needs 1 or 2 levels and a conv layer before the last one")
            last = self.layers[-1]
            self.layers = (self.layers[:-1] + [(C, C, 1, "down")] * self.unet + [(2 * C, C, 1, "up")] * self.unet
                           + [last])
            fmt, version = "<8s7I32i", 2
        self.dil = [d for _, _, d, _ in self.layers]
        self.L = len(self.layers)
        hdr = struct.unpack_from(fmt, blob, 0)
        if hdr[0] != b"SMLW0001":
            raise ValueError("weight blob: bad magic")
        _, ver, L, C_, in_ch, nh, has_bn, growth, *dil = hdr
        if (ver, L, C_, in_ch, nh, list(dil[:L])) != (version, self.L, C, self.in_ch, self.nh, self.dil) or (
                version == 2 and growth != self.growth):
            raise ValueError("weight blob does not match net spec")
        if version == 2 and has_bn:
            raise ValueError("weight blob: BatchNorm is not supported with dense blocks")
        off = struct.calcsize(fmt)

        def take(n):
            nonlocal off
            a = np.frombuffer(blob, dtype="<f4", count=n, offset=off).astype(np.float64)
            off += 4 * n
            return a

        ws, bs, bns = [], [], []
        self.bn_eps = 0.0
        for cin, cout, _, _ in self.layers:
            ws.append(take(cout * cin * 9))
            bs.append(take(cout))
            if has_bn:
                bns.append(take(4 * cout))
                self.bn_eps = float(take(1)[0])
        self.layer_w, self.layer_b = ws, bs
        self.conv_w = np.ascontiguousarray(np.concatenate(ws))
        self.conv_b = np.ascontiguousarray(np.concatenate(bs))
        self.bn = np.ascontiguousarray(np.concatenate(bns)) if has_bn else None
        self.head_w = np.ascontiguousarray(take(self.nh * C))
        self.head_b = np.ascontiguousarray(take(self.nh))
        if off != len(blob):
            raise ValueError("weight blob: trailing bytes")

    @property
    def R(self) -> int:
        """Receptive radius (px): the sum of the dilations outside the U-Net, plus for a U-Net of
        L levels the bound 3 * 2^(L+1) on its reach (pooling and upsampling included)."""
        plain = sum(d for _, _, d, kind in self.layers if kind not in ("down", "up"))
        return plain + (3 * 2 ** (self.unet + 1) if self.unet else 0)


# ----------------------------------------------------------------------------- forward


def ingest(frames, gain=1.0, offset=100.0, gain_map=None, offset_map=None, in_scale=1e-3):
    """Network input x = (adu - offset) / gain * in_scale, float64 [T,H,W]."""
    lib = _load()
    f = np.ascontiguousarray(frames, dtype=np.uint16)
    T, H, W = f.shape
    gm = None if gain_map is None else np.ascontiguousarray(gain_map, dtype=np.float64)
    om = None if offset_map is None else np.ascontiguousarray(offset_map, dtype=np.float64)
    x0 = np.empty((T, H, W), dtype=np.float64)
    lib.orc_ingest(_ptr(f), T, H, W, _ptr(gm), _ptr(om), gain, offset, in_scale, _ptr(x0))
    return x0


def context_input(x, in_ch):
    """Network input channels from single-frame inputs x [T,H,W]: in_ch = 1 gives x itself;
    in_ch = 3 gives frames (t-1, t, t+1) as channels 0..2 (three-frame temporal context,
    Sec. 3.1 on DECODE), zero where t-1 or t+1 falls outside the stack.  Returns
    [T,in_ch,H,W] float64."""
    x = np.asarray(x, dtype=np.float64)
    T = x.shape[0]
    if in_ch == 1:
        return x[:, None].copy()
    if in_ch != 3:
        raise ValueError("in_ch must be 1 or 3")
    out = np.zeros((T, 3) + x.shape[1:], dtype=np.float64)
    out[:, 1] = x
    out[1:, 0] = x[:-1]
    out[:-1, 2] = x[1:]
    return out


QUANT = {None: 0, "fp32": 0, "bf16": 1, "fp8": 2}


def round_to(a, fmt):
    """Round float64 values through float32 to bf16 or e4m3 (saturating at +-448), both
    round-to-nearest-even; returns float64."""
    lib = _load()
    out = np.array(a, dtype=np.float64, copy=True, order="C")
    lib.orc_round_array(_ptr(out), out.size, {"bf16": 1, "fp8": 2}[fmt])
    return out


def input_producers(net: Net):
    """For every conv layer in execution order, the layer that produced each of its input
    channels (-1: the network input).  A plain layer reads its predecessor; a dense layer
    (Sec. 3.2.1) reads the block input and the block's earlier outputs, so its channels come
    from several layers; a transition reads the whole concatenation; a U-Net down conv reads
    the pooled features of the level above, an up conv the level's skip features followed by
    the upsampled deeper features (Sec. 3.2).  Pooling and upsampling move stored values, so
    they keep the producer."""
    prods = []
    buf = []  # producer of each channel of the current block's concatenation
    li = 0
    while li < net.L:
        cin, cout, _, kind = net.layers[li]
        if kind == "down":
            skips = [buf[: net.C]]
            for _ in range(net.unet):
                prods.append(list(skips[-1]))
                skips.append([li] * net.C)
                li += 1
            up = skips.pop()
            while skips:
                skip = skips.pop()
                prods.append(list(skip) + list(up))
                up = [li] * net.C
                li += 1
            buf = list(up)
            continue
        prods.append([-1] * cin if li == 0 else list(buf[:cin]))
        if kind == "dense":
            buf = buf + [li] * cout
        else:
            buf = [li] * cout
        li += 1
    return [np.asarray(p, dtype=np.int64) for p in prods]


def quantized(net: Net, fmt, scales=None):
    """Copy of net whose conv weights of layers 1..L-1 are rounded as the tensor-core path
    stores them: bf16, or e4m3 of w / s[co] times s[co] with s[co] = max |w[co,:,:,:]| / 448
    (float32).  Layer 0 (the SIMT first layer) and the heads keep their float32 weights.
    Nets with dense blocks or a U-Net in e4m3 need the activation scales (scales[l + 1]: the
    output scale of layer l, as act_scales returns them): a layer's input channels come from
    several layers with their own scales, so each weight is first multiplied by the scale of
    its input channel, w'[co,ci] = w[co,ci] s_in[ci] (float32), then rounded per output channel
    as above, and divided by s_in[ci] again, so that the float64 forward on the dequantised
    activations computes what the tensor cores compute on the stored e4m3 codes."""
    import copy

    if net.bn is not None:
        raise ValueError("quantized oracle modes need a net without BatchNorm")
    q = copy.copy(net)
    if net.growth or net.unet:  # per-layer arrays (layers 1.. run on the tensor cores)
        if fmt == "bf16":
            q.layer_w = [net.layer_w[0]] + [round_to(wl, "bf16") for wl in net.layer_w[1:]]
            return q
        if fmt != "fp8" or scales is None:
            raise ValueError("dense blocks and the U-Net: bf16, or fp8 with the activation scales")
        sc = np.asarray(scales, dtype=np.float32)
        prods = input_producers(net)
        q.layer_w = [net.layer_w[0]]
        for li in range(1, net.L):
            cin, cout, _, _ = net.layers[li]
            s_in = sc[prods[li] + 1]  # float32 [cin]
            wf = net.layer_w[li].reshape(cout, cin, 9).astype(np.float32) * s_in[None, :, None]
            amax = np.abs(wf).max(axis=(1, 2))
            sw = np.where(amax > 0, amax / np.float32(448.0), np.float32(1.0)).astype(np.float32)
            wq = round_to((wf / sw[:, None, None]).astype(np.float64), "fp8")
            q.layer_w.append((wq * sw[:, None, None].astype(np.float64) / s_in[None, :, None].astype(np.float64)).ravel())
        return q
    w = net.conv_w.copy()
    off = net.C * net.in_ch * 9
    n = net.C * net.C * 9
    for layer in range(1, net.L):
        blk = w[off : off + n].reshape(net.C, net.C * 9)
        if fmt == "bf16":
            blk[:] = round_to(blk, "bf16")
        elif fmt == "fp8":
            amax = np.abs(blk.astype(np.float32)).max(axis=1)
            s = np.where(amax > 0, amax / np.float32(448.0), np.float32(1.0)).astype(np.float32)
            blk[:] = round_to((blk.astype(np.float32) / s[:, None]).astype(np.float64), "fp8") * s[:, None].astype(np.float64)
        w[off : off + n] = blk.ravel()
        off += n
    q.conv_w = w
    return q


def act_scales(net: Net, frames, gain=1.0, offset=100.0, gain_map=None, offset_map=None):
    """FP8 activation scales from this oracle's own float64 activations: [1] + [amax_l / 448]
    with amax_l the largest output of layer l = 0..L-2 over the given frames (for a plain stack
    the inputs of layers 1..L-1)."""
    x0 = context_input(ingest(frames, gain, offset, gain_map, offset_map, net.in_scale), net.in_ch)
    if net.growth or net.unet:
        amax = [0.0] * net.L
        _forward_dense(net, x0, amax=amax)
        return [1.0] + [amax[l] / 448.0 for l in range(net.L - 1)]
    _, a = forward_x(net, x0, acts=True)
    return [1.0] + [float(a[:, l - 1].max()) / 448.0 for l in range(1, net.L)]


def forward_x(net: Net, x0, acts=False, quant=None, scales=None):
    """Raw heads [T,nh,H,W] (float64) of the dilated stack on inputs x0 [T,in_ch,H,W]
    (Sec. 3.2.1 dilated convolution, zero padding at every layer; Sec. 3.2 heads).
    quant "bf16" / "fp8" rounds the input activations of layers 1..L-1 to that format
    (fp8: of a / scales[l]) before the layer, as the tensor-core path stores them; pass a
    net from quantized() to round the weights too."""
    if net.growth or net.unet:
        return _forward_dense(net, x0, acts, quant, scales)
    lib = _load()
    x0 = np.ascontiguousarray(x0, dtype=np.float64)
    if x0.ndim == 3:
        x0 = x0[:, None]
    T, cin, H, W = x0.shape
    assert cin == net.in_ch
    heads = np.empty((T, net.nh, H, W), dtype=np.float64)
    a = np.empty((T, net.L, net.C, H, W), dtype=np.float64) if acts else None
    dil = np.asarray(net.dil, dtype=np.int32)
    sc = None if scales is None else np.ascontiguousarray(scales, dtype=np.float64)
    lib.orc_forward_xqh(_ptr(x0), T, H, W, net.L, net.C, net.in_ch, _ptr(dil), _ptr(net.conv_w),
                        _ptr(net.conv_b), _ptr(net.bn), net.bn_eps, net.nh, _ptr(net.head_w), _ptr(net.head_b),
                        _ptr(heads), _ptr(a), QUANT[quant], _ptr(sc))
    return (heads, a) if acts else heads


def pool2(a):
    """2x2 max pooling with stride 2 of [C,H,W] to [C,ceil(H/2),ceil(W/2)]; a window that
    overhangs the frame's last row or column takes the max of its in-frame pixels."""
    C, H, W = a.shape
    p = np.full((C, H + H % 2, W + W % 2), -np.inf)
    p[:, :H, :W] = a
    return p.reshape(C, p.shape[1] // 2, 2, p.shape[2] // 2, 2).max(axis=(2, 4))


def upsample2(a, H, W):
    """Nearest-neighbour 2x upsampling of [C,h,w] cropped to [C,H,W]: out[c,i,j] = a[c,i//2,j//2]."""
    return a.repeat(2, axis=1).repeat(2, axis=2)[:, :H, :W]


def _forward_dense(net: Net, x0, acts=False, quant=None, scales=None, amax=None):
    """Forward of a net with dense connection dilated blocks (Sec. 3.2.1) and/or a U-Net fine
    stage (Sec. 3.2): each conv is the C oracle's conv (float64) on a channel range of a
    buffer that concatenates the block input and the block's outputs so far; the U-Net
    pools, convolves, upsamples and concatenates with numpy.  quant "bf16" rounds every conv
    layer's stored output to bf16 (what the tensor-core path stores; pooling and upsampling
    move stored values unchanged; the stem's input frames stay float); quant "fp8" rounds
    layer l's stored output a to e4m3 of a * (1 / scales[l + 1]) (float32) times scales[l + 1].
    With amax (a list of L floats), amax[l] becomes the largest output of layer l.  Returns raw
    heads [T,nh,H,W] (and, with acts, the last layer's activations)."""
    lib = _load()
    x0 = np.ascontiguousarray(x0, dtype=np.float64)
    if x0.ndim == 3:
        x0 = x0[:, None]
    T, cin0, H, W = x0.shape
    assert cin0 == net.in_ch
    if quant not in (None, "fp32", "bf16", "fp8") or (quant == "fp8" and scales is None):
        raise ValueError("dense blocks and the U-Net: bf16, or fp8 with the activation scales")

    def rnd(a, li):
        if quant == "bf16":
            return round_to(a, "bf16")
        if quant == "fp8":
            inv = np.float32(1.0 / scales[li + 1])
            return round_to((a.astype(np.float32) * inv).astype(np.float64), "fp8") * scales[li + 1]
        return a
    C, g = net.C, net.growth
    widest = max(cin for cin, _, _, _ in net.layers)

    def conv(li, inp):
        cin, cout, d, _ = net.layers[li]
        inp = np.ascontiguousarray(inp)
        h, w = inp.shape[1:]
        out = np.empty((cout, h, w), dtype=np.float64)
        lib.orc_conv(_ptr(inp), cin, h, w, _ptr(np.ascontiguousarray(net.layer_w[li])),
                     _ptr(np.ascontiguousarray(net.layer_b[li])), cout, d, _ptr(out))
        if amax is not None:
            amax[li] = max(amax[li], float(out.max()))
        return out if li == net.L - 1 else rnd(out, li)  # the last layer's output feeds the heads in FP32

    heads = np.empty((T, net.nh, H, W), dtype=np.float64)
    last = np.empty((T, C, H, W), dtype=np.float64) if acts else None
    for t in range(T):
        buf = np.zeros((widest, H, W), dtype=np.float64)  # the current block's concatenation
        used = 0  # channels of buf filled
        src = np.ascontiguousarray(x0[t])
        li = 0
        while li < net.L:
            cin, cout, d, kind = net.layers[li]
            if kind == "down":  # the U-Net: levels down, then up (2 * levels conv layers)
                skips = [buf[:C].copy()]
                for _ in range(net.unet):
                    skips.append(conv(li, pool2(skips[-1])))
                    li += 1
                up = skips.pop()
                while skips:
                    skip = skips.pop()
                    up = conv(li, np.concatenate([skip, upsample2(up, *skip.shape[1:])]))
                    li += 1
                buf[:C] = up
                used = C
                continue
            out = conv(li, src if li == 0 else buf[:cin])  # the first layer reads the network input
            if kind == "dense":  # appended to the block's concatenation
                buf[used : used + cout] = out
                used += cout
            else:  # stem, transition, plain: a new C-channel block input
                buf[:cout] = out
                used = cout
            li += 1
        a = buf[:C]
        if acts:
            last[t] = a
        heads[t] = net.head_b[:, None, None] + np.einsum("kc,chw->khw", net.head_w.reshape(net.nh, C), a)
    return (heads, last) if acts else heads


def forward(net: Net, frames, gain=1.0, offset=100.0, gain_map=None, offset_map=None, quant=None, scales=None):
    """Raw heads [T,5,H,W] float64 from uint16 frames through the camera transform (and,
    for in_ch = 3, the three-frame context of context_input)."""
    x0 = context_input(ingest(frames, gain, offset, gain_map, offset_map, net.in_scale), net.in_ch)
    return forward_x(net, x0, quant=quant, scales=scales)


def sigmoid(h):
    """p = 1 / (1 + exp(-h)) in float64."""
    return 1.0 / (1.0 + np.exp(-np.asarray(h, dtype=np.float64)))


def softplus(h):
    """Uncertainty-head activation softplus(h) = log(1 + exp(h)) in float64 (the C oracle's
    overflow-free form of that definition)."""
    lib = _load()
    h = np.ascontiguousarray(h, dtype=np.float64)
    out = np.empty_like(h)
    lib.orc_softplus(_ptr(h), h.size, _ptr(out))
    return out


def maps_f32(heads):
    """Decode input [T,nh,H,W] float32: channel 0 = sigmoid(logit), channels 1-4 unchanged,
    channels 5-8 (uncertainty heads, nh = 9) = softplus of the raw heads."""
    m = np.array(heads, dtype=np.float64, copy=True)
    m[:, 0] = sigmoid(m[:, 0])
    if m.shape[1] > NH:
        m[:, NH:] = softplus(m[:, NH:])
    return m.astype(np.float32)


def decode(maps, p_min, z_scale, ph_scale, cap=None, with_sigma=False):
    """Float32 decode (Sec. 2.2 post-processing): records ordered by (frame, row, col).
    maps [T,nh,H,W] with nh 5 or 9; with_sigma (nh = 9) also returns the uncertainties of
    each record (sigma_x, sigma_y px, sigma_z = z_scale*sz nm, sigma_photons = ph_scale*sN)."""
    lib = _load()
    m = np.ascontiguousarray(maps, dtype=np.float32)
    T, nh, H, W = m.shape
    assert nh in (NH, NH_SIGMA) and (nh == NH_SIGMA or not with_sigma)
    n = lib.orc_decode_h(_ptr(m), T, nh, H, W, p_min, z_scale, ph_scale, None, None, 0)
    out = np.zeros(n if cap is None else min(n, cap), dtype=RECORD_DTYPE)
    sig = np.zeros(out.size, dtype=SIGMA_DTYPE) if with_sigma else None
    lib.orc_decode_h(_ptr(m), T, nh, H, W, p_min, z_scale, ph_scale, _ptr(out), _ptr(sig), out.size)
    return (out, sig) if with_sigma else out


def localize(net: Net, frames, p_min, gain=1.0, offset=100.0, gain_map=None, offset_map=None):
    heads = forward(net, frames, gain, offset, gain_map, offset_map)
    maps = maps_f32(heads)
    return decode(maps, p_min, net.z_scale, net.ph_scale), heads, maps


def forward_window(net: Net, frames, i0, i1, j0, j1, gain=1.0, offset=100.0, gain_map=None,
                   offset_map=None, quant=None, scales=None):
    """Exact heads [T,nh,i1-i0,j1-j0] of the block [i0,i1) x [j0,j1) of full frames.

    The crop extends the block by the receptive radius R (clipped at the frame border).
    Every output inside the block depends only on inputs within R of it, and layer l's
    outputs are wrong only within its reach of a crop edge that is not a frame edge, so the
    block's values equal those of the whole-frame forward.  With a U-Net of L levels the
    crop starts on a multiple of 2^L, so that its pooling windows are the whole frame's.
    """
    T, H, W = frames.shape
    R = net.R
    a = 2 ** net.unet
    ci0, ci1 = max(0, i0 - R) // a * a, min(H, i1 + R)
    cj0, cj1 = max(0, j0 - R) // a * a, min(W, j1 + R)
    crop = np.ascontiguousarray(frames[:, ci0:ci1, cj0:cj1])
    gm = None if gain_map is None else gain_map[ci0:ci1, cj0:cj1]
    om = None if offset_map is None else offset_map[ci0:ci1, cj0:cj1]
    h = forward(net, crop, gain, offset, gm, om, quant=quant, scales=scales)
    return h[:, :, i0 - ci0 : i1 - ci0, j0 - cj0 : j1 - cj0]


# ----------------------------------------------------------------------------- training


def loss(heads, targets):
    lib = _load()
    h = np.ascontiguousarray(heads, dtype=np.float64)
    y = np.ascontiguousarray(targets, dtype=np.float64)
    B, _, H, W = h.shape
    dh = np.empty_like(h)
    val = lib.orc_loss(_ptr(h), _ptr(y), B, H, W, _ptr(dh))
    return val, dh


def loss_grad(net: Net, x0, targets):
    """Loss (BCE on p, Sec. 3.3, + masked L2) and its exact gradient w.r.t. every weight.

    Returns (loss, g_conv_w (flat, blob order), g_conv_b [L*C], g_head_w [5*C], g_head_b [5],
    heads)."""
    if net.bn is not None:
        raise ValueError("training gradient is defined for nets without BatchNorm")
    lib = _load()
    x0 = np.ascontiguousarray(x0, dtype=np.float64)
    if x0.ndim == 3:
        x0 = x0[:, None]
    B, cin, H, W = x0.shape
    y = np.ascontiguousarray(targets, dtype=np.float64)
    gw = np.empty_like(net.conv_w)
    gb = np.empty_like(net.conv_b)
    ghw = np.empty_like(net.head_w)
    ghb = np.empty_like(net.head_b)
    heads = np.empty((B, NH, H, W), dtype=np.float64)
    dil = np.asarray(net.dil, dtype=np.int32)
    val = lib.orc_loss_grad(_ptr(x0), _ptr(y), B, H, W, net.L, net.C, net.in_ch, _ptr(dil),
                            _ptr(net.conv_w), _ptr(net.conv_b), _ptr(net.head_w), _ptr(net.head_b),
                            _ptr(gw), _ptr(gb), _ptr(ghw), _ptr(ghb), _ptr(heads))
    return val, gw, gb, ghw, ghb, heads
