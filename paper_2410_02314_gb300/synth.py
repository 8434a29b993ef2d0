"""Seeded synthetic inputs: network specs, weight blobs, simulated camera frames.

This module draws random numbers and renders synthetic microscope frames.  It holds
none of the localization method's arithmetic (no convolution, no heads, no decode):
both the CUDA path and the CPU oracle receive what it produces as plain inputs.

* Weight blobs follow the byte layout documented in ``include/sml.h`` (``SMLW`` blobs).
  Weights are Kaiming-uniform (bound sqrt(6/fan_in)) and biases U(+-1/sqrt(fan_in)),
  drawn from a splitmix64 stream in the fixed order layer -> co -> ci -> ky -> kx.
* Frames are pixel-integrated Gaussian PSFs (optionally astigmatic), plus a constant
  background, Poisson shot noise and the camera's ADU conversion
  ``adu = round(gain * electrons + offset)`` clamped to [0, 65535].  The paper only says
  that its training and test data are simulated (Sec. 3.4, Sec. 4.1); the PSF model,
  emitter statistics and camera model here are this project's reading of those silences.
"""
from __future__ import annotations

import json
import math
import struct
from dataclasses import dataclass, field

import numpy as np

MAGIC = b"SMLW0001"
MAX_LAYERS = 16
N_HEADS = 5  # position heads: p logit, dx, dy, zhat, Nhat
# head names of the net spec: the position heads, then the uncertainty heads (Sec. 3.2)
HEAD_NAMES = ("p", "dx", "dy", "z", "N", "sx", "sy", "sz", "sN")
HEADER_FMT = "<8s7I16i"  # magic, version, L, C, in_ch, n_heads, has_bn, reserved, dil[16]
HEADER_BYTES = struct.calcsize(HEADER_FMT)
# version 2 (nets with dense connection dilated blocks): reserved = growth, dil[32] per layer
MAX_LAYERS_V2 = 32
HEADER_FMT_V2 = "<8s7I32i"
HEADER_BYTES_V2 = struct.calcsize(HEADER_FMT_V2)

_M64 = np.uint64(0xFFFFFFFFFFFFFFFF)


def splitmix64(seed: int, n: int) -> np.ndarray:
    """First ``n`` outputs of splitmix64 started at ``seed`` (uint64 array)."""
    with np.errstate(over="ignore"):
        k = np.arange(1, n + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + k * np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return z


class _Stream:
    """Sequential uniform draws from one splitmix64 stream."""

    def __init__(self, seed: int):
        self.seed = seed
        self.pos = 0

    def uniform(self, n: int, lo: float, hi: float) -> np.ndarray:
        with np.errstate(over="ignore"):
            z = splitmix64(self.seed + self.pos * 0x9E3779B97F4A7C15, n)
        self.pos += n
        u = (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
        return lo + (hi - lo) * u


# --------------------------------------------------------------------------- net spec


@dataclass
class NetSpec:
    in_ch: int = 1
    channels: int = 48
    dilations: tuple = (1, 2, 4, 8, 16, 8, 4, 1)
    precision: str = "fp32"
    in_scale: float = 1e-3
    z_scale: float = 1000.0
    ph_scale: float = 10000.0
    act_scales: tuple = ()  # fp8 only, one per conv layer: [l] = scale of what layer l-1 stores
    # Dense connection dilated blocks, or None for the plain stack: {"growth": g, "blocks":
    # [[d, ...], ...]}.  The net is then: stem conv (dilations[0], in_ch -> C); per block, one
    # dense layer per listed dilation (input: the block input and every earlier layer's
    # output, concatenated; output: g channels) and a transition conv (d = 1, C + k*g -> C);
    # then the plain C -> C layers dilations[1:], the last of which feeds the heads.
    dcd: dict | None = None
    # 5 (position heads) or 9 (and the uncertainty heads sx, sy, sz, sN)
    n_heads: int = N_HEADS
    # U-Net fine stage: number of levels (0 = none, 1 or 2), inserted before the last layer.
    # Per level down: 2x2 max pool, then a 3x3 conv C -> C; per level up: nearest 2x
    # upsample concatenated after the level's skip features, then a 3x3 conv 2C -> C.
    unet: int = 0

    def layers(self) -> list:
        """(cin, cout, dilation) of every conv layer in execution order."""
        C = self.channels
        if not self.dcd:
            out = [(self.in_ch if l == 0 else C, C, d) for l, d in enumerate(self.dilations)]
        else:
            g = int(self.dcd["growth"])
            out = [(self.in_ch, C, self.dilations[0])]
            for block in self.dcd["blocks"]:
                for j, d in enumerate(block):
                    out.append((C + j * g, g, int(d)))
                out.append((C + len(block) * g, C, 1))
            out += [(C, C, d) for d in self.dilations[1:]]
        if self.unet:
            out = out[:-1] + [(C, C, 1)] * self.unet + [(2 * C, C, 1)] * self.unet + out[-1:]
        return out

    def to_json(self) -> str:
        d = {
            "in_ch": self.in_ch,
            "channels": self.channels,
            "dilations": list(self.dilations),
            "heads": list(HEAD_NAMES[: self.n_heads]),
            "precision": self.precision,
            "in_scale": self.in_scale,
            "z_scale": self.z_scale,
            "ph_scale": self.ph_scale,
        }
        if self.act_scales:
            d["act_scales"] = [float(s) for s in self.act_scales]
        if self.dcd:
            d["dcd"] = {"growth": int(self.dcd["growth"]), "blocks": [[int(x) for x in b] for b in self.dcd["blocks"]]}
        if self.unet:
            d["unet"] = {"levels": int(self.unet)}
        return json.dumps(d)

    @property
    def L(self) -> int:
        return len(self.layers())

    @property
    def R(self) -> int:
        """Receptive radius of the net in pixels: the sum of the dilations outside the U-Net,
        plus 3 * 2^(levels+1) for a U-Net (a bound on its reach, pooling included)."""
        n = 2 * self.unet
        lay = self.layers()
        plain = lay[: len(lay) - 1 - n] + lay[-1:] if n else lay
        return int(sum(d for _, _, d in plain) + (3 * 2 ** (self.unet + 1) if self.unet else 0))


def spec_small(precision="fp32") -> NetSpec:
    """32-channel, 6-layer net with dilations 1,2,4,8,4,1 (the small 64x64 workload)."""
    return NetSpec(in_ch=1, channels=32, dilations=(1, 2, 4, 8, 4, 1), precision=precision)


def spec_48(precision="bf16") -> NetSpec:
    """48-channel, 8-layer net with dilations 1,2,4,8,16,8,4,1."""
    return NetSpec(in_ch=1, channels=48, dilations=(1, 2, 4, 8, 16, 8, 4, 1), precision=precision)


def spec_dcd(precision="bf16") -> NetSpec:
    """32-channel net with dense connection dilated blocks: stem (d = 1); one coarse block and
    three context blocks, each of four dense layers (growth 16, dilations 2, 4, 8, 16) and a
    transition back to 32 channels; then a last 32-channel layer (d = 1) feeding the heads.
    22 conv layers, receptive radius 126 px."""
    return NetSpec(in_ch=1, channels=32, dilations=(1, 1), precision=precision,
                   dcd={"growth": 16, "blocks": [[2, 4, 8, 16] for _ in range(4)]})


def spec_dilatedloc(precision="bf16") -> NetSpec:
    """The paper's full topology with our widths (Sec. 3.2): the dense-block feature extractor of
    spec_dcd (one coarse and three context blocks), a two-level U-Net fine stage and the nine
    heads (positions and their uncertainties).  26 conv layers."""
    return NetSpec(in_ch=1, channels=32, dilations=(1, 1), precision=precision, n_heads=9, unet=2,
                   dcd={"growth": 16, "blocks": [[2, 4, 8, 16] for _ in range(4)]})


# --------------------------------------------------------------------------- weights


@dataclass
class Weights:
    """Float64 copies of every parameter, in the blob's order."""

    conv_w: list  # L arrays [Cout, Cin, 3, 3]
    conv_b: list  # L arrays [Cout]
    bn: list | None  # L arrays [4, Cout] (gamma, beta, mean, var) or None
    bn_eps: float
    head_w: np.ndarray  # [5, C]
    head_b: np.ndarray  # [5]


def init_weights(spec: NetSpec, seed: int, bn: bool = False) -> Weights:
    s = _Stream(seed)
    C = spec.channels
    ws, bs, bns = [], [], []
    for cin, cout, _ in spec.layers():
        fan_in = cin * 9
        bound = math.sqrt(6.0 / fan_in)
        w = s.uniform(cout * cin * 9, -bound, bound).reshape(cout, cin, 3, 3)
        b = s.uniform(cout, -1.0 / math.sqrt(fan_in), 1.0 / math.sqrt(fan_in))
        ws.append(w)
        bs.append(b)
        if bn:
            if spec.dcd or spec.unet:
                raise ValueError("BatchNorm is not supported with dense blocks or a U-Net")
            gamma = s.uniform(C, 0.5, 1.5)
            beta = s.uniform(C, -0.1, 0.1)
            mean = s.uniform(C, -0.1, 0.1)
            var = s.uniform(C, 0.5, 1.5)
            bns.append(np.stack([gamma, beta, mean, var]))
    bound = math.sqrt(6.0 / C)
    nh = spec.n_heads
    hw = s.uniform(nh * C, -bound, bound).reshape(nh, C)
    hb = s.uniform(nh, -1.0 / math.sqrt(C), 1.0 / math.sqrt(C))
    return Weights(ws, bs, bns if bn else None, 1e-5, hw, hb)


def pack_blob(spec: NetSpec, w: Weights) -> bytes:
    """Serialise weights into an SMLW blob (little endian, float32 payload).  Plain stacks of up
    to 16 layers use version 1 (dil[16]); nets with dense blocks or a U-Net, and plain stacks of
    17 to 32 layers, version 2 (reserved = growth, dil[32] = every layer's dilation in execution
    order)."""
    L, C = spec.L, spec.channels
    has_bn = 1 if w.bn is not None else 0
    nh = int(np.asarray(w.head_b).size)
    if spec.dcd or spec.unet or L > MAX_LAYERS:
        if has_bn:
            raise ValueError("version-2 blobs carry no BatchNorm")
        if L > MAX_LAYERS_V2:
            raise ValueError(f"{L} conv layers (at most {MAX_LAYERS_V2})")
        dil = [d for _, _, d in spec.layers()] + [0] * (MAX_LAYERS_V2 - L)
        growth = int(spec.dcd["growth"]) if spec.dcd else 0
        parts = [struct.pack(HEADER_FMT_V2, MAGIC, 2, L, C, spec.in_ch, nh, has_bn, growth, *dil)]
    else:
        dil = list(spec.dilations) + [0] * (MAX_LAYERS - L)
        parts = [struct.pack(HEADER_FMT, MAGIC, 1, L, C, spec.in_ch, nh, has_bn, 0, *dil)]
    for layer in range(L):
        parts.append(np.ascontiguousarray(w.conv_w[layer], dtype="<f4").tobytes())
        parts.append(np.ascontiguousarray(w.conv_b[layer], dtype="<f4").tobytes())
        if has_bn:
            parts.append(np.ascontiguousarray(w.bn[layer], dtype="<f4").tobytes())
            parts.append(struct.pack("<f", w.bn_eps))
    parts.append(np.ascontiguousarray(w.head_w, dtype="<f4").tobytes())
    parts.append(np.ascontiguousarray(w.head_b, dtype="<f4").tobytes())
    return b"".join(parts)


def unpack_blob(blob: bytes, spec: NetSpec | None = None) -> tuple[dict, Weights]:
    """Parse an SMLW blob back into float64 arrays (header dict, Weights).  A version-2 blob
    (dense blocks, a U-Net or more than 16 layers) needs its spec for the layers' channel counts."""
    head = struct.unpack_from(HEADER_FMT, blob, 0)
    if head[0] != MAGIC:
        raise ValueError("bad magic")
    version = head[1]
    if version == 2:
        head = struct.unpack_from(HEADER_FMT_V2, blob, 0)
    _, version, L, C, in_ch, n_heads, has_bn, _, *dil = head
    off = HEADER_BYTES_V2 if version == 2 else HEADER_BYTES
    if version == 2:
        if spec is None:
            raise ValueError("a version-2 blob needs its net spec")
        shapes = [(cout, cin) for cin, cout, _ in spec.layers()]
    else:
        shapes = [(C, in_ch if layer == 0 else C) for layer in range(L)]

    def take(n):
        nonlocal off
        a = np.frombuffer(blob, dtype="<f4", count=n, offset=off).astype(np.float64)
        off += 4 * n
        return a

    ws, bs, bns, eps = [], [], [], 1e-5
    for cout, cin in shapes:
        ws.append(take(cout * cin * 9).reshape(cout, cin, 3, 3))
        bs.append(take(cout))
        if has_bn:
            bns.append(take(4 * C).reshape(4, C))
            eps = float(take(1)[0])
    hw = take(n_heads * C).reshape(n_heads, C)
    hb = take(n_heads)
    if off != len(blob):
        raise ValueError("trailing bytes in blob")
    hdr = dict(version=version, L=L, C=C, in_ch=in_ch, n_heads=n_heads, has_bn=has_bn, dil=dil[:L])
    return hdr, Weights(ws, bs, bns if has_bn else None, eps, hw, hb)


def blob_f32_weights(blob: bytes, spec: NetSpec | None = None) -> Weights:
    """The weights exactly as stored (float32-rounded), as float64 arrays."""
    return unpack_blob(blob, spec)[1]


# --------------------------------------------------------------------------- camera + frames


@dataclass
class Camera:
    gain: float = 1.0
    offset: float = 100.0
    gain_map: np.ndarray | None = None  # [H, W] float32 ADU per electron
    offset_map: np.ndarray | None = None  # [H, W] float32 ADU


@dataclass
class Emitters:
    frame: np.ndarray  # int32 [n]
    x: np.ndarray  # px, pixel centre = integer index
    y: np.ndarray
    z: np.ndarray  # nm
    photons: np.ndarray
    bg: np.ndarray = field(default_factory=lambda: np.zeros(0))  # per frame background (photons / px)


def sigma_xy(z: np.ndarray, astig: bool, sigma0: float = 1.3) -> tuple[np.ndarray, np.ndarray]:
    """PSF widths in px: constant sigma0, or the astigmatic model
    sigma_{x,y}(z) = sigma0 * sqrt(1 + ((z -+ 400 nm) / 500 nm)^2)."""
    if not astig:
        s = np.full_like(np.asarray(z, dtype=np.float64), sigma0)
        return s, s
    z = np.asarray(z, dtype=np.float64)
    sx = sigma0 * np.sqrt(1.0 + ((z + 400.0) / 500.0) ** 2)
    sy = sigma0 * np.sqrt(1.0 + ((z - 400.0) / 500.0) ** 2)
    return sx, sy


def _erf(x):
    from scipy.special import erf

    return erf(x)


def render_expected(em: Emitters, T: int, H: int, W: int, astig: bool, sigma0: float = 1.3) -> np.ndarray:
    """Expected photo-electrons per pixel [T, H, W] (float64): background plus, for every
    emitter, photons times the pixel-integrated Gaussian."""
    mu = np.zeros((T, H, W), dtype=np.float64)
    if em.bg.size:
        mu += em.bg.reshape(T, 1, 1)
    n = em.x.size
    if n == 0:
        return mu
    sx, sy = sigma_xy(em.z, astig, sigma0)
    r = int(math.ceil(4.0 * float(max(sx.max(), sy.max())))) + 1
    off = np.arange(-r, r + 1)
    cx = np.rint(em.x).astype(np.int64)
    cy = np.rint(em.y).astype(np.int64)
    jj = cx[:, None] + off[None, :]  # [n, 2r+1]
    ii = cy[:, None] + off[None, :]
    s2x = (math.sqrt(2.0) * sx)[:, None]
    s2y = (math.sqrt(2.0) * sy)[:, None]
    ex = 0.5 * (_erf((jj + 0.5 - em.x[:, None]) / s2x) - _erf((jj - 0.5 - em.x[:, None]) / s2x))
    ey = 0.5 * (_erf((ii + 0.5 - em.y[:, None]) / s2y) - _erf((ii - 0.5 - em.y[:, None]) / s2y))
    val = em.photons[:, None, None] * ey[:, :, None] * ex[:, None, :]
    I = np.broadcast_to(ii[:, :, None], val.shape)
    J = np.broadcast_to(jj[:, None, :], val.shape)
    F = np.broadcast_to(em.frame.astype(np.int64)[:, None, None], val.shape)
    ok = (I >= 0) & (I < H) & (J >= 0) & (J < W)
    flat = (F[ok] * H + I[ok]) * W + J[ok]
    mu += np.bincount(flat, weights=val[ok], minlength=T * H * W).reshape(T, H, W)
    return mu


def to_adu(electrons: np.ndarray, cam: Camera) -> np.ndarray:
    """Camera ADU conversion: round(gain * e + offset), clamped to uint16."""
    g = cam.gain_map if cam.gain_map is not None else cam.gain
    o = cam.offset_map if cam.offset_map is not None else cam.offset
    adu = np.rint(electrons * g + o)
    return np.clip(adu, 0, 65535).astype(np.uint16)


def simulate(em: Emitters, T, H, W, cam: Camera, astig: bool, rng: np.random.Generator, noise=True):
    mu = render_expected(em, T, H, W, astig)
    e = rng.poisson(mu).astype(np.float64) if noise else mu
    return to_adu(e, cam)


# --------------------------------------------------------------------------- workloads


@dataclass
class Workload:
    name: str
    frames: np.ndarray  # uint16 [T, H, W]
    cam: Camera
    emitters: Emitters
    spec: NetSpec
    blob: bytes
    astig: bool


def _uniform_positions(rng, n, H, W):
    return rng.uniform(-0.5, W - 0.5, n), rng.uniform(-0.5, H - 0.5, n)


def emitters_small(rng, T, H, W, per_frame=10):
    n = T * per_frame
    x, y = _uniform_positions(rng, n, H, W)
    return Emitters(
        frame=np.repeat(np.arange(T, dtype=np.int32), per_frame),
        x=x,
        y=y,
        z=np.zeros(n),
        photons=rng.uniform(1000.0, 5000.0, n),
        bg=np.full(T, 100.0),
    )


def emitters_density(rng, T, H, W, density_um2, px_nm=100.0, astig=False):
    area = (H * px_nm / 1000.0) * (W * px_nm / 1000.0)
    counts = rng.poisson(density_um2 * area, T)
    n = int(counts.sum())
    x, y = _uniform_positions(rng, n, H, W)
    return Emitters(
        frame=np.repeat(np.arange(T, dtype=np.int32), counts),
        x=x,
        y=y,
        z=rng.uniform(-600.0, 600.0, n) if astig else np.zeros(n),
        photons=rng.lognormal(math.log(3000.0), 0.5, n),
        bg=rng.uniform(50.0, 200.0, T),
    )


def scmos_camera(rng, H, W):
    return Camera(
        gain=2.0,
        offset=100.0,
        gain_map=rng.normal(2.0, 0.1, (H, W)).astype(np.float32),
        offset_map=rng.normal(100.0, 5.0, (H, W)).astype(np.float32),
    )


def workload_small(T=4, H=64, W=64, precision="fp32", frame_seed=1, weight_seed=2) -> Workload:
    """4 frames 64x64: 10 emitters per frame, sigma 1.3 px, photons U(1000,5000),
    background 100, gain 1, offset 100; 32-channel 6-layer net."""
    rng = np.random.default_rng(frame_seed)
    em = emitters_small(rng, T, H, W)
    cam = Camera(1.0, 100.0)
    frames = simulate(em, T, H, W, cam, False, rng)
    spec = spec_small(precision)
    blob = pack_blob(spec, init_weights(spec, weight_seed))
    return Workload("small_64", frames, cam, em, spec, blob, False)


def workload_batched(T=256, H=256, W=256, precision="bf16", seed=3) -> Workload:
    """256 frames 256x256: 1 emitter/um^2 at 100 nm px, sigma 1.3 px, photons
    LogNormal(ln 3000, 0.5), background U(50,200); 48-channel 8-layer net."""
    rng = np.random.default_rng(seed)
    em = emitters_density(rng, T, H, W, 1.0)
    cam = Camera(1.0, 100.0)
    frames = simulate(em, T, H, W, cam, False, rng)
    spec = spec_48(precision)
    blob = pack_blob(spec, init_weights(spec, seed + 1000))
    return Workload("batched_256", frames, cam, em, spec, blob, False)


def workload_dcd(T=256, H=256, W=256, precision="bf16", seed=3) -> Workload:
    """The frames of workload_batched (same seed) through the dense-block net of spec_dcd."""
    rng = np.random.default_rng(seed)
    em = emitters_density(rng, T, H, W, 1.0)
    cam = Camera(1.0, 100.0)
    frames = simulate(em, T, H, W, cam, False, rng)
    spec = spec_dcd(precision)
    blob = pack_blob(spec, init_weights(spec, seed + 2000))
    return Workload("dcd_256", frames, cam, em, spec, blob, False)


def workload_dilatedloc(T=256, H=256, W=256, precision="bf16", seed=3) -> Workload:
    """The frames of workload_batched (same seed) through the full-topology net of spec_dilatedloc."""
    rng = np.random.default_rng(seed)
    em = emitters_density(rng, T, H, W, 1.0)
    cam = Camera(1.0, 100.0)
    frames = simulate(em, T, H, W, cam, False, rng)
    spec = spec_dilatedloc(precision)
    blob = pack_blob(spec, init_weights(spec, seed + 3000))
    return Workload("dilatedloc_256", frames, cam, em, spec, blob, False)


def workload_large_fov(T=2, H=2048, W=2048, precision="bf16", seed=4) -> Workload:
    """2048x2048 sCMOS frames: per-pixel gain N(2,0.1), offset N(100,5), 2 emitters/um^2,
    astigmatic PSF with z ~ U(-600,600) nm; 48-channel 8-layer net."""
    rng = np.random.default_rng(seed)
    cam = scmos_camera(rng, H, W)
    em = emitters_density(rng, T, H, W, 2.0, astig=True)
    frames = simulate(em, T, H, W, cam, True, rng)
    spec = spec_48(precision)
    blob = pack_blob(spec, init_weights(spec, seed + 1000))
    return Workload("large_fov_2048", frames, cam, em, spec, blob, True)


# --------------------------------------------------------------------------- training data


def training_emitters(rng, B=256, H=64, W=64, max_emitters=10, astig=True, min_emitters=0) -> Emitters:
    """Emitters of a batch of training patches: U{min..max} per patch, uniform positions,
    z ~ U(-600, 600) nm (astigmatic), photons LogNormal(ln 3000, 0.5), background U(50, 200)."""
    counts = rng.integers(min_emitters, max_emitters + 1, B)
    n = int(counts.sum())
    x, y = _uniform_positions(rng, n, H, W)
    return Emitters(
        frame=np.repeat(np.arange(B, dtype=np.int32), counts),
        x=x,
        y=y,
        z=rng.uniform(-600.0, 600.0, n) if astig else np.zeros(n),
        photons=rng.lognormal(math.log(3000.0), 0.5, n),
        bg=rng.uniform(50.0, 200.0, B),
    )


def training_target_entries(em: Emitters, H: int, W: int, z_scale=1000.0, ph_scale=10000.0):
    """The nonzero entries of the per-pixel targets [B,5,H,W] of a batch, as (flat indices,
    float32 values): channel 0 is 1 at the pixel containing an emitter (the brighter emitter
    wins a shared pixel); channels 1-4 hold dx, dy (emitter minus pixel centre, px),
    z / z_scale and photons / ph_scale there."""
    j = np.clip(np.rint(em.x).astype(np.int64), 0, W - 1)
    i = np.clip(np.rint(em.y).astype(np.int64), 0, H - 1)
    f = em.frame.astype(np.int64)
    order = np.argsort(em.photons, kind="stable")  # ascending: the last write of a pixel is the brightest
    px = (f * 5 * H + i) * W + j  # flat index of channel 0
    last = {}
    for k in order:
        last[px[k]] = k
    win = np.array(sorted(last.values()), dtype=np.int64)
    idx = np.concatenate([px[win] + c * H * W for c in range(5)])
    val = np.concatenate([np.ones(win.size), em.x[win] - j[win], em.y[win] - i[win], em.z[win] / z_scale,
                          em.photons[win] / ph_scale]).astype(np.float32)
    return idx, val


def training_batch(rng, B=256, H=64, W=64, max_emitters=10, astig=True, z_scale=1000.0, ph_scale=10000.0,
                   min_emitters=0):
    """Simulated training patches and per-pixel targets.

    Returns (frames u16 [B,H,W], targets f32 [B,5,H,W], emitters, camera); targets as
    training_target_entries describes them."""
    em = training_emitters(rng, B, H, W, max_emitters, astig, min_emitters)
    cam = Camera(1.0, 100.0)
    frames = simulate(em, B, H, W, cam, astig, rng)
    tgt = np.zeros((B, 5, H, W), dtype=np.float32)
    idx, val = training_target_entries(em, H, W, z_scale, ph_scale)
    tgt.reshape(-1)[idx] = val
    return frames, tgt, em, cam
