"""GB300 single-molecule localization: Python binding of the C ABI in include/sml.h.

The functions below carry the C names and only marshal arguments (ctypes); every step of
the path runs in the CUDA library ``_lib/libsml.so``.  There is no CPU fallback: if the
library is missing or the device is not an sm_103 GPU, calls raise.

Arrays may be numpy arrays (host memory) or torch tensors (host or CUDA memory); device
entry points (``*_async``, ``sml_forward_maps``, ``sml_decode_maps``) need CUDA tensors.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libsml.so")

SML_OK = 0
SML_ERR_BAD_ARG = -1
SML_ERR_BAD_SPEC = -2
SML_ERR_BAD_WEIGHTS = -3
SML_ERR_OOM = -4
SML_ERR_CUDA = -5
SML_ERR_CAPACITY = -6
SML_ERR_UNSUPPORTED = -7

RECORD_DTYPE = np.dtype(
    [("frame", "<i4"), ("x", "<f4"), ("y", "<f4"), ("z", "<f4"), ("photons", "<f4"), ("p", "<f4")]
)
# sml_sigma: uncertainties of one record (nets with 9 heads)
SIGMA_DTYPE = np.dtype([("sigma_x", "<f4"), ("sigma_y", "<f4"), ("sigma_z", "<f4"), ("sigma_photons", "<f4")])

# every symbol the headers in include/ declare
EXPORTS = (
    "sml_create",
    "sml_destroy",
    "sml_last_error",
    "sml_localize",
    "sml_num_heads",
    "sml_num_layers",
    "sml_workspace_bytes",
    "sml_error_word",
    "sml_localize_sigma",
    "sml_localize_async",
    "sml_forward_maps",
    "sml_decode_maps",
    "sml_decode_maps_static",
    "sml_last_launch_count",
    "sml_activation_amax",
    "sml_calibrate_fp8",
    "sml_profile_enable",
    "sml_profile_read",
    "sml_debug_umma",
    "sml_debug_set_error_word",
    "sml_debug_umma_mn",
    "sml_train_ingest",
    "sml_train_conv_fwd",
    "sml_train_conv_bwd_work_bytes",
    "sml_train_conv_bwd",
    "sml_train_heads_work_bytes",
    "sml_train_heads_loss",
    "sml_train_bf16_bimg_bytes",
    "sml_train_bf16_pack",
    "sml_train_bf16_layer0",
    "sml_train_bf16_conv_fwd",
    "sml_train_bf16_conv_dgrad",
    "sml_train_bf16_wgrad_work_bytes",
    "sml_train_bf16_conv_wgrad",
    "sml_train_bf16_heads_loss",
    "sml_train_bf16_l0_wgrad",
    "sml_reader_open",
    "sml_reader_next",
    "sml_reader_release",
    "sml_reader_stats",
    "sml_reader_close",
    "sml_localize_file",
    "sml_sim_frames",
)
SML_KERNEL_LAYER1, SML_KERNEL_CONV, SML_KERNEL_CONV_HEADS, SML_KERNEL_DECODE = 0, 1, 2, 3


class IoStats(ctypes.Structure):
    """Mirror of sml_io_stats (include/sml_io.h)."""

    _fields_ = [("bytes_read", ctypes.c_double), ("read_seconds", ctypes.c_double),
                ("wall_seconds", ctypes.c_double), ("frames", ctypes.c_longlong)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class SmlError(RuntimeError):
    def __init__(self, code, msg, needed=None):
        super().__init__(f"sml error {code}: {msg}")
        self.code = code
        self.needed = needed


class _Camera(ctypes.Structure):
    _fields_ = [("gain", ctypes.c_float), ("offset", ctypes.c_float), ("gain_map", ctypes.c_void_p),
                ("offset_map", ctypes.c_void_p)]


class _Thresholds(ctypes.Structure):
    _fields_ = [("p_min", ctypes.c_float)]


_lib = None


def lib():
    """Load libsml.so (built in-tree by ``__graft_entry__.build()`` / ``_build.build()``)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"CUDA library not built: {LIB_PATH} is missing (run __graft_entry__.build())")
        L = ctypes.CDLL(LIB_PATH)
        P, I, F, S = ctypes.c_void_p, ctypes.c_int, ctypes.c_float, ctypes.c_size_t
        L.sml_create.argtypes = [ctypes.c_char_p, P, S, ctypes.POINTER(P)]
        L.sml_create.restype = I
        L.sml_destroy.argtypes = [P]
        L.sml_destroy.restype = None
        L.sml_last_error.argtypes = [P]
        L.sml_last_error.restype = ctypes.c_char_p
        L.sml_localize.argtypes = [P, P, I, I, I, ctypes.POINTER(_Camera), ctypes.POINTER(_Thresholds), P, S,
                                   ctypes.POINTER(S)]
        L.sml_localize.restype = I
        L.sml_num_heads.argtypes = [P]
        L.sml_num_heads.restype = I
        L.sml_num_layers.argtypes = [P]
        L.sml_num_layers.restype = I
        L.sml_workspace_bytes.argtypes = [P, I, I, I, ctypes.POINTER(S), ctypes.POINTER(I), ctypes.POINTER(S)]
        L.sml_workspace_bytes.restype = I
        L.sml_error_word.argtypes = [P, P, P]
        L.sml_error_word.restype = I
        L.sml_localize_sigma.argtypes = [P, P, I, I, I, ctypes.POINTER(_Camera), ctypes.POINTER(_Thresholds), P, P, S,
                                         ctypes.POINTER(S)]
        L.sml_localize_sigma.restype = I
        L.sml_localize_async.argtypes = [P, P, I, I, I, ctypes.POINTER(_Camera), ctypes.POINTER(_Thresholds), P, S,
                                         P, P]
        L.sml_localize_async.restype = I
        L.sml_forward_maps.argtypes = [P, P, I, I, I, ctypes.POINTER(_Camera), P, P, P]
        L.sml_forward_maps.restype = I
        L.sml_decode_maps.argtypes = [P, P, I, I, I, ctypes.POINTER(_Thresholds), P, S, P, P]
        L.sml_decode_maps.restype = I
        L.sml_decode_maps_static.argtypes = [P, I, I, I, F, F, F, P, S, P, P]
        L.sml_decode_maps_static.restype = I
        L.sml_last_launch_count.argtypes = [P]
        L.sml_last_launch_count.restype = I
        L.sml_activation_amax.argtypes = [P, P, I, I, I, ctypes.POINTER(_Camera), P]
        L.sml_activation_amax.restype = I
        L.sml_calibrate_fp8.argtypes = [P, P, I, I, I, ctypes.POINTER(_Camera), F, P]
        L.sml_calibrate_fp8.restype = I
        L.sml_profile_enable.argtypes = [P, I]
        L.sml_profile_enable.restype = I
        L.sml_profile_read.argtypes = [P, I, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(I)]
        L.sml_profile_read.restype = I
        L.sml_debug_umma.argtypes = [P, P, P, I, I, I, I, P]
        L.sml_debug_umma.restype = I
        L.sml_debug_set_error_word.argtypes = [P, I]
        L.sml_debug_set_error_word.restype = I
        L.sml_debug_umma_mn.argtypes = [P, P, P, I, I, I, I, I, I, I, I, P]
        L.sml_debug_umma_mn.restype = I
        LL = ctypes.c_longlong
        L.sml_reader_open.argtypes = [ctypes.c_char_p, LL, I, I, I, I, I, ctypes.POINTER(P)]
        L.sml_reader_open.restype = I
        L.sml_reader_next.argtypes = [P, ctypes.POINTER(P), ctypes.POINTER(I), ctypes.POINTER(LL), I]
        L.sml_reader_next.restype = I
        L.sml_reader_release.argtypes = [P, P]
        L.sml_reader_release.restype = I
        L.sml_reader_stats.argtypes = [P, ctypes.POINTER(IoStats)]
        L.sml_reader_stats.restype = I
        L.sml_reader_close.argtypes = [P]
        L.sml_reader_close.restype = None
        L.sml_localize_file.argtypes = [P, ctypes.c_char_p, LL, I, I, I, ctypes.POINTER(_Camera),
                                        ctypes.POINTER(_Thresholds), I, P, S, ctypes.POINTER(S), ctypes.POINTER(IoStats)]
        L.sml_localize_file.restype = I
        L.sml_sim_frames.argtypes = [P, P, P, P, P, LL, P, I, I, I, I, F, ctypes.POINTER(_Camera), ctypes.c_ulonglong,
                                     LL, I, P, P]
        L.sml_sim_frames.restype = I
        _lib = L
    return _lib


def _ptr(a):
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return a.data_ptr()
    return a.ctypes.data


def _stream(stream):
    if stream is None:
        import torch

        return torch.cuda.current_stream().cuda_stream
    return getattr(stream, "cuda_stream", stream)


def _camera(gain=1.0, offset=100.0, gain_map=None, offset_map=None):
    return _Camera(float(gain), float(offset), _ptr(gain_map), _ptr(offset_map))


def _check(ctx, code):
    if code != SML_OK:
        raise SmlError(code, sml_last_error(ctx))


# ----------------------------------------------------------------------------- C names


def sml_create(net_spec: str, weights: bytes):
    h = ctypes.c_void_p()
    buf = ctypes.create_string_buffer(weights, len(weights))
    code = lib().sml_create(net_spec.encode(), buf, len(weights), ctypes.byref(h))
    if code != SML_OK:
        raise SmlError(code, sml_last_error(None))
    return h


def sml_destroy(ctx):
    lib().sml_destroy(ctx)


def sml_last_error(ctx) -> str:
    m = lib().sml_last_error(ctx)
    return m.decode() if m else ""


def sml_last_launch_count(ctx) -> int:
    return lib().sml_last_launch_count(ctx)


def sml_localize(ctx, frames, p_min, gain=1.0, offset=100.0, gain_map=None, offset_map=None, capacity=None,
                 out=None):
    """Synchronous localization.  frames: uint16 [T,H,W] (numpy, or torch host/CUDA tensor).
    Returns a numpy record array (RECORD_DTYPE); when ``out`` is a torch byte tensor (host,
    pinned or CUDA) the records are written there and its first n*24 bytes are returned."""
    T, H, W = (int(s) for s in frames.shape)
    if isinstance(frames, np.ndarray):
        frames = np.ascontiguousarray(frames, dtype=np.uint16)
    if out is None:
        cap = int(capacity if capacity is not None else max(16, T * H * W // 9 + 16))
        out_arr = np.empty(cap, dtype=RECORD_DTYPE)
    elif hasattr(out, "data_ptr"):  # torch byte tensor (host, pinned or CUDA)
        out_arr = out
        cap = int(out.numel() * out.element_size() // RECORD_DTYPE.itemsize)
    else:
        out_arr = out
        cap = len(out)
    n = ctypes.c_size_t(0)
    cam = _camera(gain, offset, gain_map, offset_map)
    thr = _Thresholds(float(p_min))
    code = lib().sml_localize(ctx, _ptr(frames), T, H, W, ctypes.byref(cam), ctypes.byref(thr), _ptr(out_arr), cap,
                              ctypes.byref(n))
    if code == SML_ERR_CAPACITY:
        raise SmlError(code, sml_last_error(ctx), needed=int(n.value))
    _check(ctx, code)
    if hasattr(out_arr, "data_ptr"):
        return out_arr[: n.value * RECORD_DTYPE.itemsize]
    return out_arr[: n.value]


def sml_sim_frames(emitters, T, H, W, astig=False, sigma0=1.3, gain=1.0, offset=100.0, gain_map=None,
                   offset_map=None, seed=0, frame0=0, noise=True, d_adu=None, d_mu=None):
    """Simulated frames on the device (include/sml_sim.h).  emitters: an object with numpy
    arrays frame, x, y, z, photons (one entry per emitter) and bg (one per frame), e.g.
    synth.Emitters.  Returns d_adu: a CUDA int16 tensor [T,H,W] holding the uint16 ADU bits
    (view it as uint16 on the host), allocated unless given; d_mu (optional CUDA float32
    [T,H,W]) receives the expected image."""
    import torch

    fr = np.ascontiguousarray(emitters.frame, dtype=np.int32)
    xs = np.ascontiguousarray(emitters.x, dtype=np.float32)
    ys = np.ascontiguousarray(emitters.y, dtype=np.float32)
    zs = np.ascontiguousarray(emitters.z, dtype=np.float32)
    ph = np.ascontiguousarray(emitters.photons, dtype=np.float32)
    bg = np.ascontiguousarray(emitters.bg, dtype=np.float32)
    if bg.size != T:
        raise ValueError("bg needs one entry per frame")
    if d_adu is None:
        d_adu = torch.empty((T, H, W), dtype=torch.int16, device="cuda")
    cam = _camera(gain, offset, gain_map, offset_map)
    code = lib().sml_sim_frames(fr.ctypes.data, xs.ctypes.data, ys.ctypes.data, zs.ctypes.data, ph.ctypes.data,
                                int(fr.size), bg.ctypes.data, int(T), int(H), int(W), int(bool(astig)), float(sigma0),
                                ctypes.byref(cam), int(seed) & 0xFFFFFFFFFFFFFFFF, int(frame0), int(bool(noise)),
                                _ptr(d_adu), _ptr(d_mu))
    if code != SML_OK:
        raise SmlError(code, "sml_sim_frames failed")
    return d_adu


def sml_num_heads(ctx) -> int:
    return lib().sml_num_heads(ctx)


def sml_num_layers(ctx) -> int:
    return lib().sml_num_layers(ctx)


def sml_workspace_bytes(ctx, T, H, W):
    """(bytes of the plan a call on T frames of H x W uses, whether the context holds it now,
    bytes of all plans the context holds)."""
    pb, res, tot = ctypes.c_size_t(0), ctypes.c_int(0), ctypes.c_size_t(0)
    _check(ctx, lib().sml_workspace_bytes(ctx, int(T), int(H), int(W), ctypes.byref(pb), ctypes.byref(res),
                                          ctypes.byref(tot)))
    return int(pb.value), bool(res.value), int(tot.value)


def sml_error_word(ctx, d_word, stream=None):
    """Enqueue the copy of the context's device error word into d_word (CUDA int32 tensor) and
    clear it (stream ordered)."""
    _check(ctx, lib().sml_error_word(ctx, _ptr(d_word), _stream(stream)))


def sml_localize_sigma(ctx, frames, p_min, gain=1.0, offset=100.0, gain_map=None, offset_map=None, capacity=None):
    """sml_localize plus the uncertainties of each record (9-head nets): returns (records,
    sigmas) as numpy arrays of RECORD_DTYPE and SIGMA_DTYPE, sigmas[k] belonging to records[k]."""
    T, H, W = (int(s) for s in frames.shape)
    if isinstance(frames, np.ndarray):
        frames = np.ascontiguousarray(frames, dtype=np.uint16)
    cap = int(capacity if capacity is not None else max(16, T * H * W // 9 + 16))
    out = np.empty(cap, dtype=RECORD_DTYPE)
    sig = np.empty(cap, dtype=SIGMA_DTYPE)
    n = ctypes.c_size_t(0)
    cam = _camera(gain, offset, gain_map, offset_map)
    thr = _Thresholds(float(p_min))
    code = lib().sml_localize_sigma(ctx, _ptr(frames), T, H, W, ctypes.byref(cam), ctypes.byref(thr), out.ctypes.data,
                                    sig.ctypes.data, cap, ctypes.byref(n))
    if code == SML_ERR_CAPACITY:
        raise SmlError(code, sml_last_error(ctx), needed=int(n.value))
    _check(ctx, code)
    return out[: n.value], sig[: n.value]


def sml_localize_file(ctx, path, T, H, W, p_min, batch=64, gain=1.0, offset=100.0, gain_map=None, offset_map=None,
                      capacity=None, file_offset=0):
    """Localize a raw uint16 stack file (include/sml_io.h): returns (records, stats dict)."""
    cap = int(capacity if capacity is not None else max(16, T * ((H + 1) // 2) * ((W + 1) // 2)))
    out = np.empty(cap, dtype=RECORD_DTYPE)
    n = ctypes.c_size_t(0)
    st = IoStats()
    cam = _camera(gain, offset, gain_map, offset_map)
    thr = _Thresholds(float(p_min))
    code = lib().sml_localize_file(ctx, os.fsencode(path), int(file_offset), int(T), int(H), int(W), ctypes.byref(cam),
                                   ctypes.byref(thr), int(batch), out.ctypes.data, cap, ctypes.byref(n),
                                   ctypes.byref(st))
    if code == SML_ERR_CAPACITY:
        raise SmlError(code, sml_last_error(ctx), needed=int(n.value))
    _check(ctx, code)
    return out[: n.value], st.as_dict()


class StackReader:
    """Read-ahead over a raw uint16 stack file (include/sml_io.h).  Iterating yields
    (first_frame, frames) with frames a numpy uint16 [n, H, W] view of a pinned buffer that
    stays valid until the next iteration step (the buffer is then given back)."""

    def __init__(self, path, T, H, W, batch=64, n_buffers=3, file_offset=0, timeout_ms=60000):
        self.H, self.W, self.timeout_ms = int(H), int(W), int(timeout_ms)
        h = ctypes.c_void_p()
        code = lib().sml_reader_open(os.fsencode(path), int(file_offset), int(T), int(H), int(W), int(batch),
                                     int(n_buffers), ctypes.byref(h))
        if code != SML_OK:
            raise SmlError(code, f"cannot open stack {path}")
        self.handle = h.value

    def __iter__(self):
        held = None
        try:
            while True:
                p, n, first = ctypes.c_void_p(), ctypes.c_int(0), ctypes.c_longlong(0)
                code = lib().sml_reader_next(self.handle, ctypes.byref(p), ctypes.byref(n), ctypes.byref(first),
                                             self.timeout_ms)
                if held is not None:
                    lib().sml_reader_release(self.handle, held)
                    held = None
                if code != SML_OK:
                    raise SmlError(code, "stack read failed")
                if n.value == 0:
                    return
                held = p.value
                buf = (ctypes.c_uint16 * (n.value * self.H * self.W)).from_address(p.value)
                yield int(first.value), np.frombuffer(buf, dtype=np.uint16).reshape(n.value, self.H, self.W)
        finally:
            if held is not None and self.handle is not None:
                lib().sml_reader_release(self.handle, held)

    def stats(self):
        st = IoStats()
        lib().sml_reader_stats(self.handle, ctypes.byref(st))
        return st.as_dict()

    def close(self):
        if self.handle is not None:
            lib().sml_reader_close(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def sml_localize_async(ctx, d_frames, p_min, d_out, d_n, gain=1.0, offset=100.0, gain_map=None, offset_map=None,
                       stream=None):
    """Device-resident localization on a stream.  d_out: CUDA uint8 tensor holding records;
    d_n: CUDA int64 tensor (1 element) receiving the detection count."""
    T, H, W = (int(s) for s in d_frames.shape)
    cap = int(d_out.numel() * d_out.element_size() // RECORD_DTYPE.itemsize)
    cam = _camera(gain, offset, gain_map, offset_map)
    thr = _Thresholds(float(p_min))
    _check(ctx, lib().sml_localize_async(ctx, _ptr(d_frames), T, H, W, ctypes.byref(cam), ctypes.byref(thr),
                                         _ptr(d_out), cap, _ptr(d_n), _stream(stream)))


def sml_forward_maps(ctx, d_frames, d_maps, d_logits=None, gain=1.0, offset=100.0, gain_map=None, offset_map=None,
                     stream=None):
    T, H, W = (int(s) for s in d_frames.shape)
    cam = _camera(gain, offset, gain_map, offset_map)
    _check(ctx, lib().sml_forward_maps(ctx, _ptr(d_frames), T, H, W, ctypes.byref(cam), _ptr(d_maps),
                                       _ptr(d_logits), _stream(stream)))


def sml_decode_maps(ctx, d_maps, p_min, d_out, d_n, stream=None):
    T, _, H, W = (int(s) for s in d_maps.shape)
    cap = int(d_out.numel() * d_out.element_size() // RECORD_DTYPE.itemsize)
    thr = _Thresholds(float(p_min))
    _check(ctx, lib().sml_decode_maps(ctx, _ptr(d_maps), T, H, W, ctypes.byref(thr), _ptr(d_out), cap, _ptr(d_n),
                                      _stream(stream)))


def sml_activation_amax(ctx, d_frames, gain=1.0, offset=100.0, gain_map=None, offset_map=None):
    """Per-layer maxima of the activations entering each conv layer (numpy float32 [L])."""
    T, H, W = (int(s) for s in d_frames.shape)
    out = np.zeros(64, dtype=np.float32)
    cam = _camera(gain, offset, gain_map, offset_map)
    _check(ctx, lib().sml_activation_amax(ctx, _ptr(d_frames), T, H, W, ctypes.byref(cam), out.ctypes.data))
    return out


def sml_calibrate_fp8(ctx, d_frames, margin=1.0, gain=1.0, offset=100.0, gain_map=None, offset_map=None):
    """Activation scales of the fp8 precision from a calibration pass (numpy float32 [L])."""
    T, H, W = (int(s) for s in d_frames.shape)
    out = np.zeros(64, dtype=np.float32)
    cam = _camera(gain, offset, gain_map, offset_map)
    _check(ctx, lib().sml_calibrate_fp8(ctx, _ptr(d_frames), T, H, W, ctypes.byref(cam), float(margin),
                                        out.ctypes.data))
    return out


def calibrate_fp8(net_spec: str, weights: bytes, d_frames, margin=1.0, **cam):
    """The fp8 net spec of a net: its act_scales come from sml_calibrate_fp8 on a bf16 context
    of the same net over the calibration frames."""
    import json

    spec = json.loads(net_spec)
    ctx = sml_create(json.dumps(dict(spec, precision="bf16")), weights)
    try:
        L = sml_num_layers(ctx)
        scales = sml_calibrate_fp8(ctx, d_frames, margin, **cam)[:L]
    finally:
        sml_destroy(ctx)
    return json.dumps(dict(spec, precision="fp8", act_scales=[float(x) for x in scales]))


def sml_profile_enable(ctx, on: bool):
    _check(ctx, lib().sml_profile_enable(ctx, int(bool(on))))


def sml_profile_read(ctx, kernel_class: int):
    """(summed device milliseconds, number of timed launches) for one kernel class."""
    ms = ctypes.c_double(0.0)
    n = ctypes.c_int(0)
    _check(ctx, lib().sml_profile_read(ctx, int(kernel_class), ctypes.byref(ms), ctypes.byref(n)))
    return ms.value, n.value


def sml_decode_maps_static(d_maps, p_min, z_scale, ph_scale, d_out, d_n, stream=None):
    """Allocation-free decode (see include/sml.h): same records as sml_decode_maps."""
    T, _, H, W = (int(s) for s in d_maps.shape)
    cap = int(d_out.numel() * d_out.element_size() // RECORD_DTYPE.itemsize)
    code = lib().sml_decode_maps_static(_ptr(d_maps), T, H, W, float(p_min), float(z_scale), float(ph_scale),
                                        _ptr(d_out), cap, _ptr(d_n), _stream(stream))
    if code != SML_OK:
        raise SmlError(code, "sml_decode_maps_static failed")


def sml_debug_umma(d_a, d_b, d_d, n, k, kind="bf16", d_col=0, stream=None):
    """kind: "bf16", "e4m3" or "tf32" (see include/sml_debug.h)."""
    code = lib().sml_debug_umma(_ptr(d_a), _ptr(d_b), _ptr(d_d), int(n), int(k), {"bf16": 0, "e4m3": 1, "tf32": 2}[kind],
                                int(d_col), _stream(stream))
    if code != SML_OK:
        raise SmlError(code, "umma self-test failed")


# ----------------------------------------------------------------------------- helpers


def records_from_bytes(t, n):
    """View the first n records of a CUDA/CPU uint8 tensor as a numpy record array."""
    raw = t[: n * RECORD_DTYPE.itemsize].cpu().numpy()
    return raw.view(RECORD_DTYPE).copy()


class Localizer:
    """Owns one context: ``Localizer(spec_json, blob).localize(frames, p_min)``."""

    def __init__(self, net_spec: str, weights: bytes):
        self.ctx = sml_create(net_spec, weights)

    def close(self):
        if self.ctx is not None:
            sml_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def localize(self, frames, p_min, **kw):
        return sml_localize(self.ctx, frames, p_min, **kw)

    def localize_sigma(self, frames, p_min, **kw):
        return sml_localize_sigma(self.ctx, frames, p_min, **kw)

    @property
    def num_heads(self):
        return sml_num_heads(self.ctx)

    def localize_file(self, path, T, H, W, p_min, **kw):
        return sml_localize_file(self.ctx, path, T, H, W, p_min, **kw)

    def forward_maps(self, d_frames, d_maps, d_logits=None, **kw):
        sml_forward_maps(self.ctx, d_frames, d_maps, d_logits, **kw)

    def decode_maps(self, d_maps, p_min, d_out, d_n, **kw):
        sml_decode_maps(self.ctx, d_maps, p_min, d_out, d_n, **kw)

    def localize_async(self, d_frames, p_min, d_out, d_n, **kw):
        sml_localize_async(self.ctx, d_frames, p_min, d_out, d_n, **kw)

    @property
    def last_launch_count(self):
        return sml_last_launch_count(self.ctx)
