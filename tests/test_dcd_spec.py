"""Host logic of the net spec's extensions: dense connection dilated blocks (Sec. 3.2.1, the
"dcd" key and version-2 weight blobs) and the uncertainty heads (Sec. 3.2, the "heads" list).
The library checks spec and blob before it touches a device, so a malformed or unsupported
request is refused the same way with or without a GPU."""
import json
import struct

import pytest
import torch

import oracle
import paper_2410_02314_gb300 as sml
from paper_2410_02314_gb300 import synth


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2410_02314_gb300 import _build

    _build.build()


def _net(C=32, g=16, blocks=((2, 4), (1, 8, 3)), dil=(1, 2, 1), prec="bf16", in_ch=1, seed=3):
    spec = synth.NetSpec(in_ch=in_ch, channels=C, dilations=tuple(dil), precision=prec,
                         dcd={"growth": g, "blocks": [list(b) for b in blocks]})
    return spec, spec.to_json(), synth.pack_blob(spec, synth.init_weights(spec, seed))


def _code(js, blob):
    with pytest.raises(sml.SmlError) as e:
        sml.sml_create(js, blob)
    return e.value.code


def _edit(js, **kw):
    d = json.loads(js)
    d["dcd"].update(kw.pop("dcd", {}))
    d.update(kw)
    return json.dumps(d)


def test_layer_plan_of_the_dcd_spec():
    """Execution order and channel counts: stem, dense layers with inputs C + j g, transition
    C + k g -> C at d = 1, then the plain layers."""
    spec, _, _ = _net()
    assert spec.layers() == [(1, 32, 1), (32, 16, 2), (48, 16, 4), (64, 32, 1), (32, 16, 1), (48, 16, 8),
                             (64, 16, 3), (80, 32, 1), (32, 32, 2), (32, 32, 1)]
    assert spec.R == 1 + 2 + 4 + 1 + 1 + 8 + 3 + 1 + 2 + 1
    big = synth.spec_dcd()
    assert big.L == 22 and big.R == 126 and max(c for c, _, _ in big.layers()) == 96


@pytest.mark.parametrize("edit,code", [
    (dict(dcd={"growth": 8}), sml.SML_ERR_BAD_SPEC),                       # growth not a multiple of 16
    (dict(dcd={"blocks": []}), sml.SML_ERR_BAD_SPEC),                      # no block
    (dict(dcd={"blocks": [[2, 4], []]}), sml.SML_ERR_BAD_SPEC),            # empty block
    (dict(dcd={"blocks": [[2, 0]]}), sml.SML_ERR_BAD_SPEC),                # dilation 0
    (dict(dcd={"blocks": [[2, 65]]}), sml.SML_ERR_BAD_SPEC),               # dilation beyond 64
    (dict(dilations=[1]), sml.SML_ERR_BAD_SPEC),                            # no plain layer for the heads
    (dict(dcd={"growth": 32, "blocks": [[1, 2, 4, 8]]}), sml.SML_ERR_BAD_SPEC),  # 160-channel concatenation
    (dict(dcd={"blocks": [[1]] * 16}), sml.SML_ERR_BAD_SPEC),              # 35 conv layers (at most 32)
    (dict(precision="fp8"), sml.SML_ERR_BAD_SPEC),                          # fp8 without activation scales
    (dict(precision="fp8", act_scales=[1.0] * 9), sml.SML_ERR_BAD_SPEC),   # one scale short of the 10 layers
])
def test_bad_dcd_specs_are_refused(edit, code):
    _, js, blob = _net()
    assert _code(_edit(js, **edit), blob) == code


@pytest.mark.parametrize("prec", ["bf16", "fp32"])
def test_layers_beyond_shared_memory_are_unsupported(prec):
    """C = 64 with four dense layers of growth 16: the 128 -> 64 transition's weights do not fit
    one CTA's shared memory next to a four-stage ring (BF16) or as FP32 (128 x 64 x 9 floats)."""
    _, js, blob = _net(C=64, g=16, blocks=((1, 2, 4, 8),), dil=(1, 1), prec=prec)
    assert _code(js, blob) == sml.SML_ERR_UNSUPPORTED


def test_blob_must_match_the_dense_spec():
    spec, js, blob = _net()
    # a version-1 blob of a plain net of the same C and layer count
    plain = synth.NetSpec(in_ch=1, channels=32, dilations=(1,) * spec.L, precision="bf16")
    assert _code(js, synth.pack_blob(plain, synth.init_weights(plain, 1))) == sml.SML_ERR_BAD_WEIGHTS
    # another growth in the header
    _, _, blob32 = _net(g=32)
    assert _code(js, blob32) == sml.SML_ERR_BAD_WEIGHTS
    # another dilation of one dense layer
    _, _, other = _net(blocks=((2, 4), (1, 8, 5)))
    assert _code(js, other) == sml.SML_ERR_BAD_WEIGHTS
    # truncated payload
    assert _code(js, blob[:-4]) == sml.SML_ERR_BAD_WEIGHTS
    # a plain spec refuses the version-2 blob
    assert _code(plain.to_json(), blob) == sml.SML_ERR_BAD_WEIGHTS


def test_valid_dcd_net_reaches_the_device_check():
    """Spec and blob pass the host checks; without a GPU the call then fails loudly."""
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    for prec in ("bf16", "fp32"):
        _, js, blob = _net(prec=prec)
        assert _code(js, blob) == sml.SML_ERR_CUDA
    _, js, blob = _net()
    assert _code(_edit(js, precision="fp8", act_scales=[0.01] * 10), blob) == sml.SML_ERR_CUDA
    spec = synth.spec_dcd()
    assert _code(spec.to_json(), synth.pack_blob(spec, synth.init_weights(spec, 1))) == sml.SML_ERR_CUDA


# ----------------------------------------------------------------------------- heads


def _plain(n_heads=5, prec="bf16"):
    spec = synth.NetSpec(in_ch=1, channels=32, dilations=(1, 2, 1), precision=prec, n_heads=n_heads)
    return spec, spec.to_json(), synth.pack_blob(spec, synth.init_weights(spec, 5))


def test_heads_spec_lists_five_or_nine_named_outputs():
    _, js, blob = _plain(9)
    d = json.loads(js)
    assert d["heads"] == ["p", "dx", "dy", "z", "N", "sx", "sy", "sz", "sN"]
    for heads in (d["heads"][:7], d["heads"][:4], ["p", "dx", "dy", "z", "N", "sy", "sx", "sz", "sN"], "p"):
        assert _code(json.dumps(dict(d, heads=heads)), blob) == sml.SML_ERR_BAD_SPEC


def test_blob_head_count_must_match_the_spec():
    _, js9, blob9 = _plain(9)
    _, js5, blob5 = _plain(5)
    assert _code(js9, blob5) == sml.SML_ERR_BAD_WEIGHTS
    assert _code(js5, blob9) == sml.SML_ERR_BAD_WEIGHTS


def test_valid_nine_head_nets_reach_the_device_check():
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    for prec in ("fp32", "bf16", "fp8"):
        spec, js, blob = _plain(9, prec)
        if prec == "fp8":
            js = json.dumps(dict(json.loads(js), act_scales=[1.0] * spec.L))
        assert _code(js, blob) == sml.SML_ERR_CUDA
    spec = synth.NetSpec(in_ch=1, channels=32, dilations=(1, 1), n_heads=9, precision="bf16",
                         dcd={"growth": 16, "blocks": [[2, 4]]})
    assert _code(spec.to_json(), synth.pack_blob(spec, synth.init_weights(spec, 2))) == sml.SML_ERR_CUDA


# ----------------------------------------------------------------------------- U-Net


def _unet(levels=2, C=32, prec="bf16", dcd=None, dil=(1, 2, 1), n_heads=5):
    spec = synth.NetSpec(in_ch=1, channels=C, dilations=tuple(dil), precision=prec, unet=levels, dcd=dcd,
                         n_heads=n_heads)
    return spec, spec.to_json(), synth.pack_blob(spec, synth.init_weights(spec, 8))


def test_unet_layer_plan():
    """The U-Net sits before the last layer: levels down convs C -> C, then levels up convs
    2C -> C, all d = 1; version-2 blob with growth 0."""
    spec, js, blob = _unet(2)
    assert spec.layers() == [(1, 32, 1), (32, 32, 2), (32, 32, 1), (32, 32, 1), (64, 32, 1), (64, 32, 1), (32, 32, 1)]
    assert json.loads(js)["unet"] == {"levels": 2} and blob[8:12] == (2).to_bytes(4, "little")
    assert spec.R == 1 + 2 + 1 + 24


@pytest.mark.parametrize("edit,code", [
    (dict(unet={"levels": 3}), sml.SML_ERR_BAD_SPEC),
    (dict(unet={"levels": 0}), sml.SML_ERR_BAD_SPEC),
    (dict(unet={}), sml.SML_ERR_BAD_SPEC),
    (dict(unet=2), sml.SML_ERR_BAD_SPEC),
    (dict(precision="fp8", act_scales=[1.0] * 6), sml.SML_ERR_BAD_SPEC),  # one scale short of the 7 layers
])
def test_bad_unet_specs_are_refused(edit, code):
    _, js, blob = _unet(2)
    assert _code(json.dumps(dict(json.loads(js), **edit)), blob) == code


@pytest.mark.parametrize("prec", ["bf16", "fp32"])
def test_unet_up_conv_beyond_shared_memory_is_unsupported(prec):
    """C = 64: the 128 -> 64 up convs do not fit (as for the dense-block transition)."""
    _, js, blob = _unet(1, C=64, prec=prec)
    assert _code(js, blob) == sml.SML_ERR_UNSUPPORTED


def test_unet_blob_must_match():
    _, js, blob = _unet(2)
    _, _, blob1 = _unet(1)
    assert _code(js, blob1) == sml.SML_ERR_BAD_WEIGHTS
    plain = synth.NetSpec(in_ch=1, channels=32, dilations=(1, 2, 1), precision="bf16")
    assert _code(js, synth.pack_blob(plain, synth.init_weights(plain, 1))) == sml.SML_ERR_BAD_WEIGHTS


def test_valid_unet_nets_reach_the_device_check():
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    for kw in (dict(levels=1), dict(levels=2, prec="fp32"), dict(levels=2, dcd={"growth": 16, "blocks": [[2, 4]]}, n_heads=9),
               dict(levels=2, C=48)):
        _, js, blob = _unet(**kw)
        assert _code(js, blob) == sml.SML_ERR_CUDA, kw
    _, js, blob = _unet(2)
    assert _code(json.dumps(dict(json.loads(js), precision="fp8", act_scales=[0.01] * 7)), blob) == sml.SML_ERR_CUDA


# ----------------------------------------------------------------------------- deep plain stacks


def test_plain_stacks_beyond_16_layers_use_the_version_2_blob():
    """Plain stacks of 17..32 layers carry every dilation in the version-2 header (reserved =
    0); they pass the host checks, 33 layers do not, and a blob of another depth is refused."""
    deep = synth.NetSpec(in_ch=1, channels=48, dilations=(1,) + (1, 2, 4, 8, 16, 8, 4) * 4, precision="bf16")
    assert deep.L == 29
    blob = synth.pack_blob(deep, synth.init_weights(deep, 3))
    assert struct.unpack_from("<8s7I", blob, 0)[1] == 2
    net = oracle.Net(deep.to_json(), blob)
    assert net.L == 29 and net.dil == list(deep.dilations)
    if not torch.cuda.is_available():
        assert _code(deep.to_json(), blob) == sml.SML_ERR_CUDA
    too_deep = synth.NetSpec(in_ch=1, channels=16, dilations=(1,) * 33, precision="bf16")
    assert _code(too_deep.to_json(), blob) == sml.SML_ERR_BAD_SPEC
    shorter = synth.NetSpec(in_ch=1, channels=48, dilations=deep.dilations[:-1], precision="bf16")
    assert _code(shorter.to_json(), blob) == sml.SML_ERR_BAD_WEIGHTS
    with pytest.raises(ValueError):
        synth.pack_blob(deep, synth.init_weights(deep, 3, bn=True))
