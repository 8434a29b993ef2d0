"""The C-ABI library builds for sm_103a, loads, and exports every function the headers in
include/ declare (no compute calls: this runs without a GPU)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s*(sml_[a-z_0-9]+)\s*\(", text, re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def libsml():
    from paper_2410_02314_gb300 import _build

    path = _build.build()
    return ctypes.CDLL(path)


def test_headers_declare_the_boundary():
    names = declared_functions()
    for n in ("sml_create", "sml_destroy", "sml_last_error", "sml_localize", "sml_localize_async",
              "sml_forward_maps", "sml_decode_maps"):
        assert n in names


def test_library_exports_every_declared_symbol(libsml):
    import paper_2410_02314_gb300 as sml

    names = declared_functions()
    assert names <= set(sml.EXPORTS)
    for n in names:
        assert hasattr(libsml, n), n


def test_create_without_gpu_fails_loudly(libsml):
    """Without a usable sm_103 device sml_create returns an error: there is no CPU path."""
    import torch

    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import paper_2410_02314_gb300 as sml
    from paper_2410_02314_gb300 import synth

    spec = synth.spec_small()
    blob = synth.pack_blob(spec, synth.init_weights(spec, 1))
    with pytest.raises(sml.SmlError) as e:
        sml.sml_create(spec.to_json(), blob)
    assert e.value.code in (sml.SML_ERR_CUDA, sml.SML_ERR_BAD_SPEC)


def test_record_layout_is_24_bytes():
    import paper_2410_02314_gb300 as sml

    assert sml.RECORD_DTYPE.itemsize == 24
