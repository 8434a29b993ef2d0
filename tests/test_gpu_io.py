"""Stack-file pipeline (include/sml_io.h) on the GPU: the records of sml_localize_file over
batches equal those of one sml_localize call on all frames, byte for byte."""
import numpy as np
import pytest
import torch

import paper_2410_02314_gb300 as sml
from paper_2410_02314_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__

    __graft_entry__.build()
    torch.cuda.set_device(0)


def _stack(tmp_path, frames, header=0):
    p = tmp_path / "stack.raw"
    with open(p, "wb") as f:
        f.write(b"\x00" * header)
        f.write(np.ascontiguousarray(frames, dtype="<u2").tobytes())
    return str(p)


@pytest.mark.parametrize("prec,batch", [("fp32", 4), ("bf16", 3), ("bf16", 64)])
def test_file_pipeline_equals_one_call(tmp_path, prec, batch):
    w = synth.workload_small(T=9, precision=prec)
    path = _stack(tmp_path, w.frames, header=64)
    loc = sml.Localizer(w.spec.to_json(), w.blob)
    want = loc.localize(w.frames, 0.5, gain=w.cam.gain, offset=w.cam.offset)
    got, st = loc.localize_file(path, 9, 64, 64, 0.5, batch=batch, gain=w.cam.gain, offset=w.cam.offset,
                                file_offset=64)
    assert len(want) > 20
    assert got.tobytes() == want.tobytes()
    assert st["frames"] == 9 and st["bytes_read"] == w.frames.nbytes and st["wall_seconds"] > 0


def test_file_pipeline_scmos_maps_and_capacity(tmp_path):
    rng = np.random.default_rng(5)
    w = synth.workload_small(T=5, precision="bf16")
    gm = rng.normal(2.0, 0.1, (64, 64)).astype(np.float32)
    om = rng.normal(100.0, 5.0, (64, 64)).astype(np.float32)
    path = _stack(tmp_path, w.frames)
    loc = sml.Localizer(w.spec.to_json(), w.blob)
    want = loc.localize(w.frames, 0.5, gain_map=gm, offset_map=om)
    got, _ = loc.localize_file(path, 5, 64, 64, 0.5, batch=2, gain_map=gm, offset_map=om)
    assert got.tobytes() == want.tobytes()
    with pytest.raises(sml.SmlError) as e:
        loc.localize_file(path, 5, 64, 64, 0.5, batch=2, gain_map=gm, offset_map=om, capacity=len(want) - 1)
    assert e.value.code == sml.SML_ERR_CAPACITY and e.value.needed == len(want)


@pytest.mark.parametrize("prec,batch,T", [("fp32", 4, 9), ("bf16", 3, 10), ("bf16", 1, 4), ("bf16", 64, 7),
                                          ("bf16", 5, 5)])
def test_file_pipeline_with_three_frame_nets_equals_one_call(tmp_path, prec, batch, T):
    """Three-frame input (frames t-1, t, t+1 as channels, Sec. 3.1): each batch takes its
    context frames from the neighbouring batches (device copies, one batch of delay), so the
    records equal one sml_localize call on all frames byte for byte, for batch sizes that split
    the stack unevenly, one frame per batch, and a single batch."""
    spec = synth.NetSpec(in_ch=3, channels=16 if prec == "fp32" else 32, dilations=(1, 2, 4, 1), precision=prec)
    blob = synth.pack_blob(spec, synth.init_weights(spec, 3))
    w = synth.workload_small(T=T, precision=prec)
    path = _stack(tmp_path, w.frames, header=32)
    loc = sml.Localizer(spec.to_json(), blob)
    want = loc.localize(w.frames, 0.3, gain=w.cam.gain, offset=w.cam.offset)
    got, st = loc.localize_file(path, T, 64, 64, 0.3, batch=batch, gain=w.cam.gain, offset=w.cam.offset, file_offset=32)
    assert len(want) > 10
    assert got.tobytes() == want.tobytes()
    assert st["frames"] == T