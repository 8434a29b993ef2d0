"""Stack reader (include/sml_io.h) on the host: batches in file order with the right bytes,
a short last batch, buffers handed back in order, and errors for a missing or short file.
Needs only the built library (no GPU: buffers are ordinary host memory then)."""
import os

import numpy as np
import pytest

import paper_2410_02314_gb300 as sml


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__

    __graft_entry__.build()


def write_stack(path, frames, header=0):
    with open(path, "wb") as f:
        f.write(b"\x07" * header)
        f.write(np.ascontiguousarray(frames, dtype="<u2").tobytes())


def test_reader_yields_every_frame_in_order(tmp_path):
    rng = np.random.default_rng(3)
    frames = rng.integers(0, 65535, (7, 8, 9)).astype(np.uint16)
    p = tmp_path / "stack.raw"
    write_stack(p, frames, header=16)
    rd = sml.StackReader(str(p), 7, 8, 9, batch=3, n_buffers=2, file_offset=16)
    firsts, got = [], []
    for first, f in rd:
        firsts.append(first)
        got.append(f.copy())
    st = rd.stats()
    rd.close()
    assert firsts == [0, 3, 6]
    assert [g.shape[0] for g in got] == [3, 3, 1]
    assert np.array_equal(np.concatenate(got), frames)
    assert st["bytes_read"] == frames.nbytes


def test_reader_rejects_missing_and_short_files(tmp_path):
    with pytest.raises(sml.SmlError):
        sml.StackReader(str(tmp_path / "missing.raw"), 2, 4, 4)
    p = tmp_path / "short.raw"
    write_stack(p, np.zeros((2, 4, 4), np.uint16))
    with pytest.raises(sml.SmlError):
        sml.StackReader(str(p), 3, 4, 4)  # needs 3 frames
    with pytest.raises(sml.SmlError):
        sml.StackReader(str(p), 2, 4, 4, file_offset=2)  # the offset leaves too few bytes


def test_release_out_of_order_is_refused(tmp_path):
    p = tmp_path / "s.raw"
    write_stack(p, np.arange(4 * 2 * 2, dtype=np.uint16).reshape(4, 2, 2))
    L = sml.lib()
    import ctypes

    h = ctypes.c_void_p()
    assert L.sml_reader_open(os.fsencode(str(p)), 0, 4, 2, 2, 1, 3, ctypes.byref(h)) == sml.SML_OK
    ptrs = []
    for _ in range(2):
        q, n, first = ctypes.c_void_p(), ctypes.c_int(0), ctypes.c_longlong(0)
        assert L.sml_reader_next(h, ctypes.byref(q), ctypes.byref(n), ctypes.byref(first), 10000) == sml.SML_OK
        ptrs.append(q.value)
    assert L.sml_reader_release(h, ptrs[1]) == sml.SML_ERR_BAD_ARG  # batch 0 is still out
    assert L.sml_reader_release(h, ptrs[0]) == sml.SML_OK
    assert L.sml_reader_release(h, ptrs[1]) == sml.SML_OK
    L.sml_reader_close(h)
