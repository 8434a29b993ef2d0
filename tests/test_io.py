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


def test_ring_back_pressure_and_timeout(tmp_path):
    """With both buffers of a 2-buffer ring handed out, the reader cannot read the third batch:
    sml_reader_next times out (SML_ERR_CUDA, as documented) until the first buffer comes back,
    and the third batch then holds the right frames.  Closing with batches still out ends the
    reader thread."""
    import ctypes

    frames = np.arange(5 * 3 * 4, dtype=np.uint16).reshape(5, 3, 4)
    p = tmp_path / "ring.raw"
    write_stack(p, frames)
    L = sml.lib()
    h = ctypes.c_void_p()
    assert L.sml_reader_open(os.fsencode(str(p)), 0, 5, 3, 4, 2, 2, ctypes.byref(h)) == sml.SML_OK

    def nxt(timeout_ms):
        q, n, first = ctypes.c_void_p(), ctypes.c_int(0), ctypes.c_longlong(0)
        code = L.sml_reader_next(h, ctypes.byref(q), ctypes.byref(n), ctypes.byref(first), timeout_ms)
        return code, q.value, n.value, first.value

    c0, p0, n0, f0 = nxt(10000)
    c1, p1, n1, f1 = nxt(10000)
    assert (c0, n0, f0, c1, n1, f1) == (sml.SML_OK, 2, 0, sml.SML_OK, 2, 2)
    assert nxt(50)[0] == sml.SML_ERR_CUDA  # batch 2 needs buffer 0 back
    assert L.sml_reader_release(h, ctypes.c_void_p(p0)) == sml.SML_OK
    c2, p2, n2, f2 = nxt(10000)
    assert (c2, p2, n2, f2) == (sml.SML_OK, p0, 1, 4)
    got = np.ctypeslib.as_array(ctypes.cast(p2, ctypes.POINTER(ctypes.c_uint16)), shape=(1, 3, 4))
    assert np.array_equal(got, frames[4:5])
    assert nxt(10)[2] == 0  # past the last batch: no frames
    L.sml_reader_close(h)  # batches 1 and 2 still out
