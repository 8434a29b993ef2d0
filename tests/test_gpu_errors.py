"""Error reporting of asynchronous work, with the failure injected on the host.

A tensor-core kernel whose bounded wait gives up sets its context's device error word and
returns.  Here the word is set by the host-side test hook sml_debug_set_error_word (no kernel
is made to fail on the shared GPU); the tests check that each kind of caller learns of it:
the synchronous call fails with SML_ERR_CUDA, sml_error_word hands the word to asynchronous
callers in stream order and clears it, and the serving executor fails exactly the request
that ran while the word was set."""
import numpy as np
import pytest
import torch

import paper_2410_02314_gb300 as sml
from paper_2410_02314_gb300 import serve, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__

    __graft_entry__.build()
    torch.cuda.set_device(0)


def test_error_word_reaches_sync_and_async_callers():
    w = synth.workload_small(precision="bf16")
    loc = sml.Localizer(w.spec.to_json(), w.blob)
    word = torch.full((2,), 7, dtype=torch.int32, device="cuda")
    sml.sml_error_word(loc.ctx, word[0:])
    torch.cuda.synchronize()
    assert int(word[0]) == 0  # nothing failed
    assert sml.lib().sml_debug_set_error_word(loc.ctx, 1) == sml.SML_OK
    d = torch.from_numpy(w.frames).cuda()
    out = torch.empty(4096 * 24, dtype=torch.uint8, device="cuda")
    n = torch.zeros(1, dtype=torch.int64, device="cuda")
    loc.localize_async(d, 0.5, out, n)  # runs normally; the word stays set
    sml.sml_error_word(loc.ctx, word[0:])
    sml.sml_error_word(loc.ctx, word[1:])  # the first read cleared it
    torch.cuda.synchronize()
    assert word.tolist() == [1, 0]
    sml.lib().sml_debug_set_error_word(loc.ctx, 1)
    with pytest.raises(sml.SmlError) as e:
        loc.localize(w.frames, 0.5, gain=w.cam.gain, offset=w.cam.offset)
    assert e.value.code == sml.SML_ERR_CUDA
    # the failed call cleared the word: the next one succeeds with the usual records
    recs = loc.localize(w.frames, 0.5, gain=w.cam.gain, offset=w.cam.offset)
    assert len(recs) > 0
    loc.close()


def test_serving_fails_the_request_that_saw_the_error():
    rng = np.random.default_rng(1)
    spec = synth.spec_small("bf16")
    blob = synth.pack_blob(spec, synth.init_weights(spec, 3))
    reqs = []
    for k in range(4):
        em = synth.emitters_density(rng, 2, 64, 64, 1.0)
        fr = synth.simulate(em, 2, 64, 64, synth.Camera(), False, rng)
        reqs.append(serve.Request(rid=k, frames=torch.from_numpy(fr).pin_memory(), arrival=0.0))
    ex = serve.GpuExecutor(spec.to_json(), blob, slots=1)
    ex.warm([(2, 64, 64)])
    assert sml.lib().sml_debug_set_error_word(ex.locs[0].ctx, 1) == sml.SML_OK
    sch = serve.Scheduler(ex, 1 << 34)
    out = sch.run(reqs)
    assert [r.rid for r in out if r.error] == [0] and out[0].records is None
    alone = sml.Localizer(spec.to_json(), blob)
    for r in out[1:]:
        assert r.records.tobytes() == alone.localize(r.frames.numpy(), r.p_min).tobytes()
    assert sch.failed == 1


def test_a_conv_whose_waits_run_out_reports_it():
    """The kernels' own give-up path, in the form that leaves nothing in flight: with the test
    settings debug_poison_cta = 0 and debug_wait_ns = 5 ms, CTA 0 of every tensor-core conv
    launch loads no data, so its consumers' bounded waits run out; the kernel sets the error
    word, finishes its row sequence without waiting, drains its own MMAs, frees TMEM and
    returns.  The call reports SML_ERR_CUDA; a context without the settings then gives the
    usual records on the same device."""
    import json

    w = synth.workload_small(precision="bf16")
    js = json.loads(w.spec.to_json())
    bad = sml.Localizer(json.dumps(dict(js, debug_poison_cta=0, debug_wait_ns=5e6)), w.blob)
    with pytest.raises(sml.SmlError) as e:
        bad.localize(w.frames, 0.5, gain=w.cam.gain, offset=w.cam.offset)
    assert e.value.code == sml.SML_ERR_CUDA and "timed out" in str(e.value)
    bad.close()
    good = sml.Localizer(w.spec.to_json(), w.blob)
    recs = good.localize(w.frames, 0.5, gain=w.cam.gain, offset=w.cam.offset)
    again = good.localize(w.frames, 0.5, gain=w.cam.gain, offset=w.cam.offset)
    assert len(recs) > 0 and recs.tobytes() == again.tobytes()
    good.close()
    with pytest.raises(sml.SmlError) as e:  # the test setting needs a short, bounded wait
        sml.Localizer(json.dumps(dict(js, debug_poison_cta=0)), w.blob)
    assert e.value.code == sml.SML_ERR_BAD_SPEC
