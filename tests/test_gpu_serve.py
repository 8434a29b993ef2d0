"""Continuous-batching serving on the GPU: requests of mixed sizes arriving over time give
the same records as each request localized alone."""
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


@pytest.mark.parametrize("shapes,headroom_mb", [
    # seven frame sizes on slots that keep four: new workspaces are charged, and plans of
    # sizes beyond four are evicted between requests (each after its last use)
    ([(6, 64, 64), (3, 128, 96), (2, 256, 256), (5, 64, 200), (4, 64, 64), (1, 512, 512), (3, 128, 96)], 8192),
    # four sizes, all warm: a few MB of headroom above the resident workspaces make requests
    # wait for memory, not only for slots
    ([(6, 64, 64), (3, 128, 96), (2, 256, 256), (5, 64, 200), (4, 64, 64), (2, 256, 256), (3, 128, 96)], 6),
])
def test_mix_equals_alone(shapes, headroom_mb):
    rng = np.random.default_rng(0)
    spec = synth.spec_48("bf16")
    blob = synth.pack_blob(spec, synth.init_weights(spec, 21))
    reqs = []
    for k, (T, H, W) in enumerate(shapes):
        em = synth.emitters_density(rng, T, H, W, 1.0)
        fr = synth.simulate(em, T, H, W, synth.Camera(), False, rng)
        reqs.append(serve.Request(rid=k, frames=torch.from_numpy(fr).pin_memory(), arrival=0.004 * k))
    ex = serve.GpuExecutor(spec.to_json(), blob, slots=3)
    largest = {}
    for T, H, W in shapes:  # warm each size with its largest request
        largest[(H, W)] = max(largest.get((H, W), 0), T)
    ex.warm(sorted((T, H, W) for (H, W), T in largest.items())[:4])
    budget = ex.resident_bytes() + (headroom_mb << 20)
    sch = serve.Scheduler(ex, budget)
    out = sch.run(reqs)
    rep = serve.report(out)
    print("serving report", rep, "max queue", sch.max_queue, "peak bytes", sch.peak_in_use, "budget", budget)
    alone = sml.Localizer(spec.to_json(), blob)
    for r in out:
        assert r.error is None
        ref = alone.localize(r.frames.numpy(), r.p_min)
        assert r.records.tobytes() == ref.tobytes(), r.rid
    assert sch.peak_in_use <= budget
