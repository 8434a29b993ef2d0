"""The allocation-free decode entry point (for callers that cannot call cudaMalloc while they
run, e.g. an acquisition loop sharing the GPU with a live camera stream, or a plugin whose
host keeps all device memory in its own pool) gives the same records as sml_decode_maps.

Collected last on purpose: a failure here leaves every other test already run."""
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


def random_maps(seed, T, H, W):
    rng = np.random.default_rng(seed)
    m = rng.normal(0.0, 1.0, (T, 5, H, W)).astype(np.float32)
    m[:, 0] = rng.random((T, H, W), dtype=np.float32)
    return torch.from_numpy(m).cuda()


def test_static_decode_matches_decode_maps_on_two_calls():
    spec = synth.NetSpec(in_ch=1, channels=16, dilations=(1, 1), z_scale=850.0, ph_scale=12000.0)
    loc = sml.Localizer(spec.to_json(), synth.pack_blob(spec, synth.init_weights(spec, 1)))
    # two calls in a row; the second is smaller, so stale scratch from the first would show
    for seed, (T, H, W), p_min in [(1, (6, 200, 144), 0.5), (2, (3, 70, 33), 0.3)]:
        maps = random_maps(seed, T, H, W)
        cap = T * H * W // 4 + 16
        ref_out = torch.zeros(cap * 24, dtype=torch.uint8, device="cuda")
        ref_n = torch.zeros(1, dtype=torch.int64, device="cuda")
        loc.decode_maps(maps, p_min, ref_out, ref_n)
        got_out = torch.full((cap * 24,), 7, dtype=torch.uint8, device="cuda")
        got_n = torch.full((1,), 12345, dtype=torch.int64, device="cuda")
        sml.sml_decode_maps_static(maps, p_min, spec.z_scale, spec.ph_scale, got_out, got_n)
        torch.cuda.synchronize()
        n = int(ref_n.item())
        assert n > 0 and int(got_n.item()) == n
        assert torch.equal(got_out[: n * 24], ref_out[: n * 24])


def test_static_decode_rejects_sizes_beyond_its_scratch():
    maps = random_maps(3, 1, 8, 8)
    out = torch.zeros(24, dtype=torch.uint8, device="cuda")
    n = torch.zeros(1, dtype=torch.int64, device="cuda")
    code = sml.lib().sml_decode_maps_static(maps.data_ptr(), 257, 256, 256, 0.5, 1.0, 1.0, out.data_ptr(), 1,
                                            n.data_ptr(), torch.cuda.current_stream().cuda_stream)
    assert code == sml.SML_ERR_UNSUPPORTED


@pytest.mark.parametrize("T,H,W", [(1, 4096, 4096), (1, 4095, 4097)])
def test_static_decode_at_its_capacity_edge(T, H, W):
    """Exactly the fixed scratch's capacity (T*H*W = 16,777,216 pixels: the block count equals
    the array's entries) and one pixel under it (a size that is not a multiple of the
    1024-pixel decode block): the records equal those of sml_decode_maps byte for byte and
    those of the oracle's decode of the same maps."""
    import oracle

    spec = synth.NetSpec(in_ch=1, channels=16, dilations=(1, 1), z_scale=850.0, ph_scale=12000.0)
    loc = sml.Localizer(spec.to_json(), synth.pack_blob(spec, synth.init_weights(spec, 1)))
    maps = random_maps(5, T, H, W)
    p_min = 0.9
    cap = T * H * W // 8
    ref_out = torch.zeros(cap * 24, dtype=torch.uint8, device="cuda")
    ref_n = torch.zeros(1, dtype=torch.int64, device="cuda")
    loc.decode_maps(maps, p_min, ref_out, ref_n)
    got_out = torch.full((cap * 24,), 7, dtype=torch.uint8, device="cuda")
    got_n = torch.full((1,), 12345, dtype=torch.int64, device="cuda")
    sml.sml_decode_maps_static(maps, p_min, spec.z_scale, spec.ph_scale, got_out, got_n)
    torch.cuda.synchronize()
    n = int(ref_n.item())
    assert 0 < n <= cap and int(got_n.item()) == n
    assert torch.equal(got_out[: n * 24], ref_out[: n * 24])
    want = oracle.decode(maps.cpu().numpy(), p_min, spec.z_scale, spec.ph_scale)
    assert want.tobytes() == got_out[: n * 24].cpu().numpy().tobytes()
    loc.close()
