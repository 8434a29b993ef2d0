"""The device frame simulator (include/sml_sim.h) against the host simulator and the
published generator it is defined on:
* expected images equal synth.render_expected (float64) within float32 rounding;
* ADU conversion of the expected image is exact;
* Knuth-branch Poisson counts equal a host replay of the definition on synth.splitmix64;
* PTRS-branch counts have Poisson mean and variance;
* frames depend only on (seed, frame0 + t, pixel)."""
import math

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


def _as_f32(em):
    """The emitters as the device sees them (float32 positions, z and photons)."""
    return synth.Emitters(frame=em.frame, x=em.x.astype(np.float32).astype(np.float64),
                          y=em.y.astype(np.float32).astype(np.float64), z=em.z.astype(np.float32).astype(np.float64),
                          photons=em.photons.astype(np.float32).astype(np.float64),
                          bg=em.bg.astype(np.float32).astype(np.float64))


@pytest.mark.parametrize("astig,T,H,W", [(False, 3, 64, 64), (True, 2, 75, 130), (True, 1, 300, 17)])
def test_expected_image_matches_host_renderer(astig, T, H, W):
    rng = np.random.default_rng(H + W)
    em = synth.emitters_density(rng, T, H, W, 3.0, astig=astig)
    # a few emitters on and beyond the frame's edges
    em = synth.Emitters(frame=np.r_[em.frame, [0, 0, T - 1]].astype(np.int32), x=np.r_[em.x, [-0.49, W - 0.51, W + 2.0]],
                        y=np.r_[em.y, [H - 0.5, -1.7, 3.0]], z=np.r_[em.z, [0.0, 300.0, -500.0]],
                        photons=np.r_[em.photons, [4000.0, 2500.0, 1800.0]], bg=em.bg)
    mu = torch.empty((T, H, W), dtype=torch.float32, device="cuda")
    adu = sml.sml_sim_frames(em, T, H, W, astig=astig, gain=1.7, offset=100.0, noise=False, d_mu=mu)
    torch.cuda.synchronize()
    ref = synth.render_expected(_as_f32(em), T, H, W, astig)
    got = mu.cpu().numpy().astype(np.float64)
    err = np.abs(got - ref).max() / ref.max()
    print("expected image normalised max error", err)
    assert err <= 1e-5
    want = np.clip(np.rint(got * np.float64(np.float32(1.7)) + 100.0), 0, 65535).astype(np.uint16)
    assert np.array_equal(adu.cpu().numpy().view(np.uint16), want)


def _flat(T, bg):
    return synth.Emitters(frame=np.zeros(0, np.int32), x=np.zeros(0), y=np.zeros(0), z=np.zeros(0),
                          photons=np.zeros(0), bg=np.full(T, bg))


@pytest.mark.parametrize("lam", [0.3, 3.0, 11.5])
def test_knuth_counts_replay_the_published_generator(lam):
    """Below 12 a count is the number of uniforms multiplied before the product drops to
    exp(-lam) or below, minus one; the uniforms are splitmix64 outputs q*64 + k."""
    seed, H, W = 12345 + int(lam * 10), 32, 40
    adu = sml.sml_sim_frames(_flat(1, lam), 1, H, W, gain=1.0, offset=0.0, seed=seed).cpu().numpy().view(np.uint16)
    n_px = 600
    outs = synth.splitmix64(seed, n_px * 64)
    u = (outs >> np.uint64(11)).astype(np.float64) * 2.0 ** -53
    L = math.exp(-lam)
    want = np.empty(n_px, np.int64)
    for q in range(n_px):
        p, k = 1.0, 0
        while k < 63:
            p *= u[q * 64 + k]
            if p <= L:
                break
            k += 1
        want[q] = k
    assert np.array_equal(adu.reshape(-1)[:n_px].astype(np.int64), want)


@pytest.mark.parametrize("lam", [12.0, 47.0, 180.0, 3000.0])
def test_ptrs_counts_have_poisson_moments(lam):
    H = W = 512
    adu = sml.sml_sim_frames(_flat(1, lam), 1, H, W, gain=1.0, offset=0.0, seed=7).cpu().numpy().view(np.uint16)
    k = adu.astype(np.float64).ravel()
    n = k.size
    mean, var = k.mean(), k.var()
    print(lam, "mean", mean, "var", var)
    assert abs(mean - lam) <= 5.0 * math.sqrt(lam / n)
    assert abs(var / lam - 1.0) <= 5.0 * math.sqrt(2.0 / n) + 0.002
    if lam <= 50:  # the whole pmf: chi-square over the bulk, each bin within 5 sigma
        from scipy.stats import poisson

        lo, hi = int(lam - 4 * math.sqrt(lam)), int(lam + 4 * math.sqrt(lam))
        for v in range(max(0, lo), hi + 1):
            p = poisson.pmf(v, lam)
            assert abs(np.count_nonzero(k == v) - n * p) <= 5.0 * math.sqrt(n * p * (1 - p)) + 1


def test_frames_depend_on_seed_frame_index_and_pixel_only():
    rng = np.random.default_rng(3)
    T, H, W = 4, 48, 80
    em = synth.emitters_density(rng, T, H, W, 2.0, astig=True)
    a = sml.sml_sim_frames(em, T, H, W, astig=True, seed=99).cpu().numpy()
    b = sml.sml_sim_frames(em, T, H, W, astig=True, seed=99).cpu().numpy()
    c = sml.sml_sim_frames(em, T, H, W, astig=True, seed=100).cpu().numpy()
    assert np.array_equal(a, b) and not np.array_equal(a, c)
    # frames 2..3 alone, as frames 0..1 of a call starting at frame 2 (a fixed PSF width, so
    # that both calls have the same window)
    full = sml.sml_sim_frames(em, T, H, W, astig=False, seed=99).cpu().numpy()
    sel = em.frame >= 2
    tail = synth.Emitters(frame=(em.frame[sel] - 2).astype(np.int32), x=em.x[sel], y=em.y[sel], z=em.z[sel],
                          photons=em.photons[sel], bg=em.bg[2:])
    d = sml.sml_sim_frames(tail, 2, H, W, astig=False, seed=99, frame0=2).cpu().numpy()
    assert np.array_equal(full[2:], d)
