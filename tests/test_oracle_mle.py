"""Pins for the Gaussian-MLE fitter and the CRLB (the classical comparison method).

* the model's analytic Jacobian equals central differences of the model;
* the PSF integrates to the photon count;
* the CRLB reaches the textbook limits: sigma^2/N for small pixels and no background, and
  Mortensen et al.'s (2010) closed form for a pixelated Gaussian with background;
* the MLE is unbiased and efficient (std of estimates ~ sqrt(CRLB)) on simulated spots.
"""
import math

import numpy as np
import pytest

from oracle import mle


def test_jacobian_matches_central_differences():
    theta = np.array([6.3, 5.7, 2500.0, 80.0, 1.4, 1.9])
    mu, J = mle.model(theta, (13, 12))
    for k in range(6):
        h = 1e-5 * max(1.0, abs(theta[k]))
        tp, tm = theta.copy(), theta.copy()
        tp[k] += h
        tm[k] -= h
        fd = (mle.model(tp, (13, 12))[0] - mle.model(tm, (13, 12))[0]) / (2 * h)
        assert np.abs(fd - J[k]).max() <= 1e-6 * np.abs(J[k]).max() + 1e-9


def test_psf_mass():
    mu, _ = mle.model((20.2, 19.6, 3000.0, 0.0, 1.3, 2.1), (40, 40))
    assert abs(mu.sum() - 3000.0) < 1e-6 * 3000.0


def test_crlb_small_pixel_limit():
    s, N = 8.0, 2000.0
    var = mle.crlb((40.0, 40.0, N, 1e-9, s, s), (81, 81), free=(0, 1, 2))
    assert abs(var[0] / ((s * s + 1.0 / 12.0) / N) - 1.0) < 0.02


@pytest.mark.parametrize("N,b", [(3000.0, 100.0), (1000.0, 20.0), (5000.0, 200.0)])
def test_crlb_matches_mortensen_formula(N, b):
    s = 1.3
    sa2 = s * s + 1.0 / 12.0
    tau = 2 * math.pi * sa2 * b / N
    mort = sa2 / N * (1 + 4 * tau + math.sqrt(2 * tau / (1 + 4 * tau)))
    var = mle.crlb((12.0, 12.0, N, b, s, s), (25, 25), free=(0, 1, 2, 3))
    assert abs(var[0] / mort - 1.0) < 0.1


def test_mle_is_unbiased_and_efficient():
    rng = np.random.default_rng(4)
    truth = np.array([5.2, 4.9, 3000.0, 100.0, 1.3, 1.3])
    mu, _ = mle.model(truth, (11, 11))
    est = []
    for _ in range(300):
        img = rng.poisson(mu).astype(np.float64)
        th, ok = mle.fit(img, (5.0, 5.0, img.sum() - 100 * 121, 100.0, 1.3, 1.3), free=(0, 1, 2, 3))
        assert ok
        est.append(th[:2])
    est = np.array(est)
    crlb_x = math.sqrt(mle.crlb(truth, (11, 11), free=(0, 1, 2, 3))[0])
    assert abs(est[:, 0].std() / crlb_x - 1.0) < 0.15
    assert abs(est[:, 0].mean() - truth[0]) < 0.25 * crlb_x


def test_astigmatic_z_readout():
    from paper_2410_02314_gb300 import synth

    for z in (-500.0, -120.0, 0.0, 333.0, 600.0):
        sx, sy = synth.sigma_xy(np.array([z]), astig=True)
        assert abs(mle.z_from_widths(float(sx[0]), float(sy[0])) - z) <= 1.0


def test_detect_and_fit_finds_isolated_spots():
    rng = np.random.default_rng(9)
    H = W = 48
    truth = np.array([[10.3, 12.8], [30.6, 9.1], [22.0, 35.4], [40.2, 40.7]])
    mu = np.full((H, W), 60.0)
    for x, y in truth:
        mu += mle.model((x, y, 3000.0, 0.0, 1.3, 1.3), (H, W))[0]
    got = mle.detect_and_fit(rng.poisson(mu).astype(np.float64), 60.0, 30.0)
    s = mle.score([got], [np.c_[truth, np.zeros(4), np.full(4, 3000.0)]])
    assert s["jaccard"] == 1.0 and s["rmse_lateral_nm"] < 10.0
