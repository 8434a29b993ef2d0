"""Gaussian maximum-likelihood PSF fitting and the Cramer-Rao lower bound -- TEST
INFRASTRUCTURE ONLY (tests/ and bench.py import it; the product never does).

This is the classical localization method the learned network is compared with, and the
yardstick of localization error: the CRLB (Sec. 4.1.1) bounds the variance of any unbiased
estimator, and an efficient MLE reaches it.

Model (pixel-integrated Gaussian, unit pixels, pixel (i, j) centred on integer indices):
    mu_ij = N * Ex_j * Ey_i + bg,
    Ex_j = (erf((j + 1/2 - x) / (sqrt(2) sx)) - erf((j - 1/2 - x) / (sqrt(2) sx))) / 2,
with Poisson counts n_ij.  Parameters theta = (x, y, N, bg, sx, sy).  The Fisher
information is I = sum_ij grad(mu) grad(mu)^T / mu; the fit maximises the Poisson
log-likelihood by damped Fisher scoring (Levenberg-Marquardt on the scoring system).
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erf

SQ2 = math.sqrt(2.0)
SQ2PI = math.sqrt(2.0 * math.pi)


def _edges(c, s, idx):
    """Integrated 1-D Gaussian over unit pixels and its derivatives w.r.t. centre and width."""
    a = (idx - 0.5 - c) / s
    b = (idx + 0.5 - c) / s
    E = 0.5 * (erf(b / SQ2) - erf(a / SQ2))
    ga, gb = np.exp(-0.5 * a * a), np.exp(-0.5 * b * b)
    dEdc = (ga - gb) / (SQ2PI * s)
    dEds = (a * ga - b * gb) / (SQ2PI * s)
    return E, dEdc, dEds


def model(theta, shape):
    """Expected counts mu [H, W] and its Jacobian [6, H, W] at theta = (x, y, N, bg, sx, sy)."""
    x, y, N, bg, sx, sy = theta
    H, W = shape
    Ex, dEx, dEsx = _edges(x, sx, np.arange(W, dtype=np.float64))
    Ey, dEy, dEsy = _edges(y, sy, np.arange(H, dtype=np.float64))
    mu = N * np.outer(Ey, Ex) + bg
    J = np.empty((6, H, W))
    J[0] = N * np.outer(Ey, dEx)
    J[1] = N * np.outer(dEy, Ex)
    J[2] = np.outer(Ey, Ex)
    J[3] = 1.0
    J[4] = N * np.outer(Ey, dEsx)
    J[5] = N * np.outer(dEsy, Ex)
    return mu, J


def fisher(theta, shape, free=(0, 1, 2, 3, 4, 5)):
    mu, J = model(theta, shape)
    Jf = J[list(free)].reshape(len(free), -1)
    return (Jf / mu.reshape(1, -1)) @ Jf.T


def crlb(theta, shape, free=(0, 1, 2, 3, 4, 5)):
    """Diagonal of the inverse Fisher information (variances) for the free parameters."""
    return np.diag(np.linalg.inv(fisher(theta, shape, free)))


def fit(img, theta0, free=(0, 1, 2, 3, 4, 5), iters=40, tol=1e-7):
    """Poisson MLE by damped Fisher scoring.  img: photo-electron counts [H, W].
    Returns (theta, converged)."""
    theta = np.array(theta0, dtype=np.float64)
    free = list(free)
    n = np.asarray(img, dtype=np.float64).ravel()
    lam = 1e-3

    def loglik(th):
        mu = model(th, img.shape)[0].ravel()
        if np.any(mu <= 0):
            return -np.inf
        return float(np.sum(n * np.log(mu) - mu))

    ll = loglik(theta)
    for _ in range(iters):
        mu, J = model(theta, img.shape)
        mu = mu.ravel()
        Jf = J[free].reshape(len(free), -1)
        g = Jf @ (n / mu - 1.0)
        I = (Jf / mu) @ Jf.T
        accepted = False
        for _ in range(10):
            A = I + lam * np.diag(np.diag(I))
            try:
                step = np.linalg.solve(A, g)
            except np.linalg.LinAlgError:
                lam *= 10
                continue
            cand = theta.copy()
            cand[free] += step
            cand[2] = max(cand[2], 1e-3)
            cand[3] = max(cand[3], 1e-6)
            cand[4] = min(max(cand[4], 0.3), 10.0)
            cand[5] = min(max(cand[5], 0.3), 10.0)
            lc = loglik(cand)
            if lc >= ll:
                converged = abs(lc - ll) < tol * max(1.0, abs(ll))
                theta, ll, lam = cand, lc, max(lam / 10, 1e-7)
                accepted = True
                break
            lam *= 10
        if not accepted or converged:
            return theta, True
    return theta, False


def z_from_widths(sx, sy, sigma0=1.3, zgrid=np.linspace(-800.0, 800.0, 1601)):
    """Axial position from fitted widths by least squares against the astigmatic model
    sigma_{x,y}(z) = sigma0 sqrt(1 + ((z -+ 400 nm) / 500 nm)^2) on a 1-nm grid."""
    gx = sigma0 * np.sqrt(1.0 + ((zgrid + 400.0) / 500.0) ** 2)
    gy = sigma0 * np.sqrt(1.0 + ((zgrid - 400.0) / 500.0) ** 2)
    return float(zgrid[np.argmin((gx - sx) ** 2 + (gy - sy) ** 2)])


def detect_and_fit(electrons, bg_guess, thresh, win=4, sigma0=1.3, smooth=1.3, min_sep=2):
    """The method without a network: local maxima of the Gaussian-smoothed frame above
    bg_guess + thresh, each fitted by MLE in a (2 win + 1)^2 window.
    electrons: [H, W] photo-electrons.  Returns an array of (x, y, z, photons) rows."""
    from scipy.ndimage import gaussian_filter, maximum_filter

    img = np.asarray(electrons, dtype=np.float64)
    sm = gaussian_filter(img, smooth, mode="nearest")
    peaks = (sm == maximum_filter(sm, size=2 * min_sep + 1, mode="nearest")) & (sm > bg_guess + thresh)
    H, W = img.shape
    out = []
    for i, j in zip(*np.nonzero(peaks)):
        i0, i1 = max(0, i - win), min(H, i + win + 1)
        j0, j1 = max(0, j - win), min(W, j + win + 1)
        roi = np.clip(img[i0:i1, j0:j1], 0, None)
        n0 = max(float(roi.sum() - bg_guess * roi.size), 50.0)
        th, ok = fit(roi, (j - j0, i - i0, n0, max(bg_guess, 1.0), sigma0, sigma0))
        x, y = th[0] + j0, th[1] + i0
        if not ok or not (j0 - 0.5 <= x <= j1 - 0.5 and i0 - 0.5 <= y <= i1 - 0.5):
            continue
        out.append((x, y, z_from_widths(th[4], th[5], sigma0), th[2]))
    return np.array(out, dtype=np.float64).reshape(-1, 4)


def match(pred, truth, radius):
    """Greedy nearest-pair matching within radius (pixels) on (x, y); returns index pairs."""
    if len(pred) == 0 or len(truth) == 0:
        return []
    d = np.hypot(pred[:, None, 0] - truth[None, :, 0], pred[:, None, 1] - truth[None, :, 1])
    pairs = []
    used_p, used_t = set(), set()
    for k in np.argsort(d, axis=None):
        a, b = divmod(int(k), d.shape[1])
        if d[a, b] > radius:
            break
        if a in used_p or b in used_t:
            continue
        used_p.add(a)
        used_t.add(b)
        pairs.append((a, b))
    return pairs


def score(pred_by_frame, truth_by_frame, px_nm=100.0, radius_nm=250.0):
    """Jaccard index and lateral / axial RMSE (nm) over frames (SMLM-challenge style metrics,
    Sec. 4.1.2).  Each entry is an array of (x, y, z, photons) rows in pixels / nm."""
    tp = fp = fn = 0
    dl, dz = [], []
    for pred, truth in zip(pred_by_frame, truth_by_frame):
        pairs = match(pred, truth, radius_nm / px_nm)
        tp += len(pairs)
        fp += len(pred) - len(pairs)
        fn += len(truth) - len(pairs)
        for a, b in pairs:
            dl.append(px_nm * math.hypot(pred[a, 0] - truth[b, 0], pred[a, 1] - truth[b, 1]))
            dz.append(pred[a, 2] - truth[b, 2])
    jac = tp / max(1, tp + fp + fn)
    rl = math.sqrt(np.mean(np.square(dl))) if dl else float("nan")
    rz = math.sqrt(np.mean(np.square(dz))) if dz else float("nan")
    return {"jaccard": jac, "rmse_lateral_nm": rl, "rmse_axial_nm": rz, "tp": tp, "fp": fp, "fn": fn}
