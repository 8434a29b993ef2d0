"""Evaluation harness for trained nets: the detection and localization metrics of Sec. 4.1
and the Cramer-Rao lower bound of the astigmatic PSF model (Sec. 4.1.1).

* ``metrics``: Jaccard index, recall, precision and lateral / axial RMSE over matched pairs,
  plus the efficiency scores of Sec. 4.1.2-4.1.3.
* ``efficiency``: the lateral, axial and volume efficiencies, read after Sage et al. 2019.
  The Jaccard index is in percent and the RMSE in nm:
  E = 100 - sqrt((100 - JI)^2 + alpha^2 RMSE^2), with alpha = 1 / nm lateral and
  0.5 / nm axial (alpha^2 = 0.25, as in the axial term of the paper's equation). The volume
  efficiency is the mean of the two.
* ``astig_crlb``: the square root of the CRLB of (x, y, z).
  * PSF: the pixel-integrated Gaussian with sigma_x(z), sigma_y(z) = sigma0 sqrt(1 + ((z -+
    400 nm) / 500 nm)^2).
  * Noise: Poisson with a flat background.
  * The Fisher information is over theta = (x, y, z, N, bg).
* ``precision_vs_z``: the single-emitter experiment of Sec. 4.1.1.
  * Isolated emitters of constant brightness are placed on a flat background at a set of axial
    positions and localized by a caller-given function.
  * For each z it reports the RMSE of x, y and z next to sqrt(CRLB), plus the fraction
    detected.

Host-side numpy only; independent of the inference path and of the test oracle.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erf

from . import synth

SQ2 = math.sqrt(2.0)
SQ2PI = math.sqrt(2.0 * math.pi)


# ----------------------------------------------------------------------------- matching


def _rows(a):
    """Array of rows (n, k); an empty input gives shape (0, 3)."""
    a = np.asarray(a, dtype=np.float64)
    return a.reshape(0, 3) if a.size == 0 else a.reshape(len(a), -1)


def match(pred, truth, radius):
    """Greedy matching of nearest pairs on (x, y), distance <= radius (same units as x, y).
    Pairs are taken in increasing distance; each prediction and each truth is used once.
    Returns a list of (pred index, truth index)."""
    pred, truth = _rows(pred), _rows(truth)
    if len(pred) == 0 or len(truth) == 0:
        return []
    d = np.hypot(pred[:, None, 0] - truth[None, :, 0], pred[:, None, 1] - truth[None, :, 1])
    order = np.argsort(d, axis=None, kind="stable")
    used_p = np.zeros(len(pred), bool)
    used_t = np.zeros(len(truth), bool)
    pairs = []
    for k in order:
        a, b = divmod(int(k), d.shape[1])
        if d[a, b] > radius:
            break
        if used_p[a] or used_t[b]:
            continue
        used_p[a] = used_t[b] = True
        pairs.append((a, b))
    return pairs


def efficiency(ji_pct, rmse_lat_nm, rmse_ax_nm=None, alpha_lat=1.0, alpha_ax=0.5):
    """(E_lateral, E_axial, E_volume) in percent (Sec. 4.1.3); axial terms are None without
    an axial RMSE."""
    e_lat = 100.0 - math.sqrt((100.0 - ji_pct) ** 2 + (alpha_lat * rmse_lat_nm) ** 2)
    if rmse_ax_nm is None:
        return e_lat, None, None
    e_ax = 100.0 - math.sqrt((100.0 - ji_pct) ** 2 + (alpha_ax * rmse_ax_nm) ** 2)
    return e_lat, e_ax, 0.5 * (e_lat + e_ax)


def metrics(pred_by_frame, truth_by_frame, px_nm=100.0, radius_nm=250.0):
    """Detection and localization scores over frames.  Each entry is an array of rows
    (x px, y px, z nm, ...); predictions and truths are matched per frame within radius_nm
    laterally.  Returns JI (%), recall, precision, RMSE lateral / axial (nm) and the
    efficiencies."""
    tp = fp = fn = 0
    dl2, dz2 = [], []
    for pred, truth in zip(pred_by_frame, truth_by_frame):
        pred, truth = _rows(pred), _rows(truth)
        pairs = match(pred, truth, radius_nm / px_nm)
        tp += len(pairs)
        fp += len(pred) - len(pairs)
        fn += len(truth) - len(pairs)
        for a, b in pairs:
            dl2.append((px_nm * (pred[a, 0] - truth[b, 0])) ** 2 + (px_nm * (pred[a, 1] - truth[b, 1])) ** 2)
            dz2.append((pred[a, 2] - truth[b, 2]) ** 2)
    ji = 100.0 * tp / max(1, tp + fp + fn)
    rl = math.sqrt(float(np.mean(dl2))) if dl2 else float("nan")
    rz = math.sqrt(float(np.mean(dz2))) if dz2 else float("nan")
    e_lat, e_ax, e_vol = efficiency(ji, rl, rz) if dl2 else (float("nan"),) * 3
    return {"jaccard_pct": ji, "recall": tp / max(1, tp + fn), "precision": tp / max(1, tp + fp),
            "rmse_lateral_nm": rl, "rmse_axial_nm": rz, "eff_lateral": e_lat, "eff_axial": e_ax,
            "eff_volume": e_vol, "tp": tp, "fp": fp, "fn": fn}


# ----------------------------------------------------------------------------- CRLB


def _axis(c, s, idx):
    """Pixel-integrated 1-D Gaussian on unit pixels and its derivatives w.r.t. the centre c
    and the width s."""
    lo, hi = idx - 0.5 - c, idx + 0.5 - c
    g_lo, g_hi = np.exp(-lo * lo / (2 * s * s)), np.exp(-hi * hi / (2 * s * s))
    e = 0.5 * (erf(hi / (SQ2 * s)) - erf(lo / (SQ2 * s)))
    de_dc = (g_lo - g_hi) / (SQ2PI * s)
    de_ds = (lo * g_lo - hi * g_hi) / (SQ2PI * s * s)
    return e, de_dc, de_ds


def _widths(z, sigma0, c=400.0, d=500.0):
    """sigma_x, sigma_y and their z derivatives for the astigmatic model."""
    ux, uy = (z + c) / d, (z - c) / d
    sx, sy = sigma0 * math.sqrt(1 + ux * ux), sigma0 * math.sqrt(1 + uy * uy)
    return sx, sy, sigma0 * ux / (d * math.sqrt(1 + ux * ux)), sigma0 * uy / (d * math.sqrt(1 + uy * uy))


def astig_fisher(x, y, z, photons, bg, size=32, sigma0=1.3):
    """Fisher information of theta = (x px, y px, z nm, N, bg) for one emitter in a
    size x size patch with Poisson noise: I = sum_pixels grad(mu) grad(mu)^T / mu."""
    idx = np.arange(size, dtype=np.float64)
    sx, sy, dsx, dsy = _widths(z, sigma0)
    ex, dex_dc, dex_ds = _axis(x, sx, idx)
    ey, dey_dc, dey_ds = _axis(y, sy, idx)
    mu = photons * ey[:, None] * ex[None, :] + bg
    grads = np.stack([
        photons * ey[:, None] * dex_dc[None, :],
        photons * dey_dc[:, None] * ex[None, :],
        photons * (ey[:, None] * dex_ds[None, :] * dsx + dey_ds[:, None] * ex[None, :] * dsy),
        ey[:, None] * ex[None, :],
        np.ones_like(mu),
    ]).reshape(5, -1)
    return (grads / mu.reshape(1, -1)) @ grads.T


def astig_crlb(z, photons, bg, size=32, sigma0=1.3, px_nm=100.0):
    """sqrt(CRLB) of (x, y) in nm and of z in nm for an emitter at the patch centre."""
    c = (size - 1) / 2.0
    cov = np.linalg.inv(astig_fisher(c, c, float(z), photons, bg, size, sigma0))
    return {"x_nm": px_nm * math.sqrt(cov[0, 0]), "y_nm": px_nm * math.sqrt(cov[1, 1]), "z_nm": math.sqrt(cov[2, 2])}


# ----------------------------------------------------------------------------- experiment


def precision_vs_z(localize, zs, n_per_z=100, photons=3000.0, bg=50.0, size=32, seed=0, px_nm=100.0,
                   radius_nm=250.0, gain=1.0, offset=100.0, sigma0=1.3):
    """Single-emitter precision along z (Sec. 4.1.1).  Per z: n_per_z frames of size x size,
    each with one emitter at the centre plus a uniform sub-pixel shift, constant photons and
    background, Poisson noise, camera ADU = round(gain e + offset).  ``localize(frames)``
    returns a record array with fields frame, x, y, z.  Each frame's record nearest the truth
    (within radius_nm) counts as its localization.  Returns one dict per z: detected
    fraction, RMSE and bias of x, y (nm) and z (nm), and sqrt(CRLB)."""
    rng = np.random.default_rng(seed)
    cam = synth.Camera(gain, offset)
    out = []
    for z in zs:
        n = int(n_per_z)
        c = (size - 1) / 2.0
        em = synth.Emitters(frame=np.arange(n), x=c + rng.uniform(-0.5, 0.5, n), y=c + rng.uniform(-0.5, 0.5, n),
                            z=np.full(n, float(z)), photons=np.full(n, float(photons)), bg=np.full(n, float(bg)))
        frames = synth.simulate(em, n, size, size, cam, True, rng)
        recs = localize(frames)
        dx, dy, dz = [], [], []
        for t in range(n):
            r = recs[recs["frame"] == t]
            if len(r) == 0:
                continue
            d = np.hypot(r["x"] - em.x[t], r["y"] - em.y[t]) * px_nm
            k = int(np.argmin(d))
            if d[k] > radius_nm:
                continue
            dx.append(px_nm * (float(r["x"][k]) - em.x[t]))
            dy.append(px_nm * (float(r["y"][k]) - em.y[t]))
            dz.append(float(r["z"][k]) - float(z))
        row = {"z_nm": float(z), "detected": len(dx) / n}
        for name, v in (("x", dx), ("y", dy), ("z", dz)):
            v = np.asarray(v)
            row[f"rmse_{name}_nm"] = float(np.sqrt(np.mean(v * v))) if v.size else float("nan")
            row[f"bias_{name}_nm"] = float(np.mean(v)) if v.size else float("nan")
        row.update({f"crlb_{k}": v for k, v in astig_crlb(z, photons, bg, size, sigma0, px_nm).items()})
        out.append(row)
    return out
