"""Pins of the evaluation harness (Sec. 4.1): efficiency closed forms, matching on
hand-built cases, and the astigmatic CRLB against the test oracle's independent Fisher
information through the chain rule, its symmetry and its photon scaling."""
import math

import numpy as np
import pytest

from paper_2410_02314_gb300 import evaluate, synth


def test_efficiency_closed_forms():
    assert evaluate.efficiency(100.0, 0.0, 0.0) == (100.0, 100.0, 100.0)
    # 3-4-5 triangle: (100 - 70, 40 nm) -> 50 % lateral; axial alpha = 0.5 -> 80 nm gives the same
    e_lat, e_ax, e_vol = evaluate.efficiency(70.0, 40.0, 80.0)
    assert e_lat == pytest.approx(50.0) and e_ax == pytest.approx(50.0) and e_vol == pytest.approx(50.0)
    e_lat, e_ax, e_vol = evaluate.efficiency(100.0, 30.0, 60.0)  # perfect detection: E = 100 - alpha * RMSE
    assert (e_lat, e_ax, e_vol) == pytest.approx((70.0, 70.0, 70.0))
    assert evaluate.efficiency(0.0, 0.0, 0.0)[0] == pytest.approx(0.0)
    assert evaluate.efficiency(90.0, 10.0)[1:] == (None, None)


def test_match_takes_nearest_pairs_once():
    truth = np.array([[0.0, 0.0], [10.0, 0.0]])
    pred = np.array([[0.4, 0.0], [0.1, 0.0], [13.0, 0.0]])
    assert sorted(evaluate.match(pred, truth, 2.5)) == [(1, 0)]  # (2, 1) is 3 px away
    assert sorted(evaluate.match(pred, truth, 3.0)) == [(1, 0), (2, 1)]
    assert evaluate.match(np.zeros((0, 2)), truth, 1.0) == []


def test_metrics_counts_and_rmse():
    truth = [np.array([[5.0, 5.0, 0.0], [20.0, 5.0, 100.0]]), np.zeros((0, 3))]
    pred = [np.array([[5.3, 5.4, 30.0], [40.0, 40.0, 0.0]]), np.array([[1.0, 1.0, 0.0]])]
    m = evaluate.metrics(pred, truth, px_nm=100.0, radius_nm=250.0)
    assert (m["tp"], m["fp"], m["fn"]) == (1, 2, 1)
    assert m["jaccard_pct"] == pytest.approx(25.0)
    assert m["rmse_lateral_nm"] == pytest.approx(50.0)  # (30, 40) nm
    assert m["rmse_axial_nm"] == pytest.approx(30.0)
    assert m["eff_lateral"] == pytest.approx(100 - math.hypot(75.0, 50.0))


def test_astig_fisher_matches_oracle_fisher_by_chain_rule():
    """I_z = J^T I J with I the test oracle's Fisher information over (x, y, N, bg, sx, sy) and
    J the Jacobian of those parameters w.r.t. (x, y, z, N, bg), the widths' z derivatives
    taken by central differences of the simulator's sigma model."""
    mle = pytest.importorskip("oracle.mle")
    size, x, y, N, bg = 24, 11.3, 12.1, 2500.0, 40.0
    for z in (-500.0, -120.0, 0.0, 333.0, 600.0):
        sx, sy = (float(v[0]) for v in synth.sigma_xy(np.array([z]), True))
        h = 1e-3
        sp, sm = synth.sigma_xy(np.array([z + h, z - h]), True)
        dsx, dsy = (sp[0] - sp[1]) / (2 * h), (sm[0] - sm[1]) / (2 * h)
        I_o = mle.fisher((x, y, N, bg, sx, sy), (size, size))
        J = np.zeros((6, 5))
        J[0, 0] = J[1, 1] = J[2, 3] = J[3, 4] = 1.0
        J[4, 2], J[5, 2] = dsx, dsy
        want = J.T @ I_o @ J
        got = evaluate.astig_fisher(x, y, z, N, bg, size=size)
        assert np.allclose(got, want, rtol=1e-6, atol=1e-9 * np.abs(want).max())


def test_astig_crlb_symmetry_and_photon_scaling():
    a, b = evaluate.astig_crlb(250.0, 3000.0, 50.0), evaluate.astig_crlb(-250.0, 3000.0, 50.0)
    assert a["x_nm"] == pytest.approx(b["y_nm"], rel=1e-9)  # sigma_x(z) = sigma_y(-z)
    assert a["z_nm"] == pytest.approx(b["z_nm"], rel=1e-9)
    # scaling photons and background by k scales mu by k: the (x, y, z) CRLB drops by exactly k
    lo, hi = evaluate.astig_crlb(100.0, 1000.0, 30.0), evaluate.astig_crlb(100.0, 4000.0, 120.0)
    for k in ("x_nm", "y_nm", "z_nm"):
        assert lo[k] == pytest.approx(2.0 * hi[k], rel=1e-9)
    assert evaluate.astig_crlb(0.0, 3000.0, 200.0)["x_nm"] > evaluate.astig_crlb(0.0, 3000.0, 10.0)["x_nm"]


def test_precision_vs_z_with_exact_localizer():
    """A localizer that returns the true positions scores zero error and full detection."""
    truth = {}

    def fake(frames):
        n = frames.shape[0]
        recs = np.zeros(n, dtype=[("frame", "<i4"), ("x", "<f4"), ("y", "<f4"), ("z", "<f4")])
        recs["frame"] = np.arange(n)
        recs["x"], recs["y"], recs["z"] = truth["x"], truth["y"], truth["z"]
        return recs

    orig = synth.simulate

    def spy(em, *a, **k):
        truth.update(x=em.x.astype(np.float32), y=em.y.astype(np.float32), z=em.z.astype(np.float32))
        return orig(em, *a, **k)

    synth.simulate = spy
    try:
        rows = evaluate.precision_vs_z(fake, [-300.0, 0.0, 300.0], n_per_z=20, size=16)
    finally:
        synth.simulate = orig
    for r in rows:
        assert r["detected"] == 1.0
        assert r["rmse_x_nm"] < 1e-3 and r["rmse_y_nm"] < 1e-3 and r["rmse_z_nm"] < 1e-3
        assert r["crlb_x_nm"] > 0 and r["crlb_z_nm"] > 0
