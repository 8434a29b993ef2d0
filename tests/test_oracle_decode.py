"""Pins for the oracle's float32 decode (maps -> localization records).

* hand-written golden cases (tests/golden/decode_cases.json) for ties, plateaus,
  threshold equality, borders and frame independence;
* on random maps with distinct values the rule reduces to "strict 3x3 local maximum
  above threshold", which scipy.ndimage.maximum_filter computes independently;
* the readout values equal numpy float32 arithmetic (one rounding per value).
"""
import json
import os

import numpy as np
import pytest
from scipy.ndimage import maximum_filter

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "decode_cases.json")


def golden_cases():
    with open(GOLDEN) as f:
        return json.load(f)["cases"]


def case_maps(case):
    p = np.asarray(case["p"], dtype=np.float32)
    T, H, W = p.shape
    m = np.zeros((T, 5, H, W), dtype=np.float32)
    m[:, 0] = p
    m[:, 1] = case["dx"]
    m[:, 2] = case["dy"]
    m[:, 3] = case["zhat"]
    m[:, 4] = case["nhat"]
    return m


@pytest.mark.parametrize("case", golden_cases(), ids=lambda c: c["name"])
def test_decode_golden(case):
    recs = oracle.decode(case_maps(case), case["p_min"], case["z_scale"], case["ph_scale"])
    got = [[int(r["frame"]), float(r["x"]), float(r["y"]), float(r["z"]), float(r["photons"]), float(r["p"])]
           for r in recs]
    want = [[int(e[0])] + [float(np.float32(v)) for v in e[1:]] for e in case["expected"]]
    assert got == want


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_decode_matches_maximum_filter_on_distinct_values(seed):
    rng = np.random.default_rng(seed)
    T, H, W = 3, 37, 41
    maps = rng.normal(0.0, 1.0, (T, 5, H, W)).astype(np.float32)
    maps[:, 0] = ((rng.permutation(T * H * W) + 0.5) / (T * H * W)).reshape(T, H, W).astype(np.float32)
    assert np.unique(maps[:, 0]).size == T * H * W
    p_min = 0.3
    recs = oracle.decode(maps, p_min, 1000.0, 10000.0)
    want = []
    for t in range(T):
        p = maps[t, 0]
        mx = maximum_filter(p, size=3, mode="constant", cval=-np.inf)
        ii, jj = np.nonzero((p == mx) & (p > p_min))
        want += [(t, i, j) for i, j in zip(ii, jj)]
    got = []  # (t, i, j) of each record, found through its unique p value
    for r in recs:
        t = int(r["frame"])
        cand = np.argwhere(maps[t, 0] == r["p"])
        assert len(cand) == 1
        got.append((t, int(cand[0, 0]), int(cand[0, 1])))
    assert got == want  # same set, and raster order (frame, row, col)


def test_readout_is_single_rounded_float32():
    rng = np.random.default_rng(5)
    T, H, W = 2, 23, 19
    maps = rng.normal(0.0, 3.0, (T, 5, H, W)).astype(np.float32)
    maps[:, 0] = ((rng.permutation(T * H * W) + 0.5) / (T * H * W)).reshape(T, H, W).astype(np.float32)
    zs, ps = np.float32(987.654), np.float32(12345.678)
    recs = oracle.decode(maps, 0.2, float(zs), float(ps))
    assert len(recs) > 10
    for r in recs:
        t = int(r["frame"])
        (i, j), = np.argwhere(maps[t, 0] == r["p"])
        assert r["x"] == np.float32(j) + maps[t, 1, i, j]
        assert r["y"] == np.float32(i) + maps[t, 2, i, j]
        assert r["z"] == zs * maps[t, 3, i, j]
        assert r["photons"] == ps * maps[t, 4, i, j]


def test_decode_capacity_and_empty():
    m = case_maps(golden_cases()[0])
    full = oracle.decode(m, 0.5, 1000.0, 10000.0)
    part = oracle.decode(m, 0.5, 1000.0, 10000.0, cap=1)
    assert len(full) == 2 and len(part) == 1 and part[0] == full[0]
    empty = oracle.decode(np.zeros((0, 5, 4, 4), np.float32), 0.5, 1.0, 1.0)
    assert len(empty) == 0
