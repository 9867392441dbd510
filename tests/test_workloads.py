"""The seeded synthetic inputs follow their stated recipes (CPU only).

Each workload stands in for one of the paper's (Sec. 2.2-2.4); these checks
recompute the recipe's properties from the generated arrays, not from the
generator's code: the hot-rod phantom's cylinder, rods and 10:1 contrast,
the design sweep's parameter ranges, the request stream's arrival process and
pair counts, the sweep and sensitivity positions.  Every generated scanner is
also accepted by the library's validation (no GPU needed)."""
import ctypes as C
import math

import numpy as np
import pytest
from scipy import stats

import workloads as W


@pytest.fixture(scope="module")
def G():
    from paper_2603_07327_gb300 import build as B
    B.build()
    import paper_2603_07327_gb300 as G
    G.load()
    return G


def _accepts(G, sc):
    h = C.c_void_p()
    code = G.load().gpet_create_scanner(C.byref(G.scanner_desc(sc)), C.byref(h))
    if code == 0:
        G.load().gpet_destroy_scanner(h)
    return code


def test_hot_rod_phantom_recipe():
    ph = W.hot_rod_phantom()
    assert (ph["nx"], ph["ny"], ph["nz"]) == (60, 60, 100) and ph["voxel"] == (0.5, 0.5, 0.5)
    mat, act = ph["material"], ph["activity"]
    assert mat.shape == (100, 60, 60) and act.shape == mat.shape
    c = (np.arange(60) + 0.5) * 0.5 - 15.0
    zc = (np.arange(100) + 0.5) * 0.5 - 25.0
    X, Y = np.meshgrid(c, c, indexing="xy")
    inside = X * X + Y * Y <= 15.0 ** 2
    zin = np.abs(zc) <= 25.0
    # water cylinder of 30 mm diameter over the 50 mm length, air elsewhere
    assert np.array_equal(mat.astype(bool), zin[:, None, None] & inside[None])
    # activity: 0 outside, 1 in the background, 10 in rods, identical slices
    assert set(np.unique(act)) == {0.0, 1.0, 10.0}
    assert np.all(act[~(zin[:, None, None] & inside[None])] == 0.0)
    assert all(np.array_equal(act[k], act[50]) for k in range(100) if zin[k])
    rods = ph["rods"]
    assert sorted({d for _, _, d in rods}) == list(W.HOT_ROD_DIAMETERS)
    for x, y, d in rods:
        # inside radius 15 - d, and inside its 60 degree sector by at least d
        assert math.hypot(x, y) <= 15.0 - d + 1e-9
        k = W.HOT_ROD_DIAMETERS.index(d)
        a = math.radians(30.0 + 60.0 * k)
        ang = math.atan2(y, x) - a
        ang = (ang + math.pi) % (2 * math.pi) - math.pi
        r = math.hypot(x, y)
        assert r * math.sin(math.pi / 6 - abs(ang)) >= d - 1e-9
    # a rod's centre voxel is hot
    hot = act[50] == 10.0
    for x, y, d in rods:
        ix, iy = int((x + 15.0) // 0.5), int((y + 15.0) // 0.5)
        if abs((ix + 0.5) * 0.5 - 15.0 - x) < 0.25 * d and abs((iy + 0.5) * 0.5 - 15.0 - y) < 0.25 * d:
            assert hot[iy, ix]
    # rods of one sector sit on a triangular lattice of spacing 2d
    for d in W.HOT_ROD_DIAMETERS:
        pts = np.array([(x, y) for x, y, dd in rods if dd == d])
        if len(pts) > 1:
            dist = np.sqrt(((pts[:, None] - pts[None]) ** 2).sum(-1)) + np.eye(len(pts)) * 1e9
            np.testing.assert_allclose(dist.min(1), 2 * d, rtol=1e-9)


def test_design_sweep_recipe(G):
    designs = W.config4()
    assert len(designs) == 64
    n = np.array([d["n_decays"] for d in designs], dtype=np.float64)
    assert n.min() >= 1e5 and n.max() <= 1e7
    # log-uniform decay counts
    assert stats.kstest((np.log10(n) - 5.0) / 2.0, "uniform").pvalue > 1e-3
    for d in designs:
        sc = d["scanner"]
        assert sc["n_panels"] == 12 and 1 <= len(sc["layers"]) <= 3
        assert 40.0 <= sc["inner_radius"] <= 80.0
        pitch = sc["layers"][0]["pitch_u"]
        assert 0.8 <= pitch <= 2.0
        depth = sum(l["depth"] for l in sc["layers"])
        assert 8.0 <= depth <= 20.0
        r_off = math.hypot(*d["source"]["pos"][:2])
        assert r_off <= min(50.0, 0.75 * sc["inner_radius"]) + 1e-9
        assert _accepts(G, sc) == 0
    # the same seed gives the same designs
    again = W.config4()
    assert [d["n_decays"] for d in again] == [d["n_decays"] for d in designs]


def test_request_stream_recipe():
    reqs = W.config5()
    assert len(reqs) == 2000
    t = np.array([r["arrival_s"] for r in reqs])
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert np.all(gaps > 0)
    # exponential inter-arrival times with mean 20 ms
    assert stats.kstest(gaps, "expon", args=(0, 0.02)).pvalue > 1e-3
    n = np.array([r["n_decays"] for r in reqs], dtype=np.float64)
    assert n.min() >= 1e5 and n.max() <= 5e7
    u = (np.log10(n) - 5.0) / (math.log10(5e7) - 5.0)
    assert stats.kstest(u, "uniform").pvalue > 1e-3
    ph = np.array([r["phantom"] is not None for r in reqs])
    assert abs(ph.mean() - 0.5) < 4 * math.sqrt(0.25 / len(reqs))
    scales = np.array([r["phantom"][1] for r in reqs if r["phantom"] is not None])
    assert scales.min() >= 0.5 and scales.max() <= 1.0
    assert all(r["source"]["kind"] == 1 for r in reqs if r["phantom"] is not None)


def test_sweep_and_sensitivity_positions(G):
    z = W.config2_positions()
    assert z == [float(v) for v in range(-30, 31)]
    pos = W.sensitivity_positions()
    assert len(pos) == 32
    assert pos[:15] == [(float(r), 0.0, 0.0) for r in range(0, 75, 5)]
    assert pos[15:] == [(0.0, 0.0, float(v)) for v in range(10, 180, 10)]
    for g in ("A", "B"):
        assert _accepts(G, W.config2_scanner(g)) == 0
    assert _accepts(G, W.config3_scanner()) == 0
    for k in ("1CL", "split", "2CL"):
        assert _accepts(G, W.h2rspet(k)) == 0
    # the config-2 panels' axial half-length covers the +-30 mm sweep
    sc = W.config2_scanner("A")
    lay = sc["layers"][0]
    assert sc["modules_v"] * lay["n_v"] * lay["pitch_v"] / 2 >= max(abs(v) for v in z)
