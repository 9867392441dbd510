"""Failure paths that fault or hang no GPU, and a symmetry of the ring.

The device caps every photon at 1000 Woodcock steps per region; a photon past
the cap is abandoned and the run returns GPET_ERR_TIMEOUT, with the context
still usable.  Rotating a source by one panel angle permutes the per-panel
counts of a ring (statistically: the draws are the same, the geometry turns).
"""
import math

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    from paper_2603_07327_gb300 import build as B
    B.build()
    import paper_2603_07327_gb300 as G
    G.load()
    return G


def test_step_cap_returns_timeout_and_the_context_survives(G):
    # an unused dense material sets the Woodcock majorant (mean step 0.1 mm);
    # the 150 mm crystal layer of a light material keeps photons for > 1000 steps
    light = dict(name="light", mu_total_511_cm=0.01, photo_frac_511=0.5, electron_density_cm3=0.0)
    dense = dict(name="dense", mu_total_511_cm=100.0, photo_frac_511=0.5, electron_density_cm3=0.0)
    sc = W.scanner(8, 40.0, [W.layer(8, 8, 1.6, 0.0, 150.0, crystal_mat=1, interval_mat=1)],
                   materials=[W.AIR, light, dense])
    with pytest.raises(G.GpetError) as e:
        G.simulate(sc, W.point_source(), W.digitizer(), 2000, 1)
    assert e.value.code == -5
    # the device is still usable
    r = G.simulate(W.config1_scanner(), W.point_source(), W.digitizer(), 20_000, 1)
    assert r.counts()["status"] == 0 and r.counts()["hits"] > 0


def test_rotating_the_source_by_one_panel_permutes_panel_counts(G):
    sc = W.config1_scanner()
    n = 300_000
    cpp = 64  # crystals per panel (one module of 8 x 8), panel-major ids
    x, y, z = 9.0, -4.0, 1.5
    c, s = math.cos(2 * math.pi / 8), math.sin(2 * math.pi / 8)
    a = G.simulate(sc, W.point_source((x, y, z)), W.digitizer(), n, 11).tallies()[0]
    b = G.simulate(sc, W.point_source((c * x - s * y, s * x + c * y, z)), W.digitizer(), n, 12).tallies()[0]
    pa = a.reshape(8, cpp).sum(axis=1).astype(np.float64)
    pb = b.reshape(8, cpp).sum(axis=1).astype(np.float64)
    pb = np.roll(pb, -1)          # panel k of the rotated run sits where panel k - 1 was
    chi2 = float((((pa - pb) ** 2) / (pa + pb)).sum())
    # 8 degrees of freedom: chi2 < 26.1 is p > 0.001
    assert chi2 < 26.1, (chi2, pa, pb)
    # and it is not trivially satisfied: without the permutation the counts differ
    assert float((((pa - np.roll(pb, 1)) ** 2) / (pa + np.roll(pb, 1))).sum()) > 100.0
