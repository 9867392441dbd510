"""The offset dual-layer ring with the hot-rod water phantom as the source, at
its full size and default activity: 1e8 pairs at 1.7e4 Bq, 5.9e3 s of
acquisition, so decay times pass 2^52 ps (the sort key of a single run is the
whole 64-bit time).  Checked, by properties that hold at any size: singles in
time order with each (history, unit) once; every coincidence joins two
consecutive singles within the window in different panels; the coincidences
equal those the oracle's sorter finds in the same singles.  Against the
oracle: singles sampled across the time order, late ones included, each
recomputed from its history alone, with its time and blurred energy."""
import numpy as np
import pytest

import workloads as W
from tests import parity_util as PU

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    from paper_2603_07327_gb300 import build as B
    B.build()
    import paper_2603_07327_gb300 as G
    G.load()
    return G


def test_config3_full_size_at_default_activity(G, oracle):
    c3 = W.config3()
    assert c3["n_decays"] == 10**8 and c3["source"]["activity_bq"] == W.DEFAULT_ACTIVITY_BQ
    sc = G.Scanner(c3["scanner"], c3["phantom"])
    res = sc.simulate(c3["source"], c3["digitizer"], c3["n_decays"], c3["seed"])
    c = res.counts()
    assert c["status"] == 0 and c["phantom_steps"] > 0
    s = res.singles()
    t = s["t_ps"]
    assert len(t) > 10**6
    assert t.max() > 1 << 52                       # past the old 52-bit time field
    assert np.all(np.diff(t.astype(np.int64)) >= 0)
    key = np.sort((s["h"].astype(np.uint64) << np.uint64(16)) | s["unit"].astype(np.uint64))
    assert not np.any(key[1:] == key[:-1])
    a, b = res.coincidences()
    window = int(round(c3["digitizer"]["window_ns"] * 1000))
    assert len(a) > 10**4
    assert np.all(b == a + 1) and np.all(t[b] - t[a] <= window) and np.all(s["panel"][a] != s["panel"][b])
    st = np.zeros(len(t), dtype=[("t_ps", "<u8"), ("unit", "<i4"), ("panel", "<i4"), ("h", "<u8")])
    st["t_ps"], st["unit"], st["panel"], st["h"] = t, s["unit"], s["panel"], s["h"]
    _, oa, ob = oracle.coincidences(st, c3["digitizer"]["window_ns"])
    assert PU.coincidence_set(s["h"], s["unit"], a, b) == PU.coincidence_set(st["h"], st["unit"], oa, ob)
    # singles from anywhere in the time order, the last ones included
    rng = np.random.default_rng(33)
    idx = np.concatenate([rng.integers(0, len(t), 40), np.arange(len(t) - 5, len(t))])
    bad = 0
    for i in idx:
        h, unit = int(s["h"][i]), int(s["unit"][i])
        o = oracle.simulate(c3["scanner"], c3["source"], c3["digitizer"], c3["n_decays"], c3["seed"],
                            phantom=c3["phantom"], h_begin=h, h_end=h + 1, tallies=False)["singles"]
        o = o[(o["kept"] == 1) & (o["unit"] == unit)]
        if len(o) != 1 or abs(int(o["t_ps"][0]) - int(t[i])) > PU.T_ABS or \
                abs(float(o["e_blur"][0]) - float(s["e"][i])) > PU.E_REL * abs(float(s["e"][i])) + PU.EB_ABS:
            bad += 1
    assert bad <= 1, (bad, len(idx))
    res.free()
    sc.close()
