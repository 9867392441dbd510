"""The sweep at full size, in the launch form the benchmark times.

122 jobs (geometries A and B of the 12-panel ring, 61 axial positions, 1e7
pairs each, 1.22e9 pairs, about 2.1e8 singles) run as one graph-captured
batched launch.  At this size every CTA of the radix scatter works through
dozens of 4096-key tiles, so the bulk copies that stage each next tile are
exercised many tiles deep.  Checked, by properties that hold at any size:
- each job's singles are in time order and each (history, unit) appears once,
  and the jobs' singles add up to the launch's count;
- every coincidence joins two consecutive singles within the window, in
  different panels;
- in three jobs, the coincidences equal those the oracle's sorter finds in
  the same singles (compared as sets of (history, unit) pairs);
and, against the oracle, singles sampled across the whole launch (late tiles
included): the oracle recomputes each one's history alone, and the single's
time and blurred energy must match its own.
"""
import numpy as np
import pytest

import workloads as W
from tests import parity_util as PU

pytestmark = pytest.mark.gpu

PAIRS = 10_000_000
SCATTER_CTAS = 152 * 8  # radix scatter grid on a GB300: 8 CTAs per SM
TILE = 4096


@pytest.fixture(scope="module")
def G():
    from paper_2603_07327_gb300 import build as B
    B.build()
    import paper_2603_07327_gb300 as G
    G.load()
    return G


def _sweep_jobs(G):
    scs = {g: G.Scanner(W.config2_scanner(g)) for g in ("A", "B")}
    dg = W.digitizer()
    jobs = []
    for geo in ("A", "B"):
        for i, z in enumerate(W.config2_positions()):
            jobs.append(dict(scanner=scs[geo], source=W.point_source((0.0, 0.0, z)), digitizer=dg,
                             n_decays=PAIRS, seed=2 + i + 1000 * (geo == "B")))
    return scs, jobs


def _job_singles(G, r):
    return dict(t_ps=r.array(G.SINGLES_T_PS), h=r.array(G.SINGLES_H), unit=r.array(G.SINGLES_UNIT),
                panel=r.array(G.SINGLES_PANEL), e=r.array(G.SINGLES_E))


def test_full_sweep_launch_sort_and_coincidences(G, oracle):
    scs, jobs = _sweep_jobs(G)
    b = G.Batch(jobs)
    try:
        b.run()
        tot = b.counts()
        assert tot["status"] == 0 and tot["n_decays"] == PAIRS * len(jobs)
        assert tot["singles"] > 10 * SCATTER_CTAS * TILE, tot["singles"]  # many staged tiles per CTA
        window = int(round(W.digitizer()["window_ns"] * 1000))
        rng = np.random.default_rng(122)
        sampled = []
        n_singles = n_coinc = 0
        for j, job in enumerate(jobs):
            r = b.result(j)
            s = _job_singles(G, r)
            a, bb = r.coincidences()
            t = s["t_ps"].astype(np.int64)
            n_singles += len(t)
            n_coinc += len(a)
            assert np.all(np.diff(t) >= 0), j
            key = np.sort((s["h"].astype(np.uint64) << np.uint64(16)) | s["unit"].astype(np.uint64))
            assert not np.any(key[1:] == key[:-1]), j
            # coincidences: consecutive singles, inside the window, different panels
            assert np.all(bb == a + 1), j
            assert np.all(t[bb] - t[a] <= window), j
            assert np.all(s["panel"][a] != s["panel"][bb]), j
            if j in (0, 60, 121):
                st = np.zeros(len(t), dtype=[("t_ps", "<u8"), ("unit", "<i4"), ("panel", "<i4"), ("h", "<u8")])
                st["t_ps"], st["unit"], st["panel"], st["h"] = s["t_ps"], s["unit"], s["panel"], s["h"]
                _, oa, ob = oracle.coincidences(st, W.digitizer()["window_ns"])
                assert PU.coincidence_set(s["h"], s["unit"], a, bb) == PU.coincidence_set(st["h"], st["unit"], oa, ob), j
            # two singles of every fifth job, from anywhere in its time order
            if j % 5 == 0:
                for i in rng.integers(0, len(t), 2):
                    sampled.append((j, int(s["h"][i]), int(s["unit"][i]), int(s["t_ps"][i]), float(s["e"][i])))
            r.free()
        assert n_singles == tot["singles"] and n_coinc == tot["coincidences"]
    finally:
        b.close()
    bad = 0
    for j, h, unit, t, e in sampled:
        job = jobs[j]
        o = oracle.simulate(job["scanner"].desc, job["source"], job["digitizer"], PAIRS, job["seed"], h_begin=h,
                            h_end=h + 1, tallies=False)["singles"]
        o = o[(o["kept"] == 1) & (o["unit"] == unit)]
        if len(o) != 1 or abs(int(o["t_ps"][0]) - t) > PU.T_ABS or \
                abs(float(o["e_blur"][0]) - e) > PU.E_REL * abs(e) + PU.EB_ABS:
            bad += 1
    assert bad <= 1, (bad, len(sampled))
    for sc in scs.values():
        sc.close()
