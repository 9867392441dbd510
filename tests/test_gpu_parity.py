"""CUDA path vs FP64 oracle, element by element on the same Philox streams.

Bar (FP32 transport vs FP64): crystal / layer ids identical in >= 99.99 % of
histories; deposits within 1e-5 relative; positions within 1e-3 mm; times
within 1 ps; blurred energies within 1e-5 relative + 1e-3 keV with window
flips only at the window edges; coincidences identical outside mismatched
histories; per-crystal tallies identical outside mismatched histories.
"""
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


def run_both(G, oracle, sc, src, dg, n, seed, phantom=None, **opts):
    res = G.simulate(sc, src, dg, n, seed, phantom=phantom, keep_hits=True, **opts)
    orc = oracle.simulate(sc, src, dg, n, seed, phantom=phantom, threads=8)
    return res, orc


def check_parity(G, oracle, res, orc, n, dg, min_hist_frac=0.9999):
    c = res.counts()
    assert c["status"] == 0
    gh = PU.gpu_hits_table(res.hits())
    oh = PU.oracle_hits_table(orc["hits"])
    assert c["hits"] == len(gh)
    hc = PU.compare_hits(gh, oh, n)
    assert hc["frac_identical"] >= min_hist_frac, hc
    assert hc["max_rel_e"] <= PU.E_REL, hc
    assert hc["max_pos"] <= PU.POS_ABS, "worst hits: " + repr(hc["worst_pos"]) + f" p99.9={hc['p999_pos']}"
    assert hc["max_pos_outlier"] <= PU.POS_CAP, hc["worst_pos"]
    assert hc["max_dt"] <= PU.T_ABS, hc
    bad = hc["bad"]
    gs = res.singles()
    sc_ = PU.compare_singles(gs, orc["singles"], bad, dg["e_lo"], dg["e_hi"])
    assert sc_["edge_flips"] < 10**9, sc_
    assert sc_["max_rel_eraw"] <= PU.E_REL, sc_
    assert sc_["max_blur_dev"] <= PU.EB_ABS, sc_
    assert sc_["max_dt"] <= PU.T_ABS, sc_
    assert sc_["max_doi_dev"] <= PU.DOI_ABS, sc_
    # time order of the sorted singles
    assert np.all(np.diff(gs["t_ps"].astype(np.int64)) >= 0)
    # coincidences
    ga, gb = res.coincidences()
    osel, oa, ob = oracle.coincidences(orc["singles"], dg["window_ns"])
    cc = PU.compare_coincidences(gs, ga, gb, osel, oa, ob, bad)
    assert cc["unexplained"] <= sc_["edge_flips"], cc
    # tallies
    tc, te = res.tallies()
    badarr = np.array(sorted(bad), dtype=np.uint64)
    ob_hits = orc["hits"][np.isin(orc["hits"]["h"], badarr)]
    gb_hits = gh[np.isin(gh["h"], badarr)]
    allow_c = np.zeros(len(tc))
    np.add.at(allow_c, ob_hits["crystal"], 1)
    np.add.at(allow_c, gb_hits["crystal"], 1)
    assert np.all(np.abs(tc.astype(np.int64) - orc["tally_count"].astype(np.int64)) <= allow_c)
    allow_e = np.zeros(len(tc))
    np.add.at(allow_e, ob_hits["crystal"], ob_hits["edep"] * 2 ** 20)
    np.add.at(allow_e, gb_hits["crystal"], gb_hits["e"] * 2 ** 20)
    de = np.abs(te.astype(np.float64) - orc["tally_efx"].astype(np.float64))
    assert np.all(de <= allow_e + PU.E_REL * orc["tally_efx"] + tc + 1), (de - allow_e).max()
    return dict(hits=hc, singles=sc_, coinc=cc)


CASES = {
    "config1": (W.config1_scanner, lambda: W.point_source(), None, 100_000, 1),
    "config2A_z13": (lambda: W.config2_scanner("A"), lambda: W.point_source((0.0, 0.0, 13.0)), None, 200_000, 15),
    "config2B_zm30": (lambda: W.config2_scanner("B"), lambda: W.point_source((0.0, 0.0, -30.0)), None, 200_000, 2),
    "config3_phantom": (W.config3_scanner, W.phantom_source, W.hot_rod_phantom, 40_000, 3),
    "offcentre_h2rspet_2CL": (lambda: W.h2rspet("2CL", modules_v=2), lambda: W.point_source((21.0, -13.0, 9.0)),
                              None, 60_000, 77),
}


CASES["near_ring_offcentre"] = (lambda: W.config2_scanner("B"), lambda: W.point_source((45.0, 10.0, -12.0)), None,
                                100_000, 21)
# non-repetition mode (panels placed one by one) and a four-layer stack
CASES["box4_posed"] = (W.box_scanner, lambda: W.point_source((4.0, -3.0, 2.5)), None, 150_000, 41)
CASES["box4_posed_phantom"] = (W.box_scanner, W.phantom_source, W.hot_rod_phantom, 40_000, 43)
CASES["ring12_4layer"] = (W.four_layer_scanner, lambda: W.point_source((6.0, 2.0, -4.0)), None, 100_000, 47)
CASES["box4_posed_module_readout"] = (lambda: W.box_scanner(readout_level=W.READOUT_MODULE),
                                      lambda: W.point_source((-3.0, 5.0, -1.0)), None, 100_000, 49)

# three modules across each panel with 4 mm transaxial gaps, and an axial 2 mm gap
CASES["ring6_3x2_module_gaps"] = (lambda: W.scanner(6, 60.0, [W.layer(8, 8, 2.0, 0.2, 10.0)], modules_u=3,
                                                    modules_v=2, module_gap_u=4.0, module_gap_v=2.0),
                                  lambda: W.point_source((7.0, -4.0, 3.0)), None, 150_000, 53)

KERNELS = {"loop": 1, "wave": 2, "cta": 3}


@pytest.mark.parametrize("kernel", sorted(KERNELS))
@pytest.mark.parametrize("name", sorted(CASES))
def test_parity_small(G, oracle, name, kernel):
    mk_sc, mk_src, mk_ph, n, seed = CASES[name]
    sc, src = mk_sc(), mk_src()
    ph = mk_ph() if mk_ph else None
    dg = W.digitizer(doi_fwhm_mm=1.5)
    res, orc = run_both(G, oracle, sc, src, dg, n, seed, phantom=ph, kernel=KERNELS[kernel])
    check_parity(G, oracle, res, orc, n, dg)


@pytest.mark.parametrize("compact_every", [1, 2, 4])
def test_kernels_agree_bit_for_bit(G, compact_every):
    """The per-lane loop and the regrouping wavefront run the same events, so
    hits, singles, coincidences and tallies are identical (as sets)."""
    ph = W.hot_rod_phantom()
    for sc, src, n in ((W.config2_scanner("B"), W.point_source((3.0, -2.0, 11.0)), 300_000),
                       (W.config3_scanner(), W.phantom_source(), 60_000)):
        out = []
        for k in (1, 2, 3):
            r = G.simulate(sc, src, W.digitizer(), n, 77, phantom=ph if src["kind"] == 1 else None, keep_hits=True,
                           kernel=k, compact_every=compact_every)
            h = PU.gpu_hits_table(r.hits())
            s = r.singles()
            order = np.lexsort((s["unit"], s["h"]))
            a, b = r.coincidences()
            coinc = PU.coincidence_set(s["h"], s["unit"], a, b)
            out.append((h, {k2: v[order] for k2, v in s.items()}, coinc, r.tallies()))
        (h1, s1, c1, t1) = out[0]
        for (h2, s2, c2, t2) in out[1:]:
            assert np.array_equal(h1, h2)
            for key in s1:
                assert np.array_equal(s1[key], s2[key]), key
            assert c1 == c2
            assert np.array_equal(t1[0], t2[0]) and np.array_equal(t1[1], t2[1])


def test_module_and_panel_readout(G, oracle):
    for level in (W.READOUT_MODULE, W.READOUT_PANEL):
        sc = W.h2rspet("split", modules_v=2)
        sc["readout_level"] = level
        dg = W.digitizer()
        res, orc = run_both(G, oracle, sc, W.point_source((5.0, 5.0, -20.0)), dg, 40_000, 5)
        check_parity(G, oracle, res, orc, 40_000, dg)


@pytest.mark.parametrize("n", [1, 3, 33, 4097])
def test_ragged_and_tiny_runs(G, oracle, n):
    sc = W.config1_scanner()
    dg = W.digitizer(e_lo=0.0, e_hi=5000.0)
    res, orc = run_both(G, oracle, sc, W.point_source((1.0, 0.5, 0.0)), dg, n, 9)
    check_parity(G, oracle, res, orc, n, dg, min_hist_frac=1.0 - 1.0 / n if n < 10000 else 0.9999)


def test_no_hits_at_all(G):
    """A pencil pair along the axis never meets a panel: empty outputs."""
    res = G.simulate(W.config1_scanner(), W.pencil_source(direction=(0, 0, 1)), W.digitizer(), 5000, 3, keep_hits=True)
    c = res.counts()
    assert c["hits"] == 0 and c["singles"] == 0 and c["coincidences"] == 0
    assert c["flights"] == 10000 and c["entered"] == 0
    assert len(res.array(0)) == 0
    tc, te = res.tallies()
    assert tc.sum() == 0 and te.sum() == 0


def test_capacity_overflow_retry(G, oracle):
    """Open window on a large ring: more singles than the first capacity guess,
    so the library re-runs with exact capacities; results must still match."""
    sc = W.h2rspet("1CL", modules_v=6)
    dg = W.digitizer(e_lo=0.0, e_hi=1e4)
    res, orc = run_both(G, oracle, sc, W.point_source(), dg, 120_000, 12)
    c = res.counts()
    assert c["singles"] > 0.6 * 120_000
    check_parity(G, oracle, res, orc, 120_000, dg)


def test_singles_list_overflow_is_resimulated(G, oracle):
    """Fine crystals in a thick, nearly pure Compton scatterer: ~2.5 % of the
    histories touch more than 8 crystals; those are re-simulated by the
    fallback kernel and must still match the oracle."""
    mats = [W.AIR, dict(mu_total_511_cm=2.0, photo_frac_511=0.01, electron_density_cm3=0.0)]
    sc = W.scanner(8, 40.0, [W.layer(64, 64, 0.3, 0.02, 40.0)], materials=mats)
    dg = W.digitizer(e_lo=0.0, e_hi=5000.0)
    n = 20_000
    res, orc = run_both(G, oracle, sc, W.point_source(), dg, n, 4)
    per = np.bincount(np.unique(orc["hits"]["h"].astype(np.int64) * 10**7 + orc["hits"]["crystal"]) // 10**7)
    assert (per > 8).sum() >= 100  # the fallback path is exercised
    check_parity(G, oracle, res, orc, n, dg)


def test_full_size_sampled_histories(G, oracle):
    """The bench workload unit at full size: one sweep position of the 12-panel
    ring, 1e7 pairs, same launch configuration as the benchmark.  A sample of
    histories (all with >= 4 hits plus a random set) is recomputed by the
    oracle one by one; per-crystal totals are checked against a sum rule."""
    n = 10_000_000
    sc = W.config2_scanner("B")
    src = W.point_source((0.0, 0.0, 7.0))
    dg = W.digitizer()
    res = G.simulate(sc, src, dg, n, 9, keep_hits=True)
    c = res.counts()
    gh = PU.gpu_hits_table(res.hits())
    assert len(gh) == c["hits"]
    hs, cnt = np.unique(gh["h"], return_counts=True)
    rng = np.random.default_rng(0)
    sample = np.unique(np.concatenate([hs[cnt >= 4][:300], rng.integers(0, n, 1500).astype(np.uint64)]))
    rows = []
    for h in sample:
        o = oracle.simulate(sc, src, dg, n, 9, h_begin=int(h), h_end=int(h) + 1, tallies=False)
        rows.append(o["hits"])
    oh = PU.oracle_hits_table(np.concatenate(rows))
    gsel = gh[np.isin(gh["h"], sample)]
    hc = PU.compare_hits(gsel, oh, len(sample))
    assert hc["frac_identical"] >= 1.0 - 2.0 / len(sample), hc
    assert hc["max_rel_e"] <= PU.E_REL and hc["max_pos"] <= PU.POS_ABS and hc["max_dt"] <= PU.T_ABS, hc
    assert hc["max_pos_outlier"] <= PU.POS_CAP, hc
    tc, te = res.tallies()
    assert tc.sum() == c["hits"]
    np.testing.assert_allclose(te.sum() / 2 ** 20, gh["e"].astype(np.float64).sum(), rtol=1e-6)
    s = res.singles()
    assert np.all(np.diff(s["t_ps"].astype(np.int64)) >= 0)
    assert len(s["t_ps"]) == c["singles"]


def test_ring_written_as_poses_matches_the_ring(G, oracle):
    """Non-repetition mode with the ring's own poses takes the posed code path
    (explicit frames, all-panel flight) and must give the ring's histories:
    crystal ids identical in >= 99.99 % of histories (the two FP32 frame
    computations round differently, so rare boundary flips are allowed), and
    the posed run matches the oracle's posed run to the full bar."""
    sc = W.config2_scanner("B")
    posed = W.with_poses(sc, W.ring_poses(sc))
    src, dg, n, seed = W.point_source((7.0, -5.0, 3.0)), W.digitizer(), 100_000, 53
    a = G.simulate(sc, src, dg, n, seed, keep_hits=True)
    res, orc = run_both(G, oracle, posed, src, dg, n, seed)
    check_parity(G, oracle, res, orc, n, dg)
    hc = PU.compare_hits(PU.gpu_hits_table(res.hits()), PU.gpu_hits_table(a.hits()), n)
    assert hc["frac_identical"] >= 0.9999, hc


def test_posed_scanner_in_a_batch_keeps_its_own_poses(G):
    """Two posed scanners that differ only in their poses must not share a
    geometry entry in one batched launch: each job equals its plain run."""
    a = W.box_scanner()
    Q = np.array([[0.0, -1.0, 0.0], [1.0, 0.0, 0.0], [0.0, 0.0, 1.0]])
    b = W.rigid_motion(a, Q, (2.0, -1.0, 0.5))
    src, dg = W.point_source((1.0, 2.0, -1.0)), W.digitizer()
    jobs = [dict(scanner=G.Scanner(x), source=src, digitizer=dg, n_decays=50_000, seed=5) for x in (a, b)]
    outs = G.simulate_batch(jobs)
    plain = [j["scanner"].simulate(src, dg, 50_000, 5) for j in jobs]
    for r, p in zip(outs, plain):
        assert np.array_equal(r.tallies()[0], p.tallies()[0])
        assert np.array_equal(r.singles()["t_ps"], p.singles()["t_ps"])
    # the rotated scanner sees the source from elsewhere: its tallies differ
    assert not np.array_equal(plain[0].tallies()[0], plain[1].tallies()[0])


def test_per_crystal_counts_agree_in_distribution_on_independent_seeds(G, oracle):
    """The statistical form of the bar: GPU and oracle runs on different Philox
    keys give per-crystal counts that a two-sample chi-square test accepts at
    p > 0.01.  The counted events are singles (window opened to 0-5000 keV):
    a history adds at most one single to a crystal, so the counts are Poisson.
    (Interaction tallies are not: one photon's Compton chain often leaves
    several interactions in one crystal, which inflates their variance by about
    a quarter and fails the Poisson test on the same, correct runs.)"""
    from scipy import stats
    sc, src, n = W.config2_scanner("B"), W.point_source((0.0, 0.0, 7.0)), 400_000
    dg = W.digitizer(e_lo=0.0, e_hi=5000.0)
    n_cry = oracle.n_crystals(sc)
    gs = G.simulate(sc, src, dg, n, 101).singles()
    os_ = oracle.simulate(sc, src, dg, n, 202, threads=8, tallies=False)["singles"]
    g = np.bincount(gs["unit"].astype(np.int64), minlength=n_cry).astype(np.float64)
    o = np.bincount(os_[os_["kept"] == 1]["unit"].astype(np.int64), minlength=n_cry).astype(np.float64)
    keep = (g + o) >= 20
    chi2 = float((((g[keep] - o[keep]) ** 2) / (g[keep] + o[keep])).sum())
    dof = int(keep.sum())
    p = float(stats.chi2.sf(chi2, dof))
    assert dof > 1000 and p > 0.01, (chi2, dof, p)
