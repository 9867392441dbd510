"""Tally precision past 10^9 histories on the default launch form.

The per-crystal count and energy tallies are 64-bit integers (energy in units
of 2^-20 keV), so a run of 2^32 + 2^28 histories (4.56e9, past the 32-bit
history counter) equals, exactly, the sum of any partition of its histories;
and a sampled history range of that run, straddling history 2^32, matches the
FP64 oracle history by history, its tallies equal to the oracle's up to the
hits of the histories whose FP32 decisions flipped.  Together these state the
tallies' error against the oracle at this scale: exact integer sums of
per-deposit values within 1e-5 relative, plus the mismatched histories."""
import numpy as np
import pytest

import workloads as W
from tests import parity_util as PU

pytestmark = pytest.mark.gpu

N = (1 << 32) + (1 << 28)


@pytest.fixture(scope="module")
def G():
    from paper_2603_07327_gb300 import build as B
    B.build()
    import paper_2603_07327_gb300 as G
    G.load()
    return G


def _setup():
    sc_desc = W.config2_scanner("B")
    # the default 1.7e4 Bq: 2.7e5 s of acquisition, time stamps beyond 2^52 ps
    src = W.point_source((0.0, 0.0, 11.0))
    dg = W.digitizer(e_lo=0.0, e_hi=0.0)  # an empty window: tallies only
    dg["window_ns"] = 0.0
    return sc_desc, src, dg


def test_tallies_past_2_to_32_histories_are_exact_sums(G):
    from paper_2603_07327_gb300 import shard
    sc_desc, src, dg = _setup()
    sc = G.Scanner(sc_desc)
    full = sc.simulate(src, dg, N, 31)
    fc, fe = full.tallies()
    c = full.counts()
    assert c["status"] == 0
    assert int(fc.sum()) == c["hits"] > 4 * 10**8
    parts = []
    for rank in range(4):
        h0, h1 = shard.history_range(N, rank, 4)
        r = sc.simulate(src, dg, N, 31, h_begin=h0, h_end=h1)
        parts.append(r.tallies())
        r.free()
    pc, pe = shard.merge_tallies(parts)
    assert np.array_equal(pc, fc) and np.array_equal(pe, fe)
    # the energy tally of the whole ring stays far from 2^63 at this scale
    assert float(fe.astype(np.float64).sum()) < 2.0 ** 62
    # mean deposit per hit is physical (between the cutoff and 511 keV)
    mean_e = fe.astype(np.float64).sum() / 2 ** 20 / fc.sum()
    assert 10.0 < mean_e < 511.0
    full.free()
    sc.close()


def test_sampled_range_past_2_to_32_matches_the_oracle(G, oracle):
    sc_desc, src, dg = _setup()
    sc = G.Scanner(sc_desc)
    h0, h1 = (1 << 32) - 1_000_000, (1 << 32) + 1_000_000
    res = sc.simulate(src, dg, N, 31, h_begin=h0, h_end=h1, keep_hits=True)
    orc = oracle.simulate(sc_desc, src, dg, N, 31, h_begin=h0, h_end=h1, threads=8)
    gh = PU.gpu_hits_table(res.hits())
    oh = PU.oracle_hits_table(orc["hits"])
    assert res.counts()["hits"] == len(gh) > 10**5
    assert gh["h"].min() >= h0 and gh["h"].max() < h1 and (gh["h"] >= 1 << 32).any()
    hc = PU.compare_hits(gh, oh, h1 - h0)
    assert hc["frac_identical"] >= 0.9999, hc
    assert hc["max_rel_e"] <= PU.E_REL and hc["max_dt"] <= PU.T_ABS, hc
    tc, te = res.tallies()
    tq = PU.compare_tallies(tc, te, orc, gh, hc["bad"])
    assert tq["count_excess"] <= 0 and tq["energy_excess"] <= 0, tq
    assert tq["energy_total_rel"] < 1e-4, tq
    res.free()
    sc.close()
