#!/usr/bin/env python3
"""Measured error of every reported quantity against the FP64 oracle.

Runs the CUDA path (default launch form) and the oracle on the same seeded
inputs and Philox streams, and prints one markdown table: for each quantity the
largest deviation found over the cases below, with the quantity's bar.  Needs a
GPU.  Usage: python tests/error_table.py [--threads N]

Cases: the tiny ring (1e5 pairs), the 12-panel sweep ring with one and two
layers (2e5 pairs each), the offset dual-layer ring with the hot-rod phantom
as source (4e4 pairs), an off-centre source in the H2RSPET-2CL ring (6e4
pairs); a sampled range of 2e6 histories straddling history 2^32 of a
(2^32 + 2^28)-history run; the sensitivity map S(r, E) and Delta_sym of the
H2RSPET-1CL and -2CL rings at 4 positions x 4 windows, 2e5 pairs each.
"""
from __future__ import annotations

import argparse
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402
from tests import parity_util as PU  # noqa: E402

CASES = [
    ("tiny ring", W.config1_scanner, lambda: W.point_source(), None, 100_000, 1),
    ("sweep ring, one 10 mm layer", lambda: W.config2_scanner("A"), lambda: W.point_source((0.0, 0.0, 13.0)), None,
     200_000, 15),
    ("sweep ring, two 5 mm layers", lambda: W.config2_scanner("B"), lambda: W.point_source((0.0, 0.0, -30.0)), None,
     200_000, 2),
    ("offset dual layer, hot-rod phantom", W.config3_scanner, W.phantom_source, W.hot_rod_phantom, 40_000, 3),
    ("H2RSPET-2CL, off-centre source", lambda: W.h2rspet("2CL", modules_v=2),
     lambda: W.point_source((21.0, -13.0, 9.0)), None, 60_000, 77),
]


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--threads", type=int, default=os.cpu_count() or 1)
    args = ap.parse_args()
    from paper_2603_07327_gb300 import build as B
    B.build()
    import paper_2603_07327_gb300 as G
    from oracle import oracle as O
    O.build()

    worst = dict(ident=1.0, e_rel=0.0, pos=0.0, pos_out=0, pos_out_max=0.0, dt=0, eraw=0.0, eblur=0.0, st=0, doi=0.0,
                 flips=0, coinc_rel=0.0, coinc_unexpl=0, tally_c=0.0, tally_e=0.0, tally_cx=0.0, tally_ex=0.0)
    n_hist = 0
    for name, mk_sc, mk_src, mk_ph, n, seed in CASES:
        sc, src = mk_sc(), mk_src()
        ph = mk_ph() if mk_ph else None
        dg = W.digitizer(doi_fwhm_mm=1.5)
        res = G.simulate(sc, src, dg, n, seed, phantom=ph, keep_hits=True)
        orc = O.simulate(sc, src, dg, n, seed, phantom=ph, threads=args.threads)
        gh, oh = PU.gpu_hits_table(res.hits()), PU.oracle_hits_table(orc["hits"])
        hc = PU.compare_hits(gh, oh, n)
        n_hist += n
        worst["ident"] = min(worst["ident"], hc["frac_identical"])
        worst["e_rel"] = max(worst["e_rel"], hc["max_rel_e"])
        worst["pos"] = max(worst["pos"], hc["max_pos"])
        worst["pos_out"] += hc["pos_outliers"]
        worst["pos_out_max"] = max(worst["pos_out_max"], hc["max_pos_outlier"])
        worst["dt"] = max(worst["dt"], hc["max_dt"])
        gs = res.singles()
        sc_ = PU.compare_singles(gs, orc["singles"], hc["bad"], dg["e_lo"], dg["e_hi"])
        worst["eraw"] = max(worst["eraw"], sc_["max_rel_eraw"])
        worst["eblur"] = max(worst["eblur"], sc_["max_blur_dev"])
        worst["st"] = max(worst["st"], sc_["max_dt"])
        worst["doi"] = max(worst["doi"], sc_["max_doi_dev"])
        worst["flips"] += sc_["edge_flips"]
        ga, gb = res.coincidences()
        osel, oa, ob = O.coincidences(orc["singles"], dg["window_ns"])
        cc = PU.compare_coincidences(gs, ga, gb, osel, oa, ob, hc["bad"])
        worst["coinc_rel"] = max(worst["coinc_rel"], abs(cc["n_gpu"] - cc["n_orc"]) / max(cc["n_orc"], 1))
        worst["coinc_unexpl"] += cc["unexplained"]
        tc, te = res.tallies()
        tq = PU.compare_tallies(tc, te, orc, gh, hc["bad"])
        worst["tally_c"] = max(worst["tally_c"], tq["count_total_rel"])
        worst["tally_e"] = max(worst["tally_e"], tq["energy_total_rel"])
        worst["tally_cx"] = max(worst["tally_cx"], tq["count_excess"])
        worst["tally_ex"] = max(worst["tally_ex"], tq["energy_excess"])
        res.free()
        print(f"# {name}: {n} histories, {hc['frac_identical']:.6f} identical, {len(gh)} hits, "
              f"{sc_['n_common']} singles compared, {cc['n_gpu']} / {cc['n_orc']} coincidences", flush=True)

    # tallies past 2^32 histories: a sampled range of a 4.56e9-history run
    N = (1 << 32) + (1 << 28)
    sc = G.Scanner(W.config2_scanner("B"))
    src = W.point_source((0.0, 0.0, 11.0))
    dg = W.digitizer(e_lo=0.0, e_hi=0.0)
    dg["window_ns"] = 0.0
    h0, h1 = (1 << 32) - 1_000_000, (1 << 32) + 1_000_000
    res = sc.simulate(src, dg, N, 31, h_begin=h0, h_end=h1, keep_hits=True)
    orc = O.simulate(W.config2_scanner("B"), src, dg, N, 31, h_begin=h0, h_end=h1, threads=args.threads)
    gh, oh = PU.gpu_hits_table(res.hits()), PU.oracle_hits_table(orc["hits"])
    hc = PU.compare_hits(gh, oh, h1 - h0)
    tc, te = res.tallies()
    big = PU.compare_tallies(tc, te, orc, gh, hc["bad"])
    big["ident"] = hc["frac_identical"]
    res.free()
    sc.close()
    print(f"# tallies past 2^32: {h1 - h0} histories, {hc['frac_identical']:.6f} identical, {len(gh)} hits",
          flush=True)

    # sensitivity map and Delta_sym
    designs = [W.h2rspet("1CL"), W.h2rspet("2CL")]
    scs = [G.Scanner(d) for d in designs]
    pos = np.array([(0.0, 0.0, 0.0), (20.0, 0.0, 0.0), (50.0, 0.0, 0.0), (0.0, 0.0, 60.0)])
    sdg = W.sensitivity_digitizer()
    n = 200_000
    counts, S, _ = G.sensitivity_map(scs, pos, sdg, W.SENS_WINDOWS_KEV, n, 2603)
    oc, oS = O.sensitivity_map(designs, pos, sdg, W.SENS_WINDOWS_KEV, n, 2603, threads=args.threads)
    s_rel = np.abs(S - oS) / np.maximum(oS, 1e-30)
    s_abs = np.abs(counts.astype(np.int64) - oc.astype(np.int64))
    d_gpu, d_orc = G.delta_sym(S[0], S[1]), O.delta_sym(oS[0], oS[1])
    d_dev = float(np.nanmax(np.abs(d_gpu - d_orc)))
    for s in scs:
        s.close()
    print(f"# sensitivity map: {counts.size} cells, {int(oc.sum())} oracle coincidences", flush=True)

    rows = [
        ("histories with identical crystal / layer ids", f"{worst['ident']:.6f} (lowest case), "
         f"{n_hist} histories", ">= 0.9999"),
        ("deposited energy per hit (relative)", f"{worst['e_rel']:.2e}", "<= 1e-5"),
        ("hit position (mm)", f"{worst['pos']:.2e}; {worst['pos_out']} grazing-entry outliers "
         f"(<= {worst['pos_out_max']:.2e} mm)", "<= 1e-3 (outliers <= 0.05, within the 0.01 % budget)"),
        ("hit time (ps)", f"{worst['dt']}", "<= 1"),
        ("single: deposited energy (relative)", f"{worst['eraw']:.2e}", "<= 1e-5"),
        ("single: blurred energy (keV beyond 1e-5 relative)", f"{worst['eblur']:.2e}; {worst['flips']} window-edge "
         "flips", "<= 1e-3; flips only within 1e-3 keV of an edge"),
        ("single: time (ps)", f"{worst['st']}", "<= 1"),
        ("single: blurred depth of interaction (mm)", f"{worst['doi']:.2e}", "<= 2e-3"),
        ("coincidence count (relative)", f"{worst['coinc_rel']:.2e}; {worst['coinc_unexpl']} pairs not explained "
         "by flipped histories or edge flips", "identical outside flipped histories"),
        ("per-crystal count tally: total (relative)", f"{worst['tally_c']:.2e}; excess over the flipped histories' "
         f"hits {worst['tally_cx']:.0f}", "identical up to flipped histories"),
        ("per-crystal energy tally: total (relative)", f"{worst['tally_e']:.2e}; excess over the allowance "
         f"{worst['tally_ex']:.2e} units of 2^-20 keV", "within 1e-5 relative + flipped histories"),
        ("tallies past 2^32 histories (sampled 2e6-history range)", f"identical histories {big['ident']:.6f}; "
         f"count total {big['count_total_rel']:.2e}, energy total {big['energy_total_rel']:.2e} (relative); "
         f"excess {big['count_excess']:.0f} / {big['energy_excess']:.2e}", "as above"),
        ("sensitivity S(r, E) per cell (relative)", f"max {float(s_rel.max()):.2e}, mean {float(s_rel.mean()):.2e}; "
         f"max {int(s_abs.max())} coincidences of {int(oc.min())}..{int(oc.max())}", "flipped histories only"),
        ("Delta_sym per cell (percentage points)", f"{d_dev:.2e}", "follows S"),
    ]
    print("\n| quantity | measured deviation from the FP64 oracle | bar |")
    print("|---|---|---|")
    for q, m, b in rows:
        print(f"| {q} | {m} | {b} |")


if __name__ == "__main__":
    main()
