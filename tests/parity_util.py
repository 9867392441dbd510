"""Element-by-element comparison of the CUDA path with the FP64 oracle on the
same Philox streams (test infrastructure).

Tolerances (FP32 transport against FP64):
  * crystal / layer ids identical, history by history, in >= 99.99 % of histories;
  * deposits within 1e-5 relative; times within 1 ps;
  * positions within 1e-3 mm, except in ill-conditioned histories: where a ray
    meets a panel face at a grazing angle a, the entry point moves along the
    face by the FP32 rounding of the ray over sin(a), so a fixed bound is
    crossed by rare grazing entries whatever the arithmetic.  A history with a
    hit beyond 1e-3 mm (but within POS_CAP, and with identical ids) counts
    against the same 0.01 % budget as a decision flip;
  * blurred energies within 1e-5 relative + 1e-3 keV; window-edge flips allowed
    only within 1e-3 keV of an edge;
  * depth of interaction of a single (energy-weighted hit depth plus its blur)
    within 2e-3 mm: the hit positions' 1e-3 mm plus FP32 rounding of the blur.
"""
from __future__ import annotations

import numpy as np

E_REL = 1e-5
POS_ABS = 1e-3
POS_CAP = 0.05   # a position outlier must still lie within 5 % of a 1 mm pitch
T_ABS = 1
EB_ABS = 1e-3
DOI_ABS = 2e-3


def gpu_hits_table(h):
    g = (h["gstep"] >> 24).astype(np.int64)
    step = (h["gstep"] & 0xFFFFFF).astype(np.int64)
    t = np.zeros(len(h["h"]), dtype=[("h", "<u8"), ("gamma", "<i8"), ("step", "<i8"), ("crystal", "<i8"),
                                     ("layer", "<i8"), ("w", "<f8"), ("u", "<f8"), ("v", "<f8"), ("e", "<f8"),
                                     ("t", "<i8")])
    t["h"], t["gamma"], t["step"], t["crystal"], t["layer"] = h["h"], g, step, h["crystal"], h["layer"]
    t["w"], t["u"], t["v"] = h["wuv"][:, 0], h["wuv"][:, 1], h["wuv"][:, 2]
    t["e"], t["t"] = h["e"], h["t_ps"].astype(np.int64)
    return np.sort(t, order=["h", "gamma", "step"])


def oracle_hits_table(h):
    t = np.zeros(len(h), dtype=[("h", "<u8"), ("gamma", "<i8"), ("step", "<i8"), ("crystal", "<i8"),
                                ("layer", "<i8"), ("w", "<f8"), ("u", "<f8"), ("v", "<f8"), ("e", "<f8"),
                                ("t", "<i8")])
    for f in ("h", "gamma", "step", "crystal", "layer", "w", "u", "v"):
        t[f] = h[f]
    t["e"], t["t"] = h["edep"], h["t_ps"].astype(np.int64)
    return np.sort(t, order=["h", "gamma", "step"])


def _key(t):
    return (t["h"].astype(np.uint64) << np.uint64(20)) | (t["gamma"].astype(np.uint64) << np.uint64(19)) | \
        t["step"].astype(np.uint64)


def compare_hits(gpu, orc, n_histories):
    """Returns dict with the set of mismatched histories and the worst deviations
    over the hits of matching histories."""
    kg, ko = _key(gpu), _key(orc)
    common, ig, io = np.intersect1d(kg, ko, assume_unique=False, return_indices=True)
    bad = set(np.setdiff1d(gpu["h"], orc["h"][io]).tolist()) | set(np.setdiff1d(orc["h"], gpu["h"][ig]).tolist())
    only_g = np.setdiff1d(kg, common)
    only_o = np.setdiff1d(ko, common)
    bad |= set((only_g >> np.uint64(20)).tolist()) | set((only_o >> np.uint64(20)).tolist())
    g, o = gpu[ig], orc[io]
    diff_id = (g["crystal"] != o["crystal"]) | (g["layer"] != o["layer"])
    bad |= set(g["h"][diff_id].tolist())
    ok = ~np.isin(g["h"], np.array(sorted(bad), dtype=np.uint64))
    g, o = g[ok], o[ok]
    rel_e = np.abs(g["e"] - o["e"]) / np.maximum(o["e"], 1e-30)
    pos = np.max(np.abs(np.stack([g["w"] - o["w"], g["u"] - o["u"], g["v"] - o["v"]])), axis=0) if len(g) else np.zeros(0)
    dt = np.abs(g["t"] - o["t"])
    # ill-conditioned histories (grazing entries): counted against the budget
    out_h = set(g["h"][pos > POS_ABS].tolist())
    max_pos_outlier = float(pos[pos > POS_ABS].max()) if (pos > POS_ABS).any() else 0.0
    worst = None
    if len(g):
        k = np.argsort(pos)[-3:][::-1]
        worst = [dict(h=int(g["h"][i]), gamma=int(g["gamma"][i]), step=int(g["step"][i]), crystal=int(g["crystal"][i]),
                      gpu=(float(g["w"][i]), float(g["u"][i]), float(g["v"][i])),
                      orc=(float(o["w"][i]), float(o["u"][i]), float(o["v"][i])), e=float(o["e"][i]),
                      dev=float(pos[i])) for i in k]
    in_bound = ~np.isin(g["h"], np.array(sorted(out_h), dtype=np.uint64))
    return dict(bad=bad, frac_identical=1.0 - (len(bad) + len(out_h)) / max(n_histories, 1), n_compared=len(g),
                pos_outliers=len(out_h), max_pos_outlier=max_pos_outlier,
                max_rel_e=float(rel_e.max()) if len(g) else 0.0,
                max_pos=float(pos[in_bound].max()) if in_bound.any() else 0.0,
                max_dt=int(dt.max()) if len(g) else 0, n_gpu=len(gpu), n_orc=len(orc), worst_pos=worst,
                p999_pos=float(np.quantile(pos, 0.999)) if len(g) else 0.0)


def compare_singles(gs, os_, bad, e_lo, e_hi):
    """gs: dict of GPU singles arrays; os_: oracle structured singles (all, with kept flag)."""
    ok_o = os_[os_["kept"] == 1]
    badarr = np.array(sorted(bad), dtype=np.uint64)
    mg = ~np.isin(gs["h"], badarr)
    mo = ~np.isin(ok_o["h"], badarr)
    kg = (gs["h"][mg].astype(np.uint64) << np.uint64(32)) | gs["unit"][mg].astype(np.uint64)
    ko = (ok_o["h"][mo].astype(np.uint64) << np.uint64(32)) | ok_o["unit"][mo].astype(np.uint64)
    common, ig, io = np.intersect1d(kg, ko, return_indices=True)
    eg = gs["e"][mg][ig].astype(np.float64)
    eo = ok_o["e_blur"][mo][io]
    rg = gs["e_raw"][mg][ig].astype(np.float64)
    ro = ok_o["e_raw"][mo][io]
    dgi = gs["doi"][mg][ig].astype(np.float64)
    doo = ok_o["doi_blur"][mo][io]
    tg = gs["t_ps"][mg][ig].astype(np.int64)
    to = ok_o["t_ps"][mo][io].astype(np.int64)
    # singles on one side only must sit at a window edge (blur flips)
    all_o = os_[~np.isin(os_["h"], badarr)]
    ka = (all_o["h"].astype(np.uint64) << np.uint64(32)) | all_o["unit"].astype(np.uint64)
    edge_flips = 0
    for k in np.setdiff1d(kg, common):
        j = np.nonzero(ka == k)[0]
        if len(j) == 0:
            edge_flips += 10**9
            continue
        e = all_o["e_blur"][j[0]]
        edge_flips += 1 if min(abs(e - e_lo), abs(e - e_hi)) < EB_ABS else 10**9
    for k in np.setdiff1d(ko, common):
        j = np.nonzero(ko == k)[0][0]
        e = ok_o["e_blur"][mo][j]
        edge_flips += 1 if min(abs(e - e_lo), abs(e - e_hi)) < EB_ABS else 10**9
    return dict(n_gpu=int(mg.sum()), n_orc=int(mo.sum()), n_common=len(common), edge_flips=edge_flips,
                max_rel_eraw=float((np.abs(rg - ro) / ro).max()) if len(common) else 0.0,
                max_blur_dev=float((np.abs(eg - eo) - E_REL * eo).max()) if len(common) else 0.0,
                max_dt=int(np.abs(tg - to).max()) if len(common) else 0,
                max_doi_dev=float(np.abs(dgi - doo).max()) if len(common) else 0.0)


def coincidence_set(h, unit, a, b):
    return {frozenset(((int(h[i]), int(unit[i])), (int(h[j]), int(unit[j])))) for i, j in zip(a, b)}


def compare_coincidences(gs, ga, gb, os_sel, oa, ob, bad):
    sg = coincidence_set(gs["h"], gs["unit"], ga, gb)
    so = coincidence_set(os_sel["h"], os_sel["unit"], oa, ob)
    diff = sg ^ so
    unexplained = [c for c in diff if not any(h in bad for h, _ in c)]
    return dict(n_gpu=len(sg), n_orc=len(so), n_diff=len(diff), unexplained=len(unexplained))


def compare_tallies(tc, te, orc, gpu_hits, bad):
    """Per-crystal count and energy tallies of a GPU run against the oracle's,
    allowing each crystal the hits of the mismatched histories (`bad`) on both
    sides, plus the FP32 deposit rounding (1e-5 relative) and one quantum of
    the fixed-point energy per hit.  Returns the excess over that allowance
    (<= 0 when within it) and the relative difference of the energy totals."""
    badarr = np.array(sorted(bad), dtype=np.uint64)
    ob = orc["hits"][np.isin(orc["hits"]["h"], badarr)]
    gb = gpu_hits[np.isin(gpu_hits["h"], badarr)]
    allow_c = np.zeros(len(tc))
    np.add.at(allow_c, ob["crystal"], 1)
    np.add.at(allow_c, gb["crystal"], 1)
    dc = np.abs(tc.astype(np.int64) - orc["tally_count"].astype(np.int64))
    allow_e = np.zeros(len(tc))
    np.add.at(allow_e, ob["crystal"], ob["edep"] * 2 ** 20)
    np.add.at(allow_e, gb["crystal"], gb["e"] * 2 ** 20)
    de = np.abs(te.astype(np.float64) - orc["tally_efx"].astype(np.float64))
    e_tot = float(orc["tally_efx"].astype(np.float64).sum())
    return dict(count_excess=float((dc - allow_c).max()) if len(tc) else 0.0,
                energy_excess=float((de - allow_e - E_REL * orc["tally_efx"] - tc - 1).max()) if len(tc) else 0.0,
                crystals_differing=int((dc > 0).sum()),
                count_total_rel=abs(float(tc.sum()) - float(orc["tally_count"].sum())) / max(float(orc["tally_count"].sum()), 1.0),
                energy_total_rel=abs(float(te.astype(np.float64).sum()) - e_tot) / max(e_tot, 1.0))
