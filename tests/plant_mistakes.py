#!/usr/bin/env python3
"""Planted mistakes in the oracle: does every pin bite?

Each entry of MUTS is one plausible mistake, written as text replacements in
a copy of oracle/gpet_oracle.c (or oracle/oracle.py, marked "py").  For each
mistake the copy is compiled into its own library under tests/_mutants/ and
every pin of tests/test_oracle_pins.py runs against it; the script prints
which pins fail.  A mistake that no pin catches is either equivalent (it
cannot change any output) or a missing pin.

    python tests/plant_mistakes.py                 # all mistakes (~7 s each)
    python tests/plant_mistakes.py e3_law hit_time_c

Test infrastructure: it reads the oracle's sources and never touches the CUDA
library.  Equivalent mistakes kept here on purpose: module_gap_ignored,
voxel_pick_geq, inside_phantom_closed, passive_as_detector; sens_seed_shared
is a convention that only the GPU comparison of the map fixes.
"""
import importlib.util
import inspect
import itertools
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import tests.test_oracle_pins as T  # noqa: E402

MUTS = dict(
    coinc_sliding_window=[("        i = j + 1;\n    }\n    free(k);", "        i = i + 1;\n    }\n    free(k);")],
    coinc_multiples_kept=[("if (j - i + 1 == 2 && k[i].panel", "if (j - i + 1 >= 2 && k[i].panel")],
    coinc_same_panel_kept=[("if (j - i + 1 == 2 && k[i].panel != k[i + 1].panel)", "if (j - i + 1 == 2)")],
    time_span_in_ns=[("(double)n_decays / activity_bq * 1e12", "(double)n_decays / activity_bq * 1e9")],
    coinc_half_open_window=[("k[j + 1].t - k[i].t <= window_ps", "k[j + 1].t - k[i].t < window_ps")],
    posed_uv_swapped=[("        *u = or_dot3(p, g->ax[k][1]);\n        *v = or_dot3(p, g->ax[k][2]);",
                       "        *u = or_dot3(p, g->ax[k][2]);\n        *v = or_dot3(p, g->ax[k][1]);")],
    posed_dir_w_sign=[("        *dw = or_dot3(d, g->ax[k][0]);", "        *dw = -or_dot3(d, g->ax[k][0]);")],
    posed_origin_sign=[("const double p[3] = {x[0] - g->org[k][0], x[1] - g->org[k][1], x[2] - g->org[k][2]};",
                        "const double p[3] = {x[0] + g->org[k][0], x[1] - g->org[k][1], x[2] - g->org[k][2]};")],
    posed_global_rotation=[("                if (g->posed) {\n                    /* posed panel: the polar",
                            "                if (0) {\n                    /* posed panel: the polar")],
    doi_sigma=[("C->dg->doi_fwhm_mm / (2.0 * sqrt(2.0 * log(2.0))) * n02", "C->dg->doi_fwhm_mm / 2.0 * n02")],
    doi_unweighted=[("        s.doi = ew / s.e_raw;", "        s.doi = ew;")],
    det_free_path_units=[("-log(or_uniform(r[0])) / mu_maj * 10.0", "-log(or_uniform(r[0])) / mu_maj * 1.0", 2)],
    phantom_step_units=[("-log(or_uniform(r[0])) / mu_maj * 10.0", "-log(or_uniform(r[0])) / mu_maj * 1.0", 1)],
    kn_dropped_term=[("(t1 + t2 - t3);", "(t1 + t2);")],
    kahn_branch1=[("accept = r3 * eta * eta <= 4.0 * xm1;", "accept = r3 * eta <= 4.0 * xm1;")],
    kahn_branch2=[("accept = 2.0 * r3 <= c * c + 1.0 / eta;", "accept = 2.0 * r3 <= c * c + eta;")],
    rotate_sign=[("d[2] = dz * c - s * q * cp;", "d[2] = dz * c + s * q * cp;")],
    photo_branch=[("return u * mu_m < or_mu_photo(m, e_kev);", "return u * mu_m > or_mu_photo(m, e_kev);")],
    e3_law=[("return m->mu_total_511_cm * m->photo_frac_511 * r * r * r;",
             "return m->mu_total_511_cm * m->photo_frac_511 * r * r;")],
    crystal_index_transposed=[("g->layer_off[l] + iv * L->n_u + iu;", "g->layer_off[l] + iu * L->n_v + iv;")],
    hit_time_c=[("floor(path / OR_C_MM_PER_PS)", "floor(path * OR_C_MM_PER_PS)")],
    blur_law=[("double sigma = sig_k * sqrt(OR_E0_KEV * s.e_raw);", "double sigma = sig_k * s.e_raw;")],
    earliest_time=[("if (hh[j].t_ps < s.t_ps) s.t_ps = hh[j].t_ps;", "if (hh[j].t_ps > s.t_ps) s.t_ps = hh[j].t_ps;")],
    energy_sum=[("            s.e_raw += hh[j].edep;", "            s.e_raw = hh[j].edep;")],
    cutoff_deposit=[("if (Ep < C->dg->e_cut) { dep = E; dead = 1; }", "if (Ep < C->dg->e_cut) { dep = T; dead = 1; }")],
    module_gap_ignored=[("if (a_u >= sc->module_size_u || a_v >= sc->module_size_v) return; /* module gap */",
                         "if (0) return; /* module gap */")],
    photo_share_at_511=[("return u * mu_m < or_mu_photo(m, e_kev);",
                         "return u * mu_m < or_mu_photo(m, 511.0) * mu_m / or_mu_total(m, 511.0);")],
    det_majorant_at_511=[("double mu_maj = or_majorant(sc->materials, sc->n_materials, E);\n            double s = mu_maj > 0.0 ? -log(or_uniform(r[0])) / mu_maj * 10.0 : INFINITY;\n            if (s >= t_rem) {                                         /* leaves the panel */",
                          "double mu_maj = or_majorant(sc->materials, sc->n_materials, 511.0);\n            double s = mu_maj > 0.0 ? -log(or_uniform(r[0])) / mu_maj * 10.0 : INFINITY;\n            if (s >= t_rem) {                                         /* leaves the panel */")],
    compton_no_energy_update=[("else { dep = T; E = Ep; }", "else { dep = T; }")],
    flight_farthest=[("if (or_panel_hit(g, k, x, d, &ti, &to) && ti < bi) { best = k; bi = ti; bo = to; }",
                      "if (or_panel_hit(g, k, x, d, &ti, &to) && (best < 0 || ti > bi)) { best = k; bi = ti; bo = to; }")],
    phantom_majorant_at_511=[("double mu_maj = or_majorant(ph->materials, ph->n_materials, E);",
                              "double mu_maj = or_majorant(ph->materials, ph->n_materials, 511.0);")],
    voxel_pick_geq=[("if (P->cdf[i] > target) return i;", "if (P->cdf[i] >= target) return i;")],
    voxel_index_order=[("int64_t ix = vi % ph->nx, iy = (vi / ph->nx) % ph->ny, iz = vi / ((int64_t)ph->nx * ph->ny);",
                        "int64_t iz = vi % ph->nz, iy = (vi / ph->nz) % ph->ny, ix = vi / ((int64_t)ph->nz * ph->ny);")],
    decay_hemisphere=[("double ct = 2.0 * or_uniform(r[2]) - 1.0;", "double ct = or_uniform(r[2]);")],
    decay_time_half=[("*t0 = (uint64_t)(((unsigned __int128)C->t_span_ps * r64) >> 64);",
                      "*t0 = (uint64_t)(((unsigned __int128)C->t_span_ps * r64) >> 65);")],
    phantom_compton_at_511=[("            double mu_m = or_mu_total(m, E);\n            if (or_uniform(r[1]) * mu_maj >= mu_m) continue;          /* virtual */",
                             "            double mu_m = or_mu_total(m, 511.0);\n            if (or_uniform(r[1]) * mu_maj >= mu_m) continue;          /* virtual */")],
    flight_first_listed=[("if (or_panel_hit(g, k, x, d, &ti, &to) && ti < bi) { best = k; bi = ti; bo = to; }",
                          "if (or_panel_hit(g, k, x, d, &ti, &to) && best < 0) { best = k; bi = ti; bo = to; }")],
    panel_depth_from_far_face=[("double lo[3] = {0.0, -0.5 * g->U, -0.5 * g->V};", "double lo[3] = {0.5 * g->W, -0.5 * g->U, -0.5 * g->V};")],
    panel_tout_wrong=[("        if (tf < tmax) tmax = tf;", "        if (tf > tmax || tmax == INFINITY) tmax = tf;")],
    phantom_exit_one_axis=[("    for (int a = 0; a < 3; ++a) {\n        if (d[a] > 0.0) { double tt = (P->hi[a] - x[a]) / d[a]; if (tt < t) t = tt; }",
                            "    for (int a = 0; a < 1; ++a) {\n        if (d[a] > 0.0) { double tt = (P->hi[a] - x[a]) / d[a]; if (tt < t) t = tt; }")],
    phantom_mat_transposed=[("return ph->mat[((int64_t)i[2] * ph->ny + i[1]) * ph->nx + i[0]];",
                             "return ph->mat[((int64_t)i[0] * ph->ny + i[1]) * ph->nz + i[2]];")],
    module_unit_wrong=[("return H->panel * sc->modules_u * sc->modules_v + H->module;", "return H->module;")],
    inside_phantom_closed=[("if (!(x[a] >= P->lo[a] && x[a] < P->hi[a])) return 0;", "if (!(x[a] > P->lo[a] && x[a] < P->hi[a])) return 0;")],
    hit_uv_swapped=[("H->w = w; H->u = u; H->v = v; H->edep = dep;", "H->w = w; H->u = v; H->v = u; H->edep = dep;")],
    hit_w_from_u=[("H->w = w; H->u = u; H->v = v; H->edep = dep;", "H->w = u; H->u = u; H->v = v; H->edep = dep;")],
    tally_count_shift=[("            tc[hh[i].crystal] += 1;", "            tc[hh[i].crystal] += hh[i].layer + 1;")],
    tally_efx_scale=[("tefx[hh[i].crystal] += (uint64_t)nearbyint(hh[i].edep * OR_EFX_SCALE);",
                      "tefx[hh[i].crystal] += (uint64_t)nearbyint(hh[i].edep * OR_EFX_SCALE * 0.5);")],
    passive_as_detector=[("            } else {\n                en->passive += dep;", "            } else {\n                en->det += dep;")],
    gap_before_ignored=[("        w += sc->layers[l].gap_before;\n", "")],
    layer_off_zero=[("        g->layer_off[l] = off;", "        g->layer_off[l] = 0;")],
    ring_angle_sign=[("double phi = sc->first_angle + 2.0 * OR_PI * k / sc->n_panels;", "double phi = sc->first_angle - 2.0 * OR_PI * k / sc->n_panels;")],
    panel_U_no_gap=[("g->U = sc->modules_u * sc->module_size_u + (sc->modules_u - 1) * sc->module_gap_u;", "g->U = sc->modules_u * sc->module_size_u;")],
    sens_per_two=[("return counts, counts.astype(np.float64) / float(n_decays)", "return counts, counts.astype(np.float64) / float(2 * n_decays)", 1, "py")],
    sens_seed_shared=[("r = simulate(sc, src, dg, n_decays, seed + p,", "r = simulate(sc, src, dg, n_decays, seed,", 1, "py")],
    dsym_scale=[("out[nz] = 200.0 * (a - b)[nz] / tot[nz]", "out[nz] = 100.0 * (a - b)[nz] / tot[nz]", 1, "py")],
    crystal_gap_one_side=[("if (cu < 0.5 * L->gap_u || cu >= L->pitch_u - 0.5 * L->gap_u) return;",
                           "if (cu >= L->pitch_u - L->gap_u) return;")],
)


def cases():
    """Every pin, with its parametrisations expanded."""
    for name, f in inspect.getmembers(T, inspect.isfunction):
        if not name.startswith("test_"):
            continue
        marks = [m for m in getattr(f, "pytestmark", []) if m.name == "parametrize"]
        if not marks:
            yield name, f, {}
            continue
        grids = []
        for m in marks:
            argn = [a.strip() for a in m.args[0].split(",")] if isinstance(m.args[0], str) else list(m.args[0])
            vals = [v if len(argn) > 1 else (v,) for v in m.args[1]]
            grids.append([dict(zip(argn, v)) for v in vals])
        for combo in itertools.product(*grids):
            kw = {}
            for c in combo:
                kw.update(c)
            yield f"{name}{list(kw.values())}", f, kw


def apply(text, edits):
    for e in edits:
        a, b = e[0], e[1]
        nth = e[2] if len(e) > 2 else 1
        assert text.count(a) >= nth, a
        i = -1
        for _ in range(nth):
            i = text.index(a, i + 1)
        text = text[:i] + b + text[i + len(a):]
    return text


def run(name):
    """Build the oracle with mistake `name` planted and return the pins that fail."""
    c_src = open(os.path.join(ROOT, "oracle", "gpet_oracle.c")).read()
    py_src = open(os.path.join(ROOT, "oracle", "oracle.py")).read()
    edits = MUTS[name]
    d = os.path.join(ROOT, "tests", "_mutants", name)
    os.makedirs(d, exist_ok=True)
    with open(os.path.join(d, "oracle.py"), "w") as f:
        f.write(apply(py_src, [e for e in edits if len(e) > 3 and e[3] == "py"]))
    with open(os.path.join(d, "gpet_oracle.c"), "w") as f:
        f.write(apply(c_src, [e for e in edits if not (len(e) > 3 and e[3] == "py")]))
    spec = importlib.util.spec_from_file_location("mutant_" + name, os.path.join(d, "oracle.py"))
    O = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(O)
    O.build(force=True)
    failed = []
    for cname, f, kw in cases():
        try:
            f(O, **kw) if "oracle" in inspect.signature(f).parameters else f(**kw)
        except AssertionError:
            failed.append(cname)
        except Exception as e:  # a crash is caught too
            failed.append(f"{cname}<{type(e).__name__}>")
    return failed


def main(names):
    for name in names or sorted(MUTS):
        t0 = time.time()
        failed = run(name)
        print(f"{name:26s} caught by {len(failed)}: {failed[:4]} ({time.time() - t0:.0f} s)", flush=True)


if __name__ == "__main__":
    main(sys.argv[1:])
