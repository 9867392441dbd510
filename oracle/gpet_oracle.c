/*
 * gpet_oracle.c -- plain FP64 CPU oracle of the multi-layer gPET photon-pair
 * transport (arxiv 2603.07327).
 *
 * TEST INFRASTRUCTURE.  This file is the "obviously correct" restatement of
 * what the GPU path computes.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load it.  It shares no code, header,
 * table or constant generator with the CUDA library; the two only read the
 * same seeded input descriptions.
 *
 * What it follows (paper sections):
 *   - Sec. 2.1 / Fig. 1: four-level detector hierarchy panel -> module ->
 *     layer -> crystal; repetition mode (one panel, N rotated copies); a
 *     unique crystal / layer / module / panel index for every interaction;
 *     a photon leaving the phantom flies straight to its panel (line-plane
 *     intersection); inside a panel it is moved to the panel-local frame and
 *     tracked step by step with Woodcock free-path sampling; a layer-selection
 *     step picks the crystal layer from the local depth; the repetitive crystal
 *     structure gives material and crystal index; transport stops when the
 *     photon leaves the panel or falls below the cutoff energy; photons that
 *     leave one panel may enter another (abstract: interactions are sampled
 *     over several layers and several panels).
 *   - Sec. 2.3: point source, no positron range, annihilation at the emission
 *     site (back-to-back 511 keV pair); energy resolution; energy window;
 *     coincidence timing window.
 *   - Synthetic physics model (not in the paper, which defers to gPET's
 *     original tables): Compton by the closed-form Klein-Nishina cross
 *     section, photoelectric absorption scaling as E^-3 from its 511 keV
 *     value, no Rayleigh scattering, local energy deposition.
 *
 * Readings where the paper is silent (each one is also listed in the design
 * notes): Philox4x32-10 streams keyed by seed and addressed by (history,
 * region tag, photon, step, sub-draw); Kahn's rejection sampling of the
 * Klein-Nishina distribution; 10 keV cutoff with local deposit of the rest;
 * decay times iid uniform on [0, n/A); FWHM proportional to sqrt(E) anchored
 * at 511 keV; inclusive energy window; single-window coincidence policy that
 * keeps exactly-two-single windows in different panels.
 *
 * Parity pins (tests against closed forms, brute force and the paper's text):
 * Philox known-answer vectors; slab transmission exp(-mu L); Klein-Nishina
 * angular distribution (chi-square) and mean energy transfer; photoelectric
 * branching and its E^-3 law; geometric acceptance against the rectangle
 * solid angle; crystal-volume fraction of the offset dual-layer module (the
 * 1.94 % of Sec. 3.2); per-history energy conservation; split-with-zero-gap
 * equals single-layer hit by hit; the Gaussian width of the blur; the
 * coincidence policy against an O(n^2) brute-force sorter.
 *
 * Build: gcc -O2 -std=c11 -ffp-contract=off -fPIC -shared -pthread -lm
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------- */
/* constants of the synthetic model                                           */
/* ------------------------------------------------------------------------- */
#define OR_E0_KEV 511.0                 /* annihilation photon energy (Sec. 2.3) */
#define OR_MEC2_KEV 510.99895           /* electron rest energy (Klein-Nishina kappa) */
#define OR_RE_CM 2.8179403262e-13       /* classical electron radius */
#define OR_C_MM_PER_PS 0.299792458      /* speed of light */
#define OR_PI 3.14159265358979323846
#define OR_MAX_STEPS 1000               /* per photon and region: cap -> error */
#define OR_MAX_TRIALS 1000              /* Kahn rejection cap -> error */
#define OR_MAX_LAYERS 8
#define OR_MAX_MATERIALS 16
#define OR_MAX_PANELS 64
#define OR_EFX_SCALE 1048576.0          /* energy tallies in units of 2^-20 keV */

/* Philox stream tags (high nibble of counter word 2) */
#define OR_TAG_SOURCE 1u
#define OR_TAG_PHANTOM 2u
#define OR_TAG_DETECTOR 3u
#define OR_TAG_DIGI 4u

/* error codes (mirrors the library's meaning, defined here on its own) */
#define OR_OK 0
#define OR_ERR_INVALID -1
#define OR_ERR_GEOMETRY -2
#define OR_ERR_OOM -3
#define OR_ERR_TIMEOUT -5

/* ------------------------------------------------------------------------- */
/* input descriptions (oracle-owned layout, filled by the Python wrapper)     */
/* ------------------------------------------------------------------------- */
typedef struct {
    double mu_total_511_cm, photo_frac_511, electron_density_cm3;
} om_material;

typedef struct {
    int32_t n_u, n_v;
    double pitch_u, pitch_v, gap_u, gap_v, depth, gap_before, offset_u, offset_v;
    int32_t crystal_mat, interval_mat;
} om_layer;

typedef struct {
    int32_t n_panels;
    double inner_radius, first_angle;
    int32_t modules_u, modules_v;
    double module_size_u, module_size_v, module_gap_u, module_gap_v;
    int32_t n_layers;
    const om_layer *layers;
    int32_t n_materials;
    const om_material *materials;
    int32_t readout_level; /* 0 panel, 1 module, 3 crystal */
    /* Non-repetition mode (Sec. 2.1: panels placed one by one): NULL, or 12
     * doubles per panel -- the global unit vectors of the panel's w (depth,
     * away from the inner face), u and v axes, then the global position of the
     * centre of its inner face.  NULL = the repetition-mode ring above. */
    const double *panel_poses;
} om_scanner;

typedef struct {
    int32_t nx, ny, nz;
    double voxel[3], origin[3];
    const uint8_t *mat;      /* nx*ny*nz, x fastest */
    const float *activity;   /* nx*ny*nz or NULL    */
    int32_t n_materials;
    const om_material *materials;
} om_phantom;

typedef struct {
    int32_t kind; /* 0 point, 1 phantom activity, 2 collimated pair along dir */
    double pos[3], dir[3];
    double activity_bq;
} om_source;

typedef struct {
    double fwhm_at_511, e_lo, e_hi, window_ns, e_cut;
    double doi_fwhm_mm;  /* depth blur of a single's interaction depth (0 = none) */
} om_digitizer;

/* one interaction that deposits energy in a crystal */
typedef struct {
    uint64_t h;
    int32_t gamma, step, panel, module, layer, crystal; /* crystal = global id */
    double w, u, v, edep;                               /* local mm, keV */
    uint64_t t_ps;
} om_hit;

typedef struct {
    uint64_t t_ps, h;
    int32_t unit, panel;
    double e_raw, e_blur;
    int32_t kept;
    double doi, doi_blur;  /* energy-weighted depth of the single's hits (mm) and its blurred value */
} om_single;

typedef struct {
    /* counts */
    uint64_t n_hits, n_singles, n_kept;
    om_hit *hits;          /* malloc'd, n_hits */
    om_single *singles;    /* malloc'd, n_singles (kept and rejected, see .kept) */
    /* per-crystal tallies (caller-allocated, n_crystals_total each, may be NULL) */
    uint64_t *tally_count, *tally_efx;
    double *tally_edep;
    /* per-history energy balance (caller-allocated, h_end-h_begin, may be NULL) */
    double *balance;
    /* per-history count of real phantom interactions (caller-allocated, may be NULL) */
    uint32_t *ph_real;
    /* per-history event counters (sums) */
    uint64_t n_det_steps, n_ph_steps, n_flights, n_compton_trials, n_entered;
    int32_t status;
} om_output;

/* ------------------------------------------------------------------------- */
/* Philox4x32-10, from the definition in Salmon, Moraes, Dror and Shaw,       */
/* "Parallel random numbers: as easy as 1, 2, 3" (SC'11).                    */
/* ------------------------------------------------------------------------- */
void or_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]) {
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u; /* multipliers */
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u; /* Weyl key increments */
    uint32_t x0 = ctr_in[0], x1 = ctr_in[1], x2 = ctr_in[2], x3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k0 += W0; k1 += W1; }
        uint64_t p0 = (uint64_t)M0 * x0;
        uint64_t p1 = (uint64_t)M1 * x2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t y0 = hi1 ^ x1 ^ k0;
        uint32_t y1 = lo1;
        uint32_t y2 = hi0 ^ x3 ^ k1;
        uint32_t y3 = lo0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* uniform in (0,1) from the top 23 bits: (k + 1/2) * 2^-23 (exact in FP32 too) */
double or_uniform(uint32_t w) { return ((double)(w >> 9) + 0.5) * 0x1p-23; }

/* draw block for (history, tag, photon, step, sub) under key = seed.  The paper
 * names no generator; every draw is addressed so that one history can be
 * replayed alone and compared with the GPU's, draw for draw. */
static void or_draw(uint64_t seed, uint64_t h, uint32_t tag, uint32_t gamma, uint32_t step,
                    uint32_t sub, uint32_t out[4]) {
    uint32_t ctr[4] = {(uint32_t)h, (uint32_t)(h >> 32),
                       (tag << 28) | ((gamma & 1u) << 27) | (step & 0x07FFFFFFu), sub};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    or_philox4x32_10(ctr, key, out);
}

/* ------------------------------------------------------------------------- */
/* physics: Klein-Nishina total cross section (closed form) and the model    */
/* ------------------------------------------------------------------------- */
/* total KN cross section per electron, cm^2, at photon energy E (keV) */
double or_sigma_kn(double e_kev) {
    double k = e_kev / OR_MEC2_KEV;
    double a = 1.0 + 2.0 * k;
    double l = log(a);
    double t1 = (1.0 + k) / (k * k) * (2.0 * (1.0 + k) / a - l / k);
    double t2 = l / (2.0 * k);
    double t3 = (1.0 + 3.0 * k) / (a * a);
    return 2.0 * OR_PI * OR_RE_CM * OR_RE_CM * (t1 + t2 - t3);
}

/* linear attenuation coefficients in 1/cm of the synthetic physics model used
 * for this study (Sec. 2.1 defers the physics to gPET): photoelectric scaled
 * by (511/E)^3 from its 511 keV value, Compton by the Klein-Nishina total
 * cross section, no Rayleigh scattering */
double or_mu_photo(const om_material *m, double e_kev) {
    double r = OR_E0_KEV / e_kev;
    return m->mu_total_511_cm * m->photo_frac_511 * r * r * r;
}

double or_mu_compton(const om_material *m, double e_kev) {
    if (m->electron_density_cm3 > 0.0) return m->electron_density_cm3 * or_sigma_kn(e_kev);
    double mu_c511 = m->mu_total_511_cm * (1.0 - m->photo_frac_511);
    if (mu_c511 == 0.0) return 0.0;
    return mu_c511 * or_sigma_kn(e_kev) / or_sigma_kn(OR_E0_KEV);
}

double or_mu_total(const om_material *m, double e_kev) {
    return or_mu_photo(m, e_kev) + or_mu_compton(m, e_kev);
}

/* the kind of a real collision (Sec. 2.1): photoelectric with probability
 * mu_pe(E) / mu_total(E) (mu_m = mu_total(E) of the material), decided by the
 * uniform u; Compton otherwise */
static int or_is_photo(const om_material *m, double e_kev, double mu_m, double u) {
    return u * mu_m < or_mu_photo(m, e_kev);
}

/* Kahn's rejection sampling of the Klein-Nishina distribution (Kahn 1954, as
 * written in the Monte Carlo transport literature).  Returns the number of
 * trials used, fills eta - 1 = E/E' - 1 (>= 0).  Draws block (h, tag, gamma,
 * step, sub = 1 + trial) and uses words 0..2 of each block. */
int or_kahn(uint64_t seed, uint64_t h, uint32_t tag, uint32_t gamma, uint32_t step,
            double e_kev, double *eta_m1) {
    double k = e_kev / OR_MEC2_KEV;
    for (int trial = 0; trial < OR_MAX_TRIALS; ++trial) {
        uint32_t r[4];
        or_draw(seed, h, tag, gamma, step, 1u + (uint32_t)trial, r);
        double r1 = or_uniform(r[0]), r2 = or_uniform(r[1]), r3 = or_uniform(r[2]);
        double xm1;
        int accept;
        if (r1 * (9.0 + 2.0 * k) <= 1.0 + 2.0 * k) {
            /* branch 1: eta = 1 + 2k r2, accept with 4 (eta - 1) / eta^2 */
            xm1 = 2.0 * k * r2;
            double eta = 1.0 + xm1;
            accept = r3 * eta * eta <= 4.0 * xm1;
        } else {
            /* branch 2: eta = (1 + 2k)/(1 + 2k r2), accept with (cos^2 + 1/eta)/2 */
            double den = 1.0 + 2.0 * k * r2;
            xm1 = 2.0 * k * (1.0 - r2) / den;
            double eta = 1.0 + xm1;
            double c = 1.0 - xm1 / k;
            accept = 2.0 * r3 <= c * c + 1.0 / eta;
        }
        if (accept) { *eta_m1 = xm1; return trial + 1; }
    }
    return -1;
}

/* rotate unit vector d by polar angle (cos c, sin s) and azimuth phi = 2 pi u:
 * the direction change of a Compton scatter (Sec. 2.1, interactions sampled
 * along the photon's path) */
static void or_rotate(double d[3], double c, double s, double u_phi) {
    double cp = cos(2.0 * OR_PI * u_phi), sp = sin(2.0 * OR_PI * u_phi);
    double dx = d[0], dy = d[1], dz = d[2];
    if (fabs(dz) < 0.99999) {
        double q = sqrt(1.0 - dz * dz);
        d[0] = dx * c + s * (dx * dz * cp - dy * sp) / q;
        d[1] = dy * c + s * (dy * dz * cp + dx * sp) / q;
        d[2] = dz * c - s * q * cp;
    } else {
        d[0] = s * cp;
        d[1] = s * sp;
        d[2] = (dz > 0.0 ? 1.0 : -1.0) * c;
    }
}

/* ------------------------------------------------------------------------- */
/* detector geometry: repetition-mode ring of flat panels (Sec. 2.1)          */
/* ------------------------------------------------------------------------- */
typedef struct {
    const om_scanner *sc;
    double U, V, W;          /* panel extents: u in [-U/2,U/2], v in [-V/2,V/2], w in [0,W] */
    double cphi[OR_MAX_PANELS], sphi[OR_MAX_PANELS];
    int posed;                      /* 1: explicit panel poses (sc->panel_poses) */
    double ax[OR_MAX_PANELS][3][3]; /* posed: the w, u, v axes of each panel */
    double org[OR_MAX_PANELS][3];   /* posed: the centre of each panel's inner face */
    double layer_w0[OR_MAX_LAYERS]; /* start depth of each layer's crystals */
    int32_t layer_off[OR_MAX_LAYERS]; /* crystal-id offset of each layer inside a module */
    int32_t crystals_per_module;
    int32_t n_crystals;     /* whole scanner */
} or_geom;

typedef struct {
    int32_t layer, module, crystal, panel; /* crystal = global id, -1 when not in a crystal */
    int32_t mat;
} or_loc;

/* the detector of Sec. 2.1: panel extents from the modules, layer depths in
 * order, crystal-id offsets, and the panel placements (ring or poses) */
static int or_geom_init(or_geom *g, const om_scanner *sc) {
    if (sc->n_panels < 1 || sc->n_panels > OR_MAX_PANELS || sc->n_layers < 1 ||
        sc->n_layers > OR_MAX_LAYERS || sc->n_materials < 1 || sc->n_materials > OR_MAX_MATERIALS)
        return OR_ERR_INVALID;
    g->sc = sc;
    g->U = sc->modules_u * sc->module_size_u + (sc->modules_u - 1) * sc->module_gap_u;
    g->V = sc->modules_v * sc->module_size_v + (sc->modules_v - 1) * sc->module_gap_v;
    double w = 0.0;
    int32_t off = 0;
    for (int l = 0; l < sc->n_layers; ++l) {
        w += sc->layers[l].gap_before;
        g->layer_w0[l] = w;
        w += sc->layers[l].depth;
        g->layer_off[l] = off;
        off += sc->layers[l].n_u * sc->layers[l].n_v;
    }
    g->W = w;
    g->crystals_per_module = off;
    g->n_crystals = off * sc->modules_u * sc->modules_v * sc->n_panels;
    for (int k = 0; k < sc->n_panels; ++k) {
        double phi = sc->first_angle + 2.0 * OR_PI * k / sc->n_panels;
        g->cphi[k] = cos(phi);
        g->sphi[k] = sin(phi);
    }
    g->posed = sc->panel_poses != NULL;
    if (g->posed)
        for (int k = 0; k < sc->n_panels; ++k) {
            for (int a = 0; a < 3; ++a)
                for (int c = 0; c < 3; ++c) g->ax[k][a][c] = sc->panel_poses[12 * k + 3 * a + c];
            for (int c = 0; c < 3; ++c) g->org[k][c] = sc->panel_poses[12 * k + 9 + c];
        }
    return OR_OK;
}

static double or_dot3(const double a[3], const double b[3]) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

/* global -> panel-local (w = depth from the inner face, u tangential, v axial).
 * Ring: rotation by the panel angle about z, then the radius.  Posed panel:
 * components of x - (inner-face centre) along the panel's own axes. */
static void or_to_local(const or_geom *g, int k, const double x[3], double *w, double *u, double *v) {
    if (g->posed) {
        const double p[3] = {x[0] - g->org[k][0], x[1] - g->org[k][1], x[2] - g->org[k][2]};
        *w = or_dot3(p, g->ax[k][0]);
        *u = or_dot3(p, g->ax[k][1]);
        *v = or_dot3(p, g->ax[k][2]);
        return;
    }
    *w = x[0] * g->cphi[k] + x[1] * g->sphi[k] - g->sc->inner_radius;
    *u = -x[0] * g->sphi[k] + x[1] * g->cphi[k];
    *v = x[2];
}

/* a direction in panel k's frame (Sec. 2.1, panel-local coordinates) */
static void or_dir_local(const or_geom *g, int k, const double d[3], double *dw, double *du, double *dv) {
    if (g->posed) {
        *dw = or_dot3(d, g->ax[k][0]);
        *du = or_dot3(d, g->ax[k][1]);
        *dv = or_dot3(d, g->ax[k][2]);
        return;
    }
    *dw = d[0] * g->cphi[k] + d[1] * g->sphi[k];
    *du = -d[0] * g->sphi[k] + d[1] * g->cphi[k];
    *dv = d[2];
}

/* locate a panel-local point in the hierarchy: layer by depth, module, crystal.
 * Cells are half-open [lo, hi); a crystal occupies [gap/2, pitch - gap/2) of its cell. */
void or_locate(const or_geom *g, int k, double w, double u, double v, or_loc *out) {
    const om_scanner *sc = g->sc;
    out->panel = k;
    out->layer = -1; out->module = -1; out->crystal = -1;
    /* layer selection by local depth; a gap in front of layer j is filled with
     * layer j's interval material, depth beyond the stack with the last layer's */
    int l = -1, owner = sc->n_layers - 1;
    for (int j = 0; j < sc->n_layers; ++j) {
        if (w < g->layer_w0[j]) { owner = j; break; }
        if (w < g->layer_w0[j] + sc->layers[j].depth) { l = j; break; }
    }
    if (l < 0) {
        out->mat = sc->layers[owner].interval_mat;
        return;
    }
    const om_layer *L = &sc->layers[l];
    out->layer = l;
    out->mat = L->interval_mat;
    double au = u + 0.5 * g->U, av = v + 0.5 * g->V;
    double mpu = sc->module_size_u + sc->module_gap_u, mpv = sc->module_size_v + sc->module_gap_v;
    int mu = (int)floor(au / mpu), mv = (int)floor(av / mpv);
    if (mu < 0 || mu >= sc->modules_u || mv < 0 || mv >= sc->modules_v) return;
    double a_u = au - mu * mpu, a_v = av - mv * mpv;
    if (a_u >= sc->module_size_u || a_v >= sc->module_size_v) return; /* module gap */
    out->module = mv * sc->modules_u + mu;
    double bu = a_u - L->offset_u, bv = a_v - L->offset_v;
    int iu = (int)floor(bu / L->pitch_u), iv = (int)floor(bv / L->pitch_v);
    if (iu < 0 || iu >= L->n_u || iv < 0 || iv >= L->n_v) return;
    double cu = bu - iu * L->pitch_u, cv = bv - iv * L->pitch_v;
    if (cu < 0.5 * L->gap_u || cu >= L->pitch_u - 0.5 * L->gap_u) return;
    if (cv < 0.5 * L->gap_v || cv >= L->pitch_v - 0.5 * L->gap_v) return;
    out->mat = L->crystal_mat;
    int32_t module_global = (k * sc->modules_v + mv) * sc->modules_u + mu;
    out->crystal = module_global * g->crystals_per_module + g->layer_off[l] + iv * L->n_u + iu;
}

/* slab test of the ray (x, d) against panel k's box in the panel frame (Sec. 2.1:
 * line-plane intersection with the panel); returns 1 on a hit with t_in < t_out */
static int or_panel_hit(const or_geom *g, int k, const double x[3], const double d[3],
                        double *t_in, double *t_out) {
    double p[3], q[3];
    or_to_local(g, k, x, &p[0], &p[1], &p[2]);
    or_dir_local(g, k, d, &q[0], &q[1], &q[2]);
    double lo[3] = {0.0, -0.5 * g->U, -0.5 * g->V};
    double hi[3] = {g->W, 0.5 * g->U, 0.5 * g->V};
    double tmin = -INFINITY, tmax = INFINITY;
    for (int a = 0; a < 3; ++a) {
        if (q[a] == 0.0) {
            if (p[a] < lo[a] || p[a] > hi[a]) return 0;
            continue;
        }
        double t1 = (lo[a] - p[a]) / q[a], t2 = (hi[a] - p[a]) / q[a];
        double tn = t1 < t2 ? t1 : t2, tf = t1 < t2 ? t2 : t1;
        if (tn > tmin) tmin = tn;
        if (tf < tmax) tmax = tf;
    }
    if (tmin < 0.0) tmin = 0.0;
    if (!(tmin < tmax)) return 0;
    *t_in = tmin;
    *t_out = tmax;
    return 1;
}

/* line-plane flight (Sec. 2.1): nearest panel entered along (x, d), skipping
 * panel `skip`, by testing every panel */
int or_flight(const or_geom *g, const double x[3], const double d[3], int skip, double *t_in,
              double *t_out) {
    int best = -1;
    double bi = INFINITY, bo = 0.0;
    for (int k = 0; k < g->sc->n_panels; ++k) {
        if (k == skip) continue;
        double ti, to;
        if (or_panel_hit(g, k, x, d, &ti, &to) && ti < bi) { best = k; bi = ti; bo = to; }
    }
    if (best >= 0) { *t_in = bi; *t_out = bo; }
    return best;
}

/* ------------------------------------------------------------------------- */
/* phantom                                                                    */
/* ------------------------------------------------------------------------- */
typedef struct {
    const om_phantom *ph;
    double lo[3], hi[3];
    double *cdf;   /* activity prefix sums in voxel order (NULL without activity) */
    double total;
    int64_t last_active;
} or_phantom;

/* the voxel phantom of Sec. 2.3: grid bounds and, with an activity map, its
 * prefix sums in voxel order */
static int or_phantom_init(or_phantom *P, const om_phantom *ph) {
    memset(P, 0, sizeof(*P));
    P->ph = ph;
    if (!ph) return OR_OK;
    for (int a = 0; a < 3; ++a) {
        int n = a == 0 ? ph->nx : (a == 1 ? ph->ny : ph->nz);
        P->lo[a] = ph->origin[a];
        P->hi[a] = ph->origin[a] + n * ph->voxel[a];
    }
    if (ph->activity) {
        int64_t n = (int64_t)ph->nx * ph->ny * ph->nz;
        P->cdf = (double *)malloc(sizeof(double) * (size_t)n);
        if (!P->cdf) return OR_ERR_OOM;
        double s = 0.0;
        P->last_active = -1;
        for (int64_t i = 0; i < n; ++i) {
            double a = (double)ph->activity[i];
            if (a < 0.0) a = 0.0;
            s += a;
            P->cdf[i] = s;
            if (a > 0.0) P->last_active = i;
        }
        P->total = s;
    }
    return OR_OK;
}

/* smallest voxel i with cdf[i] > target (plain linear scan: obviously correct):
 * a voxel with probability proportional to its activity (Sec. 2.3, phantom
 * activity as the source) */
static int64_t or_pick_voxel(const or_phantom *P, double target) {
    int64_t n = (int64_t)P->ph->nx * P->ph->ny * P->ph->nz;
    if (target >= P->total) return P->last_active;
    for (int64_t i = 0; i < n; ++i)
        if (P->cdf[i] > target) return i;
    return P->last_active;
}

/* point inside the phantom grid (half-open box) */
static int or_inside_phantom(const or_phantom *P, const double x[3]) {
    for (int a = 0; a < 3; ++a)
        if (!(x[a] >= P->lo[a] && x[a] < P->hi[a])) return 0;
    return 1;
}

/* distance along d from x to the phantom grid's exit */
static double or_phantom_exit(const or_phantom *P, const double x[3], const double d[3]) {
    double t = INFINITY;
    for (int a = 0; a < 3; ++a) {
        if (d[a] > 0.0) { double tt = (P->hi[a] - x[a]) / d[a]; if (tt < t) t = tt; }
        else if (d[a] < 0.0) { double tt = (P->lo[a] - x[a]) / d[a]; if (tt < t) t = tt; }
    }
    return t < 0.0 ? 0.0 : t;
}

/* material of the voxel holding x */
static int or_phantom_mat(const or_phantom *P, const double x[3]) {
    const om_phantom *ph = P->ph;
    int i[3];
    int n[3] = {ph->nx, ph->ny, ph->nz};
    for (int a = 0; a < 3; ++a) {
        i[a] = (int)floor((x[a] - ph->origin[a]) / ph->voxel[a]);
        if (i[a] < 0) i[a] = 0;
        if (i[a] >= n[a]) i[a] = n[a] - 1;
    }
    return ph->mat[((int64_t)i[2] * ph->ny + i[1]) * ph->nx + i[0]];
}

/* ------------------------------------------------------------------------- */
/* growable per-thread output                                                 */
/* ------------------------------------------------------------------------- */
typedef struct {
    om_hit *hits; size_t n_hits, cap_hits;
    om_single *singles; size_t n_singles, cap_singles;
    uint64_t n_det_steps, n_ph_steps, n_flights, n_compton_trials, n_entered;
    int status;
} or_sink;

static int or_push_hit(or_sink *s, const om_hit *h) {
    if (s->n_hits == s->cap_hits) {
        size_t c = s->cap_hits ? 2 * s->cap_hits : 1024;
        om_hit *p = (om_hit *)realloc(s->hits, c * sizeof(om_hit));
        if (!p) return OR_ERR_OOM;
        s->hits = p; s->cap_hits = c;
    }
    s->hits[s->n_hits++] = *h;
    return OR_OK;
}

static int or_push_single(or_sink *s, const om_single *x) {
    if (s->n_singles == s->cap_singles) {
        size_t c = s->cap_singles ? 2 * s->cap_singles : 1024;
        om_single *p = (om_single *)realloc(s->singles, c * sizeof(om_single));
        if (!p) return OR_ERR_OOM;
        s->singles = p; s->cap_singles = c;
    }
    s->singles[s->n_singles++] = *x;
    return OR_OK;
}

/* ------------------------------------------------------------------------- */
/* one history                                                                */
/* ------------------------------------------------------------------------- */
typedef struct {
    const om_scanner *sc;
    const or_geom *g;
    const or_phantom *P;
    const om_source *src;
    const om_digitizer *dg;
    uint64_t seed, n_decays, t_span_ps;
} or_ctx;

typedef struct {
    double det, passive, phantom, escaped; /* energy channels for the balance */
    uint32_t ph_real;                      /* real interactions in the phantom */
} or_energy;

/* majorant over a material list at energy E (Woodcock tracking, Sec. 2.1) */
static double or_majorant(const om_material *mats, int n, double e) {
    double m = 0.0;
    for (int i = 0; i < n; ++i) {
        double v = or_mu_total(&mats[i], e);
        if (v > m) m = v;
    }
    return m;
}

/* one annihilation photon through the transport of Sec. 2.1: Woodcock steps in
 * the phantom, flight to a panel by line-plane intersection, Woodcock steps in
 * the panel with the layer-selection step, photoelectric absorption or
 * Klein-Nishina Compton scatter, hits in crystals, and on to the next panel
 * until the photon escapes, is absorbed or falls below the cutoff */
static int or_transport_photon(const or_ctx *C, uint64_t h, uint32_t gamma, double x[3], double d[3],
                               uint64_t t0_ps, or_sink *S, om_hit *hist_hits, int *n_hist_hits,
                               int cap_hist, or_energy *en) {
    const or_geom *g = C->g;
    const om_scanner *sc = C->sc;
    double E = OR_E0_KEV, path = 0.0;
    uint32_t s_ph = 0, s_det = 0;

    /* --- phantom: Woodcock tracking through the voxel grid (Sec. 2.1, last paragraph) --- */
    if (C->P->ph && or_inside_phantom(C->P, x)) {
        const om_phantom *ph = C->P->ph;
        for (;;) {
            if (s_ph >= OR_MAX_STEPS) return OR_ERR_TIMEOUT;
            uint32_t r[4];
            or_draw(C->seed, h, OR_TAG_PHANTOM, gamma, s_ph, 0u, r);
            uint32_t step_id = s_ph++;
            S->n_ph_steps++;
            double t_out = or_phantom_exit(C->P, x, d);
            double mu_maj = or_majorant(ph->materials, ph->n_materials, E);
            double s = mu_maj > 0.0 ? -log(or_uniform(r[0])) / mu_maj * 10.0 : INFINITY;
            if (s >= t_out) {
                for (int a = 0; a < 3; ++a) x[a] += t_out * d[a];
                path += t_out;
                break;
            }
            for (int a = 0; a < 3; ++a) x[a] += s * d[a];
            path += s;
            const om_material *m = &ph->materials[or_phantom_mat(C->P, x)];
            double mu_m = or_mu_total(m, E);
            if (or_uniform(r[1]) * mu_maj >= mu_m) continue;          /* virtual */
            en->ph_real++;
            if (or_is_photo(m, E, mu_m, or_uniform(r[2]))) {          /* photoelectric */
                en->phantom += E;
                return OR_OK;
            }
            double xm1;
            int nt = or_kahn(C->seed, h, OR_TAG_PHANTOM, gamma, step_id, E, &xm1);
            if (nt < 0) return OR_ERR_TIMEOUT;
            S->n_compton_trials += (uint64_t)nt;
            double k = E / OR_MEC2_KEV;
            double omc = xm1 / k;                                      /* 1 - cos(theta) */
            double c = 1.0 - omc, sn = sqrt(omc * (2.0 - omc));
            double T = E * xm1 / (1.0 + xm1), Ep = E / (1.0 + xm1);
            or_rotate(d, c, sn, or_uniform(r[3]));
            if (Ep < C->dg->e_cut) { en->phantom += E; return OR_OK; }
            en->phantom += T;
            E = Ep;
        }
    }

    /* --- detector: flight to a panel, then step-by-step transport inside it --- */
    int last = -1;
    for (;;) {
        double t_in, t_out;
        S->n_flights++;
        int k = or_flight(g, x, d, last, &t_in, &t_out);
        if (k < 0) { en->escaped += E; return OR_OK; }
        S->n_entered++;
        for (int a = 0; a < 3; ++a) x[a] += t_in * d[a];
        path += t_in;
        double t_rem = t_out - t_in;
        for (;;) {
            if (s_det >= OR_MAX_STEPS) return OR_ERR_TIMEOUT;
            uint32_t r[4];
            or_draw(C->seed, h, OR_TAG_DETECTOR, gamma, s_det, 0u, r);
            uint32_t step_id = s_det++;
            S->n_det_steps++;
            double mu_maj = or_majorant(sc->materials, sc->n_materials, E);
            double s = mu_maj > 0.0 ? -log(or_uniform(r[0])) / mu_maj * 10.0 : INFINITY;
            if (s >= t_rem) {                                         /* leaves the panel */
                for (int a = 0; a < 3; ++a) x[a] += t_rem * d[a];
                path += t_rem;
                last = k;
                break;
            }
            for (int a = 0; a < 3; ++a) x[a] += s * d[a];
            path += s;
            t_rem -= s;
            double w, u, v;
            or_to_local(g, k, x, &w, &u, &v);
            or_loc L;
            or_locate(g, k, w, u, v, &L);                              /* layer-selection step */
            const om_material *m = &sc->materials[L.mat];
            double mu_m = or_mu_total(m, E);
            if (or_uniform(r[1]) * mu_maj >= mu_m) continue;           /* virtual */
            double dep;
            int dead = 0;
            if (or_is_photo(m, E, mu_m, or_uniform(r[2]))) {           /* photoelectric */
                dep = E;
                dead = 1;
            } else {                                                   /* Compton */
                double xm1;
                int nt = or_kahn(C->seed, h, OR_TAG_DETECTOR, gamma, step_id, E, &xm1);
                if (nt < 0) return OR_ERR_TIMEOUT;
                S->n_compton_trials += (uint64_t)nt;
                double kk = E / OR_MEC2_KEV;
                double omc = xm1 / kk;
                double c = 1.0 - omc, sn = sqrt(omc * (2.0 - omc));
                double T = E * xm1 / (1.0 + xm1), Ep = E / (1.0 + xm1);
                if (g->posed) {
                    /* posed panel: the polar reference of the rotation is the
                     * panel's own v axis (for the ring, v = z and the global
                     * rotation below is the same map) */
                    double q[3];
                    or_dir_local(g, k, d, &q[0], &q[1], &q[2]);
                    or_rotate(q, c, sn, or_uniform(r[3]));
                    for (int a = 0; a < 3; ++a)
                        d[a] = q[0] * g->ax[k][0][a] + q[1] * g->ax[k][1][a] + q[2] * g->ax[k][2][a];
                } else {
                    or_rotate(d, c, sn, or_uniform(r[3]));
                }
                if (Ep < C->dg->e_cut) { dep = E; dead = 1; }
                else { dep = T; E = Ep; }
            }
            if (L.crystal >= 0) {
                en->det += dep;
                if (*n_hist_hits >= cap_hist) return OR_ERR_OOM;
                om_hit *H = &hist_hits[(*n_hist_hits)++];
                H->h = h; H->gamma = (int32_t)gamma; H->step = (int32_t)step_id;
                H->panel = k; H->module = L.module; H->layer = L.layer; H->crystal = L.crystal;
                H->w = w; H->u = u; H->v = v; H->edep = dep;
                H->t_ps = t0_ps + (uint64_t)floor(path / OR_C_MM_PER_PS);
            } else {
                en->passive += dep;
            }
            if (dead) return OR_OK;
            /* distance to the panel exit along the new direction */
            double p3[3] = {w, u, v}, q3[3];
            or_dir_local(g, k, d, &q3[0], &q3[1], &q3[2]);
            double lo[3] = {0.0, -0.5 * g->U, -0.5 * g->V}, hi[3] = {g->W, 0.5 * g->U, 0.5 * g->V};
            double te = INFINITY;
            for (int a = 0; a < 3; ++a) {
                if (q3[a] > 0.0) { double tt = (hi[a] - p3[a]) / q3[a]; if (tt < te) te = tt; }
                else if (q3[a] < 0.0) { double tt = (lo[a] - p3[a]) / q3[a]; if (tt < te) te = tt; }
            }
            t_rem = te < 0.0 ? 0.0 : te;
        }
    }
}

/* readout unit of a hit (Sec. 2.1: crystal-, module- or panel-level singles) */
static int32_t or_unit(const or_geom *g, const om_hit *H) {
    const om_scanner *sc = g->sc;
    if (sc->readout_level == 0) return H->panel;
    if (sc->readout_level == 1) return H->panel * sc->modules_u * sc->modules_v + H->module;
    return H->crystal;
}

/* decay of history h: time, annihilation point and photon-0 direction (Sec. 2.3:
 * annihilation at the emission site, no positron range, back-to-back photons) */
static void or_decay(const or_ctx *C, uint64_t h, uint64_t *t0, double x0[3], double d0[3]) {
    uint32_t r[4];
    or_draw(C->seed, h, OR_TAG_SOURCE, 0u, 0u, 0u, r);
    /* decay time: floor(T * r64 / 2^64), iid uniform on [0, T) */
    uint64_t r64 = ((uint64_t)r[0] << 32) | r[1];
    *t0 = (uint64_t)(((unsigned __int128)C->t_span_ps * r64) >> 64);
    x0[0] = C->src->pos[0]; x0[1] = C->src->pos[1]; x0[2] = C->src->pos[2];
    if (C->src->kind == 1) {
        /* voxel with probability proportional to its activity, then uniform inside it */
        const om_phantom *ph = C->P->ph;
        uint32_t q[4], z[4];
        or_draw(C->seed, h, OR_TAG_SOURCE, 0u, 0u, 1u, q);
        or_draw(C->seed, h, OR_TAG_SOURCE, 0u, 0u, 2u, z);
        uint64_t r53 = ((uint64_t)q[0] << 21) | (q[1] >> 11);
        double target = ldexp((double)r53, -53) * C->P->total;
        int64_t vi = or_pick_voxel(C->P, target);
        int64_t ix = vi % ph->nx, iy = (vi / ph->nx) % ph->ny, iz = vi / ((int64_t)ph->nx * ph->ny);
        x0[0] = ph->origin[0] + ((double)ix + or_uniform(q[2])) * ph->voxel[0];
        x0[1] = ph->origin[1] + ((double)iy + or_uniform(q[3])) * ph->voxel[1];
        x0[2] = ph->origin[2] + ((double)iz + or_uniform(z[0])) * ph->voxel[2];
    }
    if (C->src->kind == 2) {          /* collimated pair along a fixed axis */
        d0[0] = C->src->dir[0]; d0[1] = C->src->dir[1]; d0[2] = C->src->dir[2];
    } else {                          /* isotropic */
        double ct = 2.0 * or_uniform(r[2]) - 1.0;
        double st = sqrt((1.0 - ct) * (1.0 + ct));
        double ph = 2.0 * OR_PI * or_uniform(r[3]);
        d0[0] = st * cos(ph); d0[1] = st * sin(ph); d0[2] = ct;
    }
}

/* one decay (Sec. 2.3): the back-to-back pair transported photon by photon,
 * tallies, then the singles of the history per readout unit (Sec. 2.1) with
 * energy blur and window (Sec. 2.3) */
static int or_history(const or_ctx *C, uint64_t h, or_sink *S, uint64_t *tc, uint64_t *tefx,
                      double *tedep, double *balance, uint32_t *ph_real) {
    uint64_t t0;
    double x0[3], d0[3];
    or_decay(C, h, &t0, x0, d0);
    enum { CAP = 4096 };
    om_hit hh[CAP];
    int nh = 0;
    or_energy en = {0, 0, 0, 0, 0};
    for (uint32_t gamma = 0; gamma < 2; ++gamma) {
        double x[3] = {x0[0], x0[1], x0[2]};
        double sg = gamma == 0 ? 1.0 : -1.0;
        double d[3] = {sg * d0[0], sg * d0[1], sg * d0[2]};
        int st = or_transport_photon(C, h, gamma, x, d, t0, S, hh, &nh, CAP, &en);
        if (st != OR_OK) return st;
    }
    if (balance) *balance = en.det + en.passive + en.phantom + en.escaped;
    if (ph_real) *ph_real = en.ph_real;
    for (int i = 0; i < nh; ++i) {
        int st = or_push_hit(S, &hh[i]);
        if (st != OR_OK) return st;
        if (tc) {
            tc[hh[i].crystal] += 1;
            tefx[hh[i].crystal] += (uint64_t)nearbyint(hh[i].edep * OR_EFX_SCALE);
            tedep[hh[i].crystal] += hh[i].edep;
        }
    }
    /* singles: group by readout unit, energy sum, earliest time (Sec. 2.1, 2.3) */
    int used[CAP];
    memset(used, 0, sizeof(int) * (size_t)nh);
    double sig_k = C->dg->fwhm_at_511 / (2.0 * sqrt(2.0 * log(2.0)));
    for (int i = 0; i < nh; ++i) {
        if (used[i]) continue;
        int32_t unit = or_unit(C->g, &hh[i]);
        om_single s;
        s.h = h; s.unit = unit; s.panel = hh[i].panel;
        s.e_raw = 0.0; s.t_ps = hh[i].t_ps;
        double ew = 0.0;
        for (int j = i; j < nh; ++j) {
            if (used[j] || or_unit(C->g, &hh[j]) != unit) continue;
            used[j] = 1;
            s.e_raw += hh[j].edep;
            ew += hh[j].edep * hh[j].w;
            if (hh[j].t_ps < s.t_ps) s.t_ps = hh[j].t_ps;
        }
        s.doi = ew / s.e_raw;
        /* energy blur: FWHM(E) = fwhm_511 * sqrt(511 * E), Box-Muller normal */
        uint32_t q[4];
        uint32_t ctr[4] = {(uint32_t)h, (uint32_t)(h >> 32), OR_TAG_DIGI << 28, (uint32_t)unit};
        uint32_t key[2] = {(uint32_t)C->seed, (uint32_t)(C->seed >> 32)};
        or_philox4x32_10(ctr, key, q);
        /* Box-Muller pair: the cosine normal blurs the energy, the sine normal the depth */
        double rad = sqrt(-2.0 * log(or_uniform(q[0])));
        double n01 = rad * cos(2.0 * OR_PI * or_uniform(q[1]));
        double n02 = rad * sin(2.0 * OR_PI * or_uniform(q[1]));
        double sigma = sig_k * sqrt(OR_E0_KEV * s.e_raw);
        s.e_blur = s.e_raw + sigma * n01;
        s.doi_blur = s.doi + C->dg->doi_fwhm_mm / (2.0 * sqrt(2.0 * log(2.0))) * n02;
        s.kept = (s.e_blur >= C->dg->e_lo && s.e_blur <= C->dg->e_hi) ? 1 : 0;
        int st = or_push_single(S, &s);
        if (st != OR_OK) return st;
    }
    return OR_OK;
}

/* ------------------------------------------------------------------------- */
/* threaded driver over history ranges                                        */
/* ------------------------------------------------------------------------- */
typedef struct {
    const or_ctx *C;
    uint64_t h0, h1, hbase;
    or_sink sink;
    uint64_t *tc, *tefx;
    double *tedep;
    double *balance;
    uint32_t *ph_real;
} or_job;

static void *or_worker(void *arg) {
    or_job *J = (or_job *)arg;
    for (uint64_t h = J->h0; h < J->h1; ++h) {
        int st = or_history(J->C, h, &J->sink, J->tc, J->tefx, J->tedep,
                            J->balance ? &J->balance[h - J->hbase] : NULL,
                            J->ph_real ? &J->ph_real[h - J->hbase] : NULL);
        if (st != OR_OK) { J->sink.status = st; break; }
    }
    return NULL;
}

int or_scanner_crystals(const om_scanner *sc) {
    or_geom g;
    if (or_geom_init(&g, sc) != OR_OK) return -1;
    return g.n_crystals;
}

uint64_t or_time_span_ps(uint64_t n_decays, double activity_bq) {
    return (uint64_t)llround((double)n_decays / activity_bq * 1e12);
}

/* Simulate histories [h_begin, h_end) of an n_decays run.  Outputs are ordered
 * by history (then event order), independent of the thread count. */
int or_simulate(const om_scanner *sc, const om_phantom *ph, const om_source *src, const om_digitizer *dg,
                uint64_t n_decays, uint64_t seed, uint64_t h_begin, uint64_t h_end, int n_threads,
                om_output *out) {
    or_geom g;
    int st = or_geom_init(&g, sc);
    if (st != OR_OK) return st;
    if (src->kind == 1 && (!ph || !ph->activity)) return OR_ERR_INVALID;
    or_phantom P;
    st = or_phantom_init(&P, ph);
    if (st != OR_OK) return st;
    if (src->kind == 1 && !(P.total > 0.0)) { free(P.cdf); return OR_ERR_INVALID; }
    or_ctx C;
    memset(&C, 0, sizeof(C));
    C.sc = sc; C.g = &g; C.P = &P; C.src = src; C.dg = dg; C.seed = seed; C.n_decays = n_decays;
    C.t_span_ps = or_time_span_ps(n_decays, src->activity_bq);
    if (n_threads < 1) n_threads = 1;
    uint64_t n = h_end > h_begin ? h_end - h_begin : 0;
    if ((uint64_t)n_threads > n && n > 0) n_threads = (int)n;
    if (n == 0) n_threads = 1;
    or_job *jobs = (or_job *)calloc((size_t)n_threads, sizeof(or_job));
    uint64_t **tcs = (uint64_t **)calloc((size_t)n_threads, sizeof(void *));
    uint64_t **tes = (uint64_t **)calloc((size_t)n_threads, sizeof(void *));
    double **tds = (double **)calloc((size_t)n_threads, sizeof(void *));
    pthread_t *th = (pthread_t *)calloc((size_t)n_threads, sizeof(pthread_t));
    if (!jobs || !tcs || !tes || !tds || !th) return OR_ERR_OOM;
    for (int i = 0; i < n_threads; ++i) {
        jobs[i].C = &C;
        jobs[i].h0 = h_begin + n * (uint64_t)i / (uint64_t)n_threads;
        jobs[i].h1 = h_begin + n * (uint64_t)(i + 1) / (uint64_t)n_threads;
        jobs[i].hbase = h_begin;
        jobs[i].balance = out->balance;
        jobs[i].ph_real = out->ph_real;
        if (out->tally_count) {
            tcs[i] = (uint64_t *)calloc((size_t)g.n_crystals, sizeof(uint64_t));
            tes[i] = (uint64_t *)calloc((size_t)g.n_crystals, sizeof(uint64_t));
            tds[i] = (double *)calloc((size_t)g.n_crystals, sizeof(double));
            jobs[i].tc = tcs[i]; jobs[i].tefx = tes[i]; jobs[i].tedep = tds[i];
        }
    }
    for (int i = 0; i < n_threads; ++i) pthread_create(&th[i], NULL, or_worker, &jobs[i]);
    for (int i = 0; i < n_threads; ++i) pthread_join(th[i], NULL);
    /* merge in history order */
    size_t nh = 0, ns = 0;
    out->status = OR_OK;
    out->n_det_steps = out->n_ph_steps = out->n_flights = out->n_compton_trials = out->n_entered = 0;
    for (int i = 0; i < n_threads; ++i) {
        nh += jobs[i].sink.n_hits; ns += jobs[i].sink.n_singles;
        if (jobs[i].sink.status != OR_OK) out->status = jobs[i].sink.status;
        out->n_det_steps += jobs[i].sink.n_det_steps;
        out->n_ph_steps += jobs[i].sink.n_ph_steps;
        out->n_flights += jobs[i].sink.n_flights;
        out->n_compton_trials += jobs[i].sink.n_compton_trials;
        out->n_entered += jobs[i].sink.n_entered;
    }
    out->hits = (om_hit *)malloc((nh ? nh : 1) * sizeof(om_hit));
    out->singles = (om_single *)malloc((ns ? ns : 1) * sizeof(om_single));
    out->n_hits = nh; out->n_singles = ns; out->n_kept = 0;
    size_t ah = 0, as = 0;
    for (int i = 0; i < n_threads; ++i) {
        if (jobs[i].sink.n_hits) memcpy(out->hits + ah, jobs[i].sink.hits, jobs[i].sink.n_hits * sizeof(om_hit));
        if (jobs[i].sink.n_singles)
            memcpy(out->singles + as, jobs[i].sink.singles, jobs[i].sink.n_singles * sizeof(om_single));
        ah += jobs[i].sink.n_hits; as += jobs[i].sink.n_singles;
        free(jobs[i].sink.hits); free(jobs[i].sink.singles);
        if (out->tally_count) {
            for (int c = 0; c < g.n_crystals; ++c) {
                out->tally_count[c] += tcs[i][c];
                out->tally_efx[c] += tes[i][c];
                out->tally_edep[c] += tds[i][c];
            }
            free(tcs[i]); free(tes[i]); free(tds[i]);
        }
    }
    for (size_t i = 0; i < ns; ++i) out->n_kept += (uint64_t)out->singles[i].kept;
    free(jobs); free(tcs); free(tes); free(tds); free(th); free(P.cdf);
    return out->status;
}

void or_free_output(om_output *out) {
    free(out->hits); free(out->singles);
    out->hits = NULL; out->singles = NULL;
}

/* ------------------------------------------------------------------------- */
/* coincidence sorting (Sec. 2.3 timing window; policy is a stated reading)   */
/* ------------------------------------------------------------------------- */
typedef struct { uint64_t t, h; int32_t unit, panel, idx; } or_skey;

static int or_cmp_single(const void *a, const void *b) {
    const or_skey *x = (const or_skey *)a, *y = (const or_skey *)b;
    if (x->t != y->t) return x->t < y->t ? -1 : 1;
    if (x->unit != y->unit) return x->unit < y->unit ? -1 : 1;
    if (x->h != y->h) return x->h < y->h ? -1 : 1;
    return 0;
}

/* Input: n singles (time, unit, panel, history).  Sort by (t, unit, h); the
 * earliest unconsumed single opens [t0, t0 + window]; a window holding exactly
 * two singles in different panels yields one coincidence; every single in the
 * window is consumed.  Output pairs are indices into the input arrays, first
 * the earlier single (ties by unit, then history).  Returns the pair count. */
int64_t or_coincidences(int64_t n, const uint64_t *t_ps, const int32_t *unit, const int32_t *panel,
                        const uint64_t *h, uint64_t window_ps, int32_t *pair_a, int32_t *pair_b) {
    or_skey *k = (or_skey *)malloc((size_t)(n ? n : 1) * sizeof(or_skey));
    if (!k) return -1;
    for (int64_t i = 0; i < n; ++i) {
        k[i].t = t_ps[i]; k[i].h = h[i]; k[i].unit = unit[i]; k[i].panel = panel[i]; k[i].idx = (int32_t)i;
    }
    qsort(k, (size_t)n, sizeof(or_skey), or_cmp_single);
    int64_t np = 0, i = 0;
    while (i < n) {
        int64_t j = i;
        while (j + 1 < n && k[j + 1].t - k[i].t <= window_ps) ++j;
        if (j - i + 1 == 2 && k[i].panel != k[i + 1].panel) {
            pair_a[np] = k[i].idx;
            pair_b[np] = k[i + 1].idx;
            ++np;
        }
        i = j + 1;
    }
    free(k);
    return np;
}

/* ------------------------------------------------------------------------- */
/* small entry points used by the pins                                        */
/* ------------------------------------------------------------------------- */
/* photoelectric decisions of n real collisions in material m at energy E, with
 * the uniforms of the detector-step blocks of histories h0 .. h0 + n - 1 */
int64_t or_photo_count(const om_material *m, double e_kev, uint64_t seed, uint64_t h0, int64_t n) {
    const double mu_m = or_mu_total(m, e_kev);
    int64_t c = 0;
    for (int64_t i = 0; i < n; ++i) {
        uint32_t r[4];
        or_draw(seed, h0 + (uint64_t)i, OR_TAG_DETECTOR, 0u, 0u, 0u, r);
        c += or_is_photo(m, e_kev, mu_m, or_uniform(r[2]));
    }
    return c;
}

int or_kahn_batch(uint64_t seed, uint64_t h0, int64_t n, double e_kev, double *cos_theta, double *e_out,
                  int32_t *trials) {
    for (int64_t i = 0; i < n; ++i) {
        double xm1;
        int nt = or_kahn(seed, h0 + (uint64_t)i, OR_TAG_DETECTOR, 0u, 0u, e_kev, &xm1);
        if (nt < 0) return OR_ERR_TIMEOUT;
        cos_theta[i] = 1.0 - xm1 / (e_kev / OR_MEC2_KEV);
        e_out[i] = e_kev / (1.0 + xm1);
        trials[i] = nt;
    }
    return OR_OK;
}

int or_flight_batch(const om_scanner *sc, int64_t n, const double *x, const double *d, int32_t *panel,
                    double *t_in) {
    or_geom g;
    int st = or_geom_init(&g, sc);
    if (st != OR_OK) return st;
    for (int64_t i = 0; i < n; ++i) {
        double ti = 0.0, to = 0.0;
        panel[i] = or_flight(&g, &x[3 * i], &d[3 * i], -1, &ti, &to);
        t_in[i] = ti;
    }
    return OR_OK;
}

/* locate panel-local points of panel k; out: layer, module, crystal id, material */
int or_locate_batch(const om_scanner *sc, int k, int64_t n, const double *wuv, int32_t *out4) {
    or_geom g;
    int st = or_geom_init(&g, sc);
    if (st != OR_OK) return st;
    for (int64_t i = 0; i < n; ++i) {
        or_loc L;
        or_locate(&g, k, wuv[3 * i], wuv[3 * i + 1], wuv[3 * i + 2], &L);
        out4[4 * i] = L.layer; out4[4 * i + 1] = L.module; out4[4 * i + 2] = L.crystal; out4[4 * i + 3] = L.mat;
    }
    return OR_OK;
}

/* panel box extents (U, V, W) as the oracle derives them */
int or_panel_extent(const om_scanner *sc, double *uvw) {
    or_geom g;
    int st = or_geom_init(&g, sc);
    if (st != OR_OK) return st;
    uvw[0] = g.U; uvw[1] = g.V; uvw[2] = g.W;
    return OR_OK;
}

/* Box-Muller normals of the digitizer blur for (h, unit) under seed */
void or_blur_normals(uint64_t seed, int64_t n, const uint64_t *h, const int32_t *unit, double *out) {
    for (int64_t i = 0; i < n; ++i) {
        uint32_t q[4];
        uint32_t ctr[4] = {(uint32_t)h[i], (uint32_t)(h[i] >> 32), OR_TAG_DIGI << 28, (uint32_t)unit[i]};
        uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
        or_philox4x32_10(ctr, key, q);
        out[i] = sqrt(-2.0 * log(or_uniform(q[0]))) * cos(2.0 * OR_PI * or_uniform(q[1]));
    }
}

/* rotate n unit vectors by (cos theta, azimuth 2 pi u) with the transport's own routine */
void or_rotate_batch(int64_t n, double *d, const double *cos_theta, const double *u_phi) {
    for (int64_t i = 0; i < n; ++i) {
        double c = cos_theta[i];
        double s = sqrt((1.0 - c) * (1.0 + c));
        or_rotate(&d[3 * i], c, s, u_phi[i]);
    }
}

/* decays of histories [h0, h0 + n): time (ps), position (mm), photon-0 direction */
int or_decay_batch(const om_phantom *ph, const om_source *src, uint64_t n_decays, uint64_t seed, uint64_t h0,
                   int64_t n, uint64_t *t_ps, double *pos, double *dir) {
    or_phantom P;
    int st = or_phantom_init(&P, ph);
    if (st != OR_OK) return st;
    if (src->kind == 1 && !(P.total > 0.0)) { free(P.cdf); return OR_ERR_INVALID; }
    or_ctx C;
    memset(&C, 0, sizeof(C));
    C.P = &P; C.src = src; C.seed = seed; C.n_decays = n_decays;
    C.t_span_ps = or_time_span_ps(n_decays, src->activity_bq);
    for (int64_t i = 0; i < n; ++i) or_decay(&C, h0 + (uint64_t)i, &t_ps[i], &pos[3 * i], &dir[3 * i]);
    free(P.cdf);
    return OR_OK;
}
