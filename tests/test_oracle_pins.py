"""Pins of the FP64 oracle against things other than itself: published
known-answer vectors, closed forms of the physics model, brute-force
quadrature, exact invariants and numbers printed in the paper.

Each test names the plausible mistake it would catch.
"""
import math

import numpy as np
import pytest
from scipy import integrate, stats

import workloads as W
from tests.conftest import read_golden

MEC2 = 510.99895
RE = 2.8179403262e-13


# ---------------------------------------------------------------------------
# RNG
# ---------------------------------------------------------------------------
def test_philox_known_answers(oracle):
    """Philox4x32-10 against the Random123 KAT vectors (Salmon et al. SC'11).
    Catches a wrong multiplier, Weyl constant, round count or word order."""
    for row in read_golden("philox4x32_10_kat.txt"):
        v = [int(x, 16) for x in row.split()]
        assert oracle.philox(v[0:4], v[4:6]) == v[6:10]


def test_uniform_open_interval(oracle):
    """u = (k + 1/2) 2^-23 from the top 23 bits: never 0 or 1, exact ends."""
    assert oracle.uniform(0) == 0.5 * 2.0 ** -23
    assert oracle.uniform(0xFFFFFFFF) == 1.0 - 0.5 * 2.0 ** -23
    assert oracle.uniform(0x80000000) == 0.5 + 0.5 * 2.0 ** -23


# ---------------------------------------------------------------------------
# physics model
# ---------------------------------------------------------------------------
def kn_dsigma_domega(e_kev, cos_t):
    """Klein-Nishina differential cross section per electron (cm^2/sr)."""
    k = e_kev / MEC2
    p = 1.0 / (1.0 + k * (1.0 - cos_t))  # E'/E
    return 0.5 * RE * RE * p * p * (p + 1.0 / p - (1.0 - cos_t * cos_t))


@pytest.mark.parametrize("e", [10.0, 30.0, 100.0, 340.0, 511.0, 2000.0])
def test_sigma_kn_equals_integral_of_differential(oracle, e):
    """Closed-form total KN cross section == 2 pi * integral of dsigma/dOmega,
    over the transport's energy domain (cutoff 10 keV up to 511 keV).
    Catches a dropped or mis-signed term of the closed form."""
    val, _ = integrate.quad(lambda c: kn_dsigma_domega(e, c), -1.0, 1.0, epsabs=0, epsrel=1e-12)
    assert oracle.sigma_kn(e) == pytest.approx(2 * math.pi * val, rel=1e-9, abs=0)


@pytest.mark.parametrize("e", [511.0, 300.0, 200.0, 100.0])
def test_photoelectric_share_follows_the_energy(oracle, e):
    """The kind of a real collision at energy E: photoelectric with
    probability mu_pe(E) / mu_total(E), where mu_pe scales as (511/E)^3 from
    its 511 keV value and the Compton part as the Klein-Nishina total cross
    section (here from a quadrature of dsigma/dOmega, not the oracle's closed
    form).  Binomial test on the transport's own branch function; catches a
    share frozen at its 511 keV value or a wrong power of the E^-3 law."""
    mat = W.LYSO
    n = 200_000
    sig = lambda en: 2 * math.pi * integrate.quad(lambda c: kn_dsigma_domega(en, c), -1.0, 1.0, epsrel=1e-12)[0]
    mu_pe = mat["mu_total_511_cm"] * mat["photo_frac_511"] * (511.0 / e) ** 3
    mu_c = mat["mu_total_511_cm"] * (1.0 - mat["photo_frac_511"]) * sig(e) / sig(511.0)
    p = mu_pe / (mu_pe + mu_c)
    got = oracle.photo_count(dict(mat, electron_density_cm3=0.0), e, 77, 0, n)
    assert abs(got / n - p) < 5.0 * math.sqrt(p * (1 - p) / n), (got / n, p)


def test_sigma_kn_thomson_limit(oracle):
    """sigma -> (8 pi/3) r_e^2 (1 - 2k + 26/5 k^2 - 133/10 k^3 + 1144/35 k^4) at
    low energy.  (Below ~2 keV the closed form loses digits to cancellation in
    FP64; the transport never evaluates it there.)"""
    e = 2.0
    k = e / MEC2
    thomson = 8 * math.pi / 3 * RE * RE
    series = 1 - 2 * k + 26 / 5 * k ** 2 - 133 / 10 * k ** 3 + 1144 / 35 * k ** 4
    assert oracle.sigma_kn(e) == pytest.approx(thomson * series, rel=1e-8, abs=0)


def test_material_anchors(oracle):
    """The configs fix mu_total(511) = 0.87/cm and a 0.34 photoelectric share for
    LYSO, 0.096/cm for water; photoelectric scales as E^-3 from 511 keV."""
    assert oracle.mu(W.LYSO, 511.0) == pytest.approx(0.87, rel=1e-14)
    assert oracle.mu(W.LYSO, 511.0, "photo") == pytest.approx(0.87 * 0.34, rel=1e-14)
    assert oracle.mu(W.LYSO, 255.5, "photo") == pytest.approx(8 * 0.87 * 0.34, rel=1e-14)
    assert oracle.mu(W.WATER, 511.0) == pytest.approx(0.096, rel=1e-14)
    assert oracle.mu(W.WATER, 200.0, "photo") == 0.0
    # Compton part follows sigma_KN(E) / sigma_KN(511) from its 511 keV anchor
    r = oracle.mu(W.LYSO, 200.0, "compton") / oracle.mu(W.LYSO, 511.0, "compton")
    assert r == pytest.approx(oracle.sigma_kn(200.0) / oracle.sigma_kn(511.0), rel=1e-14)
    # literal electron density reading: mu_C = n_e sigma_KN
    assert oracle.mu(W.LYSO_LITERAL_NE, 511.0, "compton") == pytest.approx(0.6017, abs=1e-4)


@pytest.mark.parametrize("e", [511.0, 340.0, 100.0])
def test_kahn_sampler_matches_klein_nishina(oracle, e):
    """Chi-square of sampled cos(theta) against the closed-form dsigma/dOmega.
    Catches a wrong branch probability, acceptance test or kinematics."""
    n = 200_000
    ct, eo, tr = oracle.kahn(seed=7, h0=1000, n=n, e_kev=e)
    edges = np.linspace(-1.0, 1.0, 41)
    obs, _ = np.histogram(ct, edges)
    tot = integrate.quad(lambda c: kn_dsigma_domega(e, c), -1, 1, epsrel=1e-12)[0]
    exp = np.array([integrate.quad(lambda c: kn_dsigma_domega(e, c), a, b, epsrel=1e-12)[0]
                    for a, b in zip(edges[:-1], edges[1:])]) / tot * n
    chi2 = ((obs - exp) ** 2 / exp).sum()
    p = stats.chi2.sf(chi2, len(obs) - 1)
    assert p > 1e-3, (chi2, p)
    # Compton kinematics: E' = E / (1 + k (1 - cos theta))
    np.testing.assert_allclose(eo, e / (1.0 + e / MEC2 * (1.0 - ct)), rtol=1e-12)
    # mean energy transfer against its quadrature
    mean_t = integrate.quad(lambda c: kn_dsigma_domega(e, c) * (e - e / (1 + e / MEC2 * (1 - c))), -1, 1,
                            epsrel=1e-12)[0] / tot
    t = e - eo
    assert abs(t.mean() - mean_t) < 4 * t.std() / math.sqrt(n)
    assert tr.min() >= 1


def test_rotation_keeps_angle_and_norm(oracle):
    """New direction is a unit vector at angle theta from the old one, with the
    azimuth spread uniformly; also near the pole branch."""
    rng = np.random.default_rng(3)
    d = rng.normal(size=(2000, 3))
    d /= np.linalg.norm(d, axis=1)[:, None]
    d[:10] = [0, 0, 1]
    d[10:20] = [0, 0, -1]
    c = rng.uniform(-1, 1, len(d))
    u = rng.uniform(0, 1, len(d))
    r = oracle.rotate(d, c, u)
    np.testing.assert_allclose(np.linalg.norm(r, axis=1), 1.0, atol=1e-12)
    np.testing.assert_allclose((r * d).sum(1), c, atol=1e-12)
    # azimuth linear in u for a fixed d and theta
    d0 = np.tile([0.3, -0.4, math.sqrt(1 - 0.25)], (64, 1))
    uu = np.arange(64) / 64
    rr = oracle.rotate(d0, np.full(64, 0.2), uu)
    e1 = rr[0] - 0.2 * d0[0]
    e1 /= np.linalg.norm(e1)
    e2 = np.cross(d0[0], e1)
    ang = np.unwrap(np.arctan2((rr - 0.2 * d0) @ e2, (rr - 0.2 * d0) @ e1))
    np.testing.assert_allclose(np.abs(np.diff(ang)), 2 * math.pi / 64, atol=1e-9)


# ---------------------------------------------------------------------------
# transport against closed forms
# ---------------------------------------------------------------------------
def slab_scanner(mu_total, photo_frac, depth):
    mats = [W.AIR, dict(mu_total_511_cm=mu_total, photo_frac_511=photo_frac, electron_density_cm3=0.0)]
    return W.scanner(1, 100.0, [W.layer(1, 1, 400.0, 0.0, depth)], materials=mats, name="slab")


@pytest.mark.parametrize("mu_t,pf,depth", [(0.87, 0.34, 10.0), (0.5, 0.0, 20.0), (1.3, 1.0, 4.0)])
def test_slab_transmission(oracle, mu_t, pf, depth):
    """Pencil beam at normal incidence: uncollided fraction exp(-mu L), mean
    first-interaction depth of the truncated exponential, photoelectric share
    of first interactions.  Catches mm/cm mix-ups, a wrong majorant or a
    swapped photo/Compton branch."""
    n = 200_000
    sc = slab_scanner(mu_t, pf, depth)
    r = oracle.simulate(sc, W.pencil_source(direction=(1, 0, 0)), W.digitizer(), n, seed=11, threads=8)
    hits = r["hits"]
    g0 = hits[hits["gamma"] == 0]
    assert (hits["gamma"] == 1).sum() == 0  # photon 1 flies away from the single panel
    # first interaction of each photon 0
    first_idx = np.unique(g0["h"], return_index=True)[1]
    first = g0[first_idx]
    p_int = len(first) / n
    p_exp = 1.0 - math.exp(-mu_t * depth / 10.0)
    assert abs(p_int - p_exp) < 4.5 * math.sqrt(p_exp * (1 - p_exp) / n)
    mu_mm = mu_t / 10.0
    mean_w = 1 / mu_mm - depth * math.exp(-mu_mm * depth) / (1 - math.exp(-mu_mm * depth))
    sd_w = first["w"].std()
    assert abs(first["w"].mean() - mean_w) < 4.5 * sd_w / math.sqrt(len(first))
    n_photo = (first["edep"] == 511.0).sum()
    assert abs(n_photo / len(first) - pf) < 4.5 * math.sqrt(max(pf * (1 - pf), 1e-12) / len(first)) + 1e-12
    # all energy accounted for
    assert np.all(r["tally_edep"] >= 0)


def rect_solid_angle(a, b, d):
    """Solid angle of an a x b rectangle seen from distance d on its normal axis."""
    return 4.0 * math.atan(a * b / (2.0 * d * math.sqrt(4 * d * d + a * a + b * b)))


def box_solid_angle_quadrature(corners_fn, src, n=600):
    """Brute-force solid angle of a convex box: sum over faces that face the
    source of the integral of cos / r^2 on a fine midpoint grid."""
    total = 0.0
    for (o, e1, e2) in corners_fn():
        o, e1, e2 = map(np.asarray, (o, e1, e2))
        nrm = np.cross(e1, e2)
        nrm /= np.linalg.norm(nrm)
        s = (np.arange(n) + 0.5) / n
        P = o[None, None, :] + s[:, None, None] * e1[None, None, :] + s[None, :, None] * e2[None, None, :]
        rv = P - src
        r = np.linalg.norm(rv, axis=2)
        cosang = (rv @ nrm) / r
        dA = np.linalg.norm(np.cross(e1, e2)) / (n * n)
        val = (cosang / (r * r)).sum() * dA
        total += abs(val) if np.sign((o - src) @ nrm) != 0 and ((o - src) @ nrm) > 0 else 0.0
    return total


def test_geometric_acceptance_central(oracle):
    """Config-1 ring, source at the centre: accepted fraction of isotropic rays
    == 8 * rectangle solid angle / 4 pi (= 0.06357)."""
    sc = W.config1_scanner()
    ext = oracle.panel_extent(sc)
    assert ext[0] == pytest.approx(12.8) and ext[1] == pytest.approx(12.8) and ext[2] == pytest.approx(10.0)
    p_exp = 8 * rect_solid_angle(12.8, 12.8, 40.0) / (4 * math.pi)
    assert p_exp == pytest.approx(0.06357, abs=2e-5)
    rng = np.random.default_rng(5)
    n = 1_000_000
    d = rng.normal(size=(n, 3))
    d /= np.linalg.norm(d, axis=1)[:, None]
    pn, ti = oracle.flight(sc, np.zeros((n, 3)), d)
    p = (pn >= 0).mean()
    assert abs(p - p_exp) < 4 * math.sqrt(p_exp * (1 - p_exp) / n)
    # the front face is entered at distance R / cos(angle to the normal)
    k = pn[pn >= 0]
    phi = 2 * math.pi * k / 8
    cosn = d[pn >= 0, 0] * np.cos(phi) + d[pn >= 0, 1] * np.sin(phi)
    np.testing.assert_allclose(ti[pn >= 0], 40.0 / cosn, rtol=1e-12)


def test_geometric_acceptance_offcentre(oracle):
    """Off-centre source: MC acceptance == brute-force face quadrature of the
    panel boxes (front and visible side faces)."""
    sc = W.config1_scanner()
    src = np.array([9.0, -6.0, 3.0])
    U, V, Wd, R = 12.8, 12.8, 10.0, 40.0
    total = 0.0
    for k in range(8):
        phi = 2 * math.pi * k / 8
        n_ = np.array([math.cos(phi), math.sin(phi), 0.0])
        u_ = np.array([-math.sin(phi), math.cos(phi), 0.0])
        v_ = np.array([0.0, 0.0, 1.0])
        c0 = R * n_ - U / 2 * u_ - V / 2 * v_  # inner-face low corner

        def faces(c0=c0, n_=n_, u_=u_, v_=v_):
            return [(c0, U * u_, V * v_),                     # front (w = 0)
                    (c0 + Wd * n_, V * v_, U * u_),           # back
                    (c0, V * v_, Wd * n_),                    # side u = -U/2
                    (c0 + U * u_, Wd * n_, V * v_),           # side u = +U/2
                    (c0, Wd * n_, U * u_),                    # bottom v = -V/2
                    (c0 + V * v_, U * u_, Wd * n_)]           # top v = +V/2
        # outward normal orientation: use the box centre to orient each face
        centre = c0 + U / 2 * u_ + V / 2 * v_ + Wd / 2 * n_

        def oriented():
            for o, e1, e2 in faces():
                nn = np.cross(e1, e2)
                fc = o + 0.5 * e1 + 0.5 * e2
                if (fc - centre) @ nn < 0:
                    e1, e2 = e2, e1
                yield o, e1, e2

        # a face is visible when its outward normal points toward the source
        for o, e1, e2 in oriented():
            nn = np.cross(e1, e2)
            fc = o + 0.5 * e1 + 0.5 * e2
            if (src - fc) @ nn > 0:
                s = (np.arange(500) + 0.5) / 500
                P = o[None, None, :] + s[:, None, None] * e1 + s[None, :, None] * e2
                rv = P - src
                r = np.linalg.norm(rv, axis=2)
                nh = nn / np.linalg.norm(nn)
                total += ((-(rv @ nh)) / r ** 3).sum() * np.linalg.norm(nn) / 500 ** 2
    p_exp = total / (4 * math.pi)
    rng = np.random.default_rng(6)
    n = 1_000_000
    d = rng.normal(size=(n, 3))
    d /= np.linalg.norm(d, axis=1)[:, None]
    pn, _ = oracle.flight(sc, np.tile(src, (n, 1)), d)
    p = (pn >= 0).mean()
    assert abs(p - p_exp) < 4 * math.sqrt(p_exp * (1 - p_exp) / n) + 1e-5, (p, p_exp)


# ---------------------------------------------------------------------------
# hierarchy indexing
# ---------------------------------------------------------------------------
def test_flight_enters_the_nearest_panel(oracle):
    """Two posed heads one behind the other on the +x axis (the far one listed
    first): a ray meets the near head first, from either side, and a ray
    that misses the near head meets the far one.  Slab-test distances are
    exact.  Catches a flight that returns the first listed or the farthest
    panel it crosses."""
    base = W.scanner(2, 45.0, [W.layer(8, 8, 2.0, 0.1, 12.0)])
    sc = W.with_poses(base, np.stack([W.pose((1, 0, 0), (0, 1, 0), (70.0, 0.0, 0.0)),
                                      W.pose((1, 0, 0), (0, 1, 0), (45.0, 0.0, 0.0))]))
    x = np.array([[0.0, 0.0, 0.0], [60.0, 1.0, -2.0], [100.0, 0.5, 0.5], [0.0, 0.0, 0.0], [0.0, 0.0, 0.0]])
    d = np.array([[1.0, 0.0, 0.0], [1.0, 0.0, 0.0], [-1.0, 0.0, 0.0], [1.0, 0.1, 0.0], [1.0, 0.0, -0.3]])
    d /= np.linalg.norm(d, axis=1)[:, None]
    pn, ti = oracle.flight(sc, x, d)
    # near head: x in [45, 57]; far head: x in [70, 82]; both 16 mm wide in u and v
    assert list(pn[:3]) == [1, 0, 0]
    np.testing.assert_allclose(ti[:3], [45.0, 10.0, 18.0], atol=1e-12)
    # slope 0.1 in y: at x = 45 the ray is at y = 4.5, inside the near head
    assert pn[3] == 1 and ti[3] == pytest.approx(45.0 * math.sqrt(1.01), abs=1e-12)
    # slope -0.3 in z: it passes below the near head (z = -13.5 at x = 45) and
    # below the far one (z = -21 at x = 70): no panel
    assert pn[4] == -1


def test_locate_lattice_points(oracle):
    """Crystal centres locate to their own (layer, module, crystal) id; points in
    the inter-crystal gaps, the reflector gap and the module gap are interval."""
    sc = W.config3_scanner()   # two layers, the second offset by half a pitch
    Us, Vs = sc["module_size_u"], sc["module_size_v"]
    U = Us
    V = 4 * Vs
    cpm = sum(l["n_u"] * l["n_v"] for l in sc["layers"])
    pts, want = [], []
    w0 = 0.0
    loff = 0
    for li, l in enumerate(sc["layers"]):
        w0 += l["gap_before"]
        for mv in range(4):
            for iv in range(l["n_v"]):
                for iu in range(l["n_u"]):
                    u = -U / 2 + l["offset_u"] + (iu + 0.5) * l["pitch_u"]
                    v = -V / 2 + mv * Vs + l["offset_v"] + (iv + 0.5) * l["pitch_v"]
                    pts.append((w0 + 0.5 * l["depth"], u, v))
                    want.append((li, mv, (3 * 4 + mv) * cpm + loff + iv * l["n_u"] + iu, 1))
        w0 += l["depth"]
        loff += l["n_u"] * l["n_v"]
    got = oracle.locate(sc, 3, pts)
    assert np.array_equal(got, np.array(want, np.int32))
    # gap points: inter-crystal gap, reflector gap, outside the offset layer's grid
    gaps = [(2.5, -U / 2 + 1.0 + 0.01, 0.3 - V / 2),     # u on a cell boundary +- gap/2
            (5.025, 0.0, 0.0),                           # reflector between the layers
            (7.5, -U / 2 + 0.25, -V / 2 + 5.3)]          # below the offset grid of layer 2
    got = oracle.locate(sc, 0, gaps)
    assert np.all(got[:, 2] == -1) and np.all(got[:, 3] == 0)
    assert got[1, 0] == -1


def test_offset_dual_layer_volume_reduction(oracle):
    """Sec. 3.2: the 2CL module has 1.94 % less crystal volume than 1CL
    (50x50 + 51x51 half-depth layers vs 51x51).  Monte Carlo over the module
    with the oracle's own locate()."""
    vals = {k: float(v.split("=")[1]) if "=" in v else None
            for k, v in ((r.split("=")[0].strip(), r) for r in read_golden("paper_text_values.txt"))}
    rng = np.random.default_rng(9)
    n = 600_000
    pts = np.stack([rng.uniform(0, 10, n), rng.uniform(-25.5, 25.5, n), rng.uniform(-170.5, -170.5 + 51, n)], 1)
    frac = {}
    for kind in ("1CL", "2CL"):
        sc = W.h2rspet(kind)
        got = oracle.locate(sc, 0, pts)
        frac[kind] = (got[:, 2] >= 0).mean()
    red = 100 * (1 - frac["2CL"] / frac["1CL"])
    assert abs(red - vals["volume_reduction_2cl_percent"]) < 0.12, red
    assert frac["1CL"] == pytest.approx((0.92 / 1.0) ** 2, abs=3e-3)


def test_h2rspet_dimensions(oracle):
    """Sec. 2.2: panel 1.0 x 5.1 x 34.1 cm^3 (radial x tangential x axial)."""
    vals = {r.split("=")[0].strip(): float(r.split("=")[1]) for r in read_golden("paper_text_values.txt")}
    ext = oracle.panel_extent(W.h2rspet("1CL"))
    assert ext[0] == pytest.approx(vals["h2rspet_panel_tangential_mm"])
    assert ext[1] == pytest.approx(vals["h2rspet_panel_axial_mm"])
    assert ext[2] == pytest.approx(vals["h2rspet_depth_mm"])


# ---------------------------------------------------------------------------
# whole-history invariants
# ---------------------------------------------------------------------------
def test_energy_conservation_per_history(oracle):
    """Sum of crystal + passive + phantom deposits + escaped energy == 1022 keV."""
    r = oracle.simulate(W.config1_scanner(), W.point_source(), W.digitizer(), 20000, seed=1, threads=4,
                        balance=True)
    np.testing.assert_allclose(r["balance"], 1022.0, atol=1e-9)
    c3 = W.config3(2000)
    r = oracle.simulate(c3["scanner"], c3["source"], c3["digitizer"], 2000, seed=3, phantom=c3["phantom"],
                        threads=4, balance=True)
    np.testing.assert_allclose(r["balance"], 1022.0, atol=1e-9)
    assert r["counters"]["ph_steps"] > 0


def test_split_zero_gap_equals_single_layer(oracle):
    """Two 5 mm layers with no gap between them are the same detector as one
    10 mm layer: same hits, history by history, only the layer label differs."""
    one = W.scanner(8, 40.0, [W.layer(8, 8, 1.6, 0.1, 10.0)])
    two = W.scanner(8, 40.0, [W.layer(8, 8, 1.6, 0.1, 5.0), W.layer(8, 8, 1.6, 0.1, 5.0)])
    a = oracle.simulate(one, W.point_source((1.0, 2.0, 0.5)), W.digitizer(), 30000, seed=21, threads=4)["hits"]
    b = oracle.simulate(two, W.point_source((1.0, 2.0, 0.5)), W.digitizer(), 30000, seed=21, threads=4)["hits"]
    assert len(a) == len(b) and len(a) > 1000
    for f in ("h", "gamma", "step", "panel", "module", "w", "u", "v", "edep", "t_ps"):
        assert np.array_equal(a[f], b[f]), f
    assert np.array_equal(b["layer"], (b["w"] >= 5.0).astype(np.int32))
    # crystal index inside its layer is unchanged
    ca = a["crystal"] % 64
    cb = (b["crystal"] % 128) % 64
    assert np.array_equal(ca, cb)


def test_four_layer_stack_zero_gap_equals_single_layer(oracle):
    """Four 2.5 mm layers stacked with no gaps are one 10 mm layer: same hits
    history by history; layer l holds depths [2.5 l, 2.5 (l+1)), and each hit
    keeps its crystal position inside its layer."""
    one = W.scanner(8, 40.0, [W.layer(8, 8, 1.6, 0.1, 10.0)])
    four = W.scanner(8, 40.0, [W.layer(8, 8, 1.6, 0.1, 2.5) for _ in range(4)])
    a = oracle.simulate(one, W.point_source((-2.0, 1.0, 1.5)), W.digitizer(), 30000, seed=22, threads=4)["hits"]
    b = oracle.simulate(four, W.point_source((-2.0, 1.0, 1.5)), W.digitizer(), 30000, seed=22, threads=4)["hits"]
    assert len(a) == len(b) and len(a) > 1000
    for f in ("h", "gamma", "step", "panel", "module", "w", "u", "v", "edep", "t_ps"):
        assert np.array_equal(a[f], b[f]), f
    assert np.array_equal(b["layer"], np.floor(b["w"] / 2.5).astype(np.int32))
    assert set(np.unique(b["layer"])) == {0, 1, 2, 3}
    assert np.array_equal(a["crystal"] % 64, (b["crystal"] % 256) % 64)
    assert np.array_equal((b["crystal"] % 256) // 64, b["layer"])


def test_blur_width_and_normals(oracle):
    """Box-Muller normals of the digitizer are N(0,1) (KS test); the photopeak
    blur has sigma = 0.15 * 511 / 2.3548."""
    h = np.arange(200_000, dtype=np.uint64)
    unit = (np.arange(200_000) % 97).astype(np.int32)
    z = oracle.blur_normals(5, h, unit)
    assert stats.kstest(z, "norm").pvalue > 1e-3
    r = oracle.simulate(W.config1_scanner(), W.point_source(), W.digitizer(e_lo=0, e_hi=2000), 100000, seed=1,
                        threads=8)
    s = r["singles"]
    pk = s[s["e_raw"] == 511.0]
    sig = 0.15 * 511.0 / (2 * math.sqrt(2 * math.log(2)))
    dev = pk["e_blur"] - 511.0
    assert abs(dev.std() / sig - 1) < 4 / math.sqrt(2 * len(dev))
    assert abs(dev.mean()) < 4 * sig / math.sqrt(len(dev))


def brute_force_coincidences(t, panel, window_ps):
    """O(n^2) restatement of the window policy: repeatedly take the earliest
    unconsumed single, collect every unconsumed single within the window."""
    n = len(t)
    consumed = np.zeros(n, bool)
    pairs = set()
    order_key = sorted(range(n), key=lambda i: (t[i], i))
    while not consumed.all():
        i0 = next(i for i in order_key if not consumed[i])
        members = [j for j in range(n) if not consumed[j] and t[i0] <= t[j] <= t[i0] + window_ps]
        for j in members:
            consumed[j] = True
        if len(members) == 2 and panel[members[0]] != panel[members[1]]:
            pairs.add(frozenset(members))
    return pairs


def test_coincidence_policy_brute_force(oracle):
    """Window sorter vs O(n^2) brute force on clustered random singles
    (includes ties, multiples, same-panel pairs and isolated singles)."""
    rng = np.random.default_rng(12)
    for trial in range(20):
        n = int(rng.integers(1, 300))
        base = np.sort(rng.integers(0, 40_000, size=n // 2 + 1))
        t = np.concatenate([base, base[: n - len(base)] + rng.integers(0, 3000, size=n - len(base))])[:n]
        t = t.astype(np.uint64)
        panel = rng.integers(0, 4, n).astype(np.int32)
        unit = (panel * 100 + rng.integers(0, 3, n)).astype(np.int32)
        h = rng.permutation(n).astype(np.uint64)
        s = np.zeros(n, dtype=[("t_ps", "<u8"), ("unit", "<i4"), ("panel", "<i4"), ("h", "<u8")])
        s["t_ps"], s["unit"], s["panel"], s["h"] = t, unit, panel, h
        _, a, b = oracle.coincidences(s, 2.0)
        got = {frozenset((int(x), int(y))) for x, y in zip(a, b)}
        assert got == brute_force_coincidences(t, panel, 2000), trial


def test_window_edges(oracle):
    """The window [t, t + tau] is closed at both ends (the reading the sorter
    follows); a third single on the far edge makes a multiple; a single just
    past it opens the next window."""
    def count(times, panels):
        n = len(times)
        s = np.zeros(n, dtype=[("t_ps", "<u8"), ("unit", "<i4"), ("panel", "<i4"), ("h", "<u8")])
        s["t_ps"], s["panel"], s["unit"], s["h"] = times, panels, np.array(panels) * 10, np.arange(n)
        return len(oracle.coincidences(s, 2.0)[1])
    assert count([1000, 3000], [0, 1]) == 1
    assert count([1000, 3001], [0, 1]) == 0
    assert count([1000, 2000, 3000], [0, 1, 2]) == 0
    assert count([1000, 3000, 3001, 5001], [0, 1, 2, 3]) == 2
    assert count([1000, 3000], [1, 1]) == 0


def _renewal_coincidences(rate_per_ps, tau_ps, span_ps, p_diff):
    """Expected coincidences of the single-window, kill-multiples sorter on a
    Poisson stream: windows open at rate rate/(1 + rate tau) (the stream is
    memoryless, so each window closes and the next opens at the first later
    single), and a window holds exactly one more single with probability
    rate tau exp(-rate tau)."""
    x = rate_per_ps * tau_ps
    return span_ps * rate_per_ps / (1.0 + x) * x * math.exp(-x) * p_diff


@pytest.mark.parametrize("x", [0.05, 0.5, 2.0])
def test_window_sorter_on_poisson_singles(oracle, x):
    """Poisson singles with uniform panels: the coincidence count follows the
    renewal formula at any rate.  Catches a sliding instead of a consumed
    window, multiples kept or counted, and the same-panel rule."""
    rng = np.random.default_rng(int(x * 100))
    tau = 2000
    rate = x / tau
    n = 200_000
    span = n / rate
    t = np.sort(rng.uniform(0.0, span, n)).astype(np.uint64)
    n_panels = 4
    s = np.zeros(n, dtype=[("t_ps", "<u8"), ("unit", "<i4"), ("panel", "<i4"), ("h", "<u8")])
    s["t_ps"] = t
    s["panel"] = rng.integers(0, n_panels, n)
    s["unit"] = s["panel"] * 100
    s["h"] = np.arange(n)
    _, a, _ = oracle.coincidences(s, tau / 1000.0)
    want = _renewal_coincidences(rate, tau, span, 1.0 - 1.0 / n_panels)
    assert abs(len(a) - want) < 5.0 * math.sqrt(want), (len(a), want)


def test_randoms_rate_at_high_activity(oracle):
    """Whole chain at 1e9 Bq: coincidences of two histories (randoms) against
    the renewal form of 2 tau S_i S_j.  Histories arrive as a Poisson process
    (uniform decay times on [0, n/A], Sec. 2.3); a random needs an opening
    history with exactly one kept single in panel i, one more such history
    within tau in panel j != i, and no third.  Pins the time model (the span
    n/A in picoseconds) together with the sorter."""
    sc = W.config1_scanner()
    dg = W.digitizer()
    n, act = 10_000_000, 1e9
    r = oracle.simulate(sc, W.point_source(activity_bq=act), dg, n, seed=2024, threads=8, tallies=False)
    span = r["t_span_ps"]
    assert span == pytest.approx(n / act * 1e12, rel=1e-12)
    s, a, b = oracle.coincidences(r["singles"], dg["window_ns"])
    randoms = int((s["h"][a] != s["h"][b]).sum())
    # histories with at least one kept single, and those with exactly one, per panel
    hs, first, cnt = np.unique(s["h"], return_index=True, return_counts=True)
    lam = len(hs) / span
    one = s["panel"][first[cnt == 1]]
    R = np.bincount(one, minlength=sc["n_panels"]) / span
    tau = dg["window_ns"] * 1000.0
    x = lam * tau
    want = span * tau * math.exp(-x) / (1.0 + x) * (R.sum() ** 2 - (R ** 2).sum())
    assert x > 0.03 and want > 5000
    assert abs(randoms - want) < 5.0 * math.sqrt(want), (randoms, want)


def test_split_and_offset_relations_h2rspet(oracle):
    """Context check on the paper's Table 1 relations, centred point source on
    reduced H2RSPET rings: split == 1CL within Poisson error; 2CL lower."""
    rows = {r.split("=")[0].strip(): float(r.split("=")[1]) for r in read_golden("paper_text_values.txt")}
    assert rows["hits_split"] / rows["hits_1cl"] == pytest.approx(1.0005, abs=5e-4)
    n = 60000
    hits = {}
    for kind in ("1CL", "split", "2CL"):
        sc = W.h2rspet(kind, modules_v=2)
        r = oracle.simulate(sc, W.point_source(), W.digitizer(), n, seed=31, threads=8, tallies=False)
        hits[kind] = len(r["hits"])
    assert abs(hits["split"] - hits["1CL"]) < 4 * math.sqrt(hits["1CL"])
    assert hits["2CL"] < hits["1CL"]


def test_hit_time_is_path_over_c(oracle):
    """Back-to-back pencil pair onto two facing slabs at the same radius: the
    hit-time difference of the first hits is (w0 - w1) / c to within the 1 ps
    rounding of each time stamp."""
    mats = [W.AIR, dict(mu_total_511_cm=2.0, photo_frac_511=1.0, electron_density_cm3=0.0)]
    sc = W.scanner(2, 100.0, [W.layer(1, 1, 400.0, 0.0, 20.0)], materials=mats)
    r = oracle.simulate(sc, W.pencil_source(direction=(1, 0, 0)), W.digitizer(), 20000, seed=3, threads=4)
    h = r["hits"]
    a, b = h[h["gamma"] == 0], h[h["gamma"] == 1]
    common = np.intersect1d(a["h"], b["h"])
    a = a[np.isin(a["h"], common)]
    b = b[np.isin(b["h"], common)]
    assert len(common) > 5000
    dt = a["t_ps"].astype(np.int64) - b["t_ps"].astype(np.int64)
    want = (a["w"] - b["w"]) / 0.299792458
    assert np.all(np.abs(dt - want) <= 1.0 + 1e-9)
    # decay times are uniform on [0, n / A)
    t0 = np.minimum(a["t_ps"], b["t_ps"]).astype(np.float64)
    span = r["t_span_ps"]
    assert span == round(20000 / W.DEFAULT_ACTIVITY_BQ * 1e12)
    assert stats.kstest(t0 / span, "uniform").pvalue > 1e-3


def test_digitizer_singles_invariants(oracle):
    """Singles are per (history, readout unit): one single per distinct unit,
    energy sum of its hits, earliest hit time; the blur has sigma proportional
    to sqrt(E) (FWHM 15 % at 511 keV) at every energy."""
    for level in (W.READOUT_CRYSTAL, W.READOUT_MODULE, W.READOUT_PANEL):
        sc = W.h2rspet("2CL", modules_v=2)
        sc["readout_level"] = level
        r = oracle.simulate(sc, W.point_source((3.0, 1.0, 20.0)), W.digitizer(), 20000, seed=8, threads=4)
        hits, s = r["hits"], r["singles"]
        cpm = 51 * 51 + 50 * 50
        if level == W.READOUT_CRYSTAL:
            unit = hits["crystal"]
        elif level == W.READOUT_MODULE:
            unit = hits["crystal"] // cpm
        else:
            unit = hits["panel"]
        key_h = hits["h"].astype(np.int64) * 10_000_000 + unit
        uk, inv = np.unique(key_h, return_inverse=True)
        esum = np.bincount(inv, weights=hits["edep"])
        tmin = np.full(len(uk), np.iinfo(np.int64).max)
        np.minimum.at(tmin, inv, hits["t_ps"].astype(np.int64))
        key_s = s["h"].astype(np.int64) * 10_000_000 + s["unit"]
        assert len(key_s) == len(uk) and len(np.unique(key_s)) == len(key_s)
        order = np.argsort(key_s)
        assert np.array_equal(key_s[order], uk)
        np.testing.assert_allclose(s["e_raw"][order], esum, rtol=1e-12)
        assert np.array_equal(s["t_ps"][order].astype(np.int64), tmin)
    sig_k = 0.15 / (2 * math.sqrt(2 * math.log(2)))
    z = (s["e_blur"] - s["e_raw"]) / (sig_k * np.sqrt(511.0 * s["e_raw"]))
    low = s["e_raw"] < 400
    assert low.sum() > 1000
    assert stats.kstest(z[low], "norm").pvalue > 1e-3


def test_hits_and_tallies_agree(oracle):
    """Bookkeeping invariants on an offset dual-layer ring: every hit's recorded
    panel-local position locates to its recorded layer, module and crystal;
    the per-crystal tallies are the hit list summed (count, fixed-point energy
    in 2^-20 keV, FP64 energy).  Catches swapped position fields and tallies
    credited to the wrong crystal or scaled."""
    sc = W.h2rspet("2CL", modules_v=2)
    r = oracle.simulate(sc, W.point_source((3.0, 1.0, 20.0)), W.digitizer(), 20000, seed=12, threads=4)
    hits = r["hits"]
    assert len(hits) > 5000
    for k in np.unique(hits["panel"]):
        sel = hits[hits["panel"] == k]
        loc = oracle.locate(sc, int(k), np.stack([sel["w"], sel["u"], sel["v"]], 1))
        assert np.array_equal(loc[:, 0], sel["layer"]) and np.array_equal(loc[:, 1], sel["module"])
        assert np.array_equal(loc[:, 2], sel["crystal"])
    nc = r["n_crystals"]
    assert np.array_equal(r["tally_count"], np.bincount(hits["crystal"], minlength=nc).astype(np.uint64))
    efx = np.zeros(nc, np.uint64)
    np.add.at(efx, hits["crystal"], np.rint(hits["edep"] * 2.0 ** 20).astype(np.uint64))
    assert np.array_equal(r["tally_efx"], efx)
    np.testing.assert_allclose(r["tally_edep"], np.bincount(hits["crystal"], weights=hits["edep"], minlength=nc),
                               rtol=1e-12, atol=1e-9)


def test_module_gap_is_interval(oracle):
    """H2RSPET panel: six modules along the axis separated by 7 mm gaps."""
    sc = W.h2rspet("1CL")
    V = 6 * 51 + 5 * 7
    pts = [(5.0, 0.25, -V / 2 + 51 + 3.5), (5.0, 0.25, -V / 2 + 2 * (51 + 7) + 0.5), (5.0, 0.25, -V / 2 + 51 - 0.5)]
    got = oracle.locate(sc, 0, pts)
    assert got[0, 2] == -1 and got[0, 3] == 0
    assert got[1, 1] == 2 and got[1, 2] >= 0            # first crystal row of module 2
    assert got[2, 1] == 0 and got[2, 2] >= 0            # last crystal of module 0
    rng = np.random.default_rng(2)
    n = 400_000
    p = np.stack([rng.uniform(0, 10, n), rng.uniform(-25.5, 25.5, n), rng.uniform(-V / 2, V / 2, n)], 1)
    frac = (oracle.locate(sc, 0, p)[:, 2] >= 0).mean()
    want = 6 * 51 * 51 * 0.92 ** 2 / (51 * V)
    assert abs(frac - want) < 4 * math.sqrt(want * (1 - want) / n)


def test_transaxial_module_gap(oracle):
    """Three modules across the panel with 4 mm gaps between them: the panel is
    3 x 16 + 2 x 4 = 56 mm wide, a point in a gap is interval material, the
    modules sit where the widths put them, and crystals fill 3 x 64 x 1.8^2 mm^2
    of the 56 x 16 mm^2 face.  Catches a panel width or module origin that
    drops the transaxial gaps."""
    sc = W.scanner(6, 60.0, [W.layer(8, 8, 2.0, 0.2, 10.0)], modules_u=3, module_gap_u=4.0)
    U, V, Wd = oracle.panel_extent(sc)
    assert (U, V, Wd) == pytest.approx((56.0, 16.0, 10.0), abs=1e-12)
    got = oracle.locate(sc, 0, [(5.0, -10.0, 0.5), (5.0, -7.5, 0.5), (5.0, 27.5, 0.5), (5.0, -27.5, 0.5)])
    assert got[0, 2] == -1 and got[0, 3] == 0
    assert list(got[1:, 1]) == [1, 2, 0] and np.all(got[1:, 2] >= 0)
    # crystal columns: first of module 1, last of module 2, first of module 0
    assert list(got[1:, 2] % 8) == [0, 7, 0]
    rng = np.random.default_rng(4)
    n = 400_000
    p = np.stack([rng.uniform(0, 10, n), rng.uniform(-U / 2, U / 2, n), rng.uniform(-V / 2, V / 2, n)], 1)
    frac = (oracle.locate(sc, 0, p)[:, 2] >= 0).mean()
    want = 3 * 64 * 1.8 ** 2 / (U * V)
    assert abs(frac - want) < 4 * math.sqrt(want * (1 - want) / n)


def box_chord_pairs(lo, hi, n, rng):
    """Independent quadrature: mean of exp(-mu * chord) over uniform points in a
    box and isotropic lines through them (chord = exit distance both ways)."""
    x = rng.uniform(lo, hi, size=(n, 3))
    d = rng.normal(size=(n, 3))
    d /= np.linalg.norm(d, axis=1)[:, None]

    def exit_dist(x, d):
        t = np.full(len(x), np.inf)
        for a in range(3):
            with np.errstate(divide="ignore", invalid="ignore"):
                tp = np.where(d[:, a] > 0, (hi[a] - x[:, a]) / d[:, a], np.inf)
                tn = np.where(d[:, a] < 0, (lo[a] - x[:, a]) / d[:, a], np.inf)
            t = np.minimum(t, np.minimum(tp, tn))
        return t
    return exit_dist(x, d) + exit_dist(x, -d)


def test_phantom_no_scatter_fraction(oracle):
    """Uniform water box with uniform activity: the fraction of pairs with no
    real phantom interaction == E[exp(-mu (L1 + L2))] over points and lines
    (numpy quadrature, independent of the oracle)."""
    nx, ny, nz, vs = 20, 16, 12, 1.5
    origin = (-15.0, -12.0, -9.0)
    ph = dict(nx=nx, ny=ny, nz=nz, voxel=(vs, vs, vs), origin=origin,
              material=np.ones((nz, ny, nx), np.uint8), activity=np.ones((nz, ny, nx), np.float32),
              materials=[W.AIR, W.WATER])
    n = 100_000
    r = oracle.simulate(W.config1_scanner(), W.phantom_source(), W.digitizer(), n, seed=4, phantom=ph, threads=8,
                        phantom_real=True, balance=True)
    p_obs = (r["phantom_real"] == 0).mean()
    lo = np.array(origin)
    hi = lo + vs * np.array([nx, ny, nz])
    chord = box_chord_pairs(lo, hi, 2_000_000, np.random.default_rng(1))
    p_exp = np.exp(-0.0096 * chord).mean()
    assert abs(p_obs - p_exp) < 4 * math.sqrt(p_exp * (1 - p_exp) / n) + 3e-4, (p_obs, p_exp)
    np.testing.assert_allclose(r["balance"], 1022.0, atol=1e-9)


def test_phantom_single_scatter_escape(oracle):
    """Pencil pair from the centre of a 100 mm water cube (Compton only): a
    photon has exactly one real phantom interaction with probability
    p1 = P(first collision) x E[exp(-mu(E') L')], over the first-collision
    depth, the Klein-Nishina angle at 511 keV and the exit chord L' of the
    scattered photon, with mu(E') = mu(511) sigma(E') / sigma(511).  Computed
    here by an independent numpy Monte Carlo (its own KN rejection sampler and
    box chords); a history's count is 1 with probability 2 p0 p1.  Catches a
    Woodcock majorant or cross section taken at the wrong energy after a
    scatter, which the unscattered fraction cannot see."""
    half = 50.0
    ph = dict(nx=10, ny=10, nz=10, voxel=(10.0, 10.0, 10.0), origin=(-half, -half, -half),
              material=np.ones((10, 10, 10), np.uint8), activity=None, materials=[W.AIR, W.WATER])
    sc = W.scanner(8, 80.0, [W.layer(8, 8, 1.6, 0.1, 10.0)])
    n = 400_000
    r = oracle.simulate(sc, W.pencil_source(direction=(1, 0, 0)), W.digitizer(), n, seed=31, phantom=ph,
                        threads=8, tallies=False, phantom_real=True)
    cnt = r["phantom_real"]
    mu511 = 0.096 / 10.0                        # 1/mm
    p0 = math.exp(-mu511 * half)
    # independent Monte Carlo of p1
    rng = np.random.default_rng(5)
    m = 2_000_000
    s = -np.log(1.0 - rng.uniform(size=m) * (1.0 - p0)) / mu511          # first collision depth in [0, half)
    k = 511.0 / MEC2
    ct = np.empty(0)
    fmax = kn_dsigma_domega(511.0, 1.0)
    while len(ct) < m:
        c = rng.uniform(-1.0, 1.0, 2 * m)
        ct = np.concatenate([ct, c[rng.uniform(size=2 * m) * fmax < kn_dsigma_domega(511.0, c)]])
    ct = ct[:m]
    st = np.sqrt(1.0 - ct * ct)
    phi = rng.uniform(0.0, 2 * math.pi, m)
    d = np.stack([ct, st * np.cos(phi), st * np.sin(phi)], 1)
    x = np.stack([s, np.zeros(m), np.zeros(m)], 1)
    with np.errstate(divide="ignore", invalid="ignore"):
        t = np.min(np.where(d > 0, (half - x) / d, np.where(d < 0, (-half - x) / d, np.inf)), axis=1)
    e1 = 511.0 / (1.0 + k * (1.0 - ct))
    grid = np.linspace(160.0, 512.0, 353)
    sig = np.array([integrate.quad(lambda c: kn_dsigma_domega(e, c), -1, 1, epsrel=1e-10)[0] for e in grid])
    sig511 = integrate.quad(lambda c: kn_dsigma_domega(511.0, c), -1, 1, epsrel=1e-10)[0]
    mu1 = mu511 * np.interp(e1, grid, sig) / sig511
    surv = np.exp(-mu1 * t)
    p1 = (1.0 - p0) * surv.mean()
    p1_err = (1.0 - p0) * surv.std() / math.sqrt(m)
    want = 2.0 * p0 * p1
    got = (cnt == 1).mean()
    assert abs((cnt == 0).mean() - p0 * p0) < 5.0 * math.sqrt(p0 * p0 * (1 - p0 * p0) / n)
    assert abs(got - want) < 5.0 * math.sqrt(want * (1 - want) / n) + 2 * p0 * 5.0 * p1_err, (got, want)


def test_phantom_material_layout(oracle):
    """Voxel materials are indexed x fastest, then y, then z (the layout the
    ABI documents).  A 4 x 2 x 2 grid of 10 mm voxels holds an absorber
    (photoelectric only, 0.5/cm) only where ix >= 2, iy = 1 and iz = 1; a pencil
    pair from the centre along x crosses 20 mm of it with photon 0 and none
    with photon 1, so a pair is untouched with probability exp(-1).  Catches a
    transposed material index (which moves the absorber off the beam)."""
    absorber = dict(name="absorber", mu_total_511_cm=0.5, photo_frac_511=1.0, electron_density_cm3=0.0)
    mat = np.zeros((2, 2, 4), np.uint8)          # [iz][iy][ix]
    mat[1, 1, 2:] = 1
    ph = dict(nx=4, ny=2, nz=2, voxel=(10.0, 10.0, 10.0), origin=(-20.0, -10.0, -10.0), material=mat,
              activity=None, materials=[W.AIR, absorber])
    n = 200_000
    r = oracle.simulate(W.config1_scanner(), W.pencil_source(direction=(1, 0, 0)), W.digitizer(), n, seed=8,
                        phantom=ph, threads=8, tallies=False, phantom_real=True)
    p = math.exp(-0.5 * 2.0)
    got = (r["phantom_real"] == 0).mean()
    assert abs(got - p) < 5.0 * math.sqrt(p * (1 - p) / n), (got, p)
    assert r["phantom_real"].max() == 1                 # the absorber ends photon 0; photon 1 meets none


def test_decay_sampling_follows_activity(oracle):
    """Decay points: voxel counts follow the activity map (chi-square), the
    point is uniform inside its voxel, directions are isotropic, times uniform."""
    rng = np.random.default_rng(17)
    nx, ny, nz, vs = 6, 5, 4, 2.0
    act = rng.uniform(0, 1, size=(nz, ny, nx)).astype(np.float32)
    act[act < 0.25] = 0.0          # some empty voxels, including possibly the first
    act[0, 0, 0] = 0.0
    ph = dict(nx=nx, ny=ny, nz=nz, voxel=(vs, vs, vs), origin=(-6.0, -5.0, -4.0),
              material=np.ones((nz, ny, nx), np.uint8), activity=act, materials=[W.AIR, W.WATER])
    n = 300_000
    t, pos, d = oracle.decays(W.phantom_source(), n, 9, 0, n, phantom=ph)
    idx = np.floor((pos - np.array(ph["origin"])) / vs).astype(int)
    flat = (idx[:, 2] * ny + idx[:, 1]) * nx + idx[:, 0]
    cnt = np.bincount(flat, minlength=nx * ny * nz)
    p = act.reshape(-1).astype(np.float64) / act.sum()
    assert cnt[p == 0].sum() == 0
    m = p > 0
    chi2 = ((cnt[m] - n * p[m]) ** 2 / (n * p[m])).sum()
    assert stats.chi2.sf(chi2, m.sum() - 1) > 1e-3
    frac = (pos - np.array(ph["origin"])) / vs - idx
    assert stats.kstest(frac[:, 0], "uniform").pvalue > 1e-3
    assert stats.kstest(frac[:, 2], "uniform").pvalue > 1e-3
    # isotropy: cos(theta) uniform on [-1, 1], azimuth uniform
    assert stats.kstest((d[:, 2] + 1) / 2, "uniform").pvalue > 1e-3
    az = (np.arctan2(d[:, 1], d[:, 0]) / (2 * math.pi)) % 1.0
    assert stats.kstest(az, "uniform").pvalue > 1e-3
    np.testing.assert_allclose(np.linalg.norm(d, axis=1), 1.0, atol=1e-12)


def test_energy_conservation_high_cutoff(oracle):
    """With a 300 keV cutoff many Compton scatters end below it and the photon's
    remaining energy is deposited on the spot: every history still sums to
    1022 keV, and a photon either deposits all 511 keV or carries at least the
    cutoff energy away."""
    mats = [W.AIR, dict(mu_total_511_cm=0.9, photo_frac_511=0.0, electron_density_cm3=0.0)]
    sc = W.scanner(8, 40.0, [W.layer(8, 8, 1.6, 0.1, 10.0)], materials=mats)
    r = oracle.simulate(sc, W.point_source(), W.digitizer(e_cut=300.0), 20000, seed=2, threads=4, balance=True)
    np.testing.assert_allclose(r["balance"], 1022.0, atol=1e-9)
    # a photon that drops below 300 keV deposits everything it had left at once:
    # the last hit of such a photon is its whole remaining energy, so no photon's
    # hits sum to less than 511 - (energy carried away by a >= 300 keV photon)
    h = r["hits"]
    key = h["h"].astype(np.int64) * 2 + h["gamma"]
    _, inv = np.unique(key, return_inverse=True)
    tot = np.bincount(inv, weights=h["edep"])
    assert np.all((tot > 511.0 - 1e-9) | (tot < 511.0 - 300.0 + 1e-9))


def test_doi_blur_of_singles(oracle):
    """Depth of a single = energy-weighted depth of its hits; the depth blur is
    Gaussian with FWHM doi_fwhm_mm and independent of the energy blur (the two
    normals of one Box-Muller pair)."""
    sc = W.h2rspet("2CL", modules_v=2)
    dg = W.digitizer(e_lo=0.0, e_hi=5000.0, doi_fwhm_mm=2.0)
    r = oracle.simulate(sc, W.point_source((2.0, -1.0, 10.0)), dg, 60000, 14, threads=8)
    hits, s = r["hits"], r["singles"]
    key_h = hits["h"].astype(np.int64) * 10_000_000 + hits["crystal"]
    uk, inv = np.unique(key_h, return_inverse=True)
    ew = np.bincount(inv, weights=hits["edep"] * hits["w"]) / np.bincount(inv, weights=hits["edep"])
    key_s = s["h"].astype(np.int64) * 10_000_000 + s["unit"]
    order = np.argsort(key_s)
    np.testing.assert_allclose(s["doi"][order], ew, rtol=1e-12, atol=1e-12)
    assert np.all((s["doi"] >= 0.0) & (s["doi"] <= 10.0))
    sig = 2.0 / (2 * math.sqrt(2 * math.log(2)))
    zd = (s["doi_blur"] - s["doi"]) / sig
    ze = (s["e_blur"] - s["e_raw"]) / (0.15 / (2 * math.sqrt(2 * math.log(2))) * np.sqrt(511.0 * s["e_raw"]))
    assert stats.kstest(zd, "norm").pvalue > 1e-3
    assert abs(np.corrcoef(zd, ze)[0, 1]) < 4 / math.sqrt(len(zd))
    # no depth blur: the depth is reported as is
    r0 = oracle.simulate(sc, W.point_source((2.0, -1.0, 10.0)), W.digitizer(e_lo=0, e_hi=5000), 5000, 14, threads=4)
    assert np.array_equal(r0["singles"]["doi"], r0["singles"]["doi_blur"])


# --------------------------------------------------------------------------
# Non-repetition mode: panels placed one by one (Sec. 2.1)
# --------------------------------------------------------------------------

def _hits_key(h):
    return np.lexsort((h["step"], h["gamma"], h["h"]))


def test_ring_written_as_poses_is_the_ring(oracle):
    """The repetition-mode ring written out as explicit poses (built from the
    ring's definition in workloads.ring_poses) gives the same hits, crystal for
    crystal, as the ring itself; positions and energies agree to rounding."""
    sc = W.config3_scanner()
    posed = W.with_poses(sc, W.ring_poses(sc))
    src, dg = W.point_source((7.0, -4.0, 12.0)), W.digitizer()
    a = oracle.simulate(sc, src, dg, 20_000, 31, threads=4)["hits"]
    b = oracle.simulate(posed, src, dg, 20_000, 31, threads=4)["hits"]
    assert len(a) == len(b) > 10_000
    a, b = a[_hits_key(a)], b[_hits_key(b)]
    for f in ("h", "gamma", "step", "panel", "module", "layer", "crystal", "t_ps"):
        assert np.array_equal(a[f], b[f]), f
    for f in ("w", "u", "v", "edep"):
        np.testing.assert_allclose(a[f], b[f], rtol=0, atol=1e-9)


def _triangle_solid_angle(r1, r2, r3):
    """Solid angle of a triangle seen from the origin (Van Oosterom and
    Strackee, IEEE Trans. Biomed. Eng. 30, 1983)."""
    l1, l2, l3 = (np.linalg.norm(r) for r in (r1, r2, r3))
    num = abs(np.dot(r1, np.cross(r2, r3)))
    den = l1 * l2 * l3 + np.dot(r1, r2) * l3 + np.dot(r1, r3) * l2 + np.dot(r2, r3) * l1
    return 2.0 * math.atan2(num, den)


def _posed_box_solid_angle(pose_row, U, V, Wd, src):
    """Exact solid angle of a convex panel box: the sum over the faces the
    source sees from outside, each face split into two triangles."""
    w, u, v, o = (np.asarray(pose_row[3 * i:3 * i + 3]) for i in range(4))
    c = [o + a * Wd * w + b * U / 2 * u + e * V / 2 * v for a in (0, 1) for b in (-1, 1) for e in (-1, 1)]
    c = np.array(c)  # index = 4a + 2(b>0) + (e>0)
    faces = [((0, 2, 3, 1), -w), ((4, 5, 7, 6), w), ((0, 1, 5, 4), -u), ((2, 6, 7, 3), u),
             ((0, 4, 6, 2), -v), ((1, 3, 7, 5), v)]
    total = 0.0
    for idx, nrm in faces:
        P = c[list(idx)] - src
        if np.dot(P[0], nrm) >= 0.0:       # the source is behind this face's plane
            continue
        total += _triangle_solid_angle(P[0], P[1], P[2]) + _triangle_solid_angle(P[0], P[2], P[3])
    return total


def test_posed_panels_acceptance_exact_solid_angle(oracle):
    """Posed heads (tilted, turned, at different distances): the fraction of
    isotropic rays from an off-centre point that enter each head equals that
    box's exact solid angle / 4 pi."""
    sc = W.box_scanner()
    U, V, Wd = oracle.panel_extent(sc)
    src = np.array([4.0, -3.0, 6.0])
    rng = np.random.default_rng(17)
    n = 2_000_000
    d = rng.normal(size=(n, 3))
    d /= np.linalg.norm(d, axis=1)[:, None]
    pn, ti = oracle.flight(sc, np.tile(src, (n, 1)), d)
    for k in range(sc["n_panels"]):
        p_exp = _posed_box_solid_angle(sc["panel_poses"][k], U, V, Wd, src) / (4 * math.pi)
        p = (pn == k).mean()
        assert 0.01 < p_exp < 0.2
        assert abs(p - p_exp) < 4.5 * math.sqrt(p_exp * (1 - p_exp) / n), (k, p, p_exp)


def test_rigid_motion_of_posed_scanner_and_pencil_source(oracle):
    """Moving every panel and a pencil source by the same rotation and
    translation leaves each hit unchanged in its panel's own frame: crystal,
    local position, deposit, time (transport is equivariant, and the Compton
    rotation of a posed panel takes the panel's v axis as polar reference)."""
    sc = W.box_scanner()
    p0, d0 = np.array([2.0, 1.0, -3.0]), np.array([1.0, 0.08, 0.05])
    d0 /= np.linalg.norm(d0)
    rng = np.random.default_rng(23)
    A = rng.normal(size=(3, 3))
    Q, Rr = np.linalg.qr(A)
    Q = Q * np.sign(np.diag(Rr))
    if np.linalg.det(Q) < 0:
        Q[:, 0] = -Q[:, 0]
    t = np.array([13.0, -7.0, 21.0])
    moved = W.rigid_motion(sc, Q, t)
    dg = W.digitizer()
    a = oracle.simulate(sc, W.pencil_source(p0, d0), dg, 20_000, 41, threads=4)["hits"]
    b = oracle.simulate(moved, W.pencil_source(Q @ p0 + t, Q @ d0), dg, 20_000, 41, threads=4)["hits"]
    assert len(a) == len(b) > 20_000
    assert set(np.unique(a["panel"])) >= {0, 1}
    a, b = a[_hits_key(a)], b[_hits_key(b)]
    for f in ("h", "gamma", "step", "panel", "module", "layer", "crystal"):
        assert np.array_equal(a[f], b[f]), f
    for f in ("w", "u", "v", "edep"):
        np.testing.assert_allclose(a[f], b[f], rtol=0, atol=1e-8)
    assert np.abs(a["t_ps"].astype(np.int64) - b["t_ps"].astype(np.int64)).max() <= 1


# ---------------------------------------------------------------------------
# sensitivity map S(r, E) and the symmetric percent difference (Sec. 2.4)
# ---------------------------------------------------------------------------
def _pair_acceptance_on_axis(n_panels, R, U, V, z, n=400_000):
    """Fraction of isotropic back-to-back pairs from (0, 0, z) whose two photons
    both cross a panel's inner face, by midpoint quadrature over the azimuth.
    For an even ring a transaxial direction phi meets panel k's face iff
    |R tan(phi - phi_k)| <= U/2, and then so does phi + pi (the opposite panel),
    at the same distance rho = R / cos(phi - phi_k).  Both photons stay inside
    the axial extent iff |rho cot(theta)| <= V/2 - |z|, which for cos(theta)
    uniform on [-1, 1] has probability a / sqrt(1 + a^2), a = (V/2 - |z|) / rho."""
    phi = (np.arange(n) + 0.5) * (2 * math.pi / n)
    dphi = 2 * math.pi / n_panels
    rel = (phi + 0.5 * dphi) % dphi - 0.5 * dphi      # angle to the nearest panel normal
    hit = np.abs(R * np.tan(rel)) <= 0.5 * U
    rho = R / np.cos(rel)
    a = max(0.5 * V - abs(z), 0.0) / rho
    return float(np.mean(np.where(hit, a / np.sqrt(1 + a * a), 0.0)))


def test_sensitivity_equals_pair_acceptance_of_an_opaque_ring(oracle):
    """Opaque photoelectric crystals without gaps, no energy blur: every photon
    that crosses an inner face deposits 511 keV in one crystal, so S in any
    window holding 511 keV is the pair acceptance (quadrature above), a window
    above 511 keV counts nothing, and windows holding 511 keV agree exactly."""
    sc = W.opaque_ring()
    sc["materials"][1] = dict(sc["materials"][1], mu_total_511_cm=1000.0)
    dg = W.digitizer(fwhm_at_511=0.0, window_ns=2.0)
    zs = [0.0, 25.0, 38.0]
    n = 100_000
    counts, S = oracle.sensitivity_map([sc], [(0.0, 0.0, z) for z in zs], dg,
                                       [(150.0, 700.0), (450.0, 700.0), (600.0, 700.0)], n, 17, threads=8,
                                       activity_bq=100.0)
    for p, z in enumerate(zs):
        expect = _pair_acceptance_on_axis(12, 55.0, 20.0, 80.0, z)
        assert abs(S[0, p, 0] - expect) < 4.5 * math.sqrt(expect * (1 - expect) / n), (z, S[0, p, 0], expect)
        assert counts[0, p, 1] == counts[0, p, 0]
        assert counts[0, p, 2] == 0
    assert _pair_acceptance_on_axis(12, 55.0, 20.0, 80.0, 0.0) == pytest.approx(0.4024, abs=5e-3)


def test_sensitivity_window_changes_only_the_digitizer(oracle):
    """Draws are addressed by history, photon and step, and the energy window
    acts on singles only: the coincidences of a run with window E equal those
    of the widest-window run with its singles cut to E afterwards."""
    sc = W.h2rspet("2CL", modules_v=2)
    dg = W.sensitivity_digitizer()
    pos = (20.0, 0.0, 10.0)
    counts, _ = oracle.sensitivity_map([sc], [pos], dg, W.SENS_WINDOWS_KEV, 30_000, 5, threads=8)
    r = oracle.simulate(sc, W.point_source(pos), dict(dg, e_lo=150.0, e_hi=700.0), 30_000, 5, threads=8,
                        tallies=False)
    s = r["singles"]
    for w, (lo, hi) in enumerate(W.SENS_WINDOWS_KEV):
        cut = s[(s["e_blur"] >= lo) & (s["e_blur"] <= hi)]
        cut = cut[np.argsort(cut["t_ps"], kind="stable")]
        _, a, _ = oracle.coincidences(np.array(cut), dg["window_ns"])
        assert counts[0, 0, w] == len(a), w


def test_delta_sym_properties_and_the_paper_relation(oracle):
    """Delta_sym = 200 (S_a - S_b) / (S_a + S_b): antisymmetric, zero for equal
    sensitivities, bounded by +-200 (reached when one is zero), scale-free, and
    to first order 100 ln(S_a / S_b); NaN where both are zero.  The paper
    reports the single layer above the offset dual layer by about 2-5 % (Sec.
    3.3); the oracle's H2RSPET-1CL vs -2CL at three positions and four windows
    agrees in sign and size."""
    a = np.array([0.1, 0.2, 0.0, 0.3, 0.05])
    b = np.array([0.1, 0.1, 0.2, 0.0, 0.0501])
    d = oracle.delta_sym(a, b)
    np.testing.assert_allclose(oracle.delta_sym(b, a), -d)
    assert d[0] == 0.0 and d[2] == -200.0 and d[3] == 200.0
    np.testing.assert_allclose(oracle.delta_sym(7 * a, 7 * b), d)
    assert d[4] == pytest.approx(100 * math.log(0.05 / 0.0501), rel=1e-5)
    assert np.isnan(oracle.delta_sym(0.0, 0.0))
    scs = [W.h2rspet("1CL", modules_v=2), W.h2rspet("2CL", modules_v=2)]
    _, S = oracle.sensitivity_map(scs, [(0.0, 0.0, 0.0), (30.0, 0.0, 0.0), (0.0, 0.0, 40.0)],
                                  W.sensitivity_digitizer(), W.SENS_WINDOWS_KEV, 200_000, 11, threads=8)
    ds = oracle.delta_sym(S[0], S[1])
    assert np.all(ds > 0.0) and np.all(ds < 8.0), ds
    assert 1.5 < ds.mean() < 5.5, ds
