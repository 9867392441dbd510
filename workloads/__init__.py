"""Seeded synthetic inputs shared by the oracle and the CUDA path.

This module only *describes* inputs: scanner geometries, sources, phantoms and
request streams, as plain Python dicts of numbers and numpy arrays.  It holds
none of the method's arithmetic (no cross sections, no transport, no
digitizer); both the FP64 oracle and the GPU library read these dicts through
their own, independent code.

Units: mm, keV, ns, 1/cm.  Geometry vocabulary follows the four-level detector
hierarchy of Sec. 2.1 / Fig. 1 of the paper: panel (level 0) -> module (1) ->
layer (2) -> crystal (3).  Each layer lists its crystal count, pitch, gap,
depth, offset and the crystal / inter-crystal materials in order (Sec. 2.1).
"""
from __future__ import annotations

import math

import numpy as np

# ---------------------------------------------------------------------------
# materials (synthetic physics model; 511 keV anchors)
# ---------------------------------------------------------------------------
# mu_total_511_cm: linear attenuation at 511 keV (1/cm)
# photo_frac_511:  photoelectric share of mu_total at 511 keV
# electron_density_cm3: 0 -> Compton coefficient anchored at
#     mu_total*(1-photo_frac) with Klein-Nishina energy dependence;
#     > 0 -> mu_C(E) = n_e * sigma_KN(E) taken literally.
AIR = dict(name="air", mu_total_511_cm=0.0, photo_frac_511=0.0, electron_density_cm3=0.0)
LYSO = dict(name="LYSO", mu_total_511_cm=0.87, photo_frac_511=0.34, electron_density_cm3=0.0)
LYSO_LITERAL_NE = dict(name="LYSO-ne", mu_total_511_cm=0.87, photo_frac_511=0.34,
                       electron_density_cm3=2.1e24)
WATER = dict(name="water", mu_total_511_cm=0.096, photo_frac_511=0.0, electron_density_cm3=0.0)

READOUT_PANEL, READOUT_MODULE, READOUT_CRYSTAL = 0, 1, 3

SOURCE_POINT, SOURCE_PHANTOM, SOURCE_PENCIL = 0, 1, 2

DEFAULT_ACTIVITY_BQ = 1.7e4  # 1.70e-2 MBq NEMA point source of Sec. 2.3


def layer(n_u, n_v, pitch, gap, depth, gap_before=0.0, offset_u=0.0, offset_v=0.0,
          crystal_mat=1, interval_mat=0, pitch_v=None, gap_v=None):
    """One crystal layer inside a module (Sec. 2.1: per-layer size, spacing, offset, materials)."""
    return dict(n_u=int(n_u), n_v=int(n_v), pitch_u=float(pitch),
                pitch_v=float(pitch if pitch_v is None else pitch_v),
                gap_u=float(gap), gap_v=float(gap if gap_v is None else gap_v),
                depth=float(depth), gap_before=float(gap_before),
                offset_u=float(offset_u), offset_v=float(offset_v),
                crystal_mat=int(crystal_mat), interval_mat=int(interval_mat))


def scanner(n_panels, inner_radius, layers, modules_u=1, modules_v=1, module_gap_u=0.0,
            module_gap_v=0.0, module_size_u=None, module_size_v=None, materials=None,
            first_angle=0.0, readout_level=READOUT_CRYSTAL, name=""):
    """Repetition-mode ring: one panel definition repeated n_panels times (Sec. 2.1).

    The module size defaults to the smallest box that holds every layer's crystal
    grid (offset + n * pitch), which is how an offset layer enlarges its module.
    """
    if materials is None:
        materials = [AIR, LYSO]
    if module_size_u is None:
        module_size_u = max(l["offset_u"] + l["n_u"] * l["pitch_u"] for l in layers)
    if module_size_v is None:
        module_size_v = max(l["offset_v"] + l["n_v"] * l["pitch_v"] for l in layers)
    return dict(name=name, n_panels=int(n_panels), inner_radius=float(inner_radius),
                first_angle=float(first_angle), modules_u=int(modules_u), modules_v=int(modules_v),
                module_size_u=float(module_size_u), module_size_v=float(module_size_v),
                module_gap_u=float(module_gap_u), module_gap_v=float(module_gap_v),
                layers=list(layers), materials=list(materials), readout_level=int(readout_level))


def ring_poses(sc):
    """The repetition-mode ring of `sc` written out as explicit panel poses: per
    panel the global w (normal), u (z x normal) and v (z) axes and the centre of
    the inner face (radius R along the normal), 12 numbers."""
    out = np.zeros((sc["n_panels"], 12))
    for k in range(sc["n_panels"]):
        phi = sc["first_angle"] + 2.0 * np.pi * k / sc["n_panels"]
        w = np.array([np.cos(phi), np.sin(phi), 0.0])
        u = np.array([-np.sin(phi), np.cos(phi), 0.0])
        v = np.array([0.0, 0.0, 1.0])
        out[k] = np.concatenate([w, u, v, sc["inner_radius"] * w])
    return out


def with_poses(sc, poses, name=None):
    """Non-repetition mode (Sec. 2.1: panels placed one by one): the same panel
    definition at the given poses."""
    out = dict(sc)
    out["panel_poses"] = np.ascontiguousarray(poses, dtype=np.float64).reshape(-1, 12)
    out["n_panels"] = int(out["panel_poses"].shape[0])
    if name:
        out["name"] = name
    return out


def _axis_rotation(axis, ang):
    a = np.asarray(axis, dtype=np.float64)
    a = a / np.linalg.norm(a)
    K = np.array([[0, -a[2], a[1]], [a[2], 0, -a[0]], [-a[1], a[0], 0]])
    return np.eye(3) + np.sin(ang) * K + (1 - np.cos(ang)) * (K @ K)


def pose(normal, u_hint, centre):
    """Pose of a panel whose inner face is centred at `centre` with outward
    normal `normal`; u is `u_hint` made orthogonal to the normal, v = w x u."""
    w = np.asarray(normal, dtype=np.float64)
    w = w / np.linalg.norm(w)
    u = np.asarray(u_hint, dtype=np.float64)
    u = u - (u @ w) * w
    u = u / np.linalg.norm(u)
    v = np.cross(w, u)
    return np.concatenate([w, u, v, np.asarray(centre, dtype=np.float64)])


def four_layer_scanner(readout_level=READOUT_CRYSTAL):
    """A four-layer stack (Sec. 2.1: the number of layers is a module parameter): 12-panel
    ring at R = 60 mm, 1 x 2 modules; 4 mm LYSO layers of 1.0 mm pitch, the
    second and fourth offset by half a pitch, the third at 1.25 mm pitch with
    16 x 16 crystals, 0.05 mm reflector between layers."""
    ls = [layer(20, 20, 1.0, 0.1, 4.0),
          layer(20, 20, 1.0, 0.1, 4.0, gap_before=0.05, offset_u=0.5, offset_v=0.5),
          layer(16, 16, 1.25, 0.1, 4.0, gap_before=0.05),
          layer(20, 20, 1.0, 0.1, 4.0, gap_before=0.05, offset_u=0.5, offset_v=0.5)]
    return scanner(12, 60.0, ls, modules_u=1, modules_v=2, readout_level=readout_level, name="ring12-4layer")


def box_scanner(readout_level=READOUT_CRYSTAL):
    """A non-ring design in non-repetition mode: two opposed heads at
    different distances, a third head tilted 20 degrees out of the transaxial
    plane, a fourth turned 15 degrees about its own normal.  Modules 1 x 2 of
    16 x 16 LYSO crystals (1.25 mm pitch, 0.1 mm gap), two 6 mm layers, the
    second offset by half a pitch, 0.05 mm reflector."""
    base = scanner(4, 45.0, [layer(16, 16, 1.25, 0.1, 6.0),
                             layer(16, 16, 1.25, 0.1, 6.0, gap_before=0.05, offset_u=0.625, offset_v=0.625)],
                   modules_u=1, modules_v=2, readout_level=readout_level, name="box4-posed")
    t20 = _axis_rotation((-1, 0, 0), np.radians(20.0))  # tilts the +y head out of the transaxial plane
    r15 = _axis_rotation((-1, 0, 0), np.radians(15.0))  # turns the -x head about its normal
    poses = [pose((1, 0, 0), (0, 1, 0), (45.0, 0.0, 0.0)),
             pose((-1, 0, 0), r15 @ np.array([0.0, -1.0, 0.0]), (-60.0, 0.0, 0.0)),
             pose(t20 @ np.array([0.0, 1.0, 0.0]), (1, 0, 0), (0.0, 52.0, 3.0)),
             pose((0, -1, 0), (-1, 0, 0), (0.0, -48.0, -5.0))]
    return with_poses(base, np.stack(poses), name="box4-posed")


def rigid_motion(sc, Q, t):
    """Move every panel of a posed scanner by x -> Q x + t."""
    P = np.asarray(sc["panel_poses"], dtype=np.float64).reshape(-1, 12).copy()
    for k in range(len(P)):
        for a in range(3):
            P[k, 3 * a:3 * a + 3] = Q @ P[k, 3 * a:3 * a + 3]
        P[k, 9:12] = Q @ P[k, 9:12] + np.asarray(t, dtype=np.float64)
    return with_poses(sc, P)


def digitizer(fwhm_at_511=0.15, e_lo=350.0, e_hi=650.0, window_ns=2.0, e_cut=10.0, doi_fwhm_mm=0.0):
    return dict(fwhm_at_511=float(fwhm_at_511), e_lo=float(e_lo), e_hi=float(e_hi),
                window_ns=float(window_ns), e_cut=float(e_cut), doi_fwhm_mm=float(doi_fwhm_mm))


def point_source(pos=(0.0, 0.0, 0.0), activity_bq=DEFAULT_ACTIVITY_BQ):
    return dict(kind=SOURCE_POINT, pos=tuple(float(p) for p in pos), dir=(0.0, 0.0, 1.0),
                activity_bq=float(activity_bq))


def pencil_source(pos=(0.0, 0.0, 0.0), direction=(1.0, 0.0, 0.0), activity_bq=DEFAULT_ACTIVITY_BQ):
    """Collimated back-to-back pair along a fixed axis (used by the slab pins)."""
    d = np.asarray(direction, dtype=np.float64)
    d = d / np.linalg.norm(d)
    return dict(kind=SOURCE_PENCIL, pos=tuple(float(p) for p in pos), dir=tuple(float(x) for x in d),
                activity_bq=float(activity_bq))


def phantom_source(activity_bq=DEFAULT_ACTIVITY_BQ):
    return dict(kind=SOURCE_PHANTOM, pos=(0.0, 0.0, 0.0), dir=(0.0, 0.0, 1.0),
                activity_bq=float(activity_bq))


# ---------------------------------------------------------------------------
# the five workloads
# ---------------------------------------------------------------------------

def config1_scanner():
    """Tiny single-layer ring: 8 flat panels at 40 mm inner radius, 1 module of
    8x8 LYSO crystals, 1.6 mm pitch, 0.1 mm gaps, 10 mm deep."""
    return scanner(8, 40.0, [layer(8, 8, 1.6, 0.1, 10.0, crystal_mat=1, interval_mat=0)],
                   name="ring8-R40-8x8-p1.6-1x10mm")


def config1():
    return dict(scanner=config1_scanner(), source=point_source(), digitizer=digitizer(),
                n_decays=100_000, seed=1, phantom=None)


def config2_scanner(geometry="A"):
    """12-panel ring at 55 mm; 1x4 modules of 20x20 LYSO crystals at 1.0 mm pitch.

    The literal 4x4 modules of 20 mm do not fit 12 panels at 55 mm (maximum flat
    width 2*55*tan(15 deg) = 29.5 mm), so one tangential module is kept and the
    four modules run axially (80 mm), which covers the +-30 mm sweep.
    Geometry A: one 10 mm layer.  Geometry B: two aligned 5 mm layers behind a
    0.05 mm reflector gap (vacuum).
    """
    if geometry == "A":
        layers = [layer(20, 20, 1.0, 0.1, 10.0)]
    elif geometry == "B":
        layers = [layer(20, 20, 1.0, 0.1, 5.0), layer(20, 20, 1.0, 0.1, 5.0, gap_before=0.05)]
    else:
        raise ValueError(geometry)
    return scanner(12, 55.0, layers, modules_u=1, modules_v=4,
                   name=f"ring12-R55-1x4x(20x20)-p1.0-{geometry}")


def config2_positions():
    """Axial positions of the NEMA-style sweep: -30..30 mm in 1 mm steps (61)."""
    return [float(z) for z in range(-30, 31)]


def config2(geometry="A", n_decays=10_000_000):
    pos = config2_positions()
    return [dict(scanner=config2_scanner(geometry), source=point_source((0.0, 0.0, z)),
                 digitizer=digitizer(), n_decays=int(n_decays), seed=2 + i, phantom=None)
            for i, z in enumerate(pos)]


def config3_scanner():
    """Config-2 ring with two 5 mm layers; layer 2 shifted by half a pitch in u and v."""
    layers = [layer(20, 20, 1.0, 0.1, 5.0),
              layer(20, 20, 1.0, 0.1, 5.0, gap_before=0.05, offset_u=0.5, offset_v=0.5)]
    return scanner(12, 55.0, layers, modules_u=1, modules_v=4, name="ring12-R55-offset-dual-layer")


HOT_ROD_DIAMETERS = (0.8, 1.0, 1.2, 1.4, 1.6, 2.0)


def hot_rod_phantom(scale=1.0, nx=60, ny=60, nz=100, voxel=0.5, radius=15.0, length=50.0,
                    rod_ratio=10.0):
    """Water cylinder with a six-sector hot-rod insert (synthetic Derenzo analogue).

    Sectors are 60 deg wide, centred on 30 + 60k deg; sector k holds rods of
    diameter d_k on a triangular lattice of spacing 2 d_k.  A rod is kept when
    its disc lies inside the wedge (distance >= d to both edges) and inside
    radius (R - d).  Rods run the full length.  Voxel activity is rod_ratio in
    a rod, 1 elsewhere inside the cylinder, 0 outside.  Material 1 = water
    inside the cylinder, 0 = air (vacuum) outside.  `scale` multiplies the
    voxel size (and so every physical length).
    """
    vs = voxel * scale
    R = radius * scale
    half_len = 0.5 * length * scale
    origin = (-0.5 * nx * vs, -0.5 * ny * vs, -0.5 * nz * vs)
    xc = origin[0] + (np.arange(nx) + 0.5) * vs
    yc = origin[1] + (np.arange(ny) + 0.5) * vs
    zc = origin[2] + (np.arange(nz) + 0.5) * vs
    X, Y = np.meshgrid(xc, yc, indexing="xy")  # [iy, ix]
    r2 = X * X + Y * Y
    inside = r2 <= R * R
    rods = []
    in_rod = np.zeros_like(inside)
    for k, d0 in enumerate(HOT_ROD_DIAMETERS):
        d = d0 * scale
        a = math.radians(30.0 + 60.0 * k)
        e1 = np.array([math.cos(a), math.sin(a)]) * 2 * d
        e2 = np.array([math.cos(a + math.pi / 3), math.sin(a + math.pi / 3)]) * 2 * d
        # wedge edges at a -+ 30 deg
        n_lo = np.array([-math.sin(a - math.pi / 6), math.cos(a - math.pi / 6)])   # inward normal of lower edge
        n_hi = np.array([math.sin(a + math.pi / 6), -math.cos(a + math.pi / 6)])   # inward normal of upper edge
        nmax = int(R / (2 * d)) + 2
        for i in range(-nmax, nmax + 1):
            for j in range(-nmax, nmax + 1):
                c = i * e1 + j * e2
                if c @ n_lo < d or c @ n_hi < d:
                    continue
                if np.hypot(*c) > R - d:
                    continue
                rods.append((float(c[0]), float(c[1]), d))
                in_rod |= (X - c[0]) ** 2 + (Y - c[1]) ** 2 <= (0.5 * d) ** 2
    zmask = np.abs(zc) <= half_len
    act2d = np.where(in_rod & inside, rod_ratio, np.where(inside, 1.0, 0.0)).astype(np.float32)
    mat2d = inside.astype(np.uint8)
    activity = np.where(zmask[:, None, None], act2d[None, :, :], 0.0).astype(np.float32)
    material = np.where(zmask[:, None, None], mat2d[None, :, :], 0).astype(np.uint8)
    return dict(nx=nx, ny=ny, nz=nz, voxel=(vs, vs, vs), origin=origin,
                material=np.ascontiguousarray(material),    # [iz, iy, ix], x fastest
                activity=np.ascontiguousarray(activity),
                materials=[AIR, WATER], rods=rods)


def config3(n_decays=100_000_000):
    return dict(scanner=config3_scanner(), source=phantom_source(), digitizer=digitizer(),
                n_decays=int(n_decays), seed=3, phantom=hot_rod_phantom())


def random_design(rng):
    """One candidate scanner of the batched design sweep."""
    n_layers = int(rng.integers(1, 4))
    total_depth = float(rng.uniform(8.0, 20.0))
    pitch = float(rng.uniform(0.8, 2.0))
    radius = float(rng.uniform(40.0, 80.0))
    offset = bool(rng.integers(0, 2))
    n_panels = 12
    n_u = int(math.floor(0.9 * 2 * radius * math.tan(math.pi / n_panels) / pitch))
    n_v = int(round(20.0 / pitch))
    gap = 0.1
    layers = []
    for l in range(n_layers):
        off = 0.5 * pitch if (offset and l % 2 == 1) else 0.0
        layers.append(layer(n_u, n_v, pitch, gap, total_depth / n_layers,
                            gap_before=0.05 if l > 0 else 0.0, offset_u=off, offset_v=off))
    sc = scanner(n_panels, radius, layers, modules_u=1, modules_v=4,
                 name=f"design-L{n_layers}-p{pitch:.2f}-R{radius:.1f}-{'off' if offset else 'al'}")
    r_off = float(rng.uniform(0.0, min(50.0, 0.75 * radius)))
    phi = float(rng.uniform(0.0, 2 * math.pi))
    src = point_source((r_off * math.cos(phi), r_off * math.sin(phi), 0.0))
    n = int(round(10 ** rng.uniform(5.0, 7.0)))
    return sc, src, n


def config4(n_designs=64, seed=4, scale=1.0):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n_designs):
        sc, src, n = random_design(rng)
        out.append(dict(scanner=sc, source=src, digitizer=digitizer(),
                        n_decays=max(1, int(n * scale)), seed=1000 + i, phantom=None))
    return out


def config5(n_requests=2000, rate_hz=50.0, seed=5, pairs_lo=1e5, pairs_hi=5e7):
    """Poisson request stream: arrival times (s) and per-request workloads."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate_hz, size=n_requests)
    arrivals = np.cumsum(gaps)
    reqs = []
    for i in range(n_requests):
        sc, src, _ = random_design(rng)
        n = int(round(10 ** rng.uniform(math.log10(pairs_lo), math.log10(pairs_hi))))
        if rng.integers(0, 2) == 0:
            ph = None
        else:
            ph = ("hot_rod", float(rng.uniform(0.5, 1.0)))
            src = phantom_source()
        reqs.append(dict(arrival_s=float(arrivals[i]), scanner=sc, source=src,
                         digitizer=digitizer(), n_decays=n, seed=50_000 + i, phantom=ph))
    return reqs


# ---------------------------------------------------------------------------
# paper-like validation scanners (Sec. 2.2), used as extra test geometries
# ---------------------------------------------------------------------------

def h2rspet(kind="1CL", modules_v=6):
    """Ten-panel ring at 85 mm, six axial modules of 51x51 crystals at ~1.0 mm
    pitch (0.92 mm crystal + 0.08 mm gap), 7 mm inter-module gap (Sec. 2.2).
    1CL: one 10 mm layer; split: two aligned 5 mm layers; 2CL: inner 50x50 and
    outer 51x51 5 mm layers with a half-pitch axial offset."""
    p, g = 1.0, 0.08
    if kind == "1CL":
        layers = [layer(51, 51, p, g, 10.0)]
    elif kind == "split":
        layers = [layer(51, 51, p, g, 5.0), layer(51, 51, p, g, 5.0)]
    elif kind == "2CL":
        layers = [layer(50, 50, p, g, 5.0, offset_u=0.5 * p, offset_v=0.5 * p),
                  layer(51, 51, p, g, 5.0)]
    else:
        raise ValueError(kind)
    return scanner(10, 85.0, layers, modules_u=1, modules_v=modules_v, module_gap_v=7.0,
                   module_size_u=51 * p, module_size_v=51 * p, name=f"H2RSPET-{kind}")


# Sec. 2.4 sensitivity study: radial offsets 0..70 mm (5 mm steps), axial offsets
# 0..170 mm (10 mm steps), four energy windows with a 700 keV upper edge
SENS_WINDOWS_KEV = ((150.0, 700.0), (250.0, 700.0), (350.0, 700.0), (450.0, 700.0))


def sensitivity_positions(radial=tuple(range(0, 75, 5)), axial=tuple(range(0, 180, 10))):
    """Source positions of the sensitivity study: every radial offset along +x in
    the central slice, then every axial offset on the axis (the two profiles)."""
    pos = [(float(r), 0.0, 0.0) for r in radial]
    pos += [(0.0, 0.0, float(z)) for z in axial if z != 0]
    return pos


def sensitivity_digitizer():
    """Sec. 2.4 digitizer: 16 % energy resolution, 3 ns coincidence window."""
    return digitizer(fwhm_at_511=0.16, e_lo=150.0, e_hi=700.0, window_ns=3.0)


def opaque_ring(n_panels=12, radius=55.0):
    """Ring for the pair-acceptance pin: 1 x 4 modules of 20 x 20 crystals at 1.0
    mm pitch with no crystal or module gaps, 10 mm deep, of a photoelectric-only
    material with mu = 100 / cm (every photon entering a panel is absorbed in a
    crystal within ~0.1 mm, depositing 511 keV)."""
    opaque = dict(name="opaque", mu_total_511_cm=100.0, photo_frac_511=1.0, electron_density_cm3=0.0)
    return scanner(n_panels, radius, [layer(20, 20, 1.0, 0.0, 10.0)], modules_u=1, modules_v=4,
                   materials=[AIR, opaque], name="opaque-ring")
