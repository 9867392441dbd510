"""Python wrapper of the FP64 CPU oracle (gpet_oracle.c).

TEST INFRASTRUCTURE: only the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this module.  It never touches the
CUDA library and the CUDA library never touches it.

Inputs are the plain dicts of the ``workloads`` module; this wrapper packs them
into the oracle's own C structs.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gpet_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C, FP64, no FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
               "-pthread", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class Material(C.Structure):
    _fields_ = [("mu_total_511_cm", C.c_double), ("photo_frac_511", C.c_double),
                ("electron_density_cm3", C.c_double)]


class Layer(C.Structure):
    _fields_ = [("n_u", C.c_int32), ("n_v", C.c_int32), ("pitch_u", C.c_double), ("pitch_v", C.c_double),
                ("gap_u", C.c_double), ("gap_v", C.c_double), ("depth", C.c_double),
                ("gap_before", C.c_double), ("offset_u", C.c_double), ("offset_v", C.c_double),
                ("crystal_mat", C.c_int32), ("interval_mat", C.c_int32)]


class Scanner(C.Structure):
    _fields_ = [("n_panels", C.c_int32), ("inner_radius", C.c_double), ("first_angle", C.c_double),
                ("modules_u", C.c_int32), ("modules_v", C.c_int32), ("module_size_u", C.c_double),
                ("module_size_v", C.c_double), ("module_gap_u", C.c_double), ("module_gap_v", C.c_double),
                ("n_layers", C.c_int32), ("layers", C.POINTER(Layer)), ("n_materials", C.c_int32),
                ("materials", C.POINTER(Material)), ("readout_level", C.c_int32),
                ("panel_poses", C.POINTER(C.c_double))]


class Phantom(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32), ("voxel", C.c_double * 3),
                ("origin", C.c_double * 3), ("mat", C.POINTER(C.c_uint8)), ("activity", C.POINTER(C.c_float)),
                ("n_materials", C.c_int32), ("materials", C.POINTER(Material))]


class Source(C.Structure):
    _fields_ = [("kind", C.c_int32), ("pos", C.c_double * 3), ("dir", C.c_double * 3),
                ("activity_bq", C.c_double)]


class Digitizer(C.Structure):
    _fields_ = [("fwhm_at_511", C.c_double), ("e_lo", C.c_double), ("e_hi", C.c_double),
                ("window_ns", C.c_double), ("e_cut", C.c_double), ("doi_fwhm_mm", C.c_double)]


class Hit(C.Structure):
    _fields_ = [("h", C.c_uint64), ("gamma", C.c_int32), ("step", C.c_int32), ("panel", C.c_int32),
                ("module", C.c_int32), ("layer", C.c_int32), ("crystal", C.c_int32), ("w", C.c_double),
                ("u", C.c_double), ("v", C.c_double), ("edep", C.c_double), ("t_ps", C.c_uint64)]


class Single(C.Structure):
    _fields_ = [("t_ps", C.c_uint64), ("h", C.c_uint64), ("unit", C.c_int32), ("panel", C.c_int32),
                ("e_raw", C.c_double), ("e_blur", C.c_double), ("kept", C.c_int32), ("doi", C.c_double),
                ("doi_blur", C.c_double)]


class Output(C.Structure):
    _fields_ = [("n_hits", C.c_uint64), ("n_singles", C.c_uint64), ("n_kept", C.c_uint64),
                ("hits", C.POINTER(Hit)), ("singles", C.POINTER(Single)),
                ("tally_count", C.POINTER(C.c_uint64)), ("tally_efx", C.POINTER(C.c_uint64)),
                ("tally_edep", C.POINTER(C.c_double)), ("balance", C.POINTER(C.c_double)),
                ("ph_real", C.POINTER(C.c_uint32)),
                ("n_det_steps", C.c_uint64), ("n_ph_steps", C.c_uint64), ("n_flights", C.c_uint64),
                ("n_compton_trials", C.c_uint64), ("n_entered", C.c_uint64), ("status", C.c_int32)]


HIT_DTYPE = np.dtype([("h", "<u8"), ("gamma", "<i4"), ("step", "<i4"), ("panel", "<i4"), ("module", "<i4"),
                      ("layer", "<i4"), ("crystal", "<i4"), ("w", "<f8"), ("u", "<f8"), ("v", "<f8"),
                      ("edep", "<f8"), ("t_ps", "<u8")], align=True)
SINGLE_DTYPE = np.dtype([("t_ps", "<u8"), ("h", "<u8"), ("unit", "<i4"), ("panel", "<i4"), ("e_raw", "<f8"),
                         ("e_blur", "<f8"), ("kept", "<i4"), ("doi", "<f8"), ("doi_blur", "<f8")], align=True)
assert HIT_DTYPE.itemsize == C.sizeof(Hit)
assert SINGLE_DTYPE.itemsize == C.sizeof(Single)

_P = C.c_void_p


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            L.or_philox4x32_10.argtypes = [C.POINTER(C.c_uint32), C.POINTER(C.c_uint32), C.POINTER(C.c_uint32)]
            L.or_uniform.argtypes = [C.c_uint32]
            L.or_uniform.restype = C.c_double
            L.or_sigma_kn.argtypes = [C.c_double]
            L.or_sigma_kn.restype = C.c_double
            for f in (L.or_mu_photo, L.or_mu_compton, L.or_mu_total):
                f.argtypes = [C.POINTER(Material), C.c_double]
                f.restype = C.c_double
            L.or_simulate.argtypes = [C.POINTER(Scanner), C.POINTER(Phantom), C.POINTER(Source),
                                      C.POINTER(Digitizer), C.c_uint64, C.c_uint64, C.c_uint64, C.c_uint64,
                                      C.c_int, C.POINTER(Output)]
            L.or_free_output.argtypes = [C.POINTER(Output)]
            L.or_scanner_crystals.argtypes = [C.POINTER(Scanner)]
            L.or_time_span_ps.argtypes = [C.c_uint64, C.c_double]
            L.or_time_span_ps.restype = C.c_uint64
            L.or_coincidences.argtypes = [C.c_int64, _P, _P, _P, _P, C.c_uint64, _P, _P]
            L.or_coincidences.restype = C.c_int64
            L.or_kahn_batch.argtypes = [C.c_uint64, C.c_uint64, C.c_int64, C.c_double, _P, _P, _P]
            L.or_photo_count.restype = C.c_int64
            L.or_photo_count.argtypes = [C.POINTER(Material), C.c_double, C.c_uint64, C.c_uint64, C.c_int64]
            L.or_flight_batch.argtypes = [C.POINTER(Scanner), C.c_int64, _P, _P, _P, _P]
            L.or_locate_batch.argtypes = [C.POINTER(Scanner), C.c_int, C.c_int64, _P, _P]
            L.or_panel_extent.argtypes = [C.POINTER(Scanner), _P]
            L.or_blur_normals.argtypes = [C.c_uint64, C.c_int64, _P, _P, _P]
            L.or_rotate_batch.argtypes = [C.c_int64, _P, _P, _P]
            L.or_decay_batch.argtypes = [C.POINTER(Phantom), C.POINTER(Source), C.c_uint64, C.c_uint64, C.c_uint64,
                                         C.c_int64, _P, _P, _P]
            _lib = L
    return _lib


def _ptr(a):
    return a.ctypes.data_as(C.c_void_p)


def _materials(mats):
    arr = (Material * len(mats))()
    for i, m in enumerate(mats):
        arr[i] = Material(m["mu_total_511_cm"], m["photo_frac_511"], m.get("electron_density_cm3", 0.0))
    return arr


class _Packed:
    """Keeps ctypes buffers alive alongside the struct that points at them."""

    def __init__(self, struct, *keep):
        self.struct = struct
        self.keep = keep


def pack_scanner(sc):
    layers = (Layer * len(sc["layers"]))()
    for i, l in enumerate(sc["layers"]):
        layers[i] = Layer(l["n_u"], l["n_v"], l["pitch_u"], l["pitch_v"], l["gap_u"], l["gap_v"], l["depth"],
                          l["gap_before"], l["offset_u"], l["offset_v"], l["crystal_mat"], l["interval_mat"])
    mats = _materials(sc["materials"])
    poses = sc.get("panel_poses")
    if poses is not None:
        poses = np.ascontiguousarray(poses, dtype=np.float64).reshape(sc["n_panels"], 12)
    s = Scanner(sc["n_panels"], sc["inner_radius"], sc["first_angle"], sc["modules_u"], sc["modules_v"],
                sc["module_size_u"], sc["module_size_v"], sc["module_gap_u"], sc["module_gap_v"],
                len(sc["layers"]), layers, len(sc["materials"]), mats, sc["readout_level"],
                poses.ctypes.data_as(C.POINTER(C.c_double)) if poses is not None else None)
    return _Packed(s, layers, mats, poses)


def pack_phantom(ph):
    if ph is None:
        return None
    mat = np.ascontiguousarray(ph["material"], dtype=np.uint8).reshape(-1)
    act = ph.get("activity")
    act = None if act is None else np.ascontiguousarray(act, dtype=np.float32).reshape(-1)
    mats = _materials(ph["materials"])
    s = Phantom(ph["nx"], ph["ny"], ph["nz"], (C.c_double * 3)(*ph["voxel"]), (C.c_double * 3)(*ph["origin"]),
                mat.ctypes.data_as(C.POINTER(C.c_uint8)),
                act.ctypes.data_as(C.POINTER(C.c_float)) if act is not None else None, len(ph["materials"]), mats)
    return _Packed(s, mat, act, mats)


def pack_source(src):
    return Source(src["kind"], (C.c_double * 3)(*src["pos"]), (C.c_double * 3)(*src.get("dir", (0, 0, 1))),
                  src["activity_bq"])


def pack_digitizer(dg):
    return Digitizer(dg["fwhm_at_511"], dg["e_lo"], dg["e_hi"], dg["window_ns"], dg["e_cut"],
                     dg.get("doi_fwhm_mm", 0.0))


def n_crystals(sc) -> int:
    p = pack_scanner(sc)
    return int(lib().or_scanner_crystals(C.byref(p.struct)))


def panel_extent(sc):
    p = pack_scanner(sc)
    out = np.zeros(3)
    lib().or_panel_extent(C.byref(p.struct), _ptr(out))
    return out


def simulate(scanner, source, digitizer, n_decays, seed, phantom=None, h_begin=0, h_end=None, threads=1,
             tallies=True, balance=False, phantom_real=False):
    """Run histories [h_begin, h_end) of an n_decays simulation.  Returns dict:
    hits (structured array), singles (structured array, kept and rejected),
    tallies (count, efx, edep per global crystal id), counters, balance."""
    L = lib()
    if h_end is None:
        h_end = n_decays
    sp = pack_scanner(scanner)
    pp = pack_phantom(phantom)
    src = pack_source(source)
    dg = pack_digitizer(digitizer)
    nc = int(L.or_scanner_crystals(C.byref(sp.struct)))
    if nc < 0:
        raise ValueError("oracle rejected the scanner description")
    out = Output()
    tc = te = td = None
    if tallies:
        tc = np.zeros(nc, np.uint64)
        te = np.zeros(nc, np.uint64)
        td = np.zeros(nc, np.float64)
        out.tally_count = tc.ctypes.data_as(C.POINTER(C.c_uint64))
        out.tally_efx = te.ctypes.data_as(C.POINTER(C.c_uint64))
        out.tally_edep = td.ctypes.data_as(C.POINTER(C.c_double))
    bal = None
    if balance:
        bal = np.zeros(max(0, h_end - h_begin), np.float64)
        out.balance = bal.ctypes.data_as(C.POINTER(C.c_double))
    phr = None
    if phantom_real:
        phr = np.zeros(max(0, h_end - h_begin), np.uint32)
        out.ph_real = phr.ctypes.data_as(C.POINTER(C.c_uint32))
    st = L.or_simulate(C.byref(sp.struct), C.byref(pp.struct) if pp else None, C.byref(src), C.byref(dg),
                       int(n_decays), int(seed), int(h_begin), int(h_end), int(threads), C.byref(out))
    try:
        if st != 0:
            raise RuntimeError(f"oracle simulate failed with status {st}")
        nh, ns = int(out.n_hits), int(out.n_singles)
        hits = np.ctypeslib.as_array(C.cast(out.hits, C.POINTER(C.c_uint8)), shape=(nh * HIT_DTYPE.itemsize,))
        hits = hits.view(HIT_DTYPE).copy() if nh else np.zeros(0, HIT_DTYPE)
        sg = np.ctypeslib.as_array(C.cast(out.singles, C.POINTER(C.c_uint8)), shape=(ns * SINGLE_DTYPE.itemsize,))
        sg = sg.view(SINGLE_DTYPE).copy() if ns else np.zeros(0, SINGLE_DTYPE)
    finally:
        L.or_free_output(C.byref(out))
    return dict(hits=hits, singles=sg, tally_count=tc, tally_efx=te, tally_edep=td, balance=bal, phantom_real=phr,
                counters=dict(det_steps=int(out.n_det_steps), ph_steps=int(out.n_ph_steps),
                              flights=int(out.n_flights), compton_trials=int(out.n_compton_trials),
                              entered=int(out.n_entered)),
                n_crystals=nc, t_span_ps=int(L.or_time_span_ps(int(n_decays), float(source["activity_bq"]))))


def coincidences(singles, window_ns):
    """Coincidence sorting of kept singles (structured array as returned by simulate)."""
    s = singles[singles["kept"] == 1] if "kept" in singles.dtype.names else singles
    n = len(s)
    t = np.ascontiguousarray(s["t_ps"], np.uint64)
    u = np.ascontiguousarray(s["unit"], np.int32)
    p = np.ascontiguousarray(s["panel"], np.int32)
    h = np.ascontiguousarray(s["h"], np.uint64)
    a = np.zeros(max(n, 1), np.int32)
    b = np.zeros(max(n, 1), np.int32)
    np_ = lib().or_coincidences(n, _ptr(t), _ptr(u), _ptr(p), _ptr(h), int(round(window_ns * 1000.0)), _ptr(a),
                                _ptr(b))
    if np_ < 0:
        raise MemoryError
    return s, a[:np_].copy(), b[:np_].copy()


def philox(ctr, key):
    c = (C.c_uint32 * 4)(*[int(x) & 0xFFFFFFFF for x in ctr])
    k = (C.c_uint32 * 2)(*[int(x) & 0xFFFFFFFF for x in key])
    o = (C.c_uint32 * 4)()
    lib().or_philox4x32_10(c, k, o)
    return [int(x) for x in o]


def uniform(w):
    return float(lib().or_uniform(int(w) & 0xFFFFFFFF))


def sigma_kn(e_kev):
    return float(lib().or_sigma_kn(float(e_kev)))


def mu(material, e_kev, kind="total"):
    m = Material(material["mu_total_511_cm"], material["photo_frac_511"], material.get("electron_density_cm3", 0.0))
    f = dict(total=lib().or_mu_total, photo=lib().or_mu_photo, compton=lib().or_mu_compton)[kind]
    return float(f(C.byref(m), float(e_kev)))


def photo_count(material, e_kev, seed, h0, n):
    """Photoelectric decisions of n real collisions at energy e_kev (the
    transport's own branch function on its own draws)."""
    m = _materials([material])
    return int(lib().or_photo_count(m, float(e_kev), int(seed), int(h0), int(n)))


def kahn(seed, h0, n, e_kev):
    ct = np.zeros(n)
    eo = np.zeros(n)
    tr = np.zeros(n, np.int32)
    st = lib().or_kahn_batch(int(seed), int(h0), int(n), float(e_kev), _ptr(ct), _ptr(eo), _ptr(tr))
    if st != 0:
        raise RuntimeError(st)
    return ct, eo, tr


def flight(scanner, x, d):
    x = np.ascontiguousarray(x, np.float64).reshape(-1, 3)
    d = np.ascontiguousarray(d, np.float64).reshape(-1, 3)
    n = len(x)
    pn = np.zeros(n, np.int32)
    ti = np.zeros(n)
    sp = pack_scanner(scanner)
    lib().or_flight_batch(C.byref(sp.struct), n, _ptr(x), _ptr(d), _ptr(pn), _ptr(ti))
    return pn, ti


def locate(scanner, panel, wuv):
    wuv = np.ascontiguousarray(wuv, np.float64).reshape(-1, 3)
    n = len(wuv)
    out = np.zeros((n, 4), np.int32)
    sp = pack_scanner(scanner)
    lib().or_locate_batch(C.byref(sp.struct), int(panel), n, _ptr(wuv), _ptr(out))
    return out


def blur_normals(seed, h, unit):
    h = np.ascontiguousarray(h, np.uint64)
    unit = np.ascontiguousarray(unit, np.int32)
    out = np.zeros(len(h))
    lib().or_blur_normals(int(seed), len(h), _ptr(h), _ptr(unit), _ptr(out))
    return out


def rotate(d, cos_theta, u_phi):
    d = np.array(d, np.float64).reshape(-1, 3).copy()
    c = np.ascontiguousarray(cos_theta, np.float64)
    u = np.ascontiguousarray(u_phi, np.float64)
    lib().or_rotate_batch(len(d), _ptr(d), _ptr(c), _ptr(u))
    return d


def decays(source, n_decays, seed, h0, n, phantom=None):
    """Decay time (ps), annihilation point (mm) and photon-0 direction of histories [h0, h0+n)."""
    pp = pack_phantom(phantom)
    src = pack_source(source)
    t = np.zeros(n, np.uint64)
    pos = np.zeros((n, 3))
    d = np.zeros((n, 3))
    st = lib().or_decay_batch(C.byref(pp.struct) if pp else None, C.byref(src), int(n_decays), int(seed), int(h0),
                              int(n), _ptr(t), _ptr(pos), _ptr(d))
    if st != 0:
        raise RuntimeError(st)
    return t, pos, d


def sensitivity_map(scanners, positions, digitizer, windows, n_decays, seed, threads=1, activity_bq=None):
    """NEMA-style sensitivity S(r, E) (Sec. 2.4): for every scanner, source
    position r and energy window E = (lo, hi) keV, the coincidences counted by a
    full simulation with that window, divided by the decays.  Position p uses
    Philox key seed + p for every scanner (the same decays for each design).
    Written as the definition: one independent simulation per (scanner,
    position, window).  Returns (counts, S), both [scanner][position][window]."""
    ns, npos, nw = len(scanners), len(positions), len(windows)
    counts = np.zeros((ns, npos, nw), dtype=np.uint64)
    for i, sc in enumerate(scanners):
        for p, pos in enumerate(positions):
            src = dict(kind=0, pos=tuple(float(x) for x in pos), dir=(0.0, 0.0, 1.0),
                       activity_bq=float(activity_bq if activity_bq is not None else 1.7e4))
            for w, (lo, hi) in enumerate(windows):
                dg = dict(digitizer, e_lo=float(lo), e_hi=float(hi))
                r = simulate(sc, src, dg, n_decays, seed + p, threads=threads, tallies=False)
                _, a, _ = coincidences(r["singles"], dg["window_ns"])
                counts[i, p, w] = len(a)
    return counts, counts.astype(np.float64) / float(n_decays)


def delta_sym(s_a, s_b):
    """Symmetric percent difference of two sensitivities (Sec. 2.4):
    200 (S_a - S_b) / (S_a + S_b); NaN where both are zero."""
    a = np.asarray(s_a, dtype=np.float64)
    b = np.asarray(s_b, dtype=np.float64)
    tot = a + b
    out = np.full(np.broadcast(a, b).shape, np.nan)
    nz = tot != 0
    out[nz] = 200.0 * (a - b)[nz] / tot[nz]
    return out
