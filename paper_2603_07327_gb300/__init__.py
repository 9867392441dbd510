"""Python binding of libgpet (include/gpet.h): argument marshalling only.

Every step of the simulation runs in the CUDA library; this module packs the
plain-dict descriptions of ``workloads`` into the C structs, calls the C ABI
and copies results into numpy arrays.  There is no CPU fallback: loading fails
loudly when the library is missing or cannot be loaded.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgpet.so")

GPET_OK = 0
ERRORS = {-1: "GPET_ERR_INVALID_ARG", -2: "GPET_ERR_GEOMETRY", -3: "GPET_ERR_OOM", -4: "GPET_ERR_CUDA",
          -5: "GPET_ERR_TIMEOUT", -6: "GPET_ERR_OVERFLOW", -7: "GPET_ERR_BUSY", -8: "GPET_ERR_TOO_SMALL"}

# result array ids (gpet.h)
SINGLES_T_PS, SINGLES_H, SINGLES_UNIT, SINGLES_PANEL, SINGLES_E, SINGLES_E_RAW = range(6)
COINC_A, COINC_B, TALLY_COUNT, TALLY_EFX = 6, 7, 8, 9
HITS_H, HITS_GSTEP, HITS_CRYSTAL, HITS_LAYER, HITS_WUV, HITS_E, HITS_T_PS = range(10, 17)
SINGLES_DOI = 17
_ARRAY_DTYPE = {SINGLES_T_PS: np.uint64, SINGLES_H: np.uint64, SINGLES_UNIT: np.int32, SINGLES_PANEL: np.int32,
                SINGLES_E: np.float32, SINGLES_E_RAW: np.float32, COINC_A: np.int32, COINC_B: np.int32,
                TALLY_COUNT: np.uint64, TALLY_EFX: np.uint64, HITS_H: np.uint64, HITS_GSTEP: np.int32,
                HITS_CRYSTAL: np.int32, HITS_LAYER: np.int32, HITS_WUV: np.float32, HITS_E: np.float32,
                HITS_T_PS: np.uint64, SINGLES_DOI: np.float32}

KERNEL_DEFAULT, KERNEL_LOOP, KERNEL_WAVE = 0, 1, 2


class GpetError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class Material(C.Structure):
    _fields_ = [("mu_total_511_cm", C.c_double), ("photo_frac_511", C.c_double),
                ("electron_density_cm3", C.c_double)]


class Layer(C.Structure):
    _fields_ = [("n_u", C.c_int32), ("n_v", C.c_int32), ("pitch_u", C.c_double), ("pitch_v", C.c_double),
                ("gap_u", C.c_double), ("gap_v", C.c_double), ("depth", C.c_double), ("gap_before", C.c_double),
                ("offset_u", C.c_double), ("offset_v", C.c_double), ("crystal_mat", C.c_int32),
                ("interval_mat", C.c_int32)]


class ScannerDesc(C.Structure):
    _fields_ = [("n_panels", C.c_int32), ("inner_radius_mm", C.c_double), ("first_angle_rad", C.c_double),
                ("modules_u", C.c_int32), ("modules_v", C.c_int32), ("module_size_u", C.c_double),
                ("module_size_v", C.c_double), ("module_gap_u", C.c_double), ("module_gap_v", C.c_double),
                ("n_layers", C.c_int32), ("layers", C.POINTER(Layer)), ("n_materials", C.c_int32),
                ("materials", C.POINTER(Material)), ("readout_level", C.c_int32),
                ("panel_poses", C.POINTER(C.c_double))]


class Source(C.Structure):
    _fields_ = [("kind", C.c_int32), ("pos_mm", C.c_double * 3), ("dir", C.c_double * 3),
                ("activity_bq", C.c_double)]


class Digitizer(C.Structure):
    _fields_ = [("fwhm_at_511", C.c_double), ("e_lo_kev", C.c_double), ("e_hi_kev", C.c_double),
                ("coinc_window_ns", C.c_double), ("e_cut_kev", C.c_double), ("doi_fwhm_mm", C.c_double)]


class Options(C.Structure):
    _fields_ = [("keep_hits", C.c_int32), ("block_size", C.c_int32), ("blocks_per_sm", C.c_int32),
                ("kernel", C.c_int32), ("compact_every", C.c_int32), ("pool_depth", C.c_int32),
                ("stream", C.c_void_p), ("h_begin", C.c_uint64), ("h_end", C.c_uint64)]


class Counts(C.Structure):
    _fields_ = [("n_decays", C.c_uint64), ("hits", C.c_uint64), ("singles", C.c_uint64),
                ("coincidences", C.c_uint64), ("n_crystals", C.c_int64), ("det_steps", C.c_uint64),
                ("flights", C.c_uint64), ("compton_trials", C.c_uint64), ("entered", C.c_uint64),
                ("phantom_steps", C.c_uint64), ("status", C.c_int32), ("transport_ms", C.c_float),
                ("digitizer_ms", C.c_float), ("h2d_bytes", C.c_uint64), ("wave_iterations", C.c_uint64),
                ("wave_lanes", C.c_uint64), ("screened_flights", C.c_uint64), ("singles_formed", C.c_uint64),
                ("latency_ms", C.c_double), ("phase_events", C.c_uint64 * 7)]


def _counts_dict(c):
    """gpet_counts as a dict (arrays as lists)."""
    out = {}
    for k, _ in Counts._fields_:
        v = getattr(c, k)
        out[k] = list(v) if isinstance(v, C.Array) else v
    return out


class ServerConfig(C.Structure):
    _fields_ = [("hbm_budget_bytes", C.c_size_t), ("workers", C.c_int32), ("max_jobs_per_launch", C.c_int32),
                ("launch", Options), ("max_launch_ms", C.c_double), ("piece_decays", C.c_uint64)]


class ServerStats(C.Structure):
    _fields_ = [(n, C.c_uint64) for n in ("submitted", "completed", "rejected", "launches", "max_jobs_per_launch",
                                          "pairs_completed", "bytes_in_use", "peak_bytes", "queued",
                                          "live_appends", "pieces")] + \
              [("transport_ms", C.c_double), ("digitizer_ms", C.c_double)]


# every entry point declared in include/gpet.h: name -> (restype, argtypes)
_P = C.c_void_p
SIGNATURES = {
    "gpet_create_scanner": (C.c_int, [C.POINTER(ScannerDesc), C.POINTER(_P)]),
    "gpet_destroy_scanner": (None, [_P]),
    "gpet_scanner_crystals": (C.c_int, [_P, C.POINTER(C.c_int64)]),
    "gpet_load_phantom": (C.c_int, [_P, C.c_int32, C.c_int32, C.c_int32, C.POINTER(C.c_double),
                                    C.POINTER(C.c_double), _P, _P, C.c_int32, C.POINTER(Material)]),
    "gpet_simulate": (C.c_int, [_P, C.POINTER(Source), C.POINTER(Digitizer), C.c_uint64, C.c_uint64,
                                C.POINTER(Options), C.POINTER(_P)]),
    "gpet_result_counts": (C.c_int, [_P, C.POINTER(Counts)]),
    "gpet_result_copy": (C.c_int, [_P, C.c_int32, _P, C.c_size_t]),
    "gpet_result_device_ptr": (_P, [_P, C.c_int32]),
    "gpet_result_copy_run": (C.c_int, [_P, C.c_int32, _P, C.c_size_t, C.POINTER(C.c_size_t)]),
    "gpet_result_copy_run_async": (C.c_int, [_P, C.c_int32, _P, C.c_size_t, C.POINTER(C.c_size_t), _P]),
    "gpet_result_free": (None, [_P]),
    "gpet_batch_create": (C.c_int, [C.c_int32, C.POINTER(_P), C.POINTER(Source), C.POINTER(Digitizer),
                                    C.POINTER(C.c_uint64), C.POINTER(C.c_uint64), C.POINTER(Options), C.POINTER(_P)]),
    "gpet_batch_run": (C.c_int, [_P]),
    "gpet_batch_jobs": (C.c_int, [_P, C.POINTER(C.c_int32)]),
    "gpet_batch_counts": (C.c_int, [_P, C.POINTER(Counts)]),
    "gpet_batch_result": (C.c_int, [_P, C.c_int32, C.POINTER(_P)]),
    "gpet_batch_destroy": (None, [_P]),
    "gpet_simulate_batch": (C.c_int, [C.c_int32, C.POINTER(_P), C.POINTER(Source), C.POINTER(Digitizer),
                                      C.POINTER(C.c_uint64), C.POINTER(C.c_uint64), C.POINTER(Options),
                                      C.POINTER(_P)]),
    "gpet_autotune": (C.c_int, [_P, C.POINTER(Source), C.POINTER(Digitizer), C.c_uint64, C.c_uint64,
                                C.POINTER(Options), C.POINTER(C.c_float)]),
    "gpet_server_create": (C.c_int, [C.POINTER(ServerConfig), C.POINTER(_P)]),
    "gpet_server_submit": (C.c_int, [_P, _P, C.POINTER(Source), C.POINTER(Digitizer), C.c_uint64, C.c_uint64,
                                     C.c_int32, C.POINTER(C.c_uint64)]),
    "gpet_server_poll": (C.c_int, [_P, C.c_uint64, C.POINTER(_P)]),
    "gpet_server_wait": (C.c_int, [_P, C.c_uint64, C.POINTER(_P)]),
    "gpet_server_stats_get": (C.c_int, [_P, C.POINTER(ServerStats)]),
    "gpet_server_destroy": (None, [_P]),
    "gpet_sort_times_noalloc": (C.c_int, [_P, C.c_uint64, _P, _P, _P]),
    "gpet_event_costs": (C.c_int, [_P, C.POINTER(Source), C.POINTER(Digitizer), C.c_uint64, C.c_uint64,
                                   C.POINTER(C.c_double), C.POINTER(C.c_uint64)]),
    "gpet_sensitivity_map": (C.c_int, [C.c_int32, C.POINTER(_P), C.c_int32, C.POINTER(C.c_double), C.c_double,
                                       C.POINTER(Digitizer), C.c_int32, C.POINTER(C.c_double), C.c_uint64,
                                       C.c_uint64, C.POINTER(Options), _P, _P, C.POINTER(Counts)]),
    "gpet_delta_sym": (C.c_int, [C.c_int64, _P, _P, _P]),
    "gpet_last_error": (C.c_char_p, []),
    "gpet_version": (C.c_char_p, []),
}

_lib = None


def load(path: str = LIB_PATH):
    """Load libgpet.so (raises if it is missing: there is no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"libgpet.so not built ({path}); run __graft_entry__.build()")
    L = C.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def _check(code):
    if code != GPET_OK:
        raise GpetError(code, load().gpet_last_error().decode())


def _materials(mats):
    arr = (Material * len(mats))()
    for i, m in enumerate(mats):
        arr[i] = Material(m["mu_total_511_cm"], m["photo_frac_511"], m.get("electron_density_cm3", 0.0))
    return arr


def scanner_desc(sc):
    """gpet_scanner_desc from a workloads scanner dict (keeps buffers alive on the struct)."""
    layers = (Layer * len(sc["layers"]))()
    for i, l in enumerate(sc["layers"]):
        layers[i] = Layer(l["n_u"], l["n_v"], l["pitch_u"], l["pitch_v"], l["gap_u"], l["gap_v"], l["depth"],
                          l["gap_before"], l["offset_u"], l["offset_v"], l["crystal_mat"], l["interval_mat"])
    mats = _materials(sc["materials"])
    poses = sc.get("panel_poses")
    pp = None
    if poses is not None:
        poses = np.ascontiguousarray(poses, dtype=np.float64).reshape(sc["n_panels"], 12)
        pp = poses.ctypes.data_as(C.POINTER(C.c_double))
    d = ScannerDesc(sc["n_panels"], sc["inner_radius"], sc["first_angle"], sc["modules_u"], sc["modules_v"],
                    sc["module_size_u"], sc["module_size_v"], sc["module_gap_u"], sc["module_gap_v"],
                    len(sc["layers"]), layers, len(sc["materials"]), mats, sc["readout_level"], pp)
    d._keep = (layers, mats, poses)
    return d


def source_struct(src):
    return Source(src["kind"], (C.c_double * 3)(*src["pos"]), (C.c_double * 3)(*src.get("dir", (0, 0, 1))),
                  src["activity_bq"])


def digitizer_struct(dg):
    return Digitizer(dg["fwhm_at_511"], dg["e_lo"], dg["e_hi"], dg["window_ns"], dg["e_cut"],
                     dg.get("doi_fwhm_mm", 0.0))


def options_struct(keep_hits=False, block_size=0, blocks_per_sm=0, kernel=0, compact_every=0, pool_depth=0,
                   stream=None, h_begin=0, h_end=0):
    return Options(int(bool(keep_hits)), int(block_size), int(blocks_per_sm), int(kernel), int(compact_every),
                   int(pool_depth), C.c_void_p(stream) if stream else None, int(h_begin), int(h_end))


class Scanner:
    """A gpet_scanner handle (owned)."""

    def __init__(self, sc: dict, phantom: dict | None = None):
        L = load()
        self._h = C.c_void_p()
        self.desc = sc
        _check(L.gpet_create_scanner(C.byref(scanner_desc(sc)), C.byref(self._h)))
        if phantom is not None:
            self.load_phantom(phantom)

    def load_phantom(self, ph):
        L = load()
        mat = np.ascontiguousarray(ph["material"], np.uint8).reshape(-1)
        act = ph.get("activity")
        act = None if act is None else np.ascontiguousarray(act, np.float32).reshape(-1)
        mats = _materials(ph["materials"])
        _check(L.gpet_load_phantom(self._h, ph["nx"], ph["ny"], ph["nz"], (C.c_double * 3)(*ph["voxel"]),
                                   (C.c_double * 3)(*ph["origin"]), mat.ctypes.data_as(C.c_void_p),
                                   act.ctypes.data_as(C.c_void_p) if act is not None else None,
                                   len(ph["materials"]), mats))

    @property
    def n_crystals(self):
        n = C.c_int64()
        _check(load().gpet_scanner_crystals(self._h, C.byref(n)))
        return int(n.value)

    def simulate(self, source, digitizer, n_decays, seed, **opts):
        L = load()
        out = C.c_void_p()
        o = options_struct(**opts)
        _check(L.gpet_simulate(self._h, C.byref(source_struct(source)), C.byref(digitizer_struct(digitizer)),
                               int(n_decays), int(seed), C.byref(o), C.byref(out)))
        return Result(out)

    def autotune(self, source, digitizer, pilot_decays=2_000_000, seed=1):
        """Time the launch forms on a pilot run; returns (options dict, transport ms)."""
        o = Options()
        ms = C.c_float()
        _check(load().gpet_autotune(self._h, C.byref(source_struct(source)), C.byref(digitizer_struct(digitizer)),
                                    int(pilot_decays), int(seed), C.byref(o), C.byref(ms)))
        return dict(kernel=o.kernel, blocks_per_sm=o.blocks_per_sm, compact_every=o.compact_every,
                    pool_depth=o.pool_depth, block_size=o.block_size), ms.value

    def event_costs(self, source, digitizer, n_sample=1_000_000, seed=1):
        """GPU ns per event of each history phase when that event runs alone at
        full width (gpet_event_costs); returns (ns list of 7, states list of 7)."""
        ns = (C.c_double * 7)()
        states = (C.c_uint64 * 7)()
        _check(load().gpet_event_costs(self._h, C.byref(source_struct(source)),
                                       C.byref(digitizer_struct(digitizer)), int(n_sample), int(seed), ns, states))
        return list(ns), list(states)

    def close(self):
        if self._h:
            load().gpet_destroy_scanner(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Result:
    """A gpet_result handle (owned)."""

    def __init__(self, handle):
        self._h = handle

    def counts(self) -> dict:
        c = Counts()
        _check(load().gpet_result_counts(self._h, C.byref(c)))
        return _counts_dict(c)

    def array(self, which: int, n: int | None = None) -> np.ndarray:
        """Copy one result array to host; n = element count (derived from counts when None)."""
        dt = np.dtype(_ARRAY_DTYPE[which])
        if n is None:
            c = self.counts()
            if which <= SINGLES_E_RAW or which == SINGLES_DOI:
                n = c["singles"]
            elif which in (COINC_A, COINC_B):
                n = c["coincidences"]
            elif which in (TALLY_COUNT, TALLY_EFX):
                n = c["n_crystals"]
            else:
                n = c["hits"]
        width = 3 if which == HITS_WUV else 1
        buf = np.zeros(n * width, dt)
        _check(load().gpet_result_copy(self._h, which, buf.ctypes.data_as(C.c_void_p), buf.nbytes))
        return buf.reshape(-1, 3) if width == 3 else buf

    def nbytes(self, which: int) -> int:
        """Bytes of one result array (for sizing caller-owned buffers)."""
        c = self.counts()
        if which <= SINGLES_E_RAW or which == SINGLES_DOI:
            n = c["singles"]
        elif which in (COINC_A, COINC_B):
            n = c["coincidences"]
        elif which in (TALLY_COUNT, TALLY_EFX):
            n = c["n_crystals"]
        else:
            n = c["hits"]
        return n * np.dtype(_ARRAY_DTYPE[which]).itemsize * (3 if which == HITS_WUV else 1)

    def copy_into(self, which: int, ptr: int, cap_bytes: int) -> int:
        """gpet_result_copy into caller-owned host memory at address ptr (e.g.
        a pinned buffer); returns the bytes written."""
        nb = self.nbytes(which)
        _check(load().gpet_result_copy(self._h, which, C.c_void_p(ptr), int(cap_bytes)))
        return nb

    def run_nbytes(self, which: int) -> int:
        """Bytes of one array of the whole launch this result belongs to."""
        nb = C.c_size_t()
        _check(load().gpet_result_copy_run(self._h, which, None, 0, C.byref(nb)))
        return nb.value

    def copy_run_into(self, which: int, ptr: int, cap_bytes: int) -> int:
        """gpet_result_copy_run into caller-owned host memory at ptr; returns the bytes written."""
        nb = C.c_size_t()
        _check(load().gpet_result_copy_run(self._h, which, C.c_void_p(ptr), int(cap_bytes), C.byref(nb)))
        return nb.value

    def copy_run_into_async(self, which: int, ptr: int, cap_bytes: int, stream: int) -> int:
        """gpet_result_copy_run_async on the CUDA stream handle `stream`; returns the bytes enqueued."""
        nb = C.c_size_t()
        _check(load().gpet_result_copy_run_async(self._h, which, C.c_void_p(ptr), int(cap_bytes), C.byref(nb),
                                                 C.c_void_p(stream)))
        return nb.value

    def device_ptr(self, which: int) -> int:
        return load().gpet_result_device_ptr(self._h, which) or 0

    def singles(self) -> dict:
        return dict(t_ps=self.array(SINGLES_T_PS), h=self.array(SINGLES_H), unit=self.array(SINGLES_UNIT),
                    panel=self.array(SINGLES_PANEL), e=self.array(SINGLES_E), e_raw=self.array(SINGLES_E_RAW),
                    doi=self.array(SINGLES_DOI))

    def coincidences(self):
        return self.array(COINC_A), self.array(COINC_B)

    def tallies(self):
        return self.array(TALLY_COUNT), self.array(TALLY_EFX)

    def hits(self, n=None) -> dict:
        return dict(h=self.array(HITS_H, n), gstep=self.array(HITS_GSTEP, n), crystal=self.array(HITS_CRYSTAL, n),
                    layer=self.array(HITS_LAYER, n), wuv=self.array(HITS_WUV, n), e=self.array(HITS_E, n),
                    t_ps=self.array(HITS_T_PS, n))

    def free(self):
        if self._h:
            load().gpet_result_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def simulate(scanner: dict, source: dict, digitizer: dict, n_decays: int, seed: int, phantom: dict | None = None,
             **opts) -> Result:
    """One plain simulation through the C ABI (creates and releases the scanner)."""
    sc = Scanner(scanner, phantom)
    try:
        return sc.simulate(source, digitizer, n_decays, seed, **opts)
    finally:
        sc.close()


def _job_arrays(jobs):
    n = len(jobs)
    scs = (C.c_void_p * n)(*[j["scanner"]._h.value for j in jobs])
    srcs = (Source * n)(*[source_struct(j["source"]) for j in jobs])
    dgs = (Digitizer * n)(*[digitizer_struct(j["digitizer"]) for j in jobs])
    nd = (C.c_uint64 * n)(*[int(j["n_decays"]) for j in jobs])
    sd = (C.c_uint64 * n)(*[int(j["seed"]) for j in jobs])
    return n, scs, srcs, dgs, nd, sd


class Batch:
    """gpet_batch handle: jobs = list of dicts with keys scanner (a Scanner),
    source, digitizer, n_decays, seed.  Created once (first run + graph
    capture), replayed with run()."""

    def __init__(self, jobs, **opts):
        L = load()
        self._jobs = jobs                      # keeps the Scanner handles alive
        n, scs, srcs, dgs, nd, sd = _job_arrays(jobs)
        self._h = C.c_void_p()
        o = options_struct(**opts)
        _check(L.gpet_batch_create(n, scs, srcs, dgs, nd, sd, C.byref(o), C.byref(self._h)))
        self.n = n

    def run(self):
        _check(load().gpet_batch_run(self._h))

    def counts(self) -> dict:
        c = Counts()
        _check(load().gpet_batch_counts(self._h, C.byref(c)))
        return _counts_dict(c)

    def result(self, job: int) -> Result:
        out = C.c_void_p()
        _check(load().gpet_batch_result(self._h, int(job), C.byref(out)))
        return Result(out)

    def close(self):
        if self._h:
            load().gpet_batch_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def simulate_batch(jobs, **opts):
    """One-shot batch (no graph): returns one Result per job."""
    L = load()
    n, scs, srcs, dgs, nd, sd = _job_arrays(jobs)
    outs = (C.c_void_p * n)()
    o = options_struct(**opts)
    _check(L.gpet_simulate_batch(n, scs, srcs, dgs, nd, sd, C.byref(o), outs))
    return [Result(C.c_void_p(outs[i])) for i in range(n)]


def sensitivity_map(scanners, positions, digitizer: dict, windows, n_decays: int, seed: int,
                    activity_bq: float = 1.7e4, **opts):
    """gpet_sensitivity_map: `scanners` are Scanner handles, `positions` an
    (n, 3) array in mm, `windows` (lo, hi) keV pairs.  Returns (counts, S,
    totals): counts and S of shape [scanner][position][window], totals the
    launch-wide gpet_counts as a dict."""
    L = load()
    pos = np.ascontiguousarray(positions, dtype=np.float64).reshape(-1, 3)
    win = np.ascontiguousarray(windows, dtype=np.float64).reshape(-1, 2)
    ns, npos, nw = len(scanners), len(pos), len(win)
    scs = (C.c_void_p * ns)(*[sc._h.value for sc in scanners])
    counts = np.zeros((ns, npos, nw), dtype=np.uint64)
    sens = np.zeros((ns, npos, nw), dtype=np.float64)
    tot = Counts()
    o = options_struct(**opts)
    _check(L.gpet_sensitivity_map(ns, scs, npos, pos.ctypes.data_as(C.POINTER(C.c_double)), float(activity_bq),
                                  C.byref(digitizer_struct(digitizer)), nw,
                                  win.ctypes.data_as(C.POINTER(C.c_double)), int(n_decays), int(seed), C.byref(o),
                                  counts.ctypes.data, sens.ctypes.data, C.byref(tot)))
    return counts, sens, _counts_dict(tot)


def delta_sym(s_a, s_b):
    """gpet_delta_sym over two arrays of the same shape."""
    a = np.ascontiguousarray(s_a, dtype=np.float64)
    b = np.ascontiguousarray(s_b, dtype=np.float64)
    if a.shape != b.shape:
        raise ValueError("delta_sym needs arrays of one shape")
    out = np.empty_like(a)
    _check(load().gpet_delta_sym(a.size, a.ctypes.data, b.ctypes.data, out.ctypes.data))
    return out


class Server:
    """gpet_server handle: continuous batching of simulation requests."""

    def __init__(self, hbm_budget_bytes=150 * 10**9, workers=1, max_jobs_per_launch=256, max_launch_ms=0.0,
                 piece_decays=0, **launch_opts):
        L = load()
        cfg = ServerConfig(int(hbm_budget_bytes), int(workers), int(max_jobs_per_launch),
                           options_struct(**launch_opts), float(max_launch_ms), int(piece_decays))
        self._h = C.c_void_p()
        _check(L.gpet_server_create(C.byref(cfg), C.byref(self._h)))
        self._keep = {}

    def submit(self, scanner: Scanner, source, digitizer, n_decays, seed, block=True) -> int:
        rid = C.c_uint64()
        _check(load().gpet_server_submit(self._h, scanner._h, C.byref(source_struct(source)),
                                         C.byref(digitizer_struct(digitizer)), int(n_decays), int(seed),
                                         1 if block else 0, C.byref(rid)))
        self._keep[rid.value] = scanner       # the scanner must outlive the request
        return rid.value

    def poll(self, rid):
        out = C.c_void_p()
        _check(load().gpet_server_poll(self._h, int(rid), C.byref(out)))
        if not out.value:
            return None
        self._keep.pop(rid, None)
        return Result(out)

    def wait(self, rid):
        out = C.c_void_p()
        _check(load().gpet_server_wait(self._h, int(rid), C.byref(out)))
        self._keep.pop(rid, None)
        return Result(out)

    def stats(self) -> dict:
        st = ServerStats()
        _check(load().gpet_server_stats_get(self._h, C.byref(st)))
        return {k: getattr(st, k) for k, _ in ServerStats._fields_}

    def close(self):
        if self._h:
            load().gpet_server_destroy(self._h)
            self._h = C.c_void_p()
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
