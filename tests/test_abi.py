"""The C-ABI library loads and exports every entry point of include/gpet.h;
host-side validation of scanner descriptions (no GPU needed)."""
import ctypes as C
import os
import re

import numpy as np
import pytest

import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def G():
    from paper_2603_07327_gb300 import build as B
    B.build()
    import paper_2603_07327_gb300 as G
    G.load()
    return G


def declared_symbols():
    txt = open(os.path.join(ROOT, "include", "gpet.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(gpet_\w+)\s*\(", txt)))


def test_library_exports_every_declared_symbol(G):
    names = declared_symbols()
    assert "gpet_simulate" in names and "gpet_create_scanner" in names and len(names) >= 10
    lib = C.CDLL(G.LIB_PATH)
    for n in names:
        assert hasattr(lib, n), n
    # the binding declares exactly the header's entry points
    assert set(G.SIGNATURES) == set(names)
    assert G.load().gpet_version().decode().startswith("gpet-gb300")


def _create(G, sc):
    h = C.c_void_p()
    code = G.load().gpet_create_scanner(C.byref(G.scanner_desc(sc)), C.byref(h))
    if code == 0:
        G.load().gpet_destroy_scanner(h)
    return code


def test_scanner_validation(G, oracle):
    assert _create(G, W.config1_scanner()) == 0
    assert _create(G, W.config2_scanner("A")) == 0
    assert _create(G, W.config3_scanner()) == 0
    for k in ("1CL", "split", "2CL"):
        assert _create(G, W.h2rspet(k)) == 0
    # the literal config-2 reading (4 x 4 modules of 20 mm at 55 mm) overlaps
    lit = W.config2_scanner("A")
    lit["modules_u"] = 4
    assert _create(G, lit) == -2
    bad = W.config1_scanner()
    bad["layers"][0]["gap_u"] = 2.0         # gap >= pitch
    assert _create(G, bad) == -2
    bad = W.config1_scanner()
    bad["layers"][0]["n_u"] = 9             # grid leaves the module
    assert _create(G, bad) == -2
    bad = W.config1_scanner()
    bad["layers"][0]["crystal_mat"] = 5     # material index out of range
    assert _create(G, bad) == -1
    bad = W.config1_scanner()
    bad["readout_level"] = 2
    assert _create(G, bad) == -1
    assert "readout_level" in G.load().gpet_last_error().decode()


def test_posed_scanner_validation(G):
    """Non-repetition mode: valid poses are accepted; overlapping panels,
    non-unit, non-orthogonal or left-handed axes are GPET_ERR_GEOMETRY; a
    ring written as poses is rejected by the 3-D box test exactly where the
    ring's own transaxial test rejects it."""
    import numpy as np
    assert _create(G, W.box_scanner()) == 0
    assert _create(G, W.four_layer_scanner()) == 0
    ring = W.config2_scanner("B")
    assert _create(G, W.with_poses(ring, W.ring_poses(ring))) == 0
    box = W.box_scanner()
    P = np.array(box["panel_poses"])
    moved = P.copy()
    moved[0, 9:12] = [5.0, 45.0, 0.0]         # head 0 pushed into head 2
    assert _create(G, W.with_poses(box, moved)) == -2
    assert "overlap" in G.load().gpet_last_error().decode()
    scaled = P.copy()
    scaled[1, 0:3] *= 1.01                    # w axis not a unit vector
    assert _create(G, W.with_poses(box, scaled)) == -2
    left = P.copy()
    left[2, 3:6] *= -1.0                      # u flipped: v != w x u
    assert _create(G, W.with_poses(box, left)) == -2
    skew = P.copy()
    skew[3, 6:9] = skew[3, 3:6]               # v equal to u
    assert _create(G, W.with_poses(box, skew)) == -2
    nan = P.copy()
    nan[0, 10] = float("nan")
    assert _create(G, W.with_poses(box, nan)) == -1
    # rings too tight for the panel width: both tests reject, looser ones accept
    for R, want in ((18.0, -2), (19.0, -2), (40.0, 0), (55.0, 0)):
        r = W.config2_scanner("A")
        r["inner_radius"] = R
        assert _create(G, r) == want, R
        assert _create(G, W.with_poses(r, W.ring_poses(r))) == want, R


def test_phantom_must_clear_posed_panels(G):
    """A phantom grid that reaches into a posed panel is GPET_ERR_GEOMETRY
    (checked before any device work, so this runs without a GPU)."""
    import ctypes as C
    import numpy as np
    L = G.load()
    h = C.c_void_p()
    assert L.gpet_create_scanner(C.byref(G.scanner_desc(W.box_scanner())), C.byref(h)) == 0
    try:
        mats = G._materials([W.WATER])
        ids = np.zeros(8, dtype=np.uint8)
        vox = (C.c_double * 3)(30.0, 30.0, 30.0)
        org = (C.c_double * 3)(-10.0, -10.0, -10.0)   # reaches x = 50: the +x head starts at 45
        code = L.gpet_load_phantom(h, 2, 2, 2, vox, org, ids.ctypes.data_as(C.POINTER(C.c_uint8)), None, 1, mats)
        assert code == -2
        assert "posed panel 0" in L.gpet_last_error().decode()
    finally:
        L.gpet_destroy_scanner(h)


def test_phantom_validation(G):
    """gpet_load_phantom's argument checks, all before any device work: an
    empty grid, a material count outside [1, 8], a non-positive voxel, a voxel
    naming a missing material, a negative or non-finite activity
    (GPET_ERR_INVALID_ARG), and a grid reaching past the ring's inner radius
    (GPET_ERR_GEOMETRY)."""
    import ctypes as C
    import numpy as np
    L = G.load()
    h = C.c_void_p()
    assert L.gpet_create_scanner(C.byref(G.scanner_desc(W.config1_scanner())), C.byref(h)) == 0
    u8 = C.POINTER(C.c_uint8)
    f32 = C.POINTER(C.c_float)
    try:
        mats = G._materials([W.AIR, W.WATER])
        ids = np.ones(27, dtype=np.uint8)
        act = np.ones(27, dtype=np.float32)
        vox = (C.c_double * 3)(1.0, 1.0, 1.0)
        org = (C.c_double * 3)(-1.5, -1.5, -1.5)

        def load(nx=3, voxel=vox, origin=org, i=ids, a=act, nm=2):
            return L.gpet_load_phantom(h, nx, 3, 3, voxel, origin, i.ctypes.data_as(u8),
                                       None if a is None else a.ctypes.data_as(f32), nm, mats)
        assert load(nx=0) == -1
        assert load(nm=0) == -1 and load(nm=9) == -1
        assert load(voxel=(C.c_double * 3)(1.0, 0.0, 1.0)) == -1
        bad = ids.copy()
        bad[13] = 2
        assert load(i=bad) == -1 and "voxel 13" in L.gpet_last_error().decode()
        for v in (-1.0, float("nan"), float("inf")):
            a = act.copy()
            a[5] = v
            assert load(a=a) == -1
        assert load(origin=(C.c_double * 3)(38.0, 0.0, 0.0)) == -2   # reaches x = 41: C1 ring radius 40 mm
    finally:
        L.gpet_destroy_scanner(h)


def test_crystal_count_matches_oracle(G, oracle):
    for sc in (W.config1_scanner(), W.config2_scanner("B"), W.config3_scanner(), W.h2rspet("2CL")):
        h = C.c_void_p()
        assert G.load().gpet_create_scanner(C.byref(G.scanner_desc(sc)), C.byref(h)) == 0
        n = C.c_int64()
        assert G.load().gpet_scanner_crystals(h, C.byref(n)) == 0
        G.load().gpet_destroy_scanner(h)
        assert n.value == oracle.n_crystals(sc)


def test_null_arguments_are_errors(G):
    L = G.load()
    assert L.gpet_create_scanner(None, None) == -1
    assert L.gpet_result_counts(None, None) == -1
    assert L.gpet_simulate(None, None, None, 1, 1, None, None) == -1
    L.gpet_result_free(None)
    L.gpet_destroy_scanner(None)


def test_server_config_validation(G):
    L = G.load()
    h = C.c_void_p()
    cfg = G.ServerConfig(0, 2, 16, G.options_struct())
    assert L.gpet_server_create(C.byref(cfg), C.byref(h)) == -1
    cfg = G.ServerConfig(10**9, 99, 16, G.options_struct())
    assert L.gpet_server_create(C.byref(cfg), C.byref(h)) == -1
    cfg = G.ServerConfig(10**9, 2, 5000, G.options_struct())
    assert L.gpet_server_create(C.byref(cfg), C.byref(h)) == -1
    assert L.gpet_server_poll(None, 1, None) == -1
    L.gpet_server_destroy(None)


def test_noalloc_sort_refuses_oversize_before_any_launch(G):
    """The allocation-free time sort checks its size limit on the host."""
    L = G.load()
    assert L.gpet_sort_times_noalloc(None, (1 << 20) + 1, None, None, None) == -1
    assert "maximum" in L.gpet_last_error().decode()
    assert L.gpet_sort_times_noalloc(None, 0, None, None, None) == 0


def test_delta_sym_host_call_matches_the_oracle(G, oracle):
    """gpet_delta_sym is host arithmetic of the library: it agrees with the
    oracle's own Delta_sym, NaN where both sensitivities are zero."""
    import numpy as np
    rng = np.random.default_rng(3)
    a = rng.uniform(0, 0.2, 50)
    b = rng.uniform(0, 0.2, 50)
    a[:3] = [0.0, 0.0, 0.1]
    b[:3] = [0.0, 0.1, 0.0]
    got = G.delta_sym(a, b)
    want = oracle.delta_sym(a, b)
    assert np.isnan(got[0]) and np.isnan(want[0])
    np.testing.assert_allclose(got[1:], want[1:], rtol=1e-15, atol=0)


def test_sensitivity_map_refuses_bad_arguments_before_any_launch(G):
    """Windows out of order, too many windows or jobs, and NaN positions are
    GPET_ERR_INVALID_ARG (checked on the host, so this runs without a GPU)."""
    import numpy as np
    sc = G.Scanner(W.config1_scanner())
    dg = W.digitizer()
    try:
        for pos, win in (([(0, 0, 0)], [(500.0, 400.0)]),
                         ([(0, 0, 0)], [(-1.0, 400.0)]),
                         ([(0, 0, 0)], [(100.0, 700.0)] * 17),
                         ([(0, 0, float("nan"))], [(100.0, 700.0)]),
                         ([(0, 0, 0)] * 4096, [(100.0, 700.0)])):
            with pytest.raises(G.GpetError) as e:
                G.sensitivity_map([sc], np.array(pos, dtype=float), dg, win, 100, 1)
            assert e.value.code == -1, str(e.value)
    finally:
        sc.close()


def test_whole_launch_copy_refuses_null_arguments(G):
    """gpet_result_copy_run(_async) with a NULL result, or a NULL destination
    with a non-zero capacity, is GPET_ERR_INVALID_ARG (no device work)."""
    import ctypes as C
    L = G.load()
    nb = C.c_size_t()
    assert L.gpet_result_copy_run(None, G.SINGLES_T_PS, None, 0, C.byref(nb)) == -1
    assert L.gpet_result_copy_run_async(None, G.SINGLES_T_PS, None, 0, C.byref(nb), None) == -1
    assert L.gpet_result_copy(None, G.SINGLES_T_PS, None, 0) == -1


def test_empty_and_out_of_range_sizes_are_refused_on_the_host(G):
    """Degenerate and maximum sizes: zero decays, a shard outside the run, more
    than 64 panels, 8 layers or 8 materials, and an acquisition past 2^62 ps
    (53 days) are GPET_ERR_INVALID_ARG before any device work; the largest
    accepted descriptor sizes (64 panels, 8 layers, 8 materials) are accepted."""
    import ctypes as C
    L = G.load()
    sc = G.Scanner(W.config1_scanner())
    try:
        for n, opts in ((0, {}), (100, dict(h_begin=50, h_end=200)), (100, dict(h_begin=60, h_end=60))):
            with pytest.raises(G.GpetError) as e:
                sc.simulate(W.point_source(), W.digitizer(), n, 1, **opts)
            assert e.value.code == -1
        with pytest.raises(G.GpetError) as e:   # 1e9 decays at 1 Bq: 1e21 ps, far past 2^62 ps
            sc.simulate(W.point_source(activity_bq=1.0), W.digitizer(), 10**9, 1)
        assert e.value.code == -1
    finally:
        sc.close()
    big = W.scanner(64, 400.0, [W.layer(4, 4, 1.0, 0.1, 1.0, gap_before=0.05 if l else 0.0) for l in range(8)],
                    materials=[W.AIR] + [W.LYSO] * 7)
    assert _create(G, big) == 0
    for key, val in (("n_panels", 65),):
        bad = dict(big, **{key: val})
        assert _create(G, bad) == -1
    nine = dict(big, layers=big["layers"] + [W.layer(4, 4, 1.0, 0.1, 1.0, gap_before=0.05)])
    assert _create(G, nine) == -1
    mats = dict(big, materials=big["materials"] + [W.LYSO])
    assert _create(G, mats) == -1


def test_no_cpu_fallback_without_a_gpu(G):
    """On a machine without a usable GPU the compute calls fail with
    GPET_ERR_CUDA and a message naming the CUDA error; nothing falls back to a
    CPU path.  (Skipped where a GPU is present.)"""
    try:
        import torch
        if torch.cuda.is_available():
            pytest.skip("a GPU is present")
    except ImportError:
        pass
    sc = G.Scanner(W.config1_scanner())
    try:
        with pytest.raises(G.GpetError) as e:
            sc.simulate(W.point_source(), W.digitizer(), 1000, 1)
        assert e.value.code == -4 and "cuda" in str(e.value).lower()
        with pytest.raises(G.GpetError) as e:
            G.simulate_batch([dict(scanner=sc, source=W.point_source(), digitizer=W.digitizer(), n_decays=1000,
                                   seed=1)])
        assert e.value.code == -4
    finally:
        sc.close()
