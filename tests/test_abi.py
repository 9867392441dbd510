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
