"""The allocation-free time sort (gpet_sort_times_noalloc) against the
library's regular time sort.

Some callers cannot call cudaMalloc (their device memory is owned by another
allocator, or an allocation's implicit synchronisation is not acceptable);
the entry point serves them with a fixed scratch array inside the library.
The first test sorts, through the C ABI and twice in a row, a shuffled copy
of the time stamps that gpet_simulate returned already sorted, and requires
the exact same order back (integer keys: bit-exact), a permutation consistent
with it, and stability for equal keys.  The second sorts synthetic key sets
against numpy's stable argsort: sizes 1, 4096 and the 2^20 maximum, full-range
keys (every radix pass runs), keys that leave an odd and an even number of
passes (the result ends in either buffer), many equal keys, and a call without
the permutation output; once the first call has set the device up, a call
changes the free device memory by nothing.  The file is collected last so that
a run stopping at the first failure has run every other test first.
"""
import ctypes as C

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    from paper_2603_07327_gb300 import build as B
    B.build()
    import paper_2603_07327_gb300 as G
    G.load()
    return G


def test_noalloc_sort_matches_regular_sort(G):
    torch = pytest.importorskip("torch")
    # the regular path: singles of one sweep position come back time-sorted
    res = G.simulate(W.config2_scanner("B"), W.point_source((0.0, 0.0, 4.0)), W.digitizer(), 2_000_000, 7)
    t_ref = res.array(G.SINGLES_T_PS)
    n = len(t_ref)
    assert 100_000 < n <= 1 << 20 and n % 4096 != 0
    assert np.all(np.diff(t_ref.astype(np.int64)) >= 0)
    t_in = t_ref[np.random.default_rng(3).permutation(n)]

    dev = torch.device("cuda", 0)
    d_in = torch.from_numpy(t_in.view(np.int64).copy()).to(dev)
    d_out = torch.empty(n, dtype=torch.int64, device=dev)
    d_perm = torch.empty(n, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream(dev).cuda_stream
    L = G.load()
    for call in range(2):                 # the scratch keeps the previous call's contents
        d_out.fill_(-1)
        d_perm.fill_(-1)
        code = L.gpet_sort_times_noalloc(C.c_void_p(d_in.data_ptr()), n, C.c_void_p(d_out.data_ptr()),
                                         C.c_void_p(d_perm.data_ptr()), C.c_void_p(stream))
        assert code == 0, L.gpet_last_error().decode()
        torch.cuda.synchronize(dev)
        out = d_out.cpu().numpy().view(np.uint64)
        perm = d_perm.cpu().numpy()
        assert np.array_equal(out, t_ref), call
        assert np.array_equal(t_in[perm], out), call
        same = np.diff(out.astype(np.int64)) == 0
        assert np.all(np.diff(perm)[same] > 0), call   # stable for equal keys

    # sizes beyond the scratch array are refused before any launch
    code = L.gpet_sort_times_noalloc(C.c_void_p(d_in.data_ptr()), (1 << 20) + 1, C.c_void_p(d_out.data_ptr()),
                                     None, C.c_void_p(stream))
    assert code == -1 and "maximum" in L.gpet_last_error().decode()


def _noalloc_sort(G, torch, keys, with_perm=True):
    """Sort host keys with gpet_sort_times_noalloc; returns (sorted keys, perm or None)."""
    dev = torch.device("cuda", 0)
    n = len(keys)
    d_in = torch.from_numpy(keys.view(np.int64).copy()).to(dev)
    d_out = torch.full((max(n, 1),), -1, dtype=torch.int64, device=dev)
    d_perm = torch.full((max(n, 1),), -1, dtype=torch.int32, device=dev) if with_perm else None
    stream = torch.cuda.current_stream(dev).cuda_stream
    L = G.load()
    code = L.gpet_sort_times_noalloc(C.c_void_p(d_in.data_ptr()), n, C.c_void_p(d_out.data_ptr()),
                                     C.c_void_p(d_perm.data_ptr()) if with_perm else None, C.c_void_p(stream))
    assert code == 0, L.gpet_last_error().decode()
    torch.cuda.synchronize(dev)
    out = d_out.cpu().numpy().view(np.uint64)[:n]
    perm = d_perm.cpu().numpy()[:n] if with_perm else None
    return out, perm


def test_noalloc_sort_key_sets(G):
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(11)
    full = lambda n: rng.integers(0, 2**63, n, dtype=np.uint64) * np.uint64(2) + rng.integers(0, 2, n, dtype=np.uint64)
    cases = {
        "one_key": np.array([0xDEADBEEF12345678], dtype=np.uint64),
        "full_range_4096": full(4096),                                         # 8 passes, ends in buffer 0
        "full_range_max": full(1 << 20),                                       # the largest accepted size
        "three_passes": rng.integers(0, 1 << 24, 50_000, dtype=np.uint64),    # odd: ends in buffer 1
        "two_passes": rng.integers(0, 1 << 16, 70_001, dtype=np.uint64),      # even: ends in buffer 0
        "seven_passes": rng.integers(0, 1 << 56, 123_457, dtype=np.uint64),   # odd, top byte constant
        "many_equal": (rng.integers(0, 50, 200_000, dtype=np.uint64) << np.uint64(40)) | np.uint64(7),
    }
    for name, keys in cases.items():
        out, perm = _noalloc_sort(G, torch, keys)
        ref = np.argsort(keys, kind="stable")
        assert np.array_equal(out, keys[ref]), name
        assert np.array_equal(perm, ref.astype(np.int32)), name      # stable: the unique stable order
    # without the permutation output
    keys = full(300_000)
    out, perm = _noalloc_sort(G, torch, keys, with_perm=False)
    assert perm is None and np.array_equal(out, np.sort(keys))
    # the device is set up by now: a further call takes no device memory
    dev = torch.device("cuda", 0)
    d_in = torch.from_numpy(keys.view(np.int64)).to(dev)
    d_out = torch.empty_like(d_in)
    d_perm = torch.empty(len(keys), dtype=torch.int32, device=dev)
    torch.cuda.synchronize(dev)
    free0 = torch.cuda.mem_get_info(dev)[0]
    L = G.load()
    code = L.gpet_sort_times_noalloc(C.c_void_p(d_in.data_ptr()), len(keys), C.c_void_p(d_out.data_ptr()),
                                     C.c_void_p(d_perm.data_ptr()), C.c_void_p(torch.cuda.current_stream(dev).cuda_stream))
    assert code == 0, L.gpet_last_error().decode()
    torch.cuda.synchronize(dev)
    assert torch.cuda.mem_get_info(dev)[0] == free0
    assert np.array_equal(d_out.cpu().numpy().view(np.uint64), np.sort(keys))
