"""The allocation-free time sort (gpet_sort_times_noalloc) against the
library's regular time sort.

Some callers cannot call cudaMalloc (their device memory is owned by another
allocator, or an allocation's implicit synchronisation is not acceptable);
the entry point serves them with a fixed scratch array inside the library.
This test sorts, through the C ABI and twice in a row, a shuffled copy of the
time stamps that gpet_simulate returned already sorted, and requires the
exact same order back (integer keys: bit-exact), a permutation consistent
with it, and stability for equal keys.  It is collected last so that a run
stopping at the first failure has run every other test first.
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
