"""Batched form: many designs and sources in one persistent launch (and its
CUDA-graph replay) give, job by job, exactly the results of the plain call."""
import ctypes as C

import numpy as np
import pytest

import workloads as W
from tests import parity_util as PU

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    from paper_2603_07327_gb300 import build as B
    B.build()
    import paper_2603_07327_gb300 as G
    G.load()
    return G


def canon(r):
    s = r.singles()
    order = np.lexsort((s["unit"], s["h"]))
    a, b = r.coincidences()
    return ({k: v[order] for k, v in s.items()}, PU.coincidence_set(s["h"], s["unit"], a, b), r.tallies(),
            r.counts())


def assert_same(x, y):
    (s1, c1, t1, k1), (s2, c2, t2, k2) = x, y
    for key in s1:
        assert np.array_equal(s1[key], s2[key]), key
    assert c1 == c2
    assert np.array_equal(t1[0], t2[0]) and np.array_equal(t1[1], t2[1])
    assert k1["hits"] == k2["hits"] and k1["singles"] == k2["singles"] and k1["coincidences"] == k2["coincidences"]


@pytest.mark.parametrize("kernel", [1, 2, 3])
def test_batch_equals_alone(G, kernel):
    designs = W.config4(n_designs=6, scale=0.05)
    ph = W.hot_rod_phantom(scale=0.7)
    jobs = []
    for i, d in enumerate(designs):
        sc = G.Scanner(d["scanner"], ph if i == 2 else None)
        src = W.phantom_source() if i == 2 else d["source"]
        jobs.append(dict(scanner=sc, source=src, digitizer=d["digitizer"], n_decays=d["n_decays"], seed=d["seed"]))
    # a second job on the same scanner shares its geometry descriptor
    jobs.append(dict(jobs[0], seed=999, n_decays=33))
    alone = [canon(j["scanner"].simulate(j["source"], j["digitizer"], j["n_decays"], j["seed"], kernel=kernel))
             for j in jobs]
    one_shot = G.simulate_batch(jobs, kernel=kernel)
    for a, r in zip(alone, one_shot):
        assert_same(a, canon(r))
    b = G.Batch(jobs, kernel=kernel)
    first = [canon(b.result(i)) for i in range(len(jobs))]
    for a, f in zip(alone, first):
        assert_same(a, f)
    b.run()                              # graph replay: the same simulations again
    for a, i in zip(alone, range(len(jobs))):
        assert_same(a, canon(b.result(i)))
    tot = b.counts()
    assert tot["singles"] == sum(x[3]["singles"] for x in alone)
    assert tot["hits"] == sum(x[3]["hits"] for x in alone)
    b.close()


def test_batch_of_sweep_positions(G, oracle):
    """Two geometries x several positions in one launch, job-by-job parity
    against the oracle on sampled histories."""
    scs = {g: G.Scanner(W.config2_scanner(g)) for g in ("A", "B")}
    jobs = []
    for g in ("A", "B"):
        for i, z in enumerate((-30.0, -7.0, 0.0, 19.0)):
            jobs.append(dict(scanner=scs[g], source=W.point_source((0.0, 0.0, z)), digitizer=W.digitizer(),
                             n_decays=150_000, seed=2 + i + 1000 * (g == "B")))
    res = G.simulate_batch(jobs, kernel=2)
    for j, r in zip(jobs, res):
        s = r.singles()
        osim = oracle.simulate(j["scanner"].desc, j["source"], j["digitizer"], j["n_decays"], j["seed"], threads=8)
        sc_ = PU.compare_singles(s, osim["singles"], set(), 350.0, 650.0)
        # allow the rare FP32/FP64 history flip: singles of at most a few histories differ
        assert abs(sc_["n_gpu"] - sc_["n_orc"]) <= 4 and sc_["n_common"] >= sc_["n_orc"] - 4, sc_
        assert np.all(np.diff(s["t_ps"].astype(np.int64)) >= 0)


def test_history_shards_merge_to_the_whole_run(G):
    """Two history ranges of one run (as two ranks would run them) merge to the
    unsharded run: tallies add up, singles concatenate."""
    from paper_2603_07327_gb300 import shard
    sc = G.Scanner(W.config2_scanner("A"))
    src, dg, n = W.point_source((0.0, 0.0, -9.0)), W.digitizer(), 1_000_003
    full = sc.simulate(src, dg, n, 5, kernel=2)
    parts, tallies = [], []
    for rank in range(2):
        h0, h1 = shard.history_range(n, rank, 2)
        r = sc.simulate(src, dg, n, 5, kernel=2, h_begin=h0, h_end=h1)
        parts.append(r.singles())
        tallies.append(r.tallies())
        assert np.all((r.singles()["h"] >= h0) & (r.singles()["h"] < h1))
    c, e = shard.merge_tallies(tallies)
    fc, fe = full.tallies()
    assert np.array_equal(c, fc) and np.array_equal(e, fe)
    m = shard.merge_singles(parts)
    fs = full.singles()
    order = np.lexsort((fs["h"], fs["unit"], fs["t_ps"]))
    for f in shard.SINGLE_FIELDS:
        assert np.array_equal(m[f], fs[f][order]), f


def test_whole_launch_copy_equals_the_job_views(G):
    """gpet_result_copy_run: one copy per array for the whole batch equals the
    per-job views concatenated in job order; its coincidence indices count
    from the batch's first single (the job view's plus the job's offset)."""
    designs = W.config4(n_designs=4, scale=0.02)
    jobs = [dict(scanner=G.Scanner(d["scanner"]), source=d["source"], digitizer=d["digitizer"],
                 n_decays=d["n_decays"], seed=d["seed"]) for d in designs]
    res = G.simulate_batch(jobs)
    dtypes = {G.SINGLES_T_PS: np.uint64, G.SINGLES_UNIT: np.int32, G.SINGLES_E: np.float32,
              G.COINC_A: np.int32, G.COINC_B: np.int32, G.TALLY_COUNT: np.uint64, G.TALLY_EFX: np.uint64}
    s_off = np.cumsum([0] + [r.counts()["singles"] for r in res])
    for w, dt in dtypes.items():
        nb = res[0].run_nbytes(w)
        buf = np.zeros(nb // np.dtype(dt).itemsize + 1, dtype=dt)
        assert res[-1].copy_run_into(w, buf.ctypes.data, buf.nbytes) == nb
        whole = buf[:nb // np.dtype(dt).itemsize]
        parts = [r.array(w) for r in res]
        if w in (G.COINC_A, G.COINC_B):
            parts = [p + s_off[j] for j, p in enumerate(parts)]
        np.testing.assert_array_equal(whole, np.concatenate(parts).astype(dt))
    with pytest.raises(G.GpetError):
        res[0].copy_run_into(G.SINGLES_T_PS, buf.ctypes.data, 1)
    for r in res:
        r.free()
    for j in jobs:
        j["scanner"].close()


def test_async_whole_launch_copy_equals_the_blocking_one(G):
    """gpet_result_copy_run_async on a side stream delivers the same bytes as
    the blocking copy once the stream has passed it.  Into page-locked memory
    at a 16-byte boundary the copy is a kernel of SM stores; into pageable
    memory, or page-locked memory 4 bytes off the boundary, it is a copy-engine
    copy: every form gives the same bytes, and none writes past the array."""
    import torch
    designs = W.config4(n_designs=3, scale=0.02)
    jobs = [dict(scanner=G.Scanner(d["scanner"]), source=d["source"], digitizer=d["digitizer"],
                 n_decays=d["n_decays"], seed=d["seed"]) for d in designs]
    res = G.simulate_batch(jobs)
    st = torch.cuda.Stream()
    for w in (G.SINGLES_T_PS, G.SINGLES_UNIT, G.SINGLES_E, G.COINC_A, G.COINC_B, G.TALLY_COUNT, G.TALLY_EFX):
        nb = res[0].run_nbytes(w)
        ref = np.zeros(nb, dtype=np.uint8)
        res[2].copy_run_into(w, ref.ctypes.data, ref.nbytes)   # pageable: copy engine
        for off in (0, 4):
            pinned = torch.full((nb + 32,), 0xA5, dtype=torch.uint8, pin_memory=True)
            assert res[1].copy_run_into_async(w, pinned.data_ptr() + off, nb, st.cuda_stream) == nb
            st.synchronize()
            got = pinned.numpy()
            np.testing.assert_array_equal(got[off:off + nb], ref)
            assert (got[:off] == 0xA5).all() and (got[off + nb:] == 0xA5).all()
        blocking = torch.full((nb + 32,), 0xA5, dtype=torch.uint8, pin_memory=True)
        assert res[0].copy_run_into(w, blocking.data_ptr(), nb) == nb
        np.testing.assert_array_equal(blocking.numpy()[:nb], ref)
        assert (blocking.numpy()[nb:] == 0xA5).all()
    for r in res:
        r.free()
    for j in jobs:
        j["scanner"].close()


def test_batch_of_more_designs_than_staged_geometries(G):
    """24 distinct designs in one launch: the kernels stage at most 16 geometry
    descriptors in shared memory (fewer when the pool leaves no room) and read
    the rest through L1.  Every job must still equal its plain run."""
    designs = W.config4(n_designs=24, scale=0.01)
    jobs = [dict(scanner=G.Scanner(d["scanner"]), source=d["source"], digitizer=d["digitizer"],
                 n_decays=d["n_decays"], seed=d["seed"]) for d in designs]
    res = G.simulate_batch(jobs)
    for j, r in zip(jobs, res):
        p = j["scanner"].simulate(j["source"], j["digitizer"], j["n_decays"], j["seed"])
        assert np.array_equal(r.tallies()[0], p.tallies()[0])
        assert np.array_equal(r.tallies()[1], p.tallies()[1])
        assert r.counts()["coincidences"] == p.counts()["coincidences"]
        p.free()
        r.free()
    for j in jobs:
        j["scanner"].close()


def test_batch_job_count(G):
    """gpet_batch_jobs reports the batch's job count."""
    sc = G.Scanner(W.config2_scanner("A"))
    jobs = [dict(scanner=sc, source=W.point_source((0.0, 0.0, z)), digitizer=W.digitizer(), n_decays=200_000,
                 seed=9 + i) for i, z in enumerate((-5.0, 5.0))]
    b = G.Batch(jobs)
    try:
        n = C.c_int32()
        assert G.load().gpet_batch_jobs(b._h, C.byref(n)) == 0 and n.value == 2
    finally:
        b.close()
        sc.close()


def test_autotune_choice_gives_the_same_results(G):
    """gpet_autotune times the launch forms on a pilot and returns one of them;
    a run with the chosen form equals a run with the default one (every form
    gives the same results).  A seven-panel ring: a design class of its own,
    so the remembered choice touches no other test."""
    sc = G.Scanner(W.scanner(7, 50.0, [W.layer(8, 8, 1.6, 0.1, 10.0)]))
    try:
        opts, ms = sc.autotune(W.point_source(), W.digitizer(), pilot_decays=100_000)
        assert opts["kernel"] in (1, 2, 3) and ms > 0
        a = sc.simulate(W.point_source((1.0, 2.0, 0.0)), W.digitizer(), 200_000, 6, **opts)
        b = sc.simulate(W.point_source((1.0, 2.0, 0.0)), W.digitizer(), 200_000, 6, kernel=2)
        assert_same(canon(a), canon(b))
    finally:
        sc.close()


def test_time_key_fits_the_launch(G):
    """The sort key holds the job index in the fewest high bits that number a
    launch's jobs, the time stamp in the rest: a single run sorts on the whole
    64-bit time, while an acquisition that leaves no room for the job bits of
    a three-job batch is refused before any device work."""
    sc = G.Scanner(W.config1_scanner())
    try:
        n = 20_000
        # a span just below 2^62 ps: too long beside two job bits, fine alone
        src = W.point_source(activity_bq=n * 1e12 / float((1 << 62) - (1 << 31)))
        r = sc.simulate(src, W.digitizer(), n, 3)
        t = r.array(G.SINGLES_T_PS)
        assert len(t) > 100 and t.max() > 1 << 61 and np.all(np.diff(t) >= 0)
        r.free()
        jobs = [dict(scanner=sc, source=src if i == 1 else W.point_source(), digitizer=W.digitizer(),
                     n_decays=n, seed=i) for i in range(3)]
        with pytest.raises(G.GpetError) as e:
            G.simulate_batch(jobs)
        assert e.value.code == -1 and "job bits" in str(e.value)
    finally:
        sc.close()
