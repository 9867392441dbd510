"""Serving loop: requests submitted while others run are batched together;
every result equals the same request run alone, and sampled requests (point
and phantom sources) run alone match the FP64 oracle history by history;
admission by HBM footprint.  The server runs the default launch form, the one
the benchmark times."""
import threading
import time

import pytest

import workloads as W
from tests.test_gpu_batch import assert_same, canon
from tests.test_gpu_parity import check_parity

# a serving-loop test that waits on a request which never completes ends here
pytestmark = [pytest.mark.gpu, pytest.mark.timeout(240)]


@pytest.fixture(scope="module")
def G():
    from paper_2603_07327_gb300 import build as B
    B.build()
    import paper_2603_07327_gb300 as G
    G.load()
    return G


def _request_scanner(G, r, base):
    """The request's scanner, with the hot-rod phantom scaled as the request asks."""
    ph = None
    if r["phantom"] is not None:
        vs = 0.5 * r["phantom"][1]
        ph = dict(base, voxel=(vs, vs, vs), origin=(-30 * vs, -30 * vs, -50 * vs))
    return G.Scanner(r["scanner"], ph), ph


def test_served_results_equal_alone(G, oracle):
    reqs = W.config5(n_requests=24, pairs_lo=2e4, pairs_hi=4e5)
    base = W.hot_rod_phantom()
    made = [_request_scanner(G, r, base) for r in reqs]
    scanners = [m[0] for m in made]
    srv = G.Server(hbm_budget_bytes=8 * 10**9, workers=2)
    ids = [None] * len(reqs)

    def submit_all():
        t0 = time.perf_counter()
        for i, r in enumerate(reqs):
            # compressed arrival times: requests keep arriving while others run
            dt = (r["arrival_s"] - reqs[0]["arrival_s"]) / 20.0 - (time.perf_counter() - t0)
            if dt > 0:
                time.sleep(dt)
            ids[i] = srv.submit(scanners[i], r["source"], r["digitizer"], r["n_decays"], r["seed"])

    th = threading.Thread(target=submit_all)
    th.start()
    th.join()
    served = [srv.wait(i) for i in ids]
    st = srv.stats()
    assert st["completed"] == len(reqs) and st["submitted"] == len(reqs)
    assert st["launches"] <= len(reqs)
    for i, r in enumerate(reqs):
        alone = scanners[i].simulate(r["source"], r["digitizer"], r["n_decays"], r["seed"])
        assert_same(canon(alone), canon(served[i]))
        assert served[i].counts()["latency_ms"] > 0
    srv.close()
    # the served results against the oracle: three point-source and three
    # phantom requests, run alone with their hit lists (equal to the served
    # result, checked here again) and compared history by history
    point = [i for i, r in enumerate(reqs) if r["phantom"] is None][:3]
    phantom = [i for i, r in enumerate(reqs) if r["phantom"] is not None][:3]
    assert len(point) == 3 and len(phantom) == 3
    for i in point + phantom:
        r = reqs[i]
        res = scanners[i].simulate(r["source"], r["digitizer"], r["n_decays"], r["seed"], keep_hits=True)
        assert_same(canon(res), canon(served[i]))
        orc = oracle.simulate(r["scanner"], r["source"], r["digitizer"], r["n_decays"], r["seed"],
                              phantom=made[i][1], threads=8)
        check_parity(G, oracle, res, orc, r["n_decays"], r["digitizer"])
        res.free()


@pytest.mark.parametrize("kernel", [3, 1, 2])
def test_split_requests_equal_alone(G, oracle, kernel):
    """Requests above the piece size run as history ranges in successive live
    launches, their singles and tallies gathered in their own device buffers
    and sorted once at the end; each equals its plain run bit for bit, mixed
    with whole requests that arrive meanwhile, on every transport kernel."""
    reqs = W.config5(n_requests=10, pairs_lo=2e4, pairs_hi=3e5, seed=55)
    base = W.hot_rod_phantom()
    made = [_request_scanner(G, r, base) for r in reqs]
    srv = G.Server(hbm_budget_bytes=8 * 10**9, piece_decays=40_000, kernel=kernel)
    ids = [srv.submit(made[i][0], r["source"], r["digitizer"], r["n_decays"], r["seed"]) for i, r in enumerate(reqs)]
    served = [srv.wait(i) for i in ids]
    st = srv.stats()
    n_split = sum(r["n_decays"] > 40_000 for r in reqs)
    assert n_split >= 4 and st["pieces"] > n_split and st["completed"] == len(reqs)
    for i, r in enumerate(reqs):
        alone = made[i][0].simulate(r["source"], r["digitizer"], r["n_decays"], r["seed"], kernel=kernel)
        assert_same(canon(alone), canon(served[i]))
        alone.free()
    srv.close()
    # one split phantom request against the oracle as well
    i = next(k for k, r in enumerate(reqs) if r["n_decays"] > 40_000 and r["phantom"] is not None)
    r = reqs[i]
    res = made[i][0].simulate(r["source"], r["digitizer"], r["n_decays"], r["seed"], keep_hits=True)
    assert_same(canon(res), canon(served[i]))
    orc = oracle.simulate(r["scanner"], r["source"], r["digitizer"], r["n_decays"], r["seed"],
                          phantom=made[i][1], threads=8)
    check_parity(G, oracle, res, orc, r["n_decays"], r["digitizer"])


def test_requests_join_a_running_launch(G):
    """A launch stays open while requests keep arriving (max_launch_ms), and
    its kernel takes the appended jobs as they come: requests submitted while
    a large one runs are appended to its launch, and every result equals its
    plain run."""
    sc = G.Scanner(W.config2_scanner("B"))
    dg = W.digitizer()
    srv = G.Server(hbm_budget_bytes=16 * 10**9, max_launch_ms=500.0, piece_decays=30_000_000)
    jobs = [((0.0, 0.0, -3.0), 20_000_000, 71)] + [((0.0, 0.0, 1.0 * k), 200_000, 80 + k) for k in range(12)]
    ids = []
    for pos, n, seed in jobs:
        ids.append(srv.submit(sc, W.point_source(pos), dg, n, seed))
        time.sleep(0.0005)
    served = [srv.wait(i) for i in ids]
    st = srv.stats()
    assert st["live_appends"] >= 1 and st["max_jobs_per_launch"] >= 2, st
    for (pos, n, seed), s in zip(jobs, served):
        alone = sc.simulate(W.point_source(pos), dg, n, seed)
        assert_same(canon(alone), canon(s))
        alone.free()
    srv.close()
    sc.close()


def test_admission_by_footprint(G):
    sc = G.Scanner(W.config2_scanner("A"))
    srv = G.Server(hbm_budget_bytes=200 * 10**6, workers=1)
    # a request that alone exceeds the budget is refused outright
    with pytest.raises(G.GpetError) as e:
        srv.submit(sc, W.point_source(), W.digitizer(), 5 * 10**7, 1)
    assert e.value.code == -3
    # the server must be able to hold the largest request below (~61 MB)
    # a full budget refuses non-blocking submissions, blocking ones queue
    ids = [srv.submit(sc, W.point_source(), W.digitizer(), 10**6, 1 + i) for i in range(6)]
    busy = 0
    for i in range(20):
        try:
            ids.append(srv.submit(sc, W.point_source(), W.digitizer(), 10**6, 100 + i, block=False))
        except G.GpetError as ex:
            assert ex.code == -7
            busy += 1
    # results keep their device memory charged until freed: take and free each
    # one before waiting on the next, or queued requests cannot be admitted
    for i in ids:
        r = srv.wait(i)
        assert r.counts()["singles"] > 0
        r.free()
    st = srv.stats()
    assert st["completed"] == len(ids)
    assert st["rejected"] == busy and busy > 0
    # the budget, passed at most by the results being copied to their own memory
    assert st["peak_bytes"] <= 200 * 10**6 * 5 // 4
    srv.close()


def test_two_waiters_on_one_request(G):
    """Two callers wait on the same request: one takes the result, the other
    is told the id was taken (GPET_ERR_INVALID_ARG), and nothing reads a
    freed request."""
    sc = G.Scanner(W.config2_scanner("A"))
    srv = G.Server(hbm_budget_bytes=8 * 10**9, workers=1)
    rid = srv.submit(sc, W.point_source(), W.digitizer(), 2 * 10**6, 5)
    got, errs = [], []

    def waiter():
        try:
            got.append(srv.wait(rid))
        except G.GpetError as e:
            errs.append(e.code)

    ths = [threading.Thread(target=waiter) for _ in range(2)]
    for t in ths:
        t.start()
    for t in ths:
        t.join()
    assert len(got) == 1 and errs == [-1]
    assert got[0].counts()["singles"] > 0
    got[0].free()
    srv.close()
    sc.close()


def test_split_requests_leave_room_for_a_launch(G):
    """Many split requests at once whose own buffers together exceed the
    budget less one launch arena: their buffers are made only while a launch
    arena still fits beside them (pieces run only through launches), so every
    request completes, and each equals its plain run."""
    sc = G.Scanner(W.config2_scanner("A"))
    dg = W.digitizer()
    srv = G.Server(hbm_budget_bytes=12 * 10**8, piece_decays=200_000)
    jobs = [((0.0, 0.0, 0.5 * k), 1_000_000, 300 + k) for k in range(30)]
    ids = [srv.submit(sc, W.point_source(pos), dg, n, seed) for pos, n, seed in jobs]
    for k, i in enumerate(ids):
        r = srv.wait(i)
        if k in (0, 29):
            pos, n, seed = jobs[k]
            alone = sc.simulate(W.point_source(pos), dg, n, seed)
            assert_same(canon(alone), canon(r))
            alone.free()
        r.free()
    st = srv.stats()
    assert st["completed"] == len(jobs) and st["pieces"] >= 5 * len(jobs)
    # the budget, passed at most by the results being copied to their own memory
    assert st["peak_bytes"] <= 12 * 10**8 * 5 // 4
    srv.close()
    sc.close()


def test_in_order_client_behind_a_phantom_request(G):
    """A phantom request ahead of 200 point-source requests, under a budget
    that the point-source results alone would more than fill, and a client
    that takes results in submission order.  Admission passes put requests
    without a phantom first only while two launch arenas still fit the
    budget; past that they take arrival order, so the phantom request is
    admitted before the results held behind it fill the budget.  If the
    client stalls anyway, it releases every result in any order, so that the
    pipeline and close() still end, and the test fails."""
    dg = W.digitizer()
    sc = G.Scanner(W.config2_scanner("A"))
    scp = G.Scanner(W.config2_scanner("A"), W.hot_rod_phantom())
    budget = 12 * 10**8
    srv = G.Server(hbm_budget_bytes=budget)
    n = 200
    ids = [None] * (n + 1)

    def submit_all():
        ids[0] = srv.submit(scp, W.phantom_source(), dg, 1_000_000, 7)
        for k in range(n):
            ids[k + 1] = srv.submit(sc, W.point_source((0.0, 0.0, 0.1 * k)), dg, 1_000_000, 100 + k)

    th = threading.Thread(target=submit_all)
    th.start()
    deadline = time.perf_counter() + 90.0
    taken = 0
    held = 0
    while taken <= n and time.perf_counter() < deadline:
        r = srv.poll(ids[taken]) if ids[taken] is not None else None
        if r is None:
            time.sleep(0.002)
            continue
        assert r.counts()["singles"] > 0
        if taken == 0:
            assert r.counts()["phantom_steps"] > 0
        held = max(held, srv.stats()["bytes_in_use"])
        r.free()
        taken += 1
    stalled = taken <= n
    if stalled:
        left = set(range(taken, n + 1))
        drain = time.perf_counter() + 90.0
        while left and time.perf_counter() < drain:
            for k in sorted(left):
                r = srv.poll(ids[k]) if ids[k] is not None else None
                if r is not None:
                    r.free()
                    left.discard(k)
            time.sleep(0.01)
    th.join()
    st = srv.stats()
    srv.close()
    sc.close()
    scp.close()
    assert not stalled, f"request {taken} not done while the client held the later results"
    assert st["completed"] == n + 1
    # the budget, passed at most by the results being copied to their own memory
    assert st["peak_bytes"] <= budget * 5 // 4
