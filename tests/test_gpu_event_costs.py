"""Measurement infrastructure of the transport roofline: the CTA-synchronous
kernel counts the events it runs per history phase, and gpet_event_costs
times each event type alone on micro-kernels."""
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


def test_phase_event_counts_match_the_event_counters(G):
    """One decay event per history; one detector-step event per detector step
    and one phantom-step event per phantom step (the events' own counters);
    flight events are flights not decided at the photon's start; the other
    kernels report no phase counts."""
    n = 200_000
    c = G.simulate(W.config3_scanner(), W.phantom_source(), W.digitizer(), n, 3, phantom=W.hot_rod_phantom(),
                   kernel=3).counts()
    ev = c["phase_events"]
    assert ev[0] == 0 and ev[1] == n
    assert ev[2] == c["phantom_steps"] > 0 and ev[4] == c["det_steps"] > 0
    assert 0 < ev[3] + ev[6] <= c["flights"] and ev[6] > 0
    assert 0 < ev[5] <= n
    c2 = G.simulate(W.config3_scanner(), W.phantom_source(), W.digitizer(), n, 3, phantom=W.hot_rod_phantom(),
                    kernel=2).counts()
    assert c2["phase_events"] == [0] * 7 and c2["det_steps"] == c["det_steps"]


def test_event_costs(G):
    """Every phase a point source reaches gets a positive cost per event (a
    whole-GPU time: far below a nanosecond), the phantom step none; with the
    phantom as the source the phantom step is timed too."""
    sc = G.Scanner(W.config2_scanner("A"))
    ns, states = sc.event_costs(W.point_source(), W.digitizer(), n_sample=200_000, seed=2)
    assert ns[0] == 0 and ns[2] == 0 and states[2] == 0
    for p in (1, 3, 4, 5, 6):
        assert states[p] > 0 and 0 < ns[p] < 1.0, (p, ns, states)
    sc.close()
    ph = G.Scanner(W.config3_scanner(), W.hot_rod_phantom())
    ns, states = ph.event_costs(W.phantom_source(), W.digitizer(), n_sample=100_000, seed=3)
    assert states[2] > 0 and 0 < ns[2] < 1.0
    ph.close()
