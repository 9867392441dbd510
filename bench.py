#!/usr/bin/env python3
"""Benchmark of the photon-pair transport hot path on GB300.

Workload (default): the axial sensitivity sweep on the 12-panel ring at 55 mm
(1 x 4 modules of 20 x 20 LYSO crystals, 1.0 mm pitch): a point source at 61
axial positions (-30..30 mm, 1 mm steps), 1e7 back-to-back pairs per
position, for geometry A (one 10 mm layer) and geometry B (two 5 mm layers
with a 0.05 mm reflector gap).  One step = the whole sweep = 1.22e9 pairs
through transport, singles, energy blur and window, time sort and
coincidence sorting.  Inputs are synthetic and seeded.

Prints one JSON line.  `value` is pairs/s over the device-timed steps (CUDA
events on the launching stream, L2 flushed between steps); `e2e` is the same
metric through the C ABI with host descriptors in and coincidences, singles
and tallies copied back to host memory inside the timed region.

--impl reference times the FP64 CPU oracle on the host cores on a bounded
sample of the same workload (it is the slow baseline, not a GPU program).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads as W  # noqa: E402

METRIC = "pairs tracked/s/GB300 batched vs plain; p50/p99 served-request latency"
N_POSITIONS = 61
PAIRS_PER_POSITION = 10_000_000

# The transport is bound by instruction issue (no dense contraction, L2-resident
# working set).  Its roofline peak is the SMs' issue slots: the SM count of the
# device (queried), four warp schedulers per SM that each issue one warp
# instruction per cycle, at the maximum SM clock (generated peaks file,
# else the GB300's 2070 MHz).
SCHEDULERS_PER_SM = 4
PHASES = ("", "decay", "phantom_step", "flight", "detector_step", "finish", "flight_after_exit")


def _sm_max_mhz():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["sm_max_mhz"])
    except (OSError, KeyError, ValueError):
        return 2070.0


def sweep_jobs(rank=0, pairs=PAIRS_PER_POSITION, positions=N_POSITIONS):
    jobs = []
    for geo in ("A", "B"):
        for i, z in enumerate(W.config2_positions()[:positions]):
            jobs.append(dict(geometry=geo, source=W.point_source((0.0, 0.0, z)), n=pairs,
                             seed=2 + i + 1000 * (geo == "B") + 100_000 * rank))
    return jobs


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                                      stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return dict(sm_mhz=None, sm_max_mhz=None, reasons=["nvidia-smi unavailable"])
        self.p.terminate()
        self.p.wait()
        self.f.flush()
        self.f.seek(0)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f.read().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.f.name)
        return dict(sm_mhz=statistics.median(sm) if sm else None, sm_max_mhz=max(mx) if mx else None,
                    reasons=sorted(reasons), samples=len(sm))


# Counters of the transport kernel in the benchmark's own launch (the whole
# sweep), per simulated pair, from one ncu capture of that launch with
# smsp__inst_executed.sum (warp instructions), dram__bytes_read.sum and
# dram__bytes_write.sum.  A capture holds only for the sources it was taken on:
# each entry carries their SHA-1 and is reported as null once they differ.
# Entries are named by capture id (the summary of each capture under that id
# gives its command).
TRANSPORT_SOURCES = ("device.cuh", "transport.cuh", "transport.cu", "transport_cta.cu")
TRANSPORT_CAPTURE = dict(id="k_transport_cta_sweep_122x1e7", sha1="f4a6704d15a30fafa6a2dd16570072434011662a",
                         warp_inst_per_pair=143.306, dram_bytes_per_pair=9.798)
# Issue detail of the same kernel from one ncu --set full capture of a
# 2e6-pair sweep position: issue-active fraction of the schedulers and SIMT
# efficiency (thread instructions per warp instruction / 32).
TRANSPORT_DETAIL = dict(id="k_transport_cta_sweep_position_2e6", sha1="f4a6704d15a30fafa6a2dd16570072434011662a",
                        issue_active=0.494, simt_efficiency=0.583)
# algorithmic bytes of the digitizer back end per single (the model in run_ours)
DIGITIZER_BYTES_PER_SINGLE = 330
# DRAM bytes of the digitizer back end (make_keys .. job_stats of one step), per single.
DIGITIZER_SOURCES = ("device.cuh", "sort.cu")
DIGITIZER_TRAFFIC = dict(id="traffic_digitizer_sweep_8x1e7", sha1="6fd97e665d63322ce912e6a20bee0aebc691fc9c",
                         bytes_per_single=361.6)


def _current(entry, sources):
    """The capture entry when it was taken on the present sources, else None."""
    return entry if entry and entry.get("sha1") and entry["sha1"] == _sources_sha1(sources) else None


def _sources_sha1(names):
    """SHA-1 of the code of the named sources: comments and blank lines are
    dropped, so that editing a comment does not disown a capture."""
    import hashlib
    import re
    h = hashlib.sha1()
    for name in names:
        with open(os.path.join(ROOT, "paper_2603_07327_gb300", "csrc", name)) as f:
            text = f.read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        code = "\n".join(line.rstrip() for line in text.splitlines() if line.strip())
        h.update(code.encode())
    return h.hexdigest()


def _transport_traffic(pairs_per_launch):
    t = _current(TRANSPORT_CAPTURE, TRANSPORT_SOURCES)
    return t["dram_bytes_per_pair"] * pairs_per_launch if t and t["dram_bytes_per_pair"] else None


def _digitizer_traffic(singles_per_step):
    t = _current(DIGITIZER_TRAFFIC, DIGITIZER_SOURCES)
    return t["bytes_per_single"] * singles_per_step if t else None


def event_isolated(scanners, dg, counts, tr_ms, n_sample=1_000_000):
    """Event-isolated fraction of the transport: each phase's events of the
    timed launches (counted by the kernel) times that event's GPU time when it
    runs alone at full width (gpet_event_costs, on states of geometry A and B
    with the source at the centre, averaged: the sweep is half of each), over
    the measured transport time."""
    costs = [scanners[g].event_costs(W.point_source((0.0, 0.0, 0.0)), dg, n_sample=n_sample, seed=2)[0]
             for g in ("A", "B")]
    ns = [0.5 * (a + b) for a, b in zip(*costs)]
    events = [sum(c["phase_events"][p] for c in counts) for p in range(len(PHASES))]
    pairs = sum(c["n_decays"] for c in counts)
    ideal_ms = sum(events[p] * ns[p] for p in range(1, len(PHASES))) * 1e-6
    return dict(frac=ideal_ms / tr_ms, ideal_transport_ms=ideal_ms, transport_ms=tr_ms,
                ns_per_event={PHASES[p]: ns[p] for p in range(1, len(PHASES))},
                events_per_pair={PHASES[p]: events[p] / pairs for p in range(1, len(PHASES))},
                sample=f"{n_sample} histories of geometry A and of B, source at the centre")


def _measured_hbm_gbs():
    """Measured copy bandwidth of the GB300s (driver-written), else the
    recipe's fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"])
    except (OSError, KeyError, ValueError):
        return 6800.0


def cpu_baseline(budget_s=12.0, threads=None):
    """The FP64 oracle as it stands on the host cores, on a bounded sample of the
    sweep (geometry A and B at z = 0, blocks of histories until the budget)."""
    from oracle import oracle as O
    O.build()
    threads = threads or os.cpu_count() or 1
    dg = W.digitizer()
    done, t0 = 0, time.perf_counter()
    block = 250_000
    k = 0
    while time.perf_counter() - t0 < budget_s:
        geo = "A" if k % 2 == 0 else "B"
        h0 = (k * block) % (PAIRS_PER_POSITION - block)
        O.simulate(W.config2_scanner(geo), W.point_source((0.0, 0.0, 0.0)), dg, PAIRS_PER_POSITION, 2,
                   h_begin=h0, h_end=h0 + block, threads=threads, tallies=True)
        done += block
        k += 1
    dt = time.perf_counter() - t0
    return dict(value=done / dt, unit="pairs/s", cores=threads, kind="oracle",
                sample=f"{done} pairs of the sweep (geometry A and B alternating, source at z=0, 1e7-pair time span) "
                       f"in {dt:.1f} s"), done, dt


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    steps, warm = args.steps, args.warmup
    for _ in range(warm):
        cpu_baseline(budget_s=2.0)
    vals, dts, cb = [], [], None
    for _ in range(steps):
        cb, done, dt = cpu_baseline(budget_s=max(3.0, 20.0 / max(steps, 1)))
        vals.append(done)
        dts.append(dt)
    value = sum(vals) / sum(dts)
    line = dict(metric=METRIC, value=value, unit="pairs/s", n_gpus=args.gpus, steps=steps, warmup=warm,
                ms_per_step=1000 * sum(dts) / steps, higher_is_better=True, scaling="weak", vs_baseline=None,
                dtype="f64", data="synthetic", impl="reference",
                config=dict(workload="sensitivity sweep, 12-panel ring R=55 mm, geometry A/B, 61 positions x 1e7 pairs "
                                     "(bounded CPU sample)", l2="n/a (host)"),
                cpu_baseline=dict(kind="oracle", cores=cb["cores"], sample=cb["sample"], value=value, unit="pairs/s"),
                e2e=dict(value=value, unit="pairs/s", h2d_bytes_per_step=0, d2h_bytes_per_step=0))
    print(json.dumps(line), flush=True)
    return 0


def run_served(G, args):
    """The served stream: 2000 simulation requests, each a design drawn like
    the batched sweep, half point sources and half the hot-rod phantom scaled
    0.5-1x, 1e5-5e7 pairs, admitted under a 150 GB HBM budget.  Served twice:
    arriving as the Poisson process of the workload (50/s, about a tenth of
    the GPU's capacity: latency at that load), and with the same arrival times
    compressed `served_compress` times, so that the queue never empties
    (throughput at saturation).  Then the same requests as sequential plain
    launches, one gpet_simulate each, back to back."""
    import threading
    reqs = W.config5(n_requests=args.served_requests)
    base = W.hot_rod_phantom()

    def make(r):
        ph = None
        if r["phantom"] is not None:
            vs = 0.5 * r["phantom"][1]
            ph = dict(base, voxel=(vs, vs, vs), origin=(-30 * vs, -30 * vs, -50 * vs))
        return G.Scanner(r["scanner"], ph)

    scanners = [None] * len(reqs)

    def serve(compress):
        srv = G.Server(hbm_budget_bytes=150 * 10**9, kernel=args.kernel)
        w = scanners[0] or make(reqs[0])
        srv.wait(srv.submit(w, reqs[0]["source"], reqs[0]["digitizer"], 100_000, 1)).free()  # warm the path
        st0 = srv.stats()
        ids = [None] * len(reqs)
        t0 = time.perf_counter()

        def submit_all():
            for i, r in enumerate(reqs):
                dt = r["arrival_s"] / compress - (time.perf_counter() - t0)
                if dt > 0:
                    time.sleep(dt)
                if scanners[i] is None:
                    scanners[i] = make(r)   # the request's design (and phantom) is built at arrival
                ids[i] = srv.submit(scanners[i], r["source"], r["digitizer"], r["n_decays"], r["seed"])

        lat = []

        def collect_all():
            # results are taken (and their device memory released) as they complete
            for k in range(len(reqs)):
                while ids[k] is None:
                    time.sleep(0.001)
                res = srv.wait(ids[k])
                lat.append(res.counts()["latency_ms"])
                res.free()

        th = threading.Thread(target=submit_all)
        tc = threading.Thread(target=collect_all)
        th.start()
        tc.start()
        th.join()
        tc.join()
        wall = time.perf_counter() - t0
        st = srv.stats()
        srv.close()
        pairs = sum(r["n_decays"] for r in reqs)
        lat = sorted(lat)
        return dict(p50_ms=float(np.percentile(lat, 50)), p99_ms=float(np.percentile(lat, 99)),
                    max_ms=float(lat[-1]), pairs_per_s=pairs / wall,
                    offered_pairs_per_s=pairs / (reqs[-1]["arrival_s"] / compress), wall_s=wall,
                    launches=st["launches"] - st0["launches"], max_jobs_per_launch=st["max_jobs_per_launch"],
                    live_appends=st["live_appends"] - st0["live_appends"], pieces=st["pieces"] - st0["pieces"],
                    peak_hbm_bytes=st["peak_bytes"],
                    # GPU time of the launches' stages (CUDA events): the live kernels
                    # from open to close, and every time sort / coincidence pass
                    transport_gpu_s=(st["transport_ms"] - st0["transport_ms"]) / 1000.0,
                    digitizer_gpu_s=(st["digitizer_ms"] - st0["digitizer_ms"]) / 1000.0)

    poisson = serve(1.0)
    saturated = serve(args.served_compress)
    # the same requests as sequential plain launches, back to back
    k = min(len(reqs), args.served_plain_sample) if args.served_plain_sample > 0 else len(reqs)
    scanners[0].simulate(reqs[0]["source"], reqs[0]["digitizer"], 100_000, 1, kernel=args.kernel).free()
    tp = time.perf_counter()
    plain_tr = plain_dg = 0.0
    for i in range(k):
        res = scanners[i].simulate(reqs[i]["source"], reqs[i]["digitizer"], reqs[i]["n_decays"], reqs[i]["seed"],
                                   kernel=args.kernel)
        c = res.counts()
        plain_tr += c["transport_ms"] / 1000.0
        plain_dg += c["digitizer_ms"] / 1000.0
        res.free()
    tp = time.perf_counter() - tp
    pairs_plain = sum(reqs[i]["n_decays"] for i in range(k))
    for sc in scanners:
        if sc is not None:
            sc.close()
    pairs = sum(r["n_decays"] for r in reqs)
    return dict(requests=len(reqs), pairs=pairs, hbm_budget_bytes=150 * 10**9,
                arrivals="Poisson, mean 50 req/s, seed 5",
                poisson=poisson,
                saturated=dict(saturated, compress=args.served_compress),
                sequential_plain_pairs_per_s=pairs_plain / tp, sequential_plain_requests=k,
                sequential_plain_transport_gpu_s=plain_tr, sequential_plain_digitizer_gpu_s=plain_dg,
                sequential_plain_wall_s=tp,
                saturated_over_sequential_plain=saturated["pairs_per_s"] / (pairs_plain / tp))


def run_sensitivity(G, args):
    """Sensitivity map S(r, E) of Sec. 2.4 on H2RSPET-1CL and -2CL (ten panels
    at 85 mm, six axial modules of 51 x 51 crystals): 15 radial and 17 further
    axial source positions, four energy windows (150/250/350/450-700 keV), 2e6
    decays per position (the paper's 1.6e8-atom source over 120 s), 16 %
    resolution, 3 ns window.  One gpet_sensitivity_map call = 1.28e8 pairs in
    one batched launch with all windows counted in one pass.  Compared with the
    naive form: one plain gpet_simulate per (design, position, window)."""
    designs = [W.h2rspet("1CL"), W.h2rspet("2CL")]
    scs = [G.Scanner(d) for d in designs]
    pos = np.array(W.sensitivity_positions())
    dg = W.sensitivity_digitizer()
    n = args.sens_pairs
    pairs = n * len(pos) * len(scs)
    G.sensitivity_map(scs, pos, dg, W.SENS_WINDOWS_KEV, n, 2603, kernel=args.kernel)   # warm
    wall, dev = [], []
    for k in range(args.sens_reps):
        t0 = time.perf_counter()
        counts, S, tot = G.sensitivity_map(scs, pos, dg, W.SENS_WINDOWS_KEV, n, 2603 + 1000 * k,
                                           kernel=args.kernel)
        wall.append(time.perf_counter() - t0)
        dev.append((tot["transport_ms"] + tot["digitizer_ms"]) / 1000.0)
    # the naive form: one plain run per (design, position, window)
    tp = float("nan")
    if args.sens_plain:
        tp = time.perf_counter()
        for sc in scs:
            for p, x in enumerate(pos):
                for lo, hi in W.SENS_WINDOWS_KEV:
                    sc.simulate(W.point_source(tuple(x)), dict(dg, e_lo=lo, e_hi=hi), n, 2603 + p,
                                kernel=args.kernel).free()
        tp = time.perf_counter() - tp
    for sc in scs:
        sc.close()
    d = G.delta_sym(S[0], S[1])
    rich = counts.min(axis=0) > 20_000
    wall_s = statistics.median(wall)
    dev_s = statistics.median(dev)
    return dict(workload="H2RSPET-1CL and -2CL, 32 positions (radial 0-70 mm / 5 mm, axial 10-170 mm / 10 mm), "
                         "4 energy windows, 2e6 pairs per position", pairs=pairs,
                device_ms=1000 * dev_s, pairs_per_s=pairs / dev_s, e2e_ms=1000 * wall_s, e2e_pairs_per_s=pairs / wall_s,
                plain_per_window_ms=1000 * tp, plain_per_window_pairs_per_s=pairs * len(W.SENS_WINDOWS_KEV) / tp,
                map_over_plain_per_window=tp / wall_s, reps=args.sens_reps,
                singles_per_pair=tot["singles"] / pairs, coincidences_union_window=tot["coincidences"],
                delta_sym_centre=[round(float(x), 3) for x in d[0]],
                delta_sym_mean_rich_cells=float(np.nanmean(d[rich])), rich_cells=int(rich.sum()),
                sensitivity_centre_350_700=[float(S[0, 0, 2]), float(S[1, 0, 2])])


def run_design_sweep(G, args):
    """The batched design sweep: 64 candidate scanners drawn from seed 4 (1-3
    layers, 8-20 mm total depth, 0.8-2.0 mm pitch, 40-80 mm ring radius, layer
    offset 0 or half a pitch), each with a point source at a random radial
    offset and a log-uniform 1e5-1e7 decays.  Batched: the launch form is
    autotuned on a pilot of the largest design, then all 64 jobs run as one
    graph-captured persistent launch (gpet_batch_run, host-timed including the
    read-back of the counters).  Plain: 64 sequential gpet_simulate calls.
    The per-job coincidence counts of the two forms must agree exactly."""
    import torch
    designs = W.config4()
    scs = [G.Scanner(d["scanner"]) for d in designs]
    pairs = sum(d["n_decays"] for d in designs)
    big = max(range(len(designs)), key=lambda i: designs[i]["n_decays"])
    tuned, tuned_ms = scs[big].autotune(designs[big]["source"], designs[big]["digitizer"], pilot_decays=2_000_000)
    jobs = [dict(scanner=scs[i], source=d["source"], digitizer=d["digitizer"], n_decays=d["n_decays"],
                 seed=d["seed"]) for i, d in enumerate(designs)]
    b = G.Batch(jobs)
    for _ in range(args.warmup):
        b.run()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        b.run()
    batched_s = (time.perf_counter() - t0) / args.steps
    tot = b.counts()
    batched_coinc = []
    for i in range(len(jobs)):
        r = b.result(i)
        batched_coinc.append(r.counts()["coincidences"])
        r.free()

    def plain(collect=None):
        for d, sc in zip(designs, scs):
            r = sc.simulate(d["source"], d["digitizer"], d["n_decays"], d["seed"])
            if collect is not None:
                collect.append(r.counts()["coincidences"])
            r.free()

    plain()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    plain_coinc = []
    plain(plain_coinc)
    plain_s = time.perf_counter() - t0
    b.close()
    for sc in scs:
        sc.close()
    return dict(workload="64 designs drawn from seed 4 (1-3 layers, 8-20 mm, pitch 0.8-2.0 mm, R 40-80 mm), "
                         "point sources at 0-50 mm radial offset, log-uniform 1e5-1e7 pairs each",
                pairs=pairs, batched_ms=1000 * batched_s, batched_pairs_per_s=pairs / batched_s,
                transport_ms=tot["transport_ms"], digitizer_ms=tot["digitizer_ms"],
                plain_ms=1000 * plain_s, plain_pairs_per_s=pairs / plain_s, batched_over_plain=plain_s / batched_s,
                tuned=tuned, tuned_pilot_transport_ms=tuned_ms,
                coincidences_identical=batched_coinc == plain_coinc)


def run_variants(G, args):
    """Throughput of the other parity-tested forms, each one plain run after a
    warm-up, device-timed by the library's stage events (transport + digitizer):
    the offset dual-layer ring with the hot-rod water phantom as the source
    (1e8 pairs at the default 1.7e4 Bq: 5.9e3 s of acquisition),
    four posed heads in non-repetition mode, the four-layer ring,
    and module-level readout on the H2RSPET split ring (1e7 pairs each)."""
    dg = W.digitizer()
    split = W.h2rspet("split", modules_v=2)
    split["readout_level"] = W.READOUT_MODULE
    cases = [("offset_dual_layer_phantom", W.config3_scanner(), W.phantom_source(), W.hot_rod_phantom(),
              100_000_000, 3),
             ("posed_heads", W.box_scanner(), W.point_source((4.0, -3.0, 2.5)), None, 10_000_000, 41),
             ("four_layer_ring", W.four_layer_scanner(), W.point_source((6.0, 2.0, -4.0)), None, 10_000_000, 47),
             ("module_readout", split, W.point_source((21.0, -13.0, 9.0)), None, 10_000_000, 77)]
    out = {}
    for name, scd, src, ph, n, seed in cases:
        sc = G.Scanner(scd, ph)
        sc.simulate(src, dg, 1_000_000, seed, kernel=args.kernel).free()
        r = sc.simulate(src, dg, n, seed, kernel=args.kernel)
        c = r.counts()
        r.free()
        sc.close()
        ms = c["transport_ms"] + c["digitizer_ms"]
        out[name] = dict(pairs=n, device_ms=ms, pairs_per_s=n / (ms / 1000.0), transport_ms=c["transport_ms"],
                         hits=c["hits"], singles=c["singles"], coincidences=c["coincidences"],
                         phantom_steps=c["phantom_steps"])
    return out


def run_ours(args):
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import __graft_entry__
    __graft_entry__.build()
    import paper_2603_07327_gb300 as G

    dg = W.digitizer()
    scanners = {g: G.Scanner(W.config2_scanner(g)) for g in ("A", "B")}
    jobs = sweep_jobs(rank, pairs=args.pairs, positions=args.positions)
    pairs_per_step = sum(j["n"] for j in jobs)
    stream = torch.cuda.current_stream().cuda_stream
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device="cuda")

    def plain_step(collect=None):
        for j in jobs:
            r = scanners[j["geometry"]].simulate(j["source"], dg, j["n"], j["seed"], stream=stream,
                                                 kernel=args.kernel)
            if collect is not None:
                collect.append(r.counts())
            r.free()

    batch = None
    if args.form == "batched":
        batch = G.Batch([dict(scanner=scanners[j["geometry"]], source=j["source"], digitizer=dg, n_decays=j["n"],
                              seed=j["seed"]) for j in jobs], stream=stream, kernel=args.kernel)

    def step(collect=None):
        if batch is None:
            return plain_step(collect)
        batch.run()
        if collect is not None:
            collect.append(batch.counts())

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    clocks = Clocks(local)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    wall0 = time.perf_counter()
    clocks.start()
    dev_ms, counts = [], []
    for _ in range(args.steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        step(counts if batch is None else None)
        e1.record()
        e1.synchronize()
        dev_ms.append(e0.elapsed_time(e1))
        if batch is not None:
            counts.append(batch.counts())  # host bookkeeping, after the step's end mark
    torch.cuda.synchronize()
    clk = clocks.stop()
    wall = time.perf_counter() - wall0
    t_dev = sum(dev_ms) / 1000.0
    if dist:
        t = torch.tensor([t_dev, wall], device="cuda", dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        t_dev, wall = float(t[0]), float(t[1])
        dist.barrier()
    total_pairs = pairs_per_step * args.steps * world
    value = total_pairs / t_dev

    # dominant kernel: the transport kernel (per-launch CUDA events inside the library)
    tr_ms = sum(c["transport_ms"] for c in counts)
    dg_ms = sum(c["digitizer_ms"] for c in counts)
    kname = {1: "k_transport_loop", 2: "k_transport_wave"}.get(args.kernel, "k_transport_cta")
    pairs_per_launch = pairs_per_step if args.form == "batched" else pairs_per_step / max(len(jobs), 1)
    default_kernel = args.kernel in (0, 3)
    traffic = args.traffic if args.traffic is not None else (
        _transport_traffic(pairs_per_launch) if default_kernel else None)
    # issue slots: warp instructions per pair (ncu, the benchmark's own launch)
    # x pairs over the transport time of the timed launches (CUDA events),
    # against the device's issue slots
    sm_count = torch.cuda.get_device_properties(local).multi_processor_count
    sm_mhz = _sm_max_mhz()
    issue_peak = sm_count * SCHEDULERS_PER_SM * sm_mhz * 1e6
    cap = _current(TRANSPORT_CAPTURE, TRANSPORT_SOURCES) if default_kernel else None
    achieved = cap["warp_inst_per_pair"] * pairs_per_step * args.steps / (tr_ms / 1000.0) if cap else None
    detail = _current(TRANSPORT_DETAIL, TRANSPORT_SOURCES) if default_kernel else None
    roof = dict(bound="alu", achieved=achieved, peak=issue_peak, unit="warp-instructions/s",
                frac=(achieved / issue_peak) if achieved else None, traffic=traffic, kernel=kname,
                peak_note=f"{sm_count} SMs (device query) x {SCHEDULERS_PER_SM} warp schedulers x {sm_mhz:.0f} MHz "
                          "(maximum SM clock): issue slots",
                capture=cap["id"] if cap else None,
                warp_inst_per_pair=cap["warp_inst_per_pair"] if cap else None,
                issue_detail=dict(issue_active=detail["issue_active"], simt_efficiency=detail["simt_efficiency"],
                                  capture=detail["id"]) if detail else None,
                transport_share=tr_ms / (tr_ms + dg_ms))
    # beside it: the transport time the launch's events would take if each ran
    # alone at full width (per-event costs from micro-kernels on this GPU, on
    # states of this workload), over the measured transport time
    if default_kernel:
        try:
            roof["event_isolated"] = event_isolated(scanners, dg, counts, tr_ms)
        except Exception as exc:  # noqa: BLE001
            roof["event_isolated"] = dict(error=f"{type(exc).__name__}: {exc}")

    # digitizer back end (time sort + coincidences), HBM-bound: algorithmic bytes
    # per single = key pass 12 (the key the transport wrote read, the index
    # written) + 8 one-sweep radix passes x 25 (key and index read 12 and
    # written 12, look-back words 1) + gather 84 (index 4, 8 fields read 40 +
    # written 40) + coincidence pass 34 = 330
    singles_step = sum(c["singles"] for c in counts) / args.steps
    dig_bytes = DIGITIZER_BYTES_PER_SINGLE * singles_step
    dig_gbs = dig_bytes / (dg_ms / args.steps / 1000.0) / 1e9 if dg_ms > 0 else None
    hbm_peak = _measured_hbm_gbs()
    roof_dig = dict(bound="hbm", achieved=dig_gbs, peak=hbm_peak, unit="GB/s",
                    frac=(dig_gbs / hbm_peak) if dig_gbs else None, traffic=_digitizer_traffic(singles_step),
                    bytes_per_single=DIGITIZER_BYTES_PER_SINGLE,
                    note="time sort + coincidence sorting; peak = measured copy GB/s; traffic = DRAM bytes of "
                         "all back-end kernels of one step")

    # end to end through the C ABI: every step is one gpet_simulate_batch call
    # over the sweep from host descriptors, and the step's results -- singles'
    # times, units and energies, coincidence pairs and per-crystal tallies of
    # the whole launch -- are read into caller-owned pinned host buffers, one
    # copy per array, the arrays concurrently on their own streams
    # (gpet_result_copy_run_async), all landed before the step ends.  A first,
    # untimed pass sizes the buffers, which every timed step reuses.
    # (Overlapping a step's copies with the next step's simulation measured
    # slower: the simulation lost more than the copies took.)
    E2E_ARRAYS = (G.SINGLES_T_PS, G.SINGLES_UNIT, G.SINGLES_E, G.COINC_A, G.COINC_B, G.TALLY_COUNT, G.TALLY_EFX)

    def e2e_simulate():
        if args.form == "batched":
            return G.simulate_batch([dict(scanner=scanners[j["geometry"]], source=j["source"], digitizer=dg,
                                          n_decays=j["n"], seed=j["seed"]) for j in jobs], stream=stream,
                                    kernel=args.kernel)
        return [scanners[j["geometry"]].simulate(j["source"], dg, j["n"], j["seed"], stream=stream,
                                                 kernel=args.kernel) for j in jobs]

    def views_of(res):
        # batched: one copy per array for the whole launch; plain: one per run
        return res[:1] if args.form == "batched" else res

    res0 = e2e_simulate()
    need = {w: sum(r.run_nbytes(w) for r in views_of(res0)) for w in E2E_ARRAYS}
    for r in res0:
        r.free()
    bufs = {w: torch.empty(need[w] + 4096, dtype=torch.uint8, pin_memory=True) for w in E2E_ARRAYS}
    # one copy stream per array: the arrays travel concurrently once the step is done
    copy_streams = {w: torch.cuda.Stream() for w in E2E_ARRAYS}
    torch.cuda.synchronize()
    e2e_t0 = time.perf_counter()
    sim_s = 0.0
    copy_ms = []
    h2d = d2h = 0
    for k in range(args.steps):
        t0 = time.perf_counter()
        res = e2e_simulate()
        t1 = time.perf_counter()
        sim_s += t1 - t0
        h2d = d2h = 0
        for r in views_of(res):
            h2d += r.counts()["h2d_bytes"]
            off = {w: 0 for w in E2E_ARRAYS}
            for w in E2E_ARRAYS:
                nb = r.copy_run_into_async(w, bufs[w].data_ptr() + off[w], bufs[w].numel() - off[w],
                                           copy_streams[w].cuda_stream)
                off[w] += nb
                d2h += nb
        for cs in copy_streams.values():
            cs.synchronize()
        copy_ms.append(1000 * (time.perf_counter() - t1))
        for r in res:
            r.free()
    torch.cuda.synchronize()
    e2e_dt = (time.perf_counter() - e2e_t0) / args.steps
    e2e_sim_s = sim_s / args.steps
    # the copy leg against a plain pinned copy of 1 GiB from device memory,
    # measured here in the same process (best of 3 after one untimed copy)
    blk = torch.ones(1 << 30, dtype=torch.uint8, device="cuda")
    hb = torch.empty(1 << 30, dtype=torch.uint8, pin_memory=True)
    plain_gbs = 0.0
    for k in range(4):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        hb.copy_(blk, non_blocking=True)
        torch.cuda.synchronize()
        if k:
            plain_gbs = max(plain_gbs, (1 << 30) / (time.perf_counter() - t0) / 1e9)
    del blk, hb
    if dist:
        t = torch.tensor([e2e_dt], device="cuda", dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_dt = float(t[0])

    line = dict(metric=METRIC, value=value, unit="pairs/s", n_gpus=world, steps=args.steps, warmup=args.warmup,
                ms_per_step=1000 * t_dev / args.steps, higher_is_better=True, scaling="weak", vs_baseline=None,
                dtype="f32", data="synthetic",
                config=dict(workload="sensitivity sweep, 12-panel ring R=55 mm, 1x4 modules of 20x20 LYSO at 1.0 mm, "
                                     "geometry A (10 mm) + B (2x5 mm, 0.05 mm reflector), 61 axial positions x 1e7 pairs",
                            form=("batched: one persistent launch over all 122 positions, CUDA-graph replay"
                                  if args.form == "batched" else "plain: one gpet_simulate per position"),
                            pairs_per_step=pairs_per_step,
                            l2="flushed between steps (256 MB write)", kernel=args.kernel or "default",
                            parallelism=f"replicas x{world}" if world > 1 else "1 GPU"),
                wall_s=wall, gpu_launches=None, roofline=roof, roofline_digitizer=roof_dig, clocks=clk,
                e2e=dict(value=pairs_per_step * world / e2e_dt, unit="pairs/s", h2d_bytes_per_step=h2d,
                         d2h_bytes_per_step=d2h, ms_per_step=1000 * e2e_dt, simulate_ms_per_step=1000 * e2e_sim_s,
                         copy_ms_per_step=1000 * (e2e_dt - e2e_sim_s), copy_ms_steps=[round(c, 2) for c in copy_ms],
                         d2h_gbs=d2h / (1e-3 * min(copy_ms)) / 1e9 if copy_ms and min(copy_ms) > 0 else None,
                         plain_pinned_d2h_gbs=plain_gbs, host_buffers="pinned, caller-owned, reused",
                         copies="one async copy per array of the whole launch, arrays on concurrent streams; into page-locked "
                                "memory the library copies by SM stores over the host link"),
                stages=dict(transport_ms_per_step=tr_ms / args.steps, digitizer_ms_per_step=dg_ms / args.steps),
                per_step_counts=dict(hits=sum(c["hits"] for c in counts) // args.steps,
                                     singles=sum(c["singles"] for c in counts) // args.steps,
                                     coincidences=sum(c["coincidences"] for c in counts) // args.steps))
    # kernels per launch: transport + redo, key pass, plan, 8 one-sweep radix passes, gather,
    # 4 coincidence kernels, job statistics
    per_launch = 2 + 2 + 8 + 1 + 4 + 1
    line["gpu_launches"] = per_launch * args.steps * (1 if args.form == "batched" else len(jobs))
    if args.form == "batched" and args.compare_plain:
        # the plain per-position form on the same sweep, for the batched-vs-plain metric
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        plain_step()
        torch.cuda.synchronize()
        t0.record()
        plain_step()
        t1.record()
        t1.synchronize()
        line["plain_pairs_per_s"] = pairs_per_step / (t0.elapsed_time(t1) / 1000.0)
        line["batched_over_plain"] = value / line["plain_pairs_per_s"]
    def aux(key, fn):
        # an auxiliary measurement that fails is reported, not fatal: the main line still prints
        try:
            line[key] = fn()
        except Exception as exc:  # noqa: BLE001
            line[key] = dict(error=f"{type(exc).__name__}: {exc}")
            print(f"bench: {key} failed: {exc!r}", file=sys.stderr, flush=True)

    if rank == 0 and args.served:
        aux("served", lambda: run_served(G, args))
    if rank == 0 and args.design_sweep:
        aux("design_sweep", lambda: run_design_sweep(G, args))
    if rank == 0 and args.variants:
        aux("variants", lambda: run_variants(G, args))
    if rank == 0 and args.sensitivity:
        aux("sensitivity_map", lambda: run_sensitivity(G, args))
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        aux("cpu_baseline", lambda: cpu_baseline()[0])
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--kernel", type=int, default=0)
    ap.add_argument("--form", default="batched", choices=["batched", "plain"])
    ap.add_argument("--compare-plain", action="store_true", default=True)
    ap.add_argument("--no-compare-plain", dest="compare_plain", action="store_false")
    ap.add_argument("--pairs", type=int, default=PAIRS_PER_POSITION)
    ap.add_argument("--positions", type=int, default=N_POSITIONS)
    ap.add_argument("--traffic", type=float, default=None, help="DRAM bytes per transport launch from ncu")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--served", action="store_true", default=True)
    ap.add_argument("--no-served", dest="served", action="store_false")
    ap.add_argument("--served-requests", type=int, default=2000)
    ap.add_argument("--variants", action="store_true", default=True)
    ap.add_argument("--no-variants", dest="variants", action="store_false")
    ap.add_argument("--design-sweep", action="store_true", default=True)
    ap.add_argument("--no-design-sweep", dest="design_sweep", action="store_false")
    ap.add_argument("--sensitivity", action="store_true", default=True)
    ap.add_argument("--no-sensitivity", dest="sensitivity", action="store_false")
    ap.add_argument("--sens-pairs", type=int, default=2_000_000)
    ap.add_argument("--sens-reps", type=int, default=3)
    ap.add_argument("--no-sens-plain", dest="sens_plain", action="store_false", default=True,
                    help="skip the per-window plain runs that the map is compared with")
    ap.add_argument("--served-plain-sample", type=int, default=0,
                    help="requests of the sequential plain comparison (0 = all)")
    ap.add_argument("--served-compress", type=float, default=20.0,
                    help="arrival-time compression of the saturated served run")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
