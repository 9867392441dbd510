"""Multi-rank sharding on CPU ranks (gloo, world size 2).

Each rank simulates its history range of one run (the oracle stands in for
the GPU engine on this CPU-only path), the tallies are all-reduced and the
singles all-gathered; the merged result must equal a single-process run
exactly, and coincidence sorting of the merged singles must give the same
pairs."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import workloads as W


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, n, out_dir):
    import torch.distributed as dist

    from oracle import oracle as O
    from paper_2603_07327_gb300 import shard
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    h0, h1 = shard.history_range(n, rank, world)
    sc = W.config2_scanner("B")
    r = O.simulate(sc, W.point_source((0.0, 0.0, 3.0)), W.digitizer(), n, 21, h_begin=h0, h_end=h1, threads=2)
    kept = r["singles"][r["singles"]["kept"] == 1]
    singles = dict(t_ps=kept["t_ps"], h=kept["h"], unit=kept["unit"], panel=kept["panel"], e=kept["e_blur"],
                   e_raw=kept["e_raw"])
    counts, efx = shard.allreduce_tallies(r["tally_count"], r["tally_efx"])
    merged = shard.gather_singles(singles)
    if rank == 0:
        np.savez(os.path.join(out_dir, "merged.npz"), counts=counts, efx=efx, **merged)
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_shards_merge_exactly(tmp_path, oracle):
    n = 40_000
    port = _free_port()
    mp.start_processes(_rank, args=(2, port, n, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    m = np.load(tmp_path / "merged.npz")
    full = oracle.simulate(W.config2_scanner("B"), W.point_source((0.0, 0.0, 3.0)), W.digitizer(), n, 21, threads=4)
    assert np.array_equal(m["counts"], full["tally_count"])
    assert np.array_equal(m["efx"], full["tally_efx"])
    kept = full["singles"][full["singles"]["kept"] == 1]
    order = np.lexsort((kept["h"], kept["unit"], kept["t_ps"]))
    for f, g in (("t_ps", "t_ps"), ("h", "h"), ("unit", "unit"), ("e", "e_blur")):
        assert np.array_equal(m[f], kept[g][order]), f
    # coincidences of the merged stream equal those of the single process
    sm = np.zeros(len(m["t_ps"]), dtype=[("t_ps", "<u8"), ("unit", "<i4"), ("panel", "<i4"), ("h", "<u8")])
    sm["t_ps"], sm["unit"], sm["panel"], sm["h"] = m["t_ps"], m["unit"], m["panel"], m["h"]
    _, a1, b1 = oracle.coincidences(sm, 2.0)
    s2, a2, b2 = oracle.coincidences(full["singles"], 2.0)
    p1 = {frozenset(((int(sm["h"][i]), int(sm["unit"][i])), (int(sm["h"][j]), int(sm["unit"][j])))) for i, j in zip(a1, b1)}
    p2 = {frozenset(((int(s2["h"][i]), int(s2["unit"][i])), (int(s2["h"][j]), int(s2["unit"][j])))) for i, j in zip(a2, b2)}
    assert p1 == p2 and len(p1) > 0


def test_history_range_partition():
    from paper_2603_07327_gb300 import shard
    for n in (1, 7, 1000, 10**7 + 3):
        for world in (1, 2, 3, 8):
            rs = [shard.history_range(n, r, world) for r in range(world)]
            assert rs[0][0] == 0 and rs[-1][1] == n
            assert all(rs[i][1] == rs[i + 1][0] for i in range(world - 1))
            assert max(b - a for a, b in rs) - min(b - a for a, b in rs) <= 1
    with pytest.raises(ValueError):
        shard.history_range(10, 2, 2)
