"""The benchmark's reference arm and bookkeeping, on the CPU.

The reference arm times the FP64 oracle on the host cores and prints the
same one-line JSON record as the GPU arm, with `impl` = "reference".  Here it
runs with a shortened sample budget (the real arm samples about 20 s), and
the line's keys and types are checked.  The traffic and issue entries of the
GPU arm are keyed to the sources they were measured on; that check is pinned
too: a comment edit keeps a capture, an edit to the code disowns it.
"""
import importlib.util
import io
import json
import os
import sys
from contextlib import redirect_stdout

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    b = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(b)
    return b


def test_reference_arm_prints_one_contract_line(bench, monkeypatch):
    full = bench.cpu_baseline
    monkeypatch.setattr(bench, "cpu_baseline", lambda budget_s=12.0, threads=None: full(0.2, threads))
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference", "--steps", "2", "--warmup", "1"])
    out = io.StringIO()
    with redirect_stdout(out):
        assert bench.main() == 0
    lines = [ln for ln in out.getvalue().splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == "pairs/s"
    assert d["steps"] == 2 and d["warmup"] == 1 and d["n_gpus"] == 1 and d["higher_is_better"] is True
    assert d["value"] > 0 and d["ms_per_step"] > 0 and d["vs_baseline"] is None
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and "pairs" in cb["sample"]
    assert d["e2e"] == dict(value=d["value"], unit="pairs/s", h2d_bytes_per_step=0, d2h_bytes_per_step=0)
    assert "workload" in d["config"]


def test_reference_arm_on_other_ranks_does_no_work(bench, monkeypatch):
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setattr(bench, "cpu_baseline", lambda *a, **k: pytest.fail("rank 1 ran the oracle"))
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference", "--gpus", "2"])
    out = io.StringIO()
    with redirect_stdout(out):
        assert bench.main() == 0
    assert out.getvalue().strip() == ""


def test_captures_are_keyed_to_the_captured_sources(bench, tmp_path, monkeypatch):
    """A capture holds for the sources it names by hash: a comment edit keeps
    it, a code edit disowns it (and then `traffic` is null)."""
    csrc = os.path.join(ROOT, "paper_2603_07327_gb300", "csrc")
    fake = tmp_path / "paper_2603_07327_gb300" / "csrc"
    fake.mkdir(parents=True)
    for name in set(bench.TRANSPORT_SOURCES) | set(bench.DIGITIZER_SOURCES):
        with open(os.path.join(csrc, name)) as f:
            (fake / name).write_text(f.read())
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "TRANSPORT_CAPTURE", dict(bench.TRANSPORT_CAPTURE, dram_bytes_per_pair=8.4,
                                                         sha1=bench._sources_sha1(bench.TRANSPORT_SOURCES)))
    monkeypatch.setattr(bench, "DIGITIZER_TRAFFIC", dict(bench.DIGITIZER_TRAFFIC,
                                                         sha1=bench._sources_sha1(bench.DIGITIZER_SOURCES)))
    assert bench._transport_traffic(1.22e9) == pytest.approx(8.4 * 1.22e9)
    assert bench._digitizer_traffic(1000) == pytest.approx(bench.DIGITIZER_TRAFFIC["bytes_per_single"] * 1000)
    sort_cu = fake / "sort.cu"
    sort_cu.write_text(sort_cu.read_text() + "\n// a comment\n\n/* another */\n")
    assert bench._digitizer_traffic(1000) is not None
    sort_cu.write_text(sort_cu.read_text() + "\nnamespace gpet { constexpr int kUnused = 1; }\n")
    assert bench._digitizer_traffic(1000) is None
    assert bench._transport_traffic(1.22e9) is not None
