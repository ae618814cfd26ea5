"""bench.py's output contract, checked on the CPU through its reference arm
(the oracle timed on the host cores).

One JSON line carrying the keys the measurement contract names, with the
reference arm's own cpu_baseline and a zero-copy e2e entry; under torchrun
with two ranks (rendezvous on 127.0.0.1) rank 0 alone prints the line and
every rank exits 0.
"""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _json_lines(cmd, timeout=900):
    p = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=timeout,
                       env=dict(os.environ, MASTER_ADDR="127.0.0.1"))
    assert p.returncode == 0, p.stderr[-3000:]
    return [json.loads(ln) for ln in p.stdout.splitlines() if ln.startswith("{")]


def _check(d, n_gpus):
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "higher_is_better", "scaling",
              "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["n_gpus"] == n_gpus
    assert d["value"] > 0 and d["higher_is_better"] is True and d["unit"] == "cell-steps/s"
    assert d["config"]["workload"] == "rock256"
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0


def test_reference_arm_one_line():
    lines = _json_lines([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0"])
    assert len(lines) == 1
    _check(lines[0], 1)


def test_reference_arm_two_ranks_rank0_prints():
    pytest.importorskip("torch")
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    lines = _json_lines([sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
                         "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py", "--impl", "reference",
                         "--gpus", "2", "--steps", "1", "--warmup", "0"])
    assert len(lines) == 1
    _check(lines[0], 2)


def _bench_module():
    # imported here, not at collection: importing bench.py sets the
    # process's CUDA connection count, which only its own runs should see
    import importlib
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    return importlib.import_module("bench")


def test_clock_sampler_summary_from_samples():
    """The clocks entry of the line: median SM clock under load, the largest
    maximum clock seen, and every throttle reason seen active at least once
    (a run that saw hw_slowdown, hw_thermal_slowdown or sw_thermal_slowdown
    is not a valid measurement, sw_power_cap is noted); unparsable samples do
    not enter the median."""
    B = _bench_module()
    cs = B.ClockSampler(0)
    na, act = "Not Active", "Active"
    cs.rows = [["2070", "2070", "910.2", na, na, na, act],
               ["1995", "2070", "1013.0", na, na, na, na],
               ["[N/A]", "2070", "[N/A]", na, na, na, na],
               ["2040", "2070", "980.0", na, act, na, na]]
    out = cs.stop()
    assert out["sm_mhz"] == 2040.0 and out["sm_max_mhz"] == 2070.0 and out["samples"] == 4
    assert out["reasons"] == ["hw_thermal_slowdown", "sw_power_cap"]
    empty = B.ClockSampler(0).stop()
    assert empty["sm_mhz"] is None and empty["reasons"] == [] and empty["samples"] == 0


def test_measured_peaks_fallback(tmp_path, monkeypatch):
    """Without MEASURED_PEAKS.json the HBM roofline takes the 6.8 TB/s
    fallback and says so; with it, the file's measured copy bandwidth."""
    B = _bench_module()
    monkeypatch.setattr(B, "ROOT", str(tmp_path))
    assert B.measured_peaks() == (6800.0, "fallback")
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"hbm_gbs": 6663.2}))
    assert B.measured_peaks() == (6663.2, "measured")
