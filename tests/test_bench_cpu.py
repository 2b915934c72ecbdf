"""The benchmark's reference arm (the float64 oracle on the host) runs without a GPU
and prints one JSON line with the keys the measurement contract names.  CPU only."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_json_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--workload", "tex2d", "--steps", "1", "--warmup", "0"],
                       capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.strip().startswith("{")]
    assert len(lines) == 1
    line = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
              "cpu_baseline", "e2e"):
        assert k in line, k
    assert line["impl"] == "reference" and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0
    assert "workload" in line["config"]


def _bench():
    import importlib.util
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


def test_traffic_is_reported_only_for_the_captured_sources(monkeypatch):
    """The roofline's `traffic` comes from the committed ncu capture only while the
    kernel's sources hash to the captured ones; after any change it is null."""
    b = _bench()
    entries = json.load(open(os.path.join(ROOT, "profiles", "ncu_traffic.json")))
    e = entries["dense_stochastic_bspline3"]
    monkeypatch.setattr(b, "kernel_hash", lambda w: e["kernel_hash"])
    assert b.ncu_traffic("dense", "bspline3") == e["dram_bytes_per_launch"]
    monkeypatch.setattr(b, "kernel_hash", lambda w: "0" * 16)
    assert b.ncu_traffic("dense", "bspline3") is None
    assert b.ncu_traffic("dense", "no_such_filter") is None


def test_committed_traffic_entries_are_well_formed():
    """Every committed capture names its kernel's workload, a source hash and a summary
    under profiles/ that exists (an entry whose hash no longer matches is simply not
    reported)."""
    b = _bench()
    entries = json.load(open(os.path.join(ROOT, "profiles", "ncu_traffic.json")))
    wl = {"dense_stochastic_bspline3": "dense", "sparse_stochastic_bspline3": "sparse",
          "sparse_e4m3_stochastic_bspline3": "sparse_e4m3", "tex2d_stochastic_bspline3": "tex2d",
          "neural_stochastic_linear": "neural", "aniso_stochastic_ewa": "aniso",
          "dct_stochastic_linear": "dct"}
    assert set(entries) == set(wl)
    for key, e in entries.items():
        assert len(e["kernel_hash"]) == len(b.kernel_hash(wl[key])), key
        assert os.path.exists(os.path.join(ROOT, e["capture"])), e["capture"]
        assert e["dram_bytes_per_launch"] > 0


def test_algorithmic_bytes_per_lookup():
    """Query in + texel(s) fetched + result out, per the workloads' formats."""
    b = _bench()
    assert b.ALGO_BYTES[("dense", "stochastic")] == 12 + 2 + 4
    assert b.ALGO_BYTES[("sparse", "stochastic")] == 12 + 4 + 4
    assert b.ALGO_BYTES[("sparse_e4m3", "stochastic")] == 12 + 1 + 4 + 4
    assert b.ALGO_BYTES[("tex2d", "stochastic")] == 8 + 16 + 16
    assert b.ALGO_BYTES[("neural", "stochastic")] == 12 + 16 + 28
    assert b.stochastic_extra_bytes("dense", "stochastic_catmull_rom_positivized") == 20
    assert b.stochastic_extra_bytes("tex2d", "stochastic_linear") == 40
    assert b.stochastic_extra_bytes("dense", "deterministic_bspline3") is None
