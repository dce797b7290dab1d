"""Host-side helpers (no GPU): bench.py's clock-log summary and host
description, and the binding's marshalling of source tables."""
import importlib.util
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


class _Proc:  # stands in for the nvidia-smi process
    pass


def test_clock_summary_reads_samples_and_reasons(tmp_path):
    b = _bench()
    path = tmp_path / "clocks.csv"
    path.write_text("0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active\n"
                    "0, 1980, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active\n"
                    "0, 2055, 2070, 1200.5, 0x0, Not Active, Not Active, Not Active, Not Active\n"
                    "garbled line\n")
    c = b.ClockSampler(0, str(path))
    c.proc = _Proc()
    s = c.summary()
    assert s["sm_mhz"] == 2055.0 and s["sm_max_mhz"] == 2070.0 and s["samples"] == 3
    assert s["reasons"] == ["sw_power_cap"]


def test_clock_summary_without_samples(tmp_path):
    b = _bench()
    c = b.ClockSampler(0, str(tmp_path / "none.csv"))
    assert c.summary()["reasons"] == ["nvidia-smi unavailable"]
    c.proc = _Proc()
    (tmp_path / "none.csv").write_text("")
    assert c.summary()["reasons"] == ["no samples"]


def test_host_cpu_names_the_architecture():
    b = _bench()
    import platform
    assert b.host_cpu().startswith(platform.machine())


def test_directional_source_arguments_are_checked_before_any_call():
    """The binding's source tables: one axis and one pattern per source,
    omnidirectional when no axis is given (no GPU needed)."""
    import numpy as np
    import pytest
    from paper_1811_05784_gb300 import rt
    S, keep = rt._sources(np.zeros((2, 3)))
    assert S.n == 2 and not S.axis and not S.pattern
    S, keep = rt._sources(np.zeros((2, 3)), [[0, 0, 1], [1, 0, 0]], [0.5, 0.0])
    assert S.n == 2 and S.axis and S.pattern and len(keep) == 3
    S, keep = rt._sources(np.zeros((1, 3)), [[0, 0, 1]])          # pattern defaults to 0
    assert np.asarray(keep[2]).tolist() == [0.0]
    with pytest.raises(ValueError):
        rt._sources(np.zeros((2, 3)), [[0, 0, 1]], [0.1])


def _bench_lines(args, env=None):
    import json
    import subprocess
    import sys
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], capture_output=True, text=True,
                       timeout=600, env=env, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    return [json.loads(x) for x in r.stdout.splitlines() if x.startswith("{")]


def test_reference_arm_prints_the_contract_line():
    """bench.py --impl reference times the oracle on the host on a bounded
    sample and prints one JSON line with the contract's keys."""
    lines = _bench_lines(["--impl", "reference", "--steps", "1", "--warmup", "0", "--cpu-sample-rays", "2000"])
    assert len(lines) == 1
    d = lines[0]
    assert d["impl"] == "reference" and d["value"] > 0 and d["higher_is_better"] is True
    for key in ("metric", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "scaling", "dtype", "data", "config"):
        assert key in d, key
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert "workload" in d["config"]


def test_reference_arm_prints_nothing_on_other_ranks():
    env = dict(os.environ, RANK="1", LOCAL_RANK="1", WORLD_SIZE="2")
    assert _bench_lines(["--impl", "reference", "--steps", "1", "--warmup", "0", "--cpu-sample-rays", "2000"],
                        env=env) == []


def test_profiled_traffic_picks_the_capture_of_the_tree(tmp_path, monkeypatch):
    """A profile may hold one capture per tree; a block without traffic_tree
    was taken on the plain LBVH; a stale source or another configuration
    gives None."""
    bench = _bench()
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "k.md").write_text(
        "# summary\n\ntraffic_bytes_per_trace: 100\ntraffic_config: tail_rays=7\ntraffic_source_sha256_16: abc\n\n"
        "traffic_bytes_per_trace: 80\ntraffic_config: tail_rays=7\ntraffic_source_sha256_16: abc\n"
        "traffic_tree: sah_top\ntraffic_tree_source_sha256_16: 123\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_source_sha", lambda: "abc")
    monkeypatch.setattr(bench, "tree_source_sha", lambda: "123")
    assert bench.profiled_traffic("k.md", 7) == 100.0
    assert bench.profiled_traffic("k.md", 7, "sah_top") == 80.0
    assert bench.profiled_traffic("k.md", 8, "sah_top") is None
    # an SAH-top capture holds for the builder source it was taken with only
    monkeypatch.setattr(bench, "tree_source_sha", lambda: "456")
    assert bench.profiled_traffic("k.md", 7, "sah_top") is None
    assert bench.profiled_traffic("k.md", 7) == 100.0
    monkeypatch.setattr(bench, "kernel_source_sha", lambda: "def")
    assert bench.profiled_traffic("k.md", 7) is None
