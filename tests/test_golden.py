"""The paper's printed tables (tests/golden/, each file citing its table)
against the values the scene generators and the benchmark use."""
import importlib.util
import os

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
GOLDEN = os.path.join(ROOT, "tests", "golden")


def _rows(name):
    out = []
    for line in open(os.path.join(GOLDEN, name)):
        line = line.strip()
        if line and not line.startswith("#"):
            out.append(line.split())
    return out


def test_table1_absorption_coefficients():
    import scenes
    rows = _rows("table1_absorption.txt")
    assert len(rows) == 4
    for r in rows:
        ref, vals = int(r[0]), [float(x) for x in r[1:]]
        assert len(vals) == 8
        assert np.array_equal(np.asarray(scenes.TABLE1_ALPHA[ref], float), vals), ref
    assert sorted(scenes.TABLE1_ALPHA) == sorted(int(r[0]) for r in rows)


def test_table2_times_used_as_context():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    rows = _rows("table2_times.txt")
    assert len(rows) == len(bench.PAPER_TABLE2)
    for r in rows:
        n = int(r[0])
        without = None if r[1] == "X" else float(r[1])
        with_tree = float(r[2])
        assert bench.PAPER_TABLE2[n] == (without, with_tree), n
