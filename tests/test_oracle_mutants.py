"""The oracle's pins are not tautologies: a copy of the oracle with one
plausible mistake planted (a wrong factor or sign, a dropped term, an
exclusive edge, a misplaced rounding) fails at least one pin of its module's
pin file, and an unchanged copy passes them all.  Each
copy is a package of its own in a temporary directory (with its own build of
rt_oracle.c), first on the path of a separate pytest process."""
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# (name, file in oracle/, exact text, planted text, pin file in tests/)
MUTANTS = [
    ("reflection without its factor 2", "rt_oracle.c",
     "u[k] = u[k] - 2.0 * un * n[k];", "u[k] = u[k] - 1.0 * un * n[k];", "test_oracle_pins.py"),
    ("absorption keeps alpha instead of 1 - alpha", "rt_oracle.c",
     "E[f] = E[f] * (1.0 - al[f]);", "E[f] = E[f] * al[f];", "test_oracle_pins.py"),
    ("Fibonacci rule without the half offset", "rt_oracle.c",
     "fib_dir(int64_t i, int64_t N, double* u) {\n    double g = (3.0 - sqrt(5.0)) / 2.0;\n"
     "    double z = 1.0 - (double)(2 * i + 1) / (double)N;",
     "fib_dir(int64_t i, int64_t N, double* u) {\n    double g = (3.0 - sqrt(5.0)) / 2.0;\n"
     "    double z = 1.0 - (double)(2 * i) / (double)N;", "test_oracle_pins.py"),
    ("triangle edges exclusive", "rt_oracle.c",
     "if (border >= 0.0) {", "if (border > 0.0) {", "test_oracle_pins.py"),
    ("path length not accumulated", "rt_oracle.c",
     "L = L + d1;", "L = d1;", "test_oracle_pins.py"),
    ("image source mirrored without the factor 2", "__init__.py",
     "x = x - 2.0 * (float(nv @ x) - dd) * nv", "x = x - (float(nv @ x) - dd) * nv", "test_oracle_pins.py"),
    ("eq. 19 without air absorption", "__init__.py",
     "out.E[i] = (n / tr.N) * prod * np.exp(-beta * d)", "out.E[i] = (n / tr.N) * prod", "test_oracle_pins.py"),
    ("eq. 19 with alpha instead of 1 - alpha", "__init__.py",
     "prod = prod * (1.0 - alpha[smat[s]])", "prod = prod * alpha[smat[s]]", "test_oracle_pins.py"),
    ("arrival binned by rounding", "__init__.py",
     "b = int(math.floor(isrc.t[i] * fs))", "b = int(round(isrc.t[i] * fs))", "test_oracle_pins.py"),
    ("decay rate without the 1 / 2", "surrogate.py",
     "c * loss[k, f] / (2.0 * V)", "c * loss[k, f] / V", "test_surrogate_oracle.py"),
    ("range margin 20 % instead of 2 %", "surrogate.py",
     "(desc >= lo - 0.02 * span) & (desc <= hi + 0.02 * span)",
     "(desc >= lo - 0.2 * span) & (desc <= hi + 0.2 * span)", "test_surrogate_oracle.py"),
    ("Schroeder integral forwards", "post.py",
     "S = np.cumsum(e[::-1])[::-1]", "S = np.cumsum(e)", "test_post.py"),
    ("C80 ratio inverted", "post.py",
     "10.0 * math.log10(early80 / late80)", "10.0 * math.log10(late80 / early80)", "test_post.py"),
    ("decay time extrapolated to -30 dB", "post.py",
     "return -60.0 / slope", "return -30.0 / slope", "test_post.py"),
    ("T30 over the T20 range", "post.py",
     "out[k, f, 2] = _decay_time(L, b0, fs, -5.0, -35.0)", "out[k, f, 2] = _decay_time(L, b0, fs, -5.0, -25.0)",
     "test_post.py"),
    ("GELU derivative with the wrong sign", "mlp.py",
     "+ x * np.exp(-0.5 * x * x) / np.sqrt(2.0 * np.pi)", "- x * np.exp(-0.5 * x * x) / np.sqrt(2.0 * np.pi)",
     "test_mlp.py"),
    ("prior without the bin average", "prior.py",
     "return np.exp(-R * t) * avg", "return np.exp(-R * t)", "test_prior.py"),
]


def _run_pins(tmp, mutant, pins):
    """Run the pin file `pins` against a copy of oracle/ with `mutant` planted
    (None: an unchanged copy); True if they all pass."""
    work = os.path.join(tmp, ("control_" + pins[:-3]) if mutant is None else "m%d" % MUTANTS.index(mutant))
    pkg = os.path.join(work, "oracle")
    shutil.copytree(os.path.join(ROOT, "oracle"), pkg, ignore=shutil.ignore_patterns("_build", "__pycache__"))
    if mutant is not None:
        _, fname, old, new, _ = mutant
        p = os.path.join(pkg, fname)
        text = open(p).read()
        assert text.count(old) == 1, (mutant[0], "the planted line is no longer in the oracle")
        open(p, "w").write(text.replace(old, new))
    env = dict(os.environ, PYTHONPATH=os.pathsep.join([work, ROOT]))
    r = subprocess.run([sys.executable, "-m", "pytest", os.path.join(ROOT, "tests", pins), "-x", "-q", "-m", "not gpu",
                        "-p", "no:cacheprovider"], cwd=work,
                       env=env, capture_output=True, text=True, timeout=900)
    # the copy, not the repository's oracle, must have been imported
    probe = subprocess.run([sys.executable, "-c", "import oracle; print(oracle.__file__)"], cwd=work, env=env,
                           capture_output=True, text=True, timeout=120)
    assert probe.stdout.strip().startswith(pkg), probe.stdout + probe.stderr
    return r.returncode == 0


def test_every_planted_mistake_fails_a_pin(tmp_path):
    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    pin_files = sorted({m[4] for m in MUTANTS})
    jobs = [(None, f) for f in pin_files] + [(m, m[4]) for m in MUTANTS]
    with cf.ThreadPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 4)) as ex:
        ok = list(ex.map(lambda j: _run_pins(str(tmp_path), j[0], j[1]), jobs))
    controls = [f for (m, f), good in zip(jobs, ok) if m is None and not good]
    assert not controls, f"the unchanged copy fails {controls}"
    survivors = [m[0] for (m, f), good in zip(jobs, ok) if m is not None and good]
    assert not survivors, f"mistakes no pin catches: {survivors}"
