"""The autotuner's choices persist across processes in the file named by
RT_AUTOTUNE_CACHE: a process that tunes a workload class writes its choice,
and a later process uses the stored choice from its first call on."""
import os
import subprocess
import sys

import pytest

pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r"""
import sys
sys.path.insert(0, {root!r})
import scenes
from paper_1811_05784_gb300 import rt
sc = scenes.shoebox(n_rays=20_000, n_bounces=10)
tree = rt.rt_build_tree(sc.vertices, sc.tris, sc.material_id, sc.surface_id)
for k in range({calls}):
    isrc = rt.rt_trace(tree, tail_rays=rt.RT_TAIL_AUTOTUNE, **rt.scene_args(sc))
    print(isrc.block_size, isrc.compaction_period, isrc.stack_entries, flush=True)
"""


def _run(cache, calls):
    env = dict(os.environ, RT_AUTOTUNE_CACHE=str(cache))
    r = subprocess.run([sys.executable, "-c", SCRIPT.format(root=ROOT, calls=calls)], env=env,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    return [tuple(int(x) for x in line.split()) for line in r.stdout.splitlines() if line.strip()]


def test_the_choice_is_written_and_read_back(tmp_path):
    cache = tmp_path / "tune.txt"
    _run(cache, 2 * 9 + 2)                       # 9 candidates, each timed twice, then the choice
    lines = cache.read_text().split()
    assert len(lines) == 2 and lines[0].count("_") >= 5 and int(lines[1]) in range(9)
    # store candidate 5 (128 threads, compaction period 4, 64-entry stack) and start again
    cache.write_text(f"{lines[0]} 5\n")
    first = _run(cache, 1)[0]
    assert first == (128, 4, 64)
