"""Nearest-element queries by the per-ray stack traversal and by the paper's
level-by-level distribution of rays through the tree (Sec. 2.2), through
the C ABI: both give the trace's own hits and distances bit for bit, on the
LBVH and on the paper's median-split tree, and agree with the FP64 oracle
in lockstep."""
import numpy as np
import pytest

import oracle
import scenes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1811_05784_gb300 import rt  # noqa: E402
from test_gpu_trace import _check_lockstep, _performed  # noqa: E402


def _queries(sc, tree):
    """Every query of a trace: origins, directions, surface left, and the
    trace's hit and distance."""
    B, N = sc.n_bounces, sc.n_rays * len(sc.sources)
    ds = torch.empty((B, N, 6), dtype=torch.float32, device="cuda")
    dt = torch.empty((B, N), dtype=torch.float32, device="cuda")
    isrc = rt.rt_trace(tree, debug_state=ds, debug_t=dt, **rt.scene_args(sc))
    hist = isrc.hist.cpu().numpy()
    bq = np.argwhere(_performed(hist))
    surf = np.append(sc.surface_id, -1)
    excl = np.where(bq[:, 0] > 0, surf[hist[np.maximum(bq[:, 0] - 1, 0), bq[:, 1]]], -1).astype(np.int32)
    idx = torch.as_tensor(bq, device="cuda")
    st = ds[idx[:, 0], idx[:, 1]].contiguous()
    return (st[:, :3].contiguous(), st[:, 3:].contiguous(), torch.as_tensor(excl, device="cuda"),
            hist[bq[:, 0], bq[:, 1]], dt[idx[:, 0], idx[:, 1]].cpu().numpy(), bq, ds, dt, hist)


@pytest.mark.parametrize("scene,median", [("theatre", False), ("theatre", True), ("lroom", False),
                                          ("tetra", True)])
def test_both_methods_give_the_traced_hits(scene, median):
    sc = {"theatre": lambda: scenes.theatre(n_rays=50_000, n_bounces=30),
          "lroom": lambda: scenes.lroom(h=0.5, n_rays=20_000, n_bounces=20),
          "tetra": lambda: scenes.tetra(7)}[scene]()
    tree = rt.rt_build_tree(sc.vertices, sc.tris, sc.material_id, sc.surface_id, median=median)
    o, d, ex, h_ref, t_ref, bq, ds, dt, hist = _queries(sc, tree)
    stats = {}
    for method in (rt.RT_NEAREST_STACK, rt.RT_NEAREST_LEVELS):
        hit, t, stats[method] = rt.rt_nearest_hits(tree, o, d, ex, method=method)
        hit, t = hit.cpu().numpy(), t.cpu().numpy()
        assert np.array_equal(hit, h_ref), (method, int((hit != h_ref).sum()))
        assert np.array_equal(t[h_ref >= 0], t_ref[h_ref >= 0]) and np.all(np.isinf(t[h_ref < 0]))
    # the level method opens every box a ray meets before its hit is known
    assert stats[rt.RT_NEAREST_LEVELS][0] >= stats[rt.RT_NEAREST_STACK][0] > 0
    if scene == "tetra":                       # the paper's workload: every query against the oracle
        _check_lockstep(sc, oracle.OracleScene(sc, tree=True), ds.cpu().numpy(), dt.cpu().numpy(), hist)


def test_levels_against_the_oracle_on_sampled_queries():
    """Level-method hits on the L-room (h = 0.5 m) in lockstep with the FP64
    oracle: hit triangle exact but for near ties, distance within 1e-5."""
    sc = scenes.lroom(h=0.5, n_rays=20_000, n_bounces=20)
    tree = rt.rt_build_tree(sc.vertices, sc.tris, sc.material_id, sc.surface_id, median=True)
    o, d, ex, h_ref, t_ref, bq, ds, dt, hist = _queries(sc, tree)
    hit, t, _ = rt.rt_nearest_hits(tree, o, d, ex, method=rt.RT_NEAREST_LEVELS)
    # the level method's answers, placed where the trace's were, then lockstep
    h2 = np.full_like(hist, -1)
    t2 = np.full(dt.shape, np.inf, np.float32)
    h2[bq[:, 0], bq[:, 1]] = hit.cpu().numpy()
    t2[bq[:, 0], bq[:, 1]] = t.cpu().numpy()
    rng = np.random.default_rng(3)
    pick = bq[rng.choice(len(bq), 20_000, replace=False)]
    _check_lockstep(sc, oracle.OracleScene(sc, tree=True), ds.cpu().numpy(), t2, h2, pick)


def test_query_arguments_are_checked():
    sc = scenes.shoebox(n_rays=100, n_bounces=2)
    tree = rt.rt_build_tree(sc.vertices, sc.tris, sc.material_id, sc.surface_id)
    o = torch.zeros((4, 3), device="cuda")
    with pytest.raises(rt.RtError):
        rt.rt_nearest_hits(tree, o, o, method=7)
    with pytest.raises(ValueError):
        rt.rt_nearest_hits(tree, o[:, :2].contiguous(), o)
