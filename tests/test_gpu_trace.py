"""GPU path vs the FP64 oracle (parity), through the C ABI.

Tolerances (stated by the specification of the method's float32 path):
  hit triangle / reflection sequence   bit-exact, except rays the oracle
                                       reports as ambiguous (near ties, near
                                       edges), which are counted
  hit distance                         1e-5 relative
  band energies                        1e-4 relative
  RIR histograms                       1e-4 relative L2
  image-source positions (FP64)        1e-9 relative
"""
import math

import numpy as np
import pytest

import oracle
import scenes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1811_05784_gb300 import rt  # noqa: E402

TOL_T, TOL_E, TOL_RIR, TOL_POS = 1e-5, 1e-4, 1e-4, 1e-9


def _tree(sc):
    return rt.rt_build_tree(sc.vertices, sc.tris, sc.material_id, sc.surface_id)


def _trace(sc, tree=None, **kw):
    tree = tree or _tree(sc)
    args = rt.scene_args(sc)
    args.update(kw)
    return tree, rt.rt_trace(tree, **args)


def _gpu_as_oracle_trace(sc, isrc):
    """The GPU's sequences and crossings in the oracle's TraceResult layout."""
    n, B = isrc.n_traced, isrc.n_bounces
    hist = isrc.hist.cpu().numpy().T.copy()
    z = np.zeros(0)
    return oracle.TraceResult(np.zeros(n, np.int32), np.arange(n), hist, np.zeros((n, B)), z, z,
                              np.full(n, B, np.int32), np.zeros(n, np.int32),
                              isrc.rec_rcv.cpu().numpy(), isrc.rec_ray.cpu().numpy().astype(np.int64),
                              isrc.rec_order.cpu().numpy(), isrc.rec_length.cpu().numpy().astype(np.float64),
                              z, np.zeros((0, 3)), np.zeros((0, 3)), sc.n_rays, B)


def _gpu_is_table(sc, isrc):
    """{(rcv, surface sequence): (n, pos, dist, time, energy)} from the GPU output."""
    hist = isrc.hist.cpu().numpy()
    rep = isrc.rep_ray.cpu().numpy()
    order = isrc.order.cpu().numpy()
    rcv = isrc.rcv.cpu().numpy()
    cnt = isrc.count.cpu().numpy()
    pos, dist, tim, en = (x.cpu().numpy() for x in (isrc.pos, isrc.dist, isrc.time, isrc.energy))
    out = {}
    for k in range(isrc.n):
        seq = tuple(int(sc.surface_id[hist[j, rep[k]]]) for j in range(order[k]))
        key = (int(rcv[k]), seq)
        assert key not in out, "duplicate image source"
        out[key] = (int(cnt[k]), pos[k], dist[k], tim[k], en[k])
    return out


#: near-edge band for free-running comparisons: float32 trajectories drift from
#: the FP64 ones by a few ulps per bounce, so decisions within this band of an
#: edge may legitimately go either way
EPS_FREE = 2e-5


def _performed(hist):
    p = np.ones_like(hist, dtype=bool)
    p[1:] = hist[:-1] >= 0
    return p


def _lockstep(sc, osc, ds, dt, hist, pick=None):
    """The oracle answers GPU queries from the GPU's own float32 state.

    Returns (b, q, oracle tri, oracle delta, ambiguous, gpu tri, gpu delta)."""
    bq = np.argwhere(_performed(hist)) if pick is None else pick
    st = ds[bq[:, 0], bq[:, 1]].astype(np.float64)
    excl = np.where(bq[:, 0] > 0, hist[np.maximum(bq[:, 0] - 1, 0), bq[:, 1]], -1).astype(np.int32)
    tri, d1, d2, amb = osc.nearest(st[:, :3], st[:, 3:], exclude=excl)
    return bq, tri, d1, amb, hist[bq[:, 0], bq[:, 1]], dt[bq[:, 0], bq[:, 1]].astype(np.float64)


def _check_lockstep(sc, osc, ds, dt, hist, pick=None):
    bq, tri, d1, amb, g_tri, g_t = _lockstep(sc, osc, ds, dt, hist, pick)
    diff = (tri != g_tri) & ~amb
    assert diff.sum() == 0, f"{diff.sum()} unexplained differences of {len(bq)} queries"
    same = (tri >= 0) & (tri == g_tri)
    assert same.sum() > 0.9 * (tri >= 0).sum()
    # distance: |dt| <= 1e-5 * t (relative) + 1e-6 * |o|max (absolute), the
    # absolute part being what float32 coordinates resolve at the ray origin:
    # 50 micrometres at the theatre's 50 m radius, 20 at the L-room's 20 m
    oscale = np.abs(ds[bq[same, 0], bq[same, 1], :3]).max(1).astype(np.float64)
    bound = TOL_T * d1[same] + 0.1 * TOL_T * oscale
    rel = np.abs(g_t[same] - d1[same]) / (d1[same] + 0.1 * oscale)
    if not (np.abs(g_t[same] - d1[same]) <= bound).all():
        v = sc.vertices[sc.tris[tri[same]]]
        n = np.cross(v[:, 1] - v[:, 0], v[:, 2] - v[:, 0])
        n /= np.linalg.norm(n, axis=1, keepdims=True)
        st = ds[bq[same, 0], bq[same, 1]].astype(np.float64)
        cos = np.abs(np.einsum("ij,ij->i", n, st[:, 3:]))
        w = np.argsort(-rel)[:8]
        msg = "; ".join(f"t={d1[same][i]:.6g} rel={rel[i]:.2e} abs bound={bound[i]:.2e} cos={cos[i]:.2e} "
                        f"|o|={np.abs(st[i, :3]).max():.3g}"
                        for i in w)
        raise AssertionError("distance: " + msg)
    return bq, amb


def _length_bound(sc, L_ora, n_hits):
    """1e-5 relative, plus the float32 restart offset of the kernel: after
    each hit the next segment starts 2^-21 max|p| before the hit point along
    the incoming ray (p the hit point), so every hit may add up to that much
    to the summed length; the bound takes twice the scene's largest
    coordinate per hit (at the theatre's 50 m: 48 micrometres per hit)."""
    X = max(float(np.abs(sc.vertices).max()), 1e-3)
    return TOL_T * L_ora + n_hits * 2.0 ** -20 * X


#: free-running float32 and FP64 paths with the same triangles still drift
#: apart: a hit point moves by the drift over the cosine of the incidence, so
#: grazing reflections amplify it.  This share of the rays must meet the
#: per-query bound, and every ray this relative bound.
FREE_LENGTH_SHARE, FREE_LENGTH_REL = 0.999, 1e-3


def _check_lengths(sc, L_gpu, L_ora, n_hits):
    """Free-running path lengths of rays with the oracle's triangle sequence."""
    err = np.abs(L_gpu - L_ora)
    ok = err <= _length_bound(sc, L_ora, n_hits)
    assert ok.mean() >= FREE_LENGTH_SHARE, (ok.mean(), int((~ok).sum()))
    rel = err / np.maximum(L_ora, 1e-9)
    assert (rel[L_ora > 0] <= FREE_LENGTH_REL).all() and (L_gpu[L_ora == 0] == 0).all(), rel.max()
    return err


def _check_compensated_lengths(isrc, dt, hist):
    """The kernel's path length is the compensated float32 sum of its own
    segment lengths: within 4 ulps of their FP64 sum on every ray."""
    seg = np.where(hist >= 0, dt, 0.0).astype(np.float64).sum(0)
    L = isrc.ray_length.cpu().numpy().astype(np.float64)
    assert (np.abs(L - seg) <= 4 * np.spacing(np.float32(np.maximum(seg, 1e-30))).astype(np.float64)).all()


def _check_free_running(sc, hist, ids, tr, isrc=None):
    """Free-running float32 vs FP64 trajectories: the reflection sequences
    (surface ids) agree up to each ray's first ambiguous bounce.  Triangle
    ids inside one surface may differ once the trajectories have drifted by
    more than the near-edge band; those are counted, not failed.  With the
    GPU result `isrc`: rays whose whole surface sequence equals the oracle's
    carry its band energies (1e-4), and rays with its exact triangle
    sequence (no ambiguity) its hit counts and path lengths."""
    surf = np.append(sc.surface_id, -1)            # index -1 -> -1
    agree = tri_diff = 0
    same_tri = np.zeros(len(ids), bool)
    same_surf = np.zeros(len(ids), bool)
    for k, q in enumerate(ids):
        upto = tr.first_amb[k]
        g, o = hist[:upto, q], tr.hist[k, :upto]
        assert np.array_equal(surf[g], surf[o]), (q, g, o)
        tri_diff += int((g != o).any())
        agree += upto
        same_tri[k] = upto == tr.B and np.array_equal(hist[:, q], tr.hist[k])
        same_surf[k] = np.array_equal(surf[hist[:, q]], surf[tr.hist[k]])
    assert agree > 0.5 * len(ids) * tr.B
    assert tri_diff <= 0.01 * len(ids), tri_diff
    if isrc is not None:
        assert same_surf.mean() > 0.9, same_surf.mean()
        assert same_tri.sum() > 0.2 * len(ids), same_tri.mean()
        q = np.asarray(ids)
        E = isrc.ray_energy.cpu().numpy().astype(np.float64)[q]
        L = isrc.ray_length.cpu().numpy().astype(np.float64)[q]
        nh = isrc.ray_hits.cpu().numpy()[q]
        assert np.abs(E[same_surf] / tr.E[same_surf] - 1).max() < TOL_E
        assert np.array_equal(nh[same_tri], tr.n_hits[same_tri])
        _check_lengths(sc, L[same_tri], tr.L[same_tri], tr.n_hits[same_tri])
    return tri_diff


# ---------------------------------------------------------------------------
def test_fibonacci_directions_bitexact():
    N = 100_003
    sc = scenes.shoebox(n_rays=N, n_bounces=1)
    ds = torch.empty((1, N, 6), dtype=torch.float32, device="cuda")
    _trace(sc, debug_state=ds)
    torch.cuda.synchronize()
    d = ds[0, :, 3:].cpu().numpy().astype(np.float64)
    ref = oracle.fibonacci(N)
    mism = int((d != ref).any(1).sum())
    assert mism == 0, f"{mism} directions differ"
    o = ds[0, :, :3].cpu().numpy().astype(np.float64)
    assert np.array_equal(o, np.broadcast_to(sc.sources[0], o.shape))


@pytest.mark.parametrize("n_rays", [10_000, 4097])
def test_shoebox_trace_parity(n_rays):
    sc = scenes.shoebox(n_rays=n_rays)
    B = sc.n_bounces
    ds_t = torch.empty((B, n_rays, 6), dtype=torch.float32, device="cuda")
    dt_t = torch.empty((B, n_rays), dtype=torch.float32, device="cuda")
    tree, isrc = _trace(sc, debug_t=dt_t, debug_state=ds_t)
    ds, dt = ds_t.cpu().numpy(), dt_t.cpu().numpy()
    hist = isrc.hist.cpu().numpy()
    osc = oracle.OracleScene(sc, tree=False)
    # lockstep: every query, hit triangle exact (ambiguous excepted), distance 1e-5
    bq, amb = _check_lockstep(sc, osc, ds, dt, hist)
    assert amb.mean() < 0.01
    # lockstep crossings of every segment
    seg = np.where(hist[bq[:, 0], bq[:, 1]] >= 0, dt[bq[:, 0], bq[:, 1]], np.inf)
    st = ds[bq[:, 0], bq[:, 1]].astype(np.float64)
    k, r, margin = oracle.crossings(sc, st[:, :3], st[:, 3:], seg)
    want = {(int(bq[i, 1]), int(bq[i, 0]), int(rr)) for i, rr, mg in zip(k, r, margin) if abs(mg) > 1e-5}
    edge = {(int(bq[i, 1]), int(bq[i, 0]), int(rr)) for i, rr, mg in zip(k, r, margin) if abs(mg) <= 1e-5}
    got = set(zip(isrc.rec_ray.cpu().numpy().tolist(), isrc.rec_order.cpu().numpy().tolist(),
                  isrc.rec_rcv.cpu().numpy().tolist()))
    assert want <= got and not (got - want - edge)
    # free running from the source: sequences equal up to the first ambiguity
    tr = oracle.trace(osc, eps_edge_rel=EPS_FREE)
    ok = tr.first_amb == B
    assert ok.mean() > 0.95
    assert np.array_equal(hist.T[ok], tr.hist[ok])
    # energies and path lengths of rays with identical sequences
    E = isrc.ray_energy.cpu().numpy().astype(np.float64)
    assert np.abs(E[ok] / tr.E[ok] - 1).max() < TOL_E
    L = isrc.ray_length.cpu().numpy().astype(np.float64)
    assert np.abs(L[ok] / tr.L[ok] - 1).max() < TOL_T
    assert (isrc.ray_hits.cpu().numpy() == B).all()          # closed room, no escapes
    assert isrc.queries == n_rays * B
    assert isrc.hash_collisions == 0


def test_dedup_beyond_the_direct_prefix_path():
    """More than 983,040 records (256 sort tiles): the dedup sort finds its
    digit offsets by decoupled look-back; the grouping must still equal the
    oracle's grouping of the same crossings."""
    sc = scenes.shoebox(n_rays=400_000, n_bounces=30, radius=1.5)
    tree, isrc = _trace(sc)
    assert isrc.n_records > 983_040, isrc.n_records
    ref = oracle.image_sources(sc, _gpu_as_oracle_trace(sc, isrc))
    got = _gpu_is_table(sc, isrc)
    assert len(got) == len(ref.n)
    for k in range(len(ref.n)):
        n, pos, dist, tim, en = got[(int(ref.rcv[k]), ref.seq[k])]
        assert n == ref.n[k]
        assert np.allclose(en, ref.E[k], rtol=1e-12, atol=0)
    assert isrc.hash_collisions == 0


def test_shoebox_image_sources_and_rir_parity():
    sc = scenes.shoebox()
    tree, isrc = _trace(sc)
    # (1) dedup + FP64 reconstruction: exactly the oracle's grouping of the GPU's own crossings
    ref = oracle.image_sources(sc, _gpu_as_oracle_trace(sc, isrc))
    got = _gpu_is_table(sc, isrc)
    assert len(got) == len(ref.n)
    for k in range(len(ref.n)):
        key = (int(ref.rcv[k]), ref.seq[k])
        n, pos, dist, tim, en = got[key]
        assert n == ref.n[k]
        assert np.abs(pos - ref.pos[k]).max() <= TOL_POS * max(1.0, np.abs(ref.pos[k]).max())
        assert dist == pytest.approx(ref.d[k], rel=TOL_POS)
        assert tim == pytest.approx(ref.t[k], rel=TOL_POS)
        assert np.allclose(en, ref.E[k], rtol=1e-12, atol=0)
    # (2) histogram stage alone
    resp = rt.rt_rir(isrc, sc.fs, duration=0.5)
    H = resp.download().astype(np.float64)
    Href = oracle.rir(ref, 1, sc.fs, duration=0.5)
    assert np.linalg.norm(H - Href) / np.linalg.norm(Href) < 1e-6
    # (3) end to end against the free-running oracle
    tr = oracle.trace(oracle.OracleScene(sc, tree=False))
    Ho = oracle.rir(oracle.image_sources(sc, tr), 1, sc.fs, duration=0.5)
    assert np.linalg.norm(H - Ho) / np.linalg.norm(Ho) < TOL_RIR


def test_paper_shoebox_range_and_air():
    """Sec. 3.2 setup: Table 1 materials, ISO air, eq. 13 range."""
    sc = scenes.paper_shoebox(n_rays=20_000)
    tree, isrc = _trace(sc)
    tr = oracle.trace(oracle.OracleScene(sc, tree=False), eps_edge_rel=EPS_FREE)
    hist = isrc.hist.cpu().numpy().T
    ok = tr.first_amb == tr.B
    assert np.array_equal(hist[ok], tr.hist[ok])
    assert (isrc.rec_length.cpu().numpy() <= sc.max_distance * (1 + 1e-6)).all()
    ref = oracle.image_sources(sc, _gpu_as_oracle_trace(sc, isrc))
    got = _gpu_is_table(sc, isrc)
    for k in range(len(ref.n)):
        n, pos, dist, tim, en = got[(int(ref.rcv[k]), ref.seq[k])]
        assert n == ref.n[k]
        assert np.allclose(en, ref.E[k], rtol=1e-12, atol=0)
    H = rt.rt_rir(isrc, sc.fs).download().astype(np.float64)
    Ho = oracle.rir(oracle.image_sources(sc, tr), 1, sc.fs, duration=H.shape[-1] / sc.fs)
    assert np.linalg.norm(H - Ho) / np.linalg.norm(Ho) < TOL_RIR


@pytest.mark.parametrize("h,n_rays", [(0.5, 50_000), (0.125, 1_000_000)])
def test_lroom_watertight_energy_conserved(h, n_rays):
    sc = scenes.lroom(h=h, n_rays=n_rays, n_bounces=50, alpha=np.zeros((4, 8)))
    tree, isrc = _trace(sc)
    hits = isrc.ray_hits.cpu().numpy()
    assert (hits == 50).all(), f"{(hits < 50).sum()} rays escaped a closed room"
    E = isrc.ray_energy.cpu().numpy().astype(np.float64).sum(0)
    assert np.allclose(E, 1.0, rtol=1e-6)


def test_lroom_subset_against_oracle_tree():
    sc = scenes.lroom(n_rays=1_000_000, n_bounces=50)      # 102,400 triangles
    B, N = sc.n_bounces, sc.n_rays
    ds_t = torch.empty((B, N, 6), dtype=torch.float32, device="cuda")
    dt_t = torch.empty((B, N), dtype=torch.float32, device="cuda")
    tree, isrc = _trace(sc, debug_t=dt_t, debug_state=ds_t)
    hist = isrc.hist.cpu().numpy()
    _check_compensated_lengths(isrc, dt_t.cpu().numpy(), hist)
    osc = oracle.OracleScene(sc, tree=True)
    rng = np.random.default_rng(11)
    # lockstep on 20,000 sampled queries
    perf = np.argwhere(_performed(hist))
    pick = perf[rng.choice(len(perf), 20_000, replace=False)]
    _check_lockstep(sc, osc, ds_t.cpu().numpy(), dt_t.cpu().numpy(), hist, pick)
    # free running on a seeded 4096-ray subset: reflection (surface) sequences
    ids = np.sort(rng.choice(N, 4096, replace=False))
    tr = oracle.trace(osc, ray_ids=ids, eps_edge_rel=EPS_FREE)
    _check_free_running(sc, hist, ids, tr, isrc)


@pytest.mark.parametrize("level", [5, 9])
def test_tetra_scaling_workload_one_iteration(level):
    """The paper's scaling workload (Sec. 2.2, Table 2): one iteration with
    N = M rays from the centre of the refined unit tetrahedron.  Every query
    agrees with the oracle (brute force at 4,096 faces, its tree on a sample
    of 20,000 queries at 1,048,576 faces) except near-ties, and a closed mesh
    lets no ray escape."""
    sc = scenes.tetra(level)
    M = len(sc.tris)
    assert M == 4 * 4 ** level and sc.n_rays == M and sc.n_bounces == 1
    ds_t = torch.empty((1, M, 6), dtype=torch.float32, device="cuda")
    dt_t = torch.empty((1, M), dtype=torch.float32, device="cuda")
    tree, isrc = _trace(sc, debug_state=ds_t, debug_t=dt_t)
    hist = isrc.hist.cpu().numpy()
    assert isrc.queries == M and (hist >= 0).all()
    osc = oracle.OracleScene(sc, tree=level > 5)
    pick = None
    if level > 5:
        rng = np.random.default_rng(7)
        pick = np.stack([np.zeros(20_000, np.int64), np.sort(rng.choice(M, 20_000, replace=False))], 1)
    _check_lockstep(sc, osc, ds_t.cpu().numpy(), dt_t.cpu().numpy(), hist, pick)


def _moved_listeners(sc):
    """The scene with its receivers moved and one added (all of source 0)."""
    import copy
    m = copy.copy(sc)
    lo, hi = sc.vertices.min(0), sc.vertices.max(0)
    g = np.random.default_rng(3)
    n = len(sc.rcv_center) + 1
    m.rcv_center = g.uniform(lo + 0.25 * (hi - lo), hi - 0.25 * (hi - lo), (n, 3)).astype(np.float32)
    m.rcv_radius = g.uniform(0.3, 1.5, n).astype(np.float32)
    m.rcv_source = np.zeros(n, np.int32)
    return m


def _same_trace(a, b):
    for name in ("hist", "ray_energy", "ray_length", "ray_hits", "rcv", "order", "count", "rep_ray", "pos",
                 "dist", "time", "energy"):
        assert torch.equal(getattr(a, name), getattr(b, name)), name
    assert a.n == b.n and a.n_records == b.n_records and a.queries == b.queries


@pytest.mark.parametrize("scene,tail", [("shoebox", 0), ("shoebox", -1), ("theatre", 0)])
def test_replay_with_moved_listeners_equals_a_full_trace(scene, tail):
    """A moved listener: the recorded paths of an earlier trace replayed
    (only the recorded triangle re-tested per query) give exactly what a
    full trace with the new receivers gives."""
    sc = scenes.shoebox(n_rays=20_000, n_bounces=25) if scene == "shoebox" else scenes.theatre(n_rays=100_000)
    tree, first = _trace(sc, tail_rays=tail)
    moved = _moved_listeners(sc)
    kw = rt.scene_args(moved)
    full = rt.rt_trace(tree, tail_rays=tail, **kw)
    replay = rt.rt_trace(tree, tail_rays=tail, replay=first, **kw)
    _same_trace(full, replay)
    assert replay.n > 0
    # replaying the replay (the same rays) again changes nothing
    _same_trace(full, rt.rt_trace(tree, tail_rays=tail, replay=replay.hist.contiguous(), **kw))


def test_replay_reports_foreign_histories():
    sc = scenes.shoebox(n_rays=2_000, n_bounces=5)
    tree, first = _trace(sc)
    bad = first.hist.clone()
    bad[2, 17] = len(sc.tris) + 5                     # an id outside this mesh
    with pytest.raises(rt.RtError, match="outside the tree"):
        rt.rt_trace(tree, replay=bad, **rt.scene_args(sc))


@pytest.mark.parametrize("scene", ["shoebox", "lroom", "theatre"])
def test_median_split_tree_gives_the_same_trace(scene):
    """The paper's median-split tree (Sec. 2.2) built on the device: a trace
    over it equals the trace over the LBVH bit for bit (the nearest hit does
    not depend on the tree), and its depth is ceil(log2 M) or one more."""
    sc = {"shoebox": lambda: scenes.shoebox(n_rays=20_000, n_bounces=20),
          "lroom": lambda: scenes.lroom(h=0.5, n_rays=50_000, n_bounces=20),
          "theatre": lambda: scenes.theatre(n_rays=100_000)}[scene]()
    lbvh = rt.rt_build_tree(sc.vertices, sc.tris, sc.material_id, sc.surface_id)
    med = rt.rt_build_tree(sc.vertices, sc.tris, sc.material_id, sc.surface_id, median=True)
    M = len(sc.tris)
    assert med.info()["depth"] in (math.ceil(math.log2(M)), math.ceil(math.log2(M)) + 1)
    a = rt.rt_trace(lbvh, **rt.scene_args(sc))
    b = rt.rt_trace(med, **rt.scene_args(sc))
    _same_trace(a, b)


def _cost(tree, sc):
    """Nodes and triangles per query of a trace over `tree` (counting pass)."""
    n = sc.n_rays * len(sc.sources)
    cost = torch.zeros((sc.n_bounces, n, 2), dtype=torch.int32, device="cuda")
    isrc = rt.rt_trace(tree, debug_cost=cost, **rt.scene_args(sc))
    c = cost.double().sum((0, 1)).cpu().numpy() / isrc.queries
    return isrc, c


@pytest.mark.parametrize("scene", ["shoebox", "paper_shoebox", "tetra", "lroom", "theatre"])
def test_sah_top_tree_gives_the_same_trace(scene):
    """The LBVH with SAH top levels (rt_build_tree_sah): a trace over it equals
    the trace over the plain LBVH bit for bit, and on the scenes of uneven
    triangle density it visits fewer nodes per query (measured: theatre 16.3
    against 19.6, L-room 12.6 against 14.7)."""
    sc = {"shoebox": lambda: scenes.shoebox(n_rays=20_000, n_bounces=20),
          "paper_shoebox": lambda: scenes.paper_shoebox(n_rays=20_000),
          "tetra": lambda: scenes.tetra(7),
          "lroom": lambda: scenes.lroom(n_rays=100_000, n_bounces=20),
          "theatre": lambda: scenes.theatre(n_rays=100_000)}[scene]()
    lbvh = rt.rt_build_tree(sc.vertices, sc.tris, sc.material_id, sc.surface_id)
    sah = rt.rt_build_tree(sc.vertices, sc.tris, sc.material_id, sc.surface_id, sah=True)
    assert sah.info()["n_tris"] == len(sc.tris) and sah.info()["depth"] <= 42
    a, ca = _cost(lbvh, sc)
    b, cb = _cost(sah, sc)
    _same_trace(a, b)
    if scene in ("lroom", "theatre"):
        assert cb[0] < 0.95 * ca[0], (ca, cb)


def test_sah_top_tree_lockstep_against_the_oracle():
    """Queries over the SAH-top tree against the FP64 oracle directly: every
    query of the paper's scaling workload at 4,096 faces (brute force), and
    20,000 sampled queries plus 2,048 free-running rays of the closed L-room
    (102,400 triangles, 50 bounces)."""
    sc = scenes.tetra(5)
    M = len(sc.tris)
    tree = rt.rt_build_tree(sc.vertices, sc.tris, sc.material_id, sc.surface_id, sah=True)
    ds_t = torch.empty((1, M, 6), dtype=torch.float32, device="cuda")
    dt_t = torch.empty((1, M), dtype=torch.float32, device="cuda")
    _, isrc = _trace(sc, tree, debug_state=ds_t, debug_t=dt_t)
    hist = isrc.hist.cpu().numpy()
    assert isrc.queries == M and (hist >= 0).all()
    _check_lockstep(sc, oracle.OracleScene(sc), ds_t.cpu().numpy(), dt_t.cpu().numpy(), hist)
    sc = scenes.lroom(n_rays=1_000_000, n_bounces=50)
    B, N = sc.n_bounces, sc.n_rays
    tree = rt.rt_build_tree(sc.vertices, sc.tris, sc.material_id, sc.surface_id, sah=True)
    ds_t = torch.empty((B, N, 6), dtype=torch.float32, device="cuda")
    dt_t = torch.empty((B, N), dtype=torch.float32, device="cuda")
    _, isrc = _trace(sc, tree, debug_t=dt_t, debug_state=ds_t)
    hist = isrc.hist.cpu().numpy()
    osc = oracle.OracleScene(sc, tree=True)
    rng = np.random.default_rng(13)
    perf = np.argwhere(_performed(hist))
    pick = perf[rng.choice(len(perf), 20_000, replace=False)]
    _check_lockstep(sc, osc, ds_t.cpu().numpy(), dt_t.cpu().numpy(), hist, pick)
    ids = np.sort(rng.choice(N, 2048, replace=False))
    tr = oracle.trace(osc, ray_ids=ids, eps_edge_rel=EPS_FREE)
    _check_free_running(sc, hist, ids, tr, isrc)


def test_sah_top_and_median_flags_exclude_each_other():
    sc = scenes.shoebox(n_rays=100, n_bounces=2)
    with pytest.raises(ValueError):
        rt.rt_build_tree(sc.vertices, sc.tris, sc.material_id, sc.surface_id, median=True, sah=True)


def test_theatre_lockstep_and_free_running():
    sc = scenes.theatre()                                    # 436,796 triangles, 1M rays, 30 bounces
    B, N = sc.n_bounces, sc.n_rays
    ds_t = torch.empty((B, N, 6), dtype=torch.float32, device="cuda")
    dt_t = torch.empty((B, N), dtype=torch.float32, device="cuda")
    tree, isrc = _trace(sc, debug_state=ds_t, debug_t=dt_t)
    hist = isrc.hist.cpu().numpy()
    _check_compensated_lengths(isrc, dt_t.cpu().numpy(), hist)
    osc = oracle.OracleScene(sc, tree=True)
    rng = np.random.default_rng(5)
    perf = np.argwhere(_performed(hist))
    assert len(perf) == isrc.queries
    pick = perf[rng.choice(len(perf), 20_000, replace=False)]
    _check_lockstep(sc, osc, ds_t.cpu().numpy(), dt_t.cpu().numpy(), hist, pick)
    ids = np.sort(rng.choice(N, 4096, replace=False))
    tr = oracle.trace(osc, ray_ids=ids, eps_edge_rel=EPS_FREE)
    _check_free_running(sc, hist, ids, tr, isrc)


def test_deterministic():
    sc = scenes.shoebox(n_rays=20_000, n_bounces=20)
    tree = _tree(sc)
    a = rt.rt_trace(tree, **rt.scene_args(sc))
    b = rt.rt_trace(tree, **rt.scene_args(sc))
    assert torch.equal(a.hist, b.hist)
    assert a.n == b.n
    for x, y in ((a.pos, b.pos), (a.energy, b.energy), (a.count, b.count)):
        assert torch.equal(x, y)
    ha = rt.rt_rir(a, sc.fs).download()
    hb = rt.rt_rir(b, sc.fs).download()
    assert np.array_equal(ha, hb)


@pytest.mark.parametrize("tail,period,stack", [(-1, 1, 0), (1, 1, 0), (5000, 1, 0), (-1, 4, 0), (5000, 3, 48),
                                               (-1, 7, 48), (200_000, 1, 48)])
def test_tail_mode_matches_per_bounce_launches(tail, period, stack):
    """Finishing the last bounces in one launch, compacting every few
    bounces instead of every bounce, or a shorter traversal stack changes
    nothing per ray."""
    sc = scenes.theatre(n_rays=200_000, n_bounces=30)
    tree = _tree(sc)
    assert tree.info()["depth"] <= 32          # the 48-entry stack serves this tree
    a = rt.rt_trace(tree, tail_rays=-1, **rt.scene_args(sc))
    b = rt.rt_trace(tree, tail_rays=tail, compaction_period=period, stack_entries=stack, **rt.scene_args(sc))
    assert b.compaction_period == period and b.stack_entries == (48 if stack == 48 else 64)
    assert torch.equal(a.hist, b.hist)
    assert torch.equal(a.ray_energy, b.ray_energy) and torch.equal(a.ray_length, b.ray_length)
    assert a.queries == b.queries and a.n == b.n and a.n_records == b.n_records
    assert torch.equal(a.energy, b.energy) and torch.equal(a.count, b.count)


def test_compaction_period_lockstep_against_the_oracle():
    """Every query of an L-room trace run with a compaction period of 3 and
    the 48-entry stack, in lockstep with the FP64 oracle."""
    sc = scenes.lroom(h=0.5, n_rays=30_000, n_bounces=20)
    B, N = sc.n_bounces, sc.n_rays
    ds_t = torch.empty((B, N, 6), dtype=torch.float32, device="cuda")
    dt_t = torch.empty((B, N), dtype=torch.float32, device="cuda")
    tree, isrc = _trace(sc, debug_t=dt_t, debug_state=ds_t, tail_rays=-1, compaction_period=3, stack_entries=48)
    assert isrc.compaction_period == 3 and isrc.stack_entries == 48
    hist = isrc.hist.cpu().numpy()
    _check_lockstep(sc, oracle.OracleScene(sc, tree=True), ds_t.cpu().numpy(), dt_t.cpu().numpy(), hist)
    _check_compensated_lengths(isrc, dt_t.cpu().numpy(), hist)


def test_shards_add_up():
    sc = scenes.shoebox(n_rays=30_000, n_bounces=20)
    tree = _tree(sc)
    full = rt.rt_trace(tree, **rt.scene_args(sc))
    Hf = rt.rt_rir(full, sc.fs, duration=0.4).download().astype(np.float64)
    Hs = 0
    for b0, cnt in ((0, 10_000), (10_000, 12_345), (22_345, 7_655)):
        part = rt.rt_trace(tree, ray_begin=b0, ray_count=cnt, **rt.scene_args(sc))
        Hs = Hs + rt.rt_rir(part, sc.fs, duration=0.4).download().astype(np.float64)
    assert np.linalg.norm(Hs - Hf) / np.linalg.norm(Hf) < 1e-6


def test_device_and_host_mesh_agree():
    sc = scenes.lroom(h=0.5, n_rays=20_000, n_bounces=20)
    t_host, a = _trace(sc)
    dev = [torch.as_tensor(x).cuda() for x in (sc.vertices, sc.tris, sc.material_id, sc.surface_id)]
    t_dev = rt.rt_build_tree(*dev)
    b = rt.rt_trace(t_dev, **rt.scene_args(sc))
    assert torch.equal(a.hist, b.hist)
    assert t_host.info() == t_dev.info()


def test_record_capacity_retry():
    # a receiver that fills most of the room: far more crossings than the first buffer
    sc = scenes.shoebox(receiver=(5.0, 3.5, 1.5), radius=1.4, n_rays=200_000, n_bounces=40)
    tree, isrc = _trace(sc)
    assert isrc.n_records > 2 * sc.n_rays
    assert int(isrc.count.sum()) == isrc.n_records
    assert isrc.hash_collisions == 0


def test_errors_are_reported():
    sc = scenes.shoebox(n_rays=100, n_bounces=4)
    tree = _tree(sc)
    args = rt.scene_args(sc)
    for bad in (dict(n_rays=0), dict(n_bounces=0), dict(c=0.0), dict(ray_begin=100),
                dict(band_absorption=np.full((1, 8), 1.5)), dict(rcv_source=[3])):
        kw = dict(args)
        kw.update(bad)
        with pytest.raises(rt.RtError) as e:
            rt.rt_trace(tree, **kw)
        assert e.value.status == rt.RT_ERR_INVALID_ARG, bad
    tris = sc.tris.copy()
    tris[0, 2] = tris[0, 1]
    with pytest.raises(rt.RtError) as e:
        rt.rt_build_tree(sc.vertices, tris, sc.material_id, sc.surface_id)
    assert e.value.status == rt.RT_ERR_DEGENERATE_MESH
    tris = sc.tris.copy()
    tris[3, 0] = 10_000
    with pytest.raises(rt.RtError) as e:
        rt.rt_build_tree(sc.vertices, tris, sc.material_id, sc.surface_id)
    assert e.value.status == rt.RT_ERR_INVALID_ARG
    v = sc.vertices.copy()
    v[0, 0] = np.nan
    with pytest.raises(rt.RtError) as e:
        rt.rt_build_tree(v, sc.tris, sc.material_id, sc.surface_id)
    assert e.value.status == rt.RT_ERR_INVALID_ARG
    mixed = sc.material_id.copy()
    mixed[1] = 1
    with pytest.raises(rt.RtError) as e:
        rt.rt_build_tree(sc.vertices, sc.tris, mixed, sc.surface_id)
    assert e.value.status == rt.RT_ERR_INVALID_ARG
    neg = sc.surface_id.copy()
    neg[5] = -3
    with pytest.raises(rt.RtError) as e:
        rt.rt_build_tree(sc.vertices, sc.tris, sc.material_id, neg)
    assert e.value.status == rt.RT_ERR_INVALID_ARG
    # an empty mesh is refused before anything is launched
    with pytest.raises(rt.RtError) as e:
        rt.rt_build_tree(sc.vertices, np.zeros((0, 3), np.int32), np.zeros(0, np.int32), np.zeros(0, np.int32))
    assert e.value.status == rt.RT_ERR_INVALID_ARG


def test_sparse_surface_ids():
    """Surface ids far above the triangle count (tables sized by the largest
    id) trace exactly like the dense numbering of the same surfaces."""
    sc = scenes.shoebox(n_rays=5000, n_bounces=12)
    dense = rt.rt_trace(_tree(sc), **rt.scene_args(sc))
    t_sp = rt.rt_build_tree(sc.vertices, sc.tris, sc.material_id, sc.surface_id * 100_003 + 7)
    assert t_sp.info()["n_surfaces"] == 5 * 100_003 + 8
    sparse = rt.rt_trace(t_sp, **rt.scene_args(sc))
    assert torch.equal(dense.hist, sparse.hist) and torch.equal(dense.ray_energy, sparse.ray_energy)
    assert sparse.n == dense.n
    # image sources of equal distance exist (5^2 + 15^2 = 9^2 + 13^2 m^2 in
    # the unfolded lattice): match them by reflection order too
    order = lambda x: np.lexsort((x.order.cpu().numpy(), x.count.cpu().numpy(), x.dist.cpu().numpy()))
    for f in ("count", "dist", "order", "energy"):
        a, b = getattr(dense, f).cpu().numpy(), getattr(sparse, f).cpu().numpy()
        assert np.array_equal(a[order(dense)], b[order(sparse)]), f


def test_node_visit_cap_is_reported():
    sc = scenes.lroom(h=0.5, n_rays=1000, n_bounces=5)
    tree = _tree(sc)
    with pytest.raises(rt.RtError) as e:
        rt.rt_trace(tree, max_node_visits=2, **rt.scene_args(sc))
    assert e.value.status == rt.RT_ERR_STEP_LIMIT
    rt.rt_trace(tree, **rt.scene_args(sc))   # the default cap passes


def test_allocation_failure_is_reported():
    sc = scenes.shoebox(n_rays=100, n_bounces=4)
    rt.rt_set_allocator(lambda nbytes, stream, ctx: None, lambda p, s, c: None)
    try:
        with pytest.raises(rt.RtError) as e:
            _tree(sc)
        assert e.value.status == rt.RT_ERR_OOM
    finally:
        rt.rt_set_allocator(None, None)
    _trace(sc)   # default allocator works again


def test_surface_grouping_when_ids_missing():
    sc = scenes.shoebox(n_rays=5000, n_bounces=10)
    t_ids = rt.rt_build_tree(sc.vertices, sc.tris, sc.material_id, None)
    assert t_ids.info()["n_surfaces"] == 6
    a = rt.rt_trace(t_ids, **rt.scene_args(sc))
    b = rt.rt_trace(_tree(sc), **rt.scene_args(sc))
    assert torch.equal(a.hist, b.hist) and a.n == b.n


# ---------------------------------------------------------------------------
# directional sources (Sec. 1.2 footnote: non-uniform sampling, equal energies)
def _two_directional_sources(n_rays, n_bounces, patterns=(0.5, 0.2)):
    """Shoebox with two sources; the second axis points down (negative z)."""
    import copy
    sc = copy.copy(scenes.shoebox(n_rays=n_rays, n_bounces=n_bounces))
    sc.sources = np.array([[2.0, 3.0, 1.5], [7.5, 2.0, 1.25]])
    sc.rcv_center = np.array([[7.0, 4.0, 1.75], [3.0, 5.0, 2.0]])
    sc.rcv_radius = np.array([0.5, 0.5])
    sc.rcv_source = np.array([0, 1], np.int32)
    return scenes.directional(sc, [[0.36, -0.48, 0.8], [0.6, 0.0, -0.8]], list(patterns))


def test_directional_directions_match_oracle():
    """Bounce-0 directions of two directional sources against the FP64
    warp + rotation; the FP64 steps are the same on both sides, so at most
    a last-bit difference of the double sine / cosine may surface."""
    N = 50_021
    sc = _two_directional_sources(N, 1)
    ds = torch.empty((1, 2 * N, 6), dtype=torch.float32, device="cuda")
    _trace(sc, debug_state=ds)
    torch.cuda.synchronize()
    d = ds[0, :, 3:].cpu().numpy().astype(np.float64)
    for s in range(2):
        ref = oracle.source_directions(N, sc.src_axis[s], sc.src_pattern[s])
        diff = np.abs(d[s * N:(s + 1) * N] - ref)
        assert (diff > 0).sum() <= 1e-4 * 3 * N, (s, int((diff > 0).sum()))
        assert diff.max() <= 1.2e-7, (s, diff.max())
        o = ds[0, s * N:(s + 1) * N, :3].cpu().numpy().astype(np.float64)
        assert np.array_equal(o, np.broadcast_to(sc.sources[s], o.shape))


def test_directional_trace_parity():
    n_rays = 6001
    sc = _two_directional_sources(n_rays, 12)
    B, n = sc.n_bounces, 2 * n_rays
    ds_t = torch.empty((B, n, 6), dtype=torch.float32, device="cuda")
    dt_t = torch.empty((B, n), dtype=torch.float32, device="cuda")
    tree, isrc = _trace(sc, debug_t=dt_t, debug_state=ds_t)
    ds, dt = ds_t.cpu().numpy(), dt_t.cpu().numpy()
    hist = isrc.hist.cpu().numpy()
    osc = oracle.OracleScene(sc, tree=False)
    bq, amb = _check_lockstep(sc, osc, ds, dt, hist)
    assert amb.mean() < 0.01
    tr = oracle.trace(osc, eps_edge_rel=EPS_FREE)       # the oracle draws its own directional rays
    ok = tr.first_amb == B
    assert ok.mean() > 0.95
    assert np.array_equal(hist.T[ok], tr.hist[ok])
    E = isrc.ray_energy.cpu().numpy().astype(np.float64)
    assert np.abs(E[ok] / tr.E[ok] - 1).max() < TOL_E
    # image sources of the GPU's crossings, grouped and rebuilt in FP64
    ref = oracle.image_sources(sc, _gpu_as_oracle_trace(sc, isrc))
    got = _gpu_is_table(sc, isrc)
    assert len(got) == len(ref.n)
    for k in range(len(ref.n)):
        c, pos, dist, tim, en = got[(int(ref.rcv[k]), ref.seq[k])]
        assert c == ref.n[k] and np.allclose(en, ref.E[k], rtol=1e-12, atol=0)


def _direct_cap_fraction(a, d, r, side):
    """Share of a source's rays, density (1 - a + a mu) / (2 (1 - a)) in mu,
    aimed into a sphere of radius r at distance d in front of (side +1:
    mu >= c) or behind (side -1: mu <= -c) the source."""
    c = math.sqrt(1.0 - (r / d) ** 2)
    return ((1 - a) * (1 - c) + side * 0.5 * a * (1 - c * c)) / (2 * (1 - a))


@pytest.mark.parametrize("a", [0.0, 0.25, 0.5])
def test_directional_direct_sound_follows_pattern(a):
    """Direct sound in front of and behind a source pointing along +x: the
    counts n (energy n / N, eq. 19) follow the cap integral of the pattern;
    the front / back ratio is about 1 / (1 - 2 a) (for a = 1/2 only the
    rim of the back cap, where 1 + mu > 0, is reached)."""
    import copy
    N = 1_000_000
    sc = copy.copy(scenes.shoebox(L=(40.0, 40.0, 40.0), source=(20.0, 20.0, 20.0), alpha=1.0,
                                  n_rays=N, n_bounces=1))
    sc.rcv_center = np.array([[23.0, 20.0, 20.0], [17.0, 20.0, 20.0]])
    sc.rcv_radius = np.array([0.5, 0.5])
    sc.rcv_source = np.array([0, 0], np.int32)
    sc = scenes.directional(sc, [1.0, 0.0, 0.0], a)
    _, isrc = _trace(sc)
    order = isrc.order.cpu().numpy()
    rcv = isrc.rcv.cpu().numpy()
    cnt = isrc.count.cpu().numpy()
    en = isrc.energy.cpu().numpy()
    direct = {int(rcv[k]): (int(cnt[k]), en[k]) for k in range(isrc.n) if order[k] == 0}
    front = _direct_cap_fraction(a, 3.0, 0.5, +1) * N
    back = _direct_cap_fraction(a, 3.0, 0.5, -1) * N
    # the warped lattice is stratified in mu about the axis, so a cap centred
    # on it holds N times its share to within a ray or two (plus float32
    # rounding of the rays that graze the sphere)
    n_f, e_f = direct[0]
    n_b = direct[1][0] if 1 in direct else 0
    assert abs(n_f - front) <= 3 + 0.002 * front, (n_f, front)
    assert abs(n_b - back) <= 3 + 0.002 * back, (n_b, back)
    assert np.allclose(e_f, n_f / N, rtol=1e-6)
    if a < 0.5:
        assert n_f / n_b == pytest.approx(1.0 / (1.0 - 2.0 * a), rel=0.02)


def test_directional_sources_are_validated():
    sc = scenes.shoebox(n_rays=1000, n_bounces=4)
    tree = _tree(sc)
    for axis, pat in (([1.0, 1.0, 0.0], 0.2), ([1.0, 0.0, 0.0], 0.6), ([1.0, 0.0, 0.0], -0.1)):
        with pytest.raises(rt.RtError) as e:
            rt.rt_trace(tree, **dict(rt.scene_args(sc), src_axis=[axis], src_pattern=[pat]))
        assert e.value.status == rt.RT_ERR_INVALID_ARG
    # a = 0 turned to +z is the omnidirectional lattice itself
    a = rt.rt_trace(tree, **dict(rt.scene_args(sc), src_axis=[[0.0, 0.0, 1.0]], src_pattern=[0.0]))
    b = rt.rt_trace(tree, **rt.scene_args(sc))
    assert torch.equal(a.hist, b.hist) and torch.equal(a.ray_energy, b.ray_energy)
