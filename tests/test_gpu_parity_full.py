"""GPU path against the FP64 oracle at the benchmark's sizes, and on the
paths whose other tests compare CUDA with CUDA (batched rooms, the moving
listener's replay, the paper's median-split tree), through the C ABI.

Tolerances (the float32 path's stated bounds, as in test_gpu_trace):
  hit triangle / reflection sequence   bit-exact except rays the oracle
                                       reports as ambiguous (counted)
  hit distance                         1e-5 relative
  band energies                        1e-4 relative
  RIR histograms                       1e-4 relative L2
  image sources (FP64)                 position, distance, time 1e-9
                                       relative; eq. 19 energies 1e-12
"""
import numpy as np
import pytest

import oracle
import scenes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1811_05784_gb300 import rt  # noqa: E402
from test_gpu_trace import (EPS_FREE, TOL_E, TOL_POS, TOL_RIR, TOL_T, _check_free_running,  # noqa: E402
                            _check_compensated_lengths, _check_lengths, _check_lockstep, _gpu_as_oracle_trace,
                            _moved_listeners, _performed)

#: crossings whose FP64 margin (r - distance) / r lies within this band of
#: the sphere are decided by rounding (float32 vs FP64 trajectories)
MARGIN_BAND = 1e-4


def _table(sc, hist, rep, order, rcv, rcv_base=0):
    """{(receiver, surface sequence): row} of image sources."""
    surf = np.append(sc.surface_id, -1)
    out = {}
    for k in range(len(rep)):
        seq = tuple(surf[hist[:order[k], rep[k]]].tolist())
        key = (int(rcv[k]) - rcv_base, seq)
        assert key not in out, "duplicate image source"
        out[key] = k
    return out


def _compare_image_sources(ref, rows, count, pos, dist, tim, en):
    """The GPU's image sources (rows aligned to the oracle's) against the
    oracle's grouping and FP64 reconstruction (Sec. 1.4, eq. 19)."""
    assert len(rows) == len(ref.n)
    rows = np.asarray(rows)
    assert np.array_equal(count[rows], ref.n)
    scale = np.maximum(1.0, np.abs(ref.pos).max(1))
    assert (np.abs(pos[rows] - ref.pos).max(1) <= TOL_POS * scale).all()
    assert (np.abs(dist[rows] - ref.d) <= TOL_POS * ref.d).all()
    assert (np.abs(tim[rows] - ref.t) <= TOL_POS * ref.t).all()
    assert (np.abs(en[rows] - ref.E) <= 1e-12 * np.abs(ref.E)).all()


def _check_image_sources(sc, isrc):
    """Every image source equals the oracle's grouping of the GPU's own
    crossings by (receiver, surface sequence), mirrored in FP64."""
    ref = oracle.image_sources(sc, _gpu_as_oracle_trace(sc, isrc))
    hist = isrc.hist.cpu().numpy()
    f = {k: getattr(isrc, k).cpu().numpy() for k in ("rep_ray", "order", "rcv", "count", "pos", "dist", "time",
                                                      "energy")}
    tab = _table(sc, hist, f["rep_ray"], f["order"], f["rcv"])
    rows = [tab[(int(ref.rcv[k]), ref.seq[k])] for k in range(len(ref.n))]
    _compare_image_sources(ref, rows, f["count"], f["pos"], f["dist"], f["time"], f["energy"])
    return ref


def _lockstep_crossings(sc, ds, dt, hist, rec_ray, rec_order, rec_rcv, ray_src=None):
    """Every (ray, bounce, receiver) crossing of the GPU's segments, in FP64
    on the GPU's own float32 states (eq. 22): the clear ones are all
    recorded, nothing else is recorded but crossings within the rounding
    band of the sphere.  Returns the FP64 margins per segment crossing."""
    bq = np.argwhere(_performed(hist))
    seg = np.where(hist[bq[:, 0], bq[:, 1]] >= 0, dt[bq[:, 0], bq[:, 1]], np.inf)
    st = ds[bq[:, 0], bq[:, 1]].astype(np.float64)
    src = None if ray_src is None else ray_src[bq[:, 1]]
    k, r, margin = oracle.crossings(sc, st[:, :3], st[:, 3:], seg, src)
    clear = np.abs(margin) > 1e-5
    want = set(zip(bq[k[clear], 1].tolist(), bq[k[clear], 0].tolist(), r[clear].tolist()))
    edge = set(zip(bq[k[~clear], 1].tolist(), bq[k[~clear], 0].tolist(), r[~clear].tolist()))
    got = set(zip(rec_ray.tolist(), rec_order.tolist(), rec_rcv.tolist()))
    assert want <= got, f"{len(want - got)} clear crossings not recorded"
    assert not (got - want - edge), f"{len(got - want - edge)} recorded crossings the oracle does not see"
    return bq[k, 1], margin


@pytest.mark.parametrize("scene", ["theatre", "lroom"])
def test_headline_image_sources_and_histograms(scene):
    """Full size, in the bounce kernel's benchmark configuration: every
    image source of every receiver (theatre: 8 bands, 6 materials, ISO air
    over tens of metres; L-room: 50 bounces), and rt_rir's 8-band histograms
    against the oracle's binning of those image sources."""
    sc = scenes.theatre() if scene == "theatre" else scenes.lroom()
    tree = rt.rt_build_tree(sc.vertices, sc.tris, sc.material_id, sc.surface_id)
    isrc = rt.rt_trace(tree, tail_rays=sc.n_rays, block_size=128, **rt.scene_args(sc))
    assert isrc.hash_collisions == 0 and isrc.n > 10_000
    ref = _check_image_sources(sc, isrc)
    dur = 2.0
    H = rt.rt_rir(isrc, sc.fs, duration=dur).download().astype(np.float64)
    Href = oracle.rir(ref, len(sc.rcv_center), sc.fs, duration=dur)
    assert np.linalg.norm(H - Href) / np.linalg.norm(Href) < 1e-6


def test_theatre_end_to_end_against_the_free_running_oracle():
    """The theatre (436,796 triangles, 1M rays x 30 bounces, 16 receivers)
    traced from the source by the FP64 oracle on every ray, and by the GPU:
      - lockstep crossings of all 3.28M GPU segments (eq. 22);
      - rays whose sequences the oracle reports ambiguous (near ties and
        near edges) or whose crossings lie within the rounding band of a
        sphere are counted and set aside; no other ray may differ in its
        surface sequence or its crossings;
      - the other rays carry the oracle's band energies and path lengths;
      - the 8-band RIR without the set-aside rays on both sides equals the
        oracle's within 1e-4 relative L2 (the GPU side: rt_rir's output
        minus those rays' shares E_s / n of their image sources)."""
    sc = scenes.theatre()
    B, N, R = sc.n_bounces, sc.n_rays, len(sc.rcv_center)
    ds_t = torch.empty((B, N, 6), dtype=torch.float32, device="cuda")
    dt_t = torch.empty((B, N), dtype=torch.float32, device="cuda")
    tree = rt.rt_build_tree(sc.vertices, sc.tris, sc.material_id, sc.surface_id)
    # wavefront bounces down to 16,384 live rays, then tail mode
    isrc = rt.rt_trace(tree, debug_state=ds_t, debug_t=dt_t, tail_rays=16384, **rt.scene_args(sc))
    dur = 2.0
    H = rt.rt_rir(isrc, sc.fs, duration=dur).download().astype(np.float64)
    hist = isrc.hist.cpu().numpy()
    ds, dt = ds_t.cpu().numpy(), dt_t.cpu().numpy()
    del ds_t, dt_t
    rec_ray = isrc.rec_ray.cpu().numpy().astype(np.int64)
    rec_m = isrc.rec_order.cpu().numpy()
    rec_r = isrc.rec_rcv.cpu().numpy()
    seg_ray, seg_margin = _lockstep_crossings(sc, ds, dt, hist, rec_ray, rec_m, rec_r)
    _check_compensated_lengths(isrc, dt, hist)
    del ds, dt

    tr = oracle.trace(oracle.OracleScene(sc, tree=True), eps_edge_rel=EPS_FREE)
    assert tr.queries == isrc.queries or abs(tr.queries - isrc.queries) < 1e-4 * isrc.queries
    aside = tr.first_amb < B
    aside[tr.rec_ray[np.abs(tr.rec_margin) <= MARGIN_BAND]] = True
    aside[seg_ray[np.abs(seg_margin) <= MARGIN_BAND]] = True
    surf = np.append(sc.surface_id, -1)
    seq_diff = (surf[hist.T] != surf[tr.hist]).any(1)
    key = lambda ray, m, r: ray * (B * R) + m * R + r
    xdiff = np.unique(np.setxor1d(key(rec_ray, rec_m, rec_r), key(tr.rec_ray, tr.rec_m, tr.rec_rcv)) // (B * R))
    differ = seq_diff.copy()
    differ[xdiff] = True
    unexplained = np.flatnonzero(differ & ~aside)
    assert len(unexplained) == 0, f"{len(unexplained)} rays differ without ambiguity, e.g. {unexplained[:5]}"
    assert aside.mean() < 0.05, aside.mean()

    # band energies of every ray with the oracle's surface sequence; hit
    # counts and path lengths of every ray with its exact triangle sequence
    same_surf = ~seq_diff
    assert same_surf.mean() > 0.99
    E = isrc.ray_energy.cpu().numpy().astype(np.float64)
    assert np.abs(E[same_surf] / tr.E[same_surf] - 1).max() < TOL_E
    same = ~aside & (hist.T == tr.hist).all(1)
    assert same.mean() > 0.9
    L = isrc.ray_length.cpu().numpy().astype(np.float64)[same]
    assert np.array_equal(isrc.ray_hits.cpu().numpy()[same], tr.n_hits[same])
    _check_lengths(sc, L, tr.L[same], tr.n_hits[same])

    # RIR without the set-aside rays: GPU output minus their shares
    tab = _table(sc, hist, *(getattr(isrc, k).cpu().numpy() for k in ("rep_ray", "order", "rcv")))
    cnt, tim, en = (getattr(isrc, k).cpu().numpy() for k in ("count", "time", "energy"))
    nb = H.shape[-1]
    for j in np.flatnonzero(aside[rec_ray]):
        q, m, r = int(rec_ray[j]), int(rec_m[j]), int(rec_r[j])
        k = tab[(r, tuple(surf[hist[:m, q]].tolist()))]
        b = int(np.floor(tim[k] * sc.fs))
        if b < nb:
            H[r, :, b] -= en[k] / cnt[k]
    Ho = oracle.rir(oracle.image_sources(sc, tr, exclude_rays=np.flatnonzero(aside)), R, sc.fs, duration=dur)
    err = np.linalg.norm(H - Ho) / np.linalg.norm(Ho)
    assert err < TOL_RIR, (err, int(aside.sum()))


# ---------------------------------------------------------------------------
# batched rooms (one launch per bounce for all rooms)
# ---------------------------------------------------------------------------
def test_batched_rooms_against_the_oracle():
    """All 64 rooms x 16 source / receiver pairs of the batched workload
    (2,048 rays per pair, 30 bounces) in one batched trace.  On seven seeded
    rooms (the largest among them), against each room's FP64 oracle:
    lockstep hits and distances on sampled queries, free-running sequences,
    energies and lengths on sampled rays, and every image source of the
    room's receivers."""
    n_rays, B = 2048, 30
    scs = scenes.batched_rooms(n_rays=n_rays, n_bounces=B)
    trees = [rt.rt_build_tree(sc.vertices, sc.tris, sc.material_id, sc.surface_id) for sc in scs]
    rooms = [dict(tree=t, sources=sc.sources, rcv_center=sc.rcv_center, rcv_radius=sc.rcv_radius,
                  rcv_source=sc.rcv_source, band_absorption=sc.alpha) for t, sc in zip(trees, scs)]
    n_src = [len(sc.sources) for sc in scs]
    n_tot = sum(n_src) * n_rays
    ds_t = torch.empty((B, n_tot, 6), dtype=torch.float32, device="cuda")
    dt_t = torch.empty((B, n_tot), dtype=torch.float32, device="cuda")
    batch = rt.rt_trace_batch(rooms, n_rays, B, tail_rays=rt.RT_TAIL_AUTOTUNE, debug_state=ds_t, debug_t=dt_t)
    assert batch.n_traced == n_tot and batch.hash_collisions == 0
    hist_all = batch.hist.cpu().numpy()
    rec = {k: getattr(batch, k).cpu().numpy() for k in ("rec_ray", "rec_order", "rec_rcv")}
    f = {k: getattr(batch, k).cpu().numpy() for k in ("rep_ray", "order", "rcv", "count", "pos", "dist", "time",
                                                      "energy")}
    ray_base = np.cumsum([0] + n_src) * n_rays
    rcv_base = np.cumsum([0] + [len(sc.rcv_center) for sc in scs])
    rng = np.random.default_rng(44)
    pick = sorted(set(rng.choice(len(scs), 6, replace=False).tolist()) |
                  {int(np.argmax([len(sc.tris) for sc in scs]))})
    for room in pick:
        sc = scs[room]
        lo, hi = ray_base[room], ray_base[room + 1]
        hist = hist_all[:, lo:hi]
        ds = ds_t[:, lo:hi].cpu().numpy()
        dt = dt_t[:, lo:hi].cpu().numpy()
        osc = oracle.OracleScene(sc, tree=True)
        # lockstep on sampled queries
        perf = np.argwhere(_performed(hist))
        sel = perf[rng.choice(len(perf), min(4000, len(perf)), replace=False)]
        _check_lockstep(sc, osc, ds, dt, hist, sel)
        # free running: traced ray q of the room is source q // n_rays, Fibonacci index q % n_rays
        qs = np.sort(rng.choice(hi - lo, 512, replace=False))
        tr = oracle.trace(osc, ray_ids=qs % n_rays, ray_src=(qs // n_rays).astype(np.int32),
                          eps_edge_rel=EPS_FREE)
        room_res = _RoomSlice(batch, lo, hi)
        _check_free_running(sc, hist, qs, tr, room_res)
        # image sources of this room's receivers: the oracle's grouping of the batch's crossings
        m = (rec["rec_rcv"] >= rcv_base[room]) & (rec["rec_rcv"] < rcv_base[room + 1])
        z = np.zeros(0)
        n = hi - lo
        mine = oracle.TraceResult(np.zeros(n, np.int32), np.arange(n), hist.T.copy(), np.zeros((n, B)), z, z,
                                  np.full(n, B, np.int32), np.zeros(n, np.int32),
                                  rec["rec_rcv"][m] - rcv_base[room], rec["rec_ray"][m].astype(np.int64) - lo,
                                  rec["rec_order"][m], np.zeros(int(m.sum())), z, np.zeros((0, 3)),
                                  np.zeros((0, 3)), n_rays, B)
        ref = oracle.image_sources(sc, mine)
        sel_is = (f["rcv"] >= rcv_base[room]) & (f["rcv"] < rcv_base[room + 1])
        idx = np.flatnonzero(sel_is)
        tab = _table(sc, hist_all, f["rep_ray"][idx], f["order"][idx], f["rcv"][idx], rcv_base[room])
        rows = [idx[tab[(int(ref.rcv[k]), ref.seq[k])]] for k in range(len(ref.n))]
        assert len(tab) == len(ref.n)
        _compare_image_sources(ref, rows, f["count"], f["pos"], f["dist"], f["time"], f["energy"])


class _RoomSlice:
    """Per-ray outputs of one room of a batched trace, indexed room-locally."""

    def __init__(self, batch, lo, hi):
        self.ray_energy = batch.ray_energy[lo:hi]
        self.ray_length = batch.ray_length[lo:hi]
        self.ray_hits = batch.ray_hits[lo:hi]


# ---------------------------------------------------------------------------
# moving listener: replayed paths with new receivers
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("scene", ["shoebox", "theatre"])
def test_replay_with_moved_listeners_against_the_oracle(scene):
    """A replay (each query re-tests the triangle an earlier trace hit) with
    moved and added receivers: its crossings equal the FP64 crossings of
    its segments with the new spheres, its image sources equal the oracle's
    grouping, and the oracle's own free-running trace with the moved
    receivers records the same crossings on every unambiguous ray."""
    sc = scenes.shoebox(n_rays=20_000, n_bounces=25) if scene == "shoebox" else scenes.theatre(n_rays=100_000)
    B, N = sc.n_bounces, sc.n_rays
    tree = rt.rt_build_tree(sc.vertices, sc.tris, sc.material_id, sc.surface_id)
    first = rt.rt_trace(tree, **rt.scene_args(sc))
    moved = _moved_listeners(sc)
    ds_t = torch.empty((B, N, 6), dtype=torch.float32, device="cuda")
    dt_t = torch.empty((B, N), dtype=torch.float32, device="cuda")
    rep = rt.rt_trace(tree, replay=first, debug_state=ds_t, debug_t=dt_t, **rt.scene_args(moved))
    hist = rep.hist.cpu().numpy()
    assert np.array_equal(hist, first.hist.cpu().numpy())
    rec_ray = rep.rec_ray.cpu().numpy().astype(np.int64)
    rec_m, rec_r = rep.rec_order.cpu().numpy(), rep.rec_rcv.cpu().numpy()
    _lockstep_crossings(moved, ds_t.cpu().numpy(), dt_t.cpu().numpy(), hist, rec_ray, rec_m, rec_r)
    assert rep.n > 0
    _check_image_sources(moved, rep)
    # the oracle traces the moved scene itself
    rng = np.random.default_rng(9)
    ids = np.sort(rng.choice(N, 2000, replace=False))
    tr = oracle.trace(oracle.OracleScene(moved, tree=scene != "shoebox"), ray_ids=ids, eps_edge_rel=EPS_FREE)
    near = set(tr.rec_ray[np.abs(tr.rec_margin) <= MARGIN_BAND].tolist())
    got = {}
    for q, m, r in zip(rec_ray.tolist(), rec_m.tolist(), rec_r.tolist()):
        got.setdefault(q, set()).add((m, r))
    want = {}
    for i, m, r in zip(tr.rec_ray.tolist(), tr.rec_m.tolist(), tr.rec_rcv.tolist()):
        want.setdefault(i, set()).add((m, r))
    checked = 0
    for i, q in enumerate(ids.tolist()):
        if tr.first_amb[i] < B or i in near:
            continue
        checked += 1
        assert got.get(q, set()) == want.get(i, set()), q
    assert checked > 0.9 * len(ids)


# ---------------------------------------------------------------------------
# the paper's median-split tree (Sec. 2.2) on the GPU
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("scene", ["lroom", "theatre"])
def test_median_split_tree_trace_against_the_oracle(scene):
    """Traces over the median-split tree against the FP64 oracle: lockstep
    hits and distances, free-running sequences, energies and lengths."""
    sc = scenes.lroom(h=0.5, n_rays=50_000, n_bounces=20) if scene == "lroom" else scenes.theatre(n_rays=100_000)
    B, N = sc.n_bounces, sc.n_rays
    med = rt.rt_build_tree(sc.vertices, sc.tris, sc.material_id, sc.surface_id, median=True)
    ds_t = torch.empty((B, N, 6), dtype=torch.float32, device="cuda")
    dt_t = torch.empty((B, N), dtype=torch.float32, device="cuda")
    isrc = rt.rt_trace(med, debug_state=ds_t, debug_t=dt_t, **rt.scene_args(sc))
    hist = isrc.hist.cpu().numpy()
    osc = oracle.OracleScene(sc, tree=True)
    rng = np.random.default_rng(21)
    perf = np.argwhere(_performed(hist))
    pick = perf[rng.choice(len(perf), min(40_000, len(perf)), replace=False)]
    _check_lockstep(sc, osc, ds_t.cpu().numpy(), dt_t.cpu().numpy(), hist, pick)
    ids = np.sort(rng.choice(N, 2048, replace=False))
    tr = oracle.trace(osc, ray_ids=ids, eps_edge_rel=EPS_FREE)
    _check_free_running(sc, hist, ids, tr, isrc)
