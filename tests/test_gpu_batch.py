"""Batched rooms in one launch, the workspace's CUDA-graph bounce loop, and
the online autotuner: none of them may change any ray's result."""
import numpy as np
import pytest

import scenes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1811_05784_gb300 import rt  # noqa: E402


def _tree(sc):
    return rt.rt_build_tree(sc.vertices, sc.tris, sc.material_id, sc.surface_id)


def _is_table(sc_list, isrc, rcv_base):
    """{(room, local receiver, surface sequence): (count, energy)} from an output."""
    hist = isrc.hist.cpu().numpy()
    rep, order, rcv = (x.cpu().numpy() for x in (isrc.rep_ray, isrc.order, isrc.rcv))
    cnt, en = isrc.count.cpu().numpy(), isrc.energy.cpu().numpy()
    out = {}
    for k in range(isrc.n):
        room = int(np.searchsorted(rcv_base, rcv[k], side="right") - 1)
        sc = sc_list[room]
        seq = tuple(int(sc.surface_id[hist[j, rep[k]]]) for j in range(order[k]))
        out[(room, int(rcv[k] - rcv_base[room]), seq)] = (int(cnt[k]), en[k])
    return out


def _check_batch_equals_single(scs, N, B):
    trees = [_tree(sc) for sc in scs]
    rooms = [dict(tree=t, sources=sc.sources, rcv_center=sc.rcv_center, rcv_radius=sc.rcv_radius,
                  rcv_source=sc.rcv_source, band_absorption=sc.alpha, src_axis=sc.src_axis,
                  src_pattern=sc.src_pattern) for t, sc in zip(trees, scs)]
    batch = rt.rt_trace_batch(rooms, N, B, tail_rays=rt.RT_TAIL_AUTOTUNE)
    rcv_base = np.cumsum([0] + [len(sc.rcv_center) for sc in scs])
    hb = batch.hist.cpu().numpy()
    eb = batch.ray_energy.cpu().numpy()
    table_b = _is_table(scs, batch, rcv_base)
    off = 0
    for r, (sc, t) in enumerate(zip(scs, trees)):
        kw = rt.scene_args(sc)
        kw.update(n_rays=N, n_bounces=B)
        single = rt.rt_trace(t, **kw)
        n = single.n_traced
        assert np.array_equal(hb[:, off:off + n], single.hist.cpu().numpy())
        assert np.array_equal(eb[off:off + n], single.ray_energy.cpu().numpy())
        ts = _is_table([sc], single, np.array([0, len(sc.rcv_center)]))
        for (room0, lr, seq), (c, e) in ts.items():
            cb, ebx = table_b[(r, lr, seq)]
            assert cb == c and np.array_equal(ebx, e)
        assert sum(1 for key in table_b if key[0] == r) == len(ts)
        off += n
    assert off == batch.n_traced
    return batch


def test_batch_matches_single_rooms():
    N, B = 20_000, 20
    scs = [scenes.shoebox(n_rays=N, n_bounces=B), scenes.lroom(h=0.5, n_rays=N, n_bounces=B),
           scenes.icosphere(level=2, n_rays=N, n_bounces=B)]
    _check_batch_equals_single(scs, N, B)


def test_batch_with_directional_rooms_matches_single_rooms():
    """Omnidirectional and directional rooms in one launch (each source keeps
    its own axis and pattern)."""
    N, B = 12_000, 16
    scs = [scenes.shoebox(n_rays=N, n_bounces=B),
           scenes.directional(scenes.lroom(h=0.5, n_rays=N, n_bounces=B), [0.0, -0.6, 0.8], 0.5),
           scenes.directional(scenes.shoebox(L=(6.0, 5.0, 3.0), source=(1.0, 1.0, 1.0), receiver=(4.0, 3.0, 1.5),
                                             n_rays=N, n_bounces=B), [-1.0, 0.0, 0.0], 0.3)]
    _check_batch_equals_single(scs, N, B)


def test_batched_config_rooms_match_single_rooms():
    """The first 8 rooms of the batched-rooms workload (12 to 200k triangles,
    shoeboxes and L-rooms, several source / receiver pairs each) in one
    launch give every room's own trace bit for bit."""
    scs = scenes.batched_rooms(n_rooms=8, pairs=4, n_rays=4096, n_bounces=12)
    batch = _check_batch_equals_single(scs, 4096, 12)
    assert batch.n > 0


def test_batch_replay_with_moved_listeners():
    scs = scenes.batched_rooms(n_rooms=6, pairs=3, n_rays=4096, n_bounces=12)
    trees = [_tree(sc) for sc in scs]

    def rooms(move):
        out = []
        for t, sc in zip(trees, scs):
            c = sc.rcv_center + (np.float32(0.4) if move else np.float32(0))
            out.append(dict(tree=t, sources=sc.sources, rcv_center=c, rcv_radius=sc.rcv_radius,
                            rcv_source=sc.rcv_source, band_absorption=sc.alpha))
        return out

    first = rt.rt_trace_batch(rooms(False), 4096, 12)
    full = rt.rt_trace_batch(rooms(True), 4096, 12)
    rep = rt.rt_trace_batch(rooms(True), 4096, 12, replay=first)
    for name in ("hist", "ray_energy", "rcv", "order", "count", "rep_ray", "pos", "time", "energy"):
        assert torch.equal(getattr(full, name), getattr(rep, name)), name


def test_workspace_graph_replays_give_identical_results():
    sc = scenes.theatre(n_rays=100_000)
    tree = _tree(sc)
    ref = rt.rt_trace(tree, **rt.scene_args(sc))
    stream = torch.cuda.Stream()
    ws = rt.Workspace()
    for k in range(3):
        got = rt.rt_trace(tree, stream=stream, workspace=ws, **rt.scene_args(sc))
        torch.cuda.synchronize()
        assert torch.equal(got.hist, ref.hist) and torch.equal(got.energy, ref.energy)
        assert got.n == ref.n and got.queries == ref.queries
    assert ws.graph_launches == 3
    ws.free()


def test_autotuner_candidates_agree():
    sc = scenes.theatre(n_rays=50_000)
    tree = _tree(sc)
    ref = rt.rt_trace(tree, tail_rays=-1, block_size=128, **rt.scene_args(sc))
    seen = set()
    for k in range(9):
        got = rt.rt_trace(tree, tail_rays=rt.RT_TAIL_AUTOTUNE, **rt.scene_args(sc))
        seen.add((got.block_size, got.tail_rays))
        assert torch.equal(got.hist, ref.hist) and torch.equal(got.ray_energy, ref.ray_energy)
        assert torch.equal(got.count, ref.count)
    assert len(seen) >= 5          # the candidates were tried, then one kept
