"""Seeded input generators (no method arithmetic): sizes, placement, determinism."""
import numpy as np

import scenes


def test_batched_rooms_workload():
    rooms = scenes.batched_rooms()
    assert len(rooms) == 64
    m = np.array([len(r.tris) for r in rooms])
    assert m.min() >= 12 and m.max() <= 200_000 and m.max() > 100_000 and m.min() < 100
    kinds = {r.meta["kind"] for r in rooms}
    assert kinds == {"shoebox", "lroom"}
    for r in rooms:
        assert len(r.sources) == 16 and len(r.rcv_center) == 16
        assert np.array_equal(r.rcv_source, np.arange(16))
        lo, hi = r.vertices.min(0), r.vertices.max(0)
        for p in np.concatenate([r.sources, r.rcv_center]):
            assert np.all(p > lo) and np.all(p < hi)
            if r.meta["kind"] == "lroom":      # inside the L, not in the cut-out quarter
                sc = (hi[0] - lo[0]) / 20.0
                assert p[0] < 10 * sc or p[1] < 7.5 * sc
        assert np.all(np.linalg.norm(r.sources - r.rcv_center, axis=1) >= 1.0)
        assert r.alpha.shape == (4, 8) and r.alpha.min() >= 0.02 and r.alpha.max() <= 0.6
        assert r.material_id.max() < 4
    again = scenes.batched_rooms(n_rooms=3)
    for a, b in zip(again, rooms[:3]):
        assert np.array_equal(a.vertices, b.vertices) and np.array_equal(a.sources, b.sources)


def test_directional_copy_normalises_and_broadcasts():
    """scenes.directional: one axis for all sources or one per source, unit
    length, one pattern per source; the scene it copies is left as it was."""
    import numpy as np
    import scenes
    sc = scenes.shoebox(n_rays=100, n_bounces=2)
    d = scenes.directional(sc, [0.0, 3.0, 4.0], 0.25)
    assert sc.src_axis is None and sc.src_pattern is None
    assert d.src_axis.shape == (len(sc.sources), 3) and d.src_pattern.shape == (len(sc.sources),)
    assert np.allclose(d.src_axis[0], [0.0, 0.6, 0.8], atol=0, rtol=1e-15)
    assert abs(np.sum(d.src_axis[0] ** 2) - 1.0) < 1e-15
    assert np.all(d.src_pattern == 0.25)
    assert d.tris is sc.tris and d.vertices is sc.vertices
