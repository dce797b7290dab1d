"""Pins of the FP64 oracle against what the paper and mathematics fix.

Each test compares the oracle with something computed another way: hand
geometry, the unfolded-lattice closed form of a rectangular room (McGovern,
paper Sec. 3.2), eq. 9's solid angle, the mirror geometry of a sphere
(Sec. 3.1), the mean free path of a rectangular room (Eyring rate), or brute
force against the paper's tree (Sec. 2.2).
"""
import math

import numpy as np
import pytest

import oracle
import scenes
from closed_form import (cone_fraction, image_source, reflections_within,
                         shoebox_image_sources)


def _mini_scene(tris_xyz, mats=None, surfs=None, alpha=None):
    tris_xyz = np.asarray(tris_xyz, float).reshape(-1, 3, 3)
    M = len(tris_xyz)
    return scenes.Scene(
        name="mini", vertices=tris_xyz.reshape(-1, 3), tris=np.arange(3 * M, dtype=np.int32).reshape(M, 3),
        material_id=np.zeros(M, np.int32) if mats is None else np.asarray(mats, np.int32),
        surface_id=np.arange(M, dtype=np.int32) if surfs is None else np.asarray(surfs, np.int32),
        alpha=np.zeros((1, 8), np.float32) if alpha is None else alpha, beta=np.zeros(8, np.float32),
        sources=np.zeros((1, 3)), rcv_center=np.zeros((0, 3)), rcv_radius=np.zeros(0),
        rcv_source=np.zeros(0, np.int32), n_rays=1, n_bounces=1)


# ---------------------------------------------------------------------------
# Sec. 2.1, eq. 20-21: one triangle, hand cases
# ---------------------------------------------------------------------------
def test_moller_trumbore_hand_cases():
    osc = oracle.OracleScene(_mini_scene([[0, 0, 0], [1, 0, 0], [0, 1, 0]]), tree=False)
    down = [0, 0, -1]
    cases = [  # (origin, direction, expected tri, expected delta, expected ambiguous)
        ([0.25, 0.25, 1], down, 0, 1.0, False),      # interior
        ([0.5, 0.5, 2], down, 0, 2.0, True),         # on lambda + mu = 1 (inclusive)
        ([0.0, 0.0, 1], down, 0, 1.0, True),         # on a vertex
        ([0.3, 0.0, 1], down, 0, 1.0, True),         # on mu = 0
        ([0.6, 0.6, 1], down, -1, math.inf, False),  # clearly outside
        ([0.5 + 1e-9, 0.5, 1], down, -1, math.inf, True),  # just outside: near edge
        ([0.25, 0.25, 1], [0, 0, 1], -1, math.inf, False),  # behind the origin (delta < 0)
        ([0.25, 0.25, 1], [1, 0, 0], -1, math.inf, False),  # parallel to the plane
        ([0.25, 0.25, 0], down, -1, math.inf, False),       # delta = 0 is not > 0
    ]
    o = np.array([c[0] for c in cases], float)
    u = np.array([c[1] for c in cases], float)
    tri, d1, d2, amb = osc.nearest(o, u, brute=True)
    for k, (_, _, et, ed, ea) in enumerate(cases):
        assert tri[k] == et, k
        if et >= 0:
            assert d1[k] == pytest.approx(ed, abs=1e-15), k
        assert bool(amb[k]) == ea, k


def test_nearest_and_ties():
    # two coplanar triangles sharing the diagonal of the unit square at z=0,
    # and a third one at z=0.5 that only covers x+y < 0.5
    tris = [[[0, 0, 0], [1, 0, 0], [1, 1, 0]],
            [[0, 0, 0], [1, 1, 0], [0, 1, 0]],
            [[0, 0, 0.5], [0.5, 0, 0.5], [0, 0.5, 0.5]]]
    osc = oracle.OracleScene(_mini_scene(tris), tree=False)
    o = np.array([[0.7, 0.7, 1], [0.8, 0.2, 1], [0.2, 0.8, 1], [0.1, 0.1, 1], [0.1, 0.1, 0.25]])
    u = np.array([[0, 0, -1]] * 5, float)
    tri, d1, d2, amb = osc.nearest(o, u, brute=True)
    assert list(tri) == [0, 0, 1, 2, 0]          # shared edge -> lowest index
    assert amb[0] and not amb[1] and not amb[2] and not amb[3]
    assert d1[3] == 0.5 and d1[4] == 0.25
    # excluding the last-hit triangle
    tri, *_ = osc.nearest(o[3:4], u[3:4], exclude=np.array([2]), brute=True)
    assert tri[0] == 0


# ---------------------------------------------------------------------------
# Sec. 1.2: Fibonacci rule
# ---------------------------------------------------------------------------
def test_fibonacci_rule():
    N = 2000
    u = oracle.fibonacci(N)
    k = np.arange(N)
    z = (1.0 - (2 * k + 1) / N).astype(np.float32).astype(np.float64)
    assert np.array_equal(u[:, 2], z)
    assert np.all(u == u.astype(np.float32).astype(np.float64))
    assert np.abs(np.linalg.norm(u, axis=1) - 1).max() < 2e-7
    # consecutive azimuths advance by the golden angle pi (3 - sqrt 5)
    phi = np.arctan2(u[:, 1], u[:, 0])
    dphi = np.mod(np.diff(phi) - math.pi * (3 - math.sqrt(5)) + math.pi, 2 * math.pi) - math.pi
    rho = np.hypot(u[:, 0], u[:, 1])
    ok = (rho[1:] > 0.1) & (rho[:-1] > 0.1)
    assert np.abs(dphi[ok]).max() < 1e-5
    # uniform: the mean direction vanishes
    assert np.abs(u.mean(0)).max() < 1e-3
    # subset ids give the same directions
    ids = np.array([0, 7, 1999, 1000])
    assert np.array_equal(oracle.fibonacci(N, ids), u[ids])


# ---------------------------------------------------------------------------
# Sec. 2.2: the median-split tree answers exactly like brute force
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("seed", [0, 1])
def test_tree_equals_brute_force(seed):
    rng = np.random.default_rng(seed)
    M = 400
    c = rng.uniform(0, 10, (M, 1, 3))
    tris = c + rng.normal(0, 0.8, (M, 3, 3))
    # a few coplanar neighbours sharing edges
    tris[:20] = np.array([[[i, 0, 0], [i + 1, 0, 0], [i, 1, 0]] for i in range(20)])
    sc = _mini_scene(scenes.f32(tris))
    osc_t = oracle.OracleScene(sc, tree=True)
    osc_b = oracle.OracleScene(sc, tree=False)
    assert osc_t.tree_nodes == 2 * M - 1          # one element per leaf
    n = 3000
    o = rng.uniform(-1, 11, (n, 3))
    u = rng.normal(size=(n, 3))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    t1, d1, _, a1 = osc_t.nearest(o, u)
    t2, e1, _, a2 = osc_b.nearest(o, u, brute=True)
    assert np.array_equal(t1, t2)
    hit = t1 >= 0
    assert np.array_equal(d1[hit], e1[hit])
    assert np.array_equal(a1, a2)
    assert hit.sum() > n // 4


def test_tree_equals_brute_force_trace_lroom():
    sc = scenes.lroom(h=0.5, n_rays=400, n_bounces=12)
    tr_t = oracle.trace(oracle.OracleScene(sc, tree=True))
    tr_b = oracle.trace(oracle.OracleScene(sc, tree=False))
    assert np.array_equal(tr_t.hist, tr_b.hist)
    assert np.array_equal(tr_t.E, tr_b.E)
    assert np.array_equal(tr_t.rec_ray, tr_b.rec_ray)


# ---------------------------------------------------------------------------
# Sec. 3.2: closed-form rectangular room (McGovern lattice, unfolded rays)
# ---------------------------------------------------------------------------
def _compare_shoebox(sc, n_check_rays=None):
    osc = oracle.OracleScene(sc, tree=False)
    tr = oracle.trace(osc)
    dirs = oracle.fibonacci(sc.n_rays)
    L = np.array(sc.meta["L"])
    cf = shoebox_image_sources(sc.sources[0], sc.rcv_center[0], sc.rcv_radius[0], L, dirs,
                               sc.n_bounces, dmax=sc.max_distance)
    amb = set(np.nonzero(tr.first_amb < tr.B)[0]) | cf["ambiguous_rays"]
    amb |= set(int(x) for x in tr.rec_ray[np.abs(tr.rec_margin) < 1e-6])
    assert len(amb) < 0.01 * sc.n_rays
    # per-ray crossings: same (m, sequence) lists
    oracle_cross = {}
    for k in range(len(tr.rec_ray)):
        i = int(tr.rec_ray[k])
        m = int(tr.rec_m[k])
        seq = tuple(int(sc.surface_id[t]) for t in tr.hist[i, :m])
        oracle_cross.setdefault(i, []).append((m, seq))
    cf_cross = {}
    for i, m, seq, cell, margin in cf["crossings"]:
        cf_cross.setdefault(i, []).append((m, seq))
    rays = set(oracle_cross) | set(cf_cross)
    for i in sorted(rays - amb):
        assert sorted(oracle_cross.get(i, [])) == sorted(cf_cross.get(i, [])), i
    # image sources: positions, arrival times, counts, energies (eq. 19)
    isrc = oracle.image_sources(sc, tr, exclude_rays=amb)
    cf_n = {}
    for i, m, seq, cell, margin in cf["crossings"]:
        if i not in amb:
            cf_n[seq] = cf_n.get(seq, 0) + 1
    assert len(isrc.n) == len(cf_n)
    alpha = sc.alpha.astype(np.float64)
    smat = oracle.surface_material(sc)
    for k in range(len(isrc.n)):
        seq = isrc.seq[k]
        n, pos, cell = cf["groups"][seq]
        assert isrc.n[k] == cf_n[seq]
        assert np.abs(isrc.pos[k] - pos).max() <= 1e-9 * max(1.0, np.abs(pos).max())
        d = float(np.linalg.norm(pos - sc.rcv_center[0]))
        assert isrc.t[k] == pytest.approx(d / sc.c, rel=1e-12)
        prod = np.prod([1.0 - alpha[smat[s]] for s in seq], axis=0) if seq else np.ones(8)
        E = cf_n[seq] / sc.n_rays * prod * np.exp(-sc.beta.astype(np.float64) * d)
        assert np.allclose(isrc.E[k], E, rtol=1e-12, atol=0)
    return tr, isrc, amb


def test_shoebox_closed_form_config1():
    sc = scenes.shoebox()   # 10x7x3 m, alpha 0.1, 1e4 rays, 20 bounces
    tr, isrc, amb = _compare_shoebox(sc)
    # direct sound: d = |x_m - x_s|, n = Fibonacci directions in the cone (eq. 9)
    k0 = np.nonzero(isrc.order == 0)[0]
    assert len(k0) == 1
    d = float(np.linalg.norm(sc.rcv_center[0] - sc.sources[0]))
    assert isrc.d[k0[0]] == pytest.approx(d, rel=1e-15)
    assert abs(isrc.n[k0[0]] - sc.n_rays * cone_fraction(0.5, d)) < 6
    # closed room: every ray makes exactly B hits, E = (1/N)(1 - 0.1)^B (eq. 18)
    assert not tr.escaped.any() and (tr.n_hits == sc.n_bounces).all()
    assert np.allclose(tr.E, 0.9 ** sc.n_bounces / sc.n_rays, rtol=1e-13)


def test_shoebox_closed_form_paper_setup():
    """Sec. 3.2: [5,4,3] m box, x_s=[4,2,1.7], sphere r=0.2 at [2,2,1.7],
    Table 1 materials, ISO 9613-1 air, iterations stopped by eq. 13."""
    sc = scenes.paper_shoebox(n_rays=20_000)
    dmax = 0.1 * math.sqrt(sc.n_rays)
    assert sc.max_distance == pytest.approx(dmax)
    tr, isrc, amb = _compare_shoebox(sc)
    assert (tr.rec_L <= dmax).all()
    assert ((tr.L > dmax) | (tr.n_hits == sc.n_bounces)).all()


def test_retro_propagation_matches_mirror_chain():
    """Sec. 1.4: a crossing ray traced back along its last direction by its
    path length lands on the image source built by mirroring x_s."""
    sc = scenes.lroom(h=0.5, n_rays=3000, n_bounces=25)
    tr = oracle.trace(oracle.OracleScene(sc))
    isrc = oracle.image_sources(sc, tr)
    where = {(int(r), s): k for k, (r, s) in enumerate(zip(isrc.rcv, isrc.seq))}
    assert len(tr.rec_ray) > 100
    for j in range(len(tr.rec_ray)):
        i, m, r = int(tr.rec_ray[j]), int(tr.rec_m[j]), int(tr.rec_rcv[j])
        seq = tuple(int(sc.surface_id[t]) for t in tr.hist[i, :m])
        x_back = tr.rec_pos[j] - tr.rec_L[j] * tr.rec_dir[j]
        x_is = isrc.pos[where[(r, seq)]]
        assert np.abs(x_back - x_is).max() <= 1e-9 * max(1.0, tr.rec_L[j])


# ---------------------------------------------------------------------------
# eq. 9 / eq. 12: direct-sound counts in free field
# ---------------------------------------------------------------------------
def test_direct_sound_cone_counts():
    N = 100_000
    r = 0.36                                     # Fig. 3 radius
    dists = [1.0, 2.0, 4.0, 8.0, 16.0]
    rng = np.random.default_rng(7)
    centres = []
    for d in dists:
        v = rng.normal(size=3)
        centres.append(scenes.f32(v / np.linalg.norm(v) * d))
    sc = scenes.Scene("free", np.zeros((0, 3)), np.zeros((0, 3), np.int32), np.zeros(0, np.int32),
                      np.zeros(0, np.int32), np.zeros((1, 8), np.float32), np.zeros(8, np.float32),
                      np.zeros((1, 3)), np.array(centres), np.full(len(dists), r),
                      np.zeros(len(dists), np.int32), N, 1)
    tr = oracle.trace(oracle.OracleScene(sc, tree=False))
    assert (tr.n_hits == 0).all() and tr.escaped.all()
    u = oracle.fibonacci(N)
    for k, c in enumerate(centres):
        d = float(np.linalg.norm(c))
        n = int((tr.rec_rcv == k).sum())
        # exact: directions inside the cone of half-angle asin(r/d)
        cosang = (u @ c) / (np.linalg.norm(u, axis=1) * d)
        cos_lim = math.sqrt(1 - (r / d) ** 2)
        inside = cosang >= cos_lim
        border = np.abs(cosang - cos_lim) < 1e-9
        assert inside.sum() - border.sum() <= n <= inside.sum() + border.sum()
        # statistical: eq. 9 solid angle, eq. 12 small-angle form
        exp = N * cone_fraction(r, d)
        assert abs(n - exp) <= 4 * math.sqrt(exp) + 2
        assert n / N == pytest.approx(r * r / (4 * d * d), rel=0.05 + 4 / math.sqrt(exp))


# ---------------------------------------------------------------------------
# Sec. 3.1: 100 % reflecting sphere (facetted), source and receiver at centre
# ---------------------------------------------------------------------------
def test_reflecting_sphere():
    sc = scenes.icosphere(level=3, n_rays=20_000, n_bounces=6, radius=0.1)
    tr = oracle.trace(oracle.OracleScene(sc))
    assert not tr.escaped.any()                      # closed mesh: energy conserved
    assert np.allclose(tr.E.sum(0), 1.0, rtol=1e-12)
    isrc = oracle.image_sources(sc, tr)
    # first order: mirror of the centre across facet j lies at 2 h_j
    tri = sc.vertices[sc.tris]
    nrm = np.cross(tri[:, 1] - tri[:, 0], tri[:, 2] - tri[:, 0])
    nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
    h = np.abs(np.einsum("ij,ij->i", nrm, tri[:, 0]))
    one = np.nonzero(isrc.order == 1)[0]
    assert len(one) > 50
    for k in one:
        assert isrc.d[k] == pytest.approx(2 * h[isrc.seq[k][0]], rel=1e-12)
    # pulses two metres apart (Dirac comb): energy-weighted distance per order
    for m in range(1, 6):
        sel = isrc.order == m
        if sel.sum() == 0:
            continue
        mean_d = float((isrc.d[sel] * isrc.n[sel]).sum() / isrc.n[sel].sum())
        assert mean_d == pytest.approx(2.0 * m, rel=0.05)


# ---------------------------------------------------------------------------
# Sec. 1.3 with a rectangular room: reflection counts and the Eyring rate
# ---------------------------------------------------------------------------
def test_reflection_counts_and_eyring_rate():
    Lr = (10.0, 7.0, 3.0)
    sc = scenes.shoebox(n_rays=2000, n_bounces=120)
    tr = oracle.trace(oracle.OracleScene(sc, tree=False))
    dirs = oracle.fibonacci(sc.n_rays)
    cum = np.cumsum(tr.hist_t, axis=1)
    length = 300.0
    m_or = (cum <= length).sum(1)
    bad = 0
    for i in range(sc.n_rays):
        m_cf = reflections_within(sc.sources[0], dirs[i], Lr, length)
        if m_cf != m_or[i]:
            bad += 1
    assert bad <= 2                                  # only exact-edge coincidences
    V = Lr[0] * Lr[1] * Lr[2]
    S = 2 * (Lr[0] * Lr[1] + Lr[1] * Lr[2] + Lr[0] * Lr[2])
    rate = m_or.mean() / length                      # reflections per metre
    assert rate == pytest.approx(S / (4 * V), rel=0.01)
    # Eyring reverberation time from the measured rate vs the formula
    alpha, c = 0.1, sc.c
    T_eyr = 60.0 / (-10 * math.log10(1 - alpha) * c * S / (4 * V))
    T_meas = 60.0 / (-10 * math.log10(1 - alpha) * c * rate)
    assert T_meas == pytest.approx(T_eyr, rel=0.01)
    # log-mean energy decays exactly at the Eyring rate
    t = np.linspace(0, 1.0, 2001)
    logm = np.array([np.mean((cum <= c * tt).sum(1)) for tt in t]) * 10 * math.log10(1 - alpha)
    k = np.polyfit(t[200:], logm[200:], 1)[0]
    assert -60.0 / k == pytest.approx(T_eyr, rel=0.01)
    # energy-mean decay (all rays): early decay near Sabine / Eyring; by Jensen's
    # inequality the energy mean lies above the log mean, so the late decay is slower
    E = np.array([np.mean(0.9 ** (cum <= c * tt).sum(1)) for tt in t])
    h = -np.diff(np.concatenate([E, [0.0]]))
    fs = 1.0 / (t[1] - t[0])
    T_sab = 0.161 * V / (S * alpha)
    assert 0.97 * T_eyr < oracle.edt(h, fs) < 1.1 * T_sab
    assert T_eyr < oracle.t30(h, fs) < 1.5 * T_sab


# ---------------------------------------------------------------------------
# Sec. 1.4: histogram and decay metrics
# ---------------------------------------------------------------------------
def test_rir_binning():
    """Arrival t goes to bin floor(t fs) (Sec. 1.4): arrivals 0.6 and 1.7 bins
    into the response land in bins 0 and 1, where rounding would move them."""
    isrc = oracle.ImageSources(np.array([0, 0, 0, 1], np.int32), np.zeros(4, np.int32), np.ones(4, np.int64),
                               np.zeros(4, np.int64), [(), (), (), ()], np.zeros((4, 3)), np.zeros(4),
                               np.array([0.0, 0.6e-4, 1.7e-4, 2.0e-4]), np.ones((4, 8)))
    H = oracle.rir(isrc, 2, fs=10_000.0, duration=0.001)
    assert H.shape == (2, 8, 10)
    assert H[0, :, 0].tolist() == [2.0] * 8 and H[0, :, 1].tolist() == [1.0] * 8
    assert H[1, :, 2].tolist() == [1.0] * 8 and H.sum() == 32


@pytest.mark.parametrize("T", [0.5, 1.326, 3.0])
def test_decay_metrics_on_exponential(T):
    fs = 1000.0
    n = np.arange(int(4 * T * fs))
    h = np.exp(-6 * math.log(10) * n / (fs * T))      # 60 dB per T seconds
    assert oracle.t30(h, fs) == pytest.approx(T, rel=1e-3)
    assert oracle.edt(h, fs) == pytest.approx(T, rel=1e-3)


def test_directional_source_sampling():
    """Directional sources (Sec. 1.2 footnote): equal-energy rays whose
    directions have density (1 - a + a cos theta) / (4 pi (1 - a)) about the
    axis.  a = 0 about +z is the Fibonacci rule itself; the mean of cos theta
    is a / (3 (1 - a)); a cardioid (a = 1/2) sends 3/4 of its rays forward;
    the mean direction lies along the axis."""
    N = 200_000
    assert np.array_equal(oracle.source_directions(N, (0, 0, 1), 0.0), oracle.fibonacci(N))
    g = np.random.default_rng(0)
    for a in (0.1, 0.3, 0.5):
        w = g.normal(size=3)
        w /= np.linalg.norm(w)
        d = oracle.source_directions(N, w, a)
        assert np.allclose(np.linalg.norm(d, axis=1), 1.0, atol=1e-6)
        mu = d @ w
        assert abs(mu.mean() - a / (3 * (1 - a))) < 2e-3
        fwd = (1 - a / 2) / (2 * (1 - a))
        assert abs((mu > 0).mean() - fwd) < 2e-3
        perp = d - np.outer(mu, w)
        assert np.linalg.norm(perp.mean(0)) < 2e-3
    assert abs((oracle.source_directions(N, (1, 0, 0), 0.5) @ np.array([1, 0, 0]) > 0).mean() - 0.75) < 2e-3


@pytest.mark.parametrize("a", [0.0, 0.25, 0.5])
def test_directional_direct_sound_counts(a):
    """Direct sound of a directional source (Sec. 1.2 footnote) through the
    whole oracle trace: the rays of a source pointing along +x that cross a
    sphere of radius r at distance d in front of / behind it number N times
    the cap integral of the density (1 - a + a mu) / (2 (1 - a)) over
    mu >= c, resp. mu <= -c, c = sqrt(1 - r^2 / d^2).  The warped lattice is
    stratified in mu about the axis, so the counts hold to a ray or two."""
    import copy
    N, d, r = 200_000, 3.0, 0.5
    sc = copy.copy(scenes.shoebox(L=(40.0, 40.0, 40.0), source=(20.0, 20.0, 20.0), alpha=1.0,
                                  n_rays=N, n_bounces=1))
    sc.rcv_center = np.array([[20.0 + d, 20.0, 20.0], [20.0 - d, 20.0, 20.0]])
    sc.rcv_radius = np.array([r, r])
    sc.rcv_source = np.array([0, 0], np.int32)
    sc = scenes.directional(sc, [1.0, 0.0, 0.0], a)
    tr = oracle.trace(oracle.OracleScene(sc, tree=False))
    direct = tr.rec_m == 0
    c = math.sqrt(1.0 - (r / d) ** 2)
    for k, side in ((0, 1.0), (1, -1.0)):
        n = int(np.sum(direct & (tr.rec_rcv == k)))
        want = N * ((1 - a) * (1 - c) + side * 0.5 * a * (1 - c * c)) / (2 * (1 - a))
        assert abs(n - want) <= 2 + 1e-3 * want, (k, n, want)
