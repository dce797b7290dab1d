"""Seeded synthetic scenes: the inputs of the ray-propagation path.

This module produces input arrays only.  It holds none of the method's
arithmetic (no ray generation, intersection, reflection, absorption decay,
image-source construction or binning); the CUDA library and the CPU oracle
both consume these arrays and nothing else from each other.

Every coordinate is rounded to a value that float32 represents exactly and
then stored as float64, so the float32 device path and the float64 oracle see
bit-identical geometry, sources and receivers.

Scenes (sizes are the workloads of the paper's experiments, rebuilt
synthetically because the paper's meshes are not published):

* ``shoebox``     -- 12-triangle rectangular room (paper Sec. 3.2, McGovern test).
* ``lroom``       -- L-shaped room on a shared grid (watertight; every edge shared).
* ``theatre``     -- procedural open-air theatre, ~436,000 triangles (paper Sec. 4).
* ``icosphere``   -- reflecting unit sphere (paper Sec. 3.1).
* ``tetra``       -- refined unit tetrahedron (paper Sec. 2.2, Table 2 workload).
* ``batched_rooms`` -- many shoeboxes / L-rooms of uneven size.

Absorption tables are per-material, 8 octave bands 62.5 Hz .. 8 kHz (paper
Table 1 lists the band layout).  ``iso9613_beta`` turns ISO 9613-1's published
atmospheric attenuation equations into the per-band energy coefficient beta(f)
(1/m) that eq. 19 uses.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

N_BANDS = 8
#: octave band centres 62.5 Hz .. 8 kHz (paper Table 1 header).
BAND_HZ = np.array([1000.0 * 2.0 ** (k - 4) for k in range(N_BANDS)])

#: paper Table 1: Odeon materials 1, 2, 107, 3000, eight bands each.
TABLE1_ALPHA = {
    1: [1, 1, 1, 1, 1, 1, 1, 1],
    2: [0, 0, 0, 0, 0, 0, 0, 0],
    107: [0.36, 0.36, 0.44, 0.31, 0.29, 0.39, 0.25, 0.25],
    3000: [0.4, 0.4, 0.3, 0.2, 0.17, 0.15, 0.1, 0.1],
}


def f32(x):
    """Round to the nearest float32 and return float64 (exactly representable)."""
    return np.asarray(x, dtype=np.float64).astype(np.float32).astype(np.float64)


@dataclass
class Scene:
    name: str
    vertices: np.ndarray          # float64 [V,3], float32-exact values
    tris: np.ndarray              # int32 [M,3]
    material_id: np.ndarray       # int32 [M]
    surface_id: np.ndarray        # int32 [M]  (coplanar, same-material groups)
    alpha: np.ndarray             # float32 [n_mat, 8] band absorption
    beta: np.ndarray              # float32 [8] air attenuation on energy (1/m)
    sources: np.ndarray           # float64 [S,3], float32-exact
    rcv_center: np.ndarray        # float64 [R,3], float32-exact
    rcv_radius: np.ndarray        # float64 [R], float32-exact
    rcv_source: np.ndarray        # int32 [R]: index of the source each receiver listens to
    n_rays: int                   # rays per source
    n_bounces: int                # nearest-hit queries per ray (cap)
    c: float = 343.2              # sound speed (m/s)
    fs: float = 48000.0           # RIR sample rate (Hz)
    max_distance: float = 0.0     # <=0: off; else eq. 13 range cap on path length
    src_axis: np.ndarray = None   # float64 [S,3] unit axes of directional sources, or None (omnidirectional)
    src_pattern: np.ndarray = None  # float64 [S] pattern a in [0, 1/2]: ray density 1 - a + a cos(theta)
    meta: dict = field(default_factory=dict)

    @property
    def n_tris(self) -> int:
        return int(self.tris.shape[0])

    @property
    def n_materials(self) -> int:
        return int(self.alpha.shape[0])

    @property
    def n_surfaces(self) -> int:
        return int(self.surface_id.max()) + 1 if self.n_tris else 0

    def tri_coords(self) -> np.ndarray:
        """[M,3,3] float64 vertex coordinates per triangle."""
        return self.vertices[self.tris]

    def diameter(self) -> float:
        if self.n_tris == 0:
            return 1.0
        v = self.vertices
        return float(np.linalg.norm(v.max(0) - v.min(0)))


# ----------------------------------------------------------------------------
# triangle-soup assembly
# ----------------------------------------------------------------------------
class _Soup:
    """Collects triangles as coordinate triples plus material / surface ids."""

    def __init__(self):
        self.coords, self.mat, self.surf = [], [], []
        self.n_surf = 0

    def new_surface(self) -> int:
        s = self.n_surf
        self.n_surf += 1
        return s

    def add(self, tri_xyz: np.ndarray, material: int, surface):
        """Triangles of one material; `surface` is one id or one id per triangle."""
        tri_xyz = np.asarray(tri_xyz, dtype=np.float64).reshape(-1, 3, 3)
        self.coords.append(tri_xyz)
        self.mat.append(np.full(len(tri_xyz), material, np.int32))
        surface = np.asarray(surface, np.int32)
        self.surf.append(np.broadcast_to(surface, (len(tri_xyz),)).astype(np.int32))

    def new_surfaces(self, n: int) -> np.ndarray:
        s = np.arange(self.n_surf, self.n_surf + n, dtype=np.int32)
        self.n_surf += n
        return s

    def grid(self, p0, a, b, na: int, nb: int, material: int, surface: int, keep=None):
        """Planar parallelogram p0 + i/na * a + j/nb * b, split into 2 triangles per cell.

        ``keep(i, j) -> bool array`` removes cells (holes).  Vertex positions
        are computed per grid index, so edges shared with another grid on the
        same lattice produce identical coordinates.
        """
        p0, a, b = (np.asarray(x, np.float64) for x in (p0, a, b))
        ii, jj = np.meshgrid(np.arange(na), np.arange(nb), indexing="ij")
        ii, jj = ii.ravel(), jj.ravel()
        if keep is not None:
            m = keep(ii, jj)
            ii, jj = ii[m], jj[m]

        def P(i, j):
            return p0 + (i[:, None] / na) * a + (j[:, None] / nb) * b

        v00, v10, v01, v11 = P(ii, jj), P(ii + 1, jj), P(ii, jj + 1), P(ii + 1, jj + 1)
        t1 = np.stack([v00, v10, v11], 1)
        t2 = np.stack([v00, v11, v01], 1)
        self.add(np.concatenate([t1, t2]), material, surface)

    def finish(self):
        coords = np.concatenate(self.coords) if self.coords else np.zeros((0, 3, 3))
        coords = f32(coords)
        flat = coords.reshape(-1, 3)
        uniq, inv = np.unique(flat.astype(np.float32), axis=0, return_inverse=True)
        tris = inv.reshape(-1, 3).astype(np.int32)
        verts = uniq.astype(np.float64)
        mat = np.concatenate(self.mat) if self.mat else np.zeros(0, np.int32)
        surf = np.concatenate(self.surf) if self.surf else np.zeros(0, np.int32)
        # drop triangles that collapsed to zero area after rounding
        d = verts[tris]
        area2 = np.linalg.norm(np.cross(d[:, 1] - d[:, 0], d[:, 2] - d[:, 0]), axis=1)
        ok = area2 > 0
        return verts, tris[ok], mat[ok], surf[ok]


def _box_faces(soup: _Soup, lo, hi, material, cells=None):
    """Six faces of an axis-aligned box, each a separate surface."""
    lo, hi = np.asarray(lo, float), np.asarray(hi, float)
    L = hi - lo
    ex, ey, ez = np.eye(3)
    faces = [
        (lo, ey * L[1], ez * L[2], 1, 2),
        (lo + ex * L[0], ey * L[1], ez * L[2], 1, 2),
        (lo, ex * L[0], ez * L[2], 0, 2),
        (lo + ey * L[1], ex * L[0], ez * L[2], 0, 2),
        (lo, ex * L[0], ey * L[1], 0, 1),
        (lo + ez * L[2], ex * L[0], ey * L[1], 0, 1),
    ]
    for k, (p0, a, b, ia, ib) in enumerate(faces):
        mat = material[k] if isinstance(material, (list, tuple, np.ndarray)) else material
        if cells is None:
            na = nb = 1
        else:
            na = max(1, int(round(L[ia] / cells)))
            nb = max(1, int(round(L[ib] / cells)))
        soup.grid(p0, a, b, na, nb, mat, soup.new_surface())


def _scene(name, soup, alpha, beta, sources, rcv_center, rcv_radius, rcv_source,
           n_rays, n_bounces, **kw) -> Scene:
    verts, tris, mat, surf = soup.finish()
    return Scene(
        name=name, vertices=verts, tris=tris, material_id=mat, surface_id=surf,
        alpha=np.asarray(alpha, np.float32).reshape(-1, N_BANDS),
        beta=np.asarray(beta, np.float32).reshape(N_BANDS),
        sources=f32(np.asarray(sources, float).reshape(-1, 3)),
        rcv_center=f32(np.asarray(rcv_center, float).reshape(-1, 3)),
        rcv_radius=f32(np.asarray(rcv_radius, float).reshape(-1)),
        rcv_source=np.asarray(rcv_source, np.int32).reshape(-1),
        n_rays=int(n_rays), n_bounces=int(n_bounces), **kw)


# ----------------------------------------------------------------------------
# air attenuation (ISO 9613-1 published equations) -> energy coefficient 1/m
# ----------------------------------------------------------------------------
def iso9613_beta(temp_c=20.0, rh_percent=50.0, pa_kpa=101.325, freqs=BAND_HZ):
    """Per-band energy attenuation beta (1/m) from ISO 9613-1's pure-tone formula.

    ISO 9613-1 gives the attenuation a in dB/m; energy decays as
    exp(-beta d) with beta = a ln(10) / 10.
    """
    T = temp_c + 273.15
    T0, T01, pr = 293.15, 273.16, 101.325
    pa = pa_kpa / pr
    C = -6.8346 * (T01 / T) ** 1.261 + 4.6151
    h = rh_percent * 10.0 ** C / pa            # molar concentration of water vapour (%)
    frO = pa * (24.0 + 4.04e4 * h * (0.02 + h) / (0.391 + h))
    frN = pa * (T / T0) ** -0.5 * (9.0 + 280.0 * h * math.exp(-4.170 * ((T / T0) ** (-1.0 / 3.0) - 1.0)))
    f = np.asarray(freqs, float)
    a_db = 8.686 * f ** 2 * (
        1.84e-11 / pa * (T / T0) ** 0.5
        + (T / T0) ** -2.5 * (
            0.01275 * math.exp(-2239.1 / T) / (frO + f ** 2 / frO)
            + 0.1068 * math.exp(-3352.0 / T) / (frN + f ** 2 / frN)))
    return (a_db * math.log(10.0) / 10.0).astype(np.float32)


def seeded_alpha(n_mat, seed, lo=0.02, hi=0.6):
    rng = np.random.default_rng(seed)
    return rng.uniform(lo, hi, size=(n_mat, N_BANDS)).astype(np.float32)


# ----------------------------------------------------------------------------
# scenes
# ----------------------------------------------------------------------------
def shoebox(L=(10.0, 7.0, 3.0), source=(2.0, 3.0, 1.5), receiver=(7.0, 4.0, 1.7),
            radius=0.5, alpha=0.1, n_rays=10_000, n_bounces=20, beta=None,
            face_materials=None, alpha_table=None, max_distance=0.0, cells=None,
            fs=48000.0) -> Scene:
    """Rectangular room [0,Lx]x[0,Ly]x[0,Lz], 2 triangles per face (fixed diagonal).

    Defaults: 10x7x3 m, alpha 0.1 in every band, no air loss, source
    (2,3,1.5), receiver sphere r=0.5 at (7,4,1.7), 10,000 rays, 20 bounces.
    Face order: x=0, x=Lx, y=0, y=Ly, z=0, z=Lz (surface ids 0..5).
    """
    soup = _Soup()
    if face_materials is None:
        face_materials = [0] * 6
        alpha_tab = np.full((1, N_BANDS), alpha, np.float32)
    else:
        alpha_tab = np.asarray(alpha_table, np.float32)
    _box_faces(soup, (0, 0, 0), L, list(face_materials), cells=cells)
    beta = np.zeros(N_BANDS, np.float32) if beta is None else beta
    return _scene("shoebox", soup, alpha_tab, beta, [source], [receiver], [radius], [0],
                  n_rays, n_bounces, max_distance=max_distance, fs=fs,
                  meta={"L": tuple(float(x) for x in L)})


def paper_shoebox(n_rays=100_000, seed=0) -> Scene:
    """The paper's Sec. 3.2 shoebox: [5,4,3] m, source [4,2,1.7], sphere r=0.2 at
    [2,2,1.7], 1e5 rays, walls drawn from Table 1's two finite materials,
    ISO 9613-1 air, iterations stopped by eq. 13 (n=1)."""
    rng = np.random.default_rng(seed)
    mats = [107, 3000]
    face_mat = rng.integers(0, 2, size=6)
    alpha_tab = np.array([TABLE1_ALPHA[m] for m in mats], np.float32)
    r = 0.2
    dmax = (r / 2.0) * math.sqrt(n_rays)          # eq. 13 with n = 1
    return shoebox(L=(5.0, 4.0, 3.0), source=(4.0, 2.0, 1.7), receiver=(2.0, 2.0, 1.7),
                   radius=r, n_rays=n_rays, n_bounces=64, beta=iso9613_beta(),
                   face_materials=face_mat, alpha_table=alpha_tab, max_distance=dmax)


def directional(sc: Scene, axis, pattern) -> Scene:
    """A copy of `sc` whose sources are directional (Sec. 1.2 footnote): rays
    of equal energy sampled with density 1 - a + a cos(theta) about `axis`
    (one [3] for all sources or [S, 3]; normalised here), a = `pattern` in
    [0, 1/2] (0 = omnidirectional lattice turned to the axis, 1/2 = cardioid)."""
    import copy
    out = copy.copy(sc)
    S = len(sc.sources)
    ax = np.broadcast_to(np.asarray(axis, np.float64).reshape(-1, 3), (S, 3)).copy()
    ax /= np.sqrt((ax * ax).sum(1, keepdims=True))
    out.src_axis = ax
    out.src_pattern = np.broadcast_to(np.asarray(pattern, np.float64).reshape(-1), (S,)).copy()
    return out


LROOM_FOOTPRINT = [(0, 0), (20, 0), (20, 7.5), (10, 7.5), (10, 15), (0, 15)]


def lroom(h=0.125, height=5.0, n_rays=1_000_000, n_bounces=50, n_receivers=4, seed=2,
          alpha=None, beta=None) -> Scene:
    """L-shaped room, footprint (0,0)(20,0)(20,7.5)(10,7.5)(10,15)(0,15), height 5 m.

    Every face is meshed on one shared h-grid (2 triangles per square), so all
    edges are shared and vertices are float32-exact: 800 m^2 / h^2 * 2
    triangles (102,400 at h = 0.125).  4 materials: floor, ceiling and two wall
    groups, alpha ~ U[0.02, 0.6] per band (seeded).  Surfaces: floor, ceiling
    and the 6 walls.
    """
    for v in (7.5, 10.0, height):
        if abs(v / h - round(v / h)) > 1e-9:
            raise ValueError("grid step h must divide 7.5, 10 and the height")
    rng = np.random.default_rng(seed)
    soup = _Soup()
    fp = np.array(LROOM_FOOTPRINT, float)

    def in_l(x, y):
        return (x < 10) | (y < 7.5)

    # floor and ceiling: h-grid over [0,20]x[0,15], keep cells inside the L
    nx, ny = int(round(20 / h)), int(round(15 / h))
    keep = lambda i, j: in_l((i + 0.5) * h, (j + 0.5) * h)
    soup.grid((0, 0, 0), (20, 0, 0), (0, 15, 0), nx, ny, 0, soup.new_surface(), keep)
    soup.grid((0, 0, height), (20, 0, 0), (0, 15, 0), nx, ny, 1, soup.new_surface(), keep)
    nz = int(round(height / h))
    for k in range(len(fp)):
        p, q = fp[k], fp[(k + 1) % len(fp)]
        length = float(np.linalg.norm(q - p))
        na = int(round(length / h))
        mat = 2 + (k % 2)
        soup.grid((p[0], p[1], 0), (q[0] - p[0], q[1] - p[1], 0), (0, 0, height),
                  na, nz, mat, soup.new_surface())
    alpha = seeded_alpha(4, seed) if alpha is None else np.asarray(alpha, np.float32)
    beta = np.zeros(N_BANDS, np.float32) if beta is None else beta
    # source and receivers: seeded points >= 1 m from every wall, in the L
    pts = []
    while len(pts) < 1 + n_receivers:
        x, y = rng.uniform(1, 19), rng.uniform(1, 14)
        if not ((x < 9) or (y < 6.5)):
            continue
        if x > 19 or y > 14 or (x > 9 and y > 6.5):
            continue
        z = rng.uniform(1.0, height - 1.0)
        pts.append((x, y, z))
    src, rcv = pts[0], pts[1:]
    return _scene("lroom", soup, alpha, beta, [src], rcv, [0.5] * n_receivers,
                  [0] * n_receivers, n_rays, n_bounces, meta={"h": h, "height": height})


def _arc(n, a0=0.0, a1=math.pi):
    """n+1 angles over [a0, a1] with exact endpoints' cos / sin snapped for 0, pi."""
    th = a0 + (a1 - a0) * np.arange(n + 1) / n
    c, s = np.cos(th), np.sin(th)
    for k, t in enumerate(th):
        if abs(t) < 1e-15 or abs(t - math.pi) < 1e-12:
            s[k] = 0.0
            c[k] = 1.0 if abs(t) < 1e-15 else -1.0
    return c, s


def _column(soup, base, radius, height, sides, nv, material):
    """Closed faceted prism: `sides` flat faces subdivided `nv` times vertically,
    plus top and bottom cap fans.  Each flat face and each cap is a surface."""
    bx, by, bz = base
    ang = 2 * math.pi * (np.arange(sides + 1) % sides) / sides
    cx, cy = bx + radius * np.cos(ang), by + radius * np.sin(ang)
    for k in range(sides):
        p0 = (cx[k], cy[k], bz)
        a = (cx[k + 1] - cx[k], cy[k + 1] - cy[k], 0.0)
        soup.grid(p0, a, (0, 0, height), 1, nv, material, soup.new_surface())
    for z, flip in ((bz, True), (bz + height, False)):
        centre = np.array([bx, by, z])
        ring = np.stack([cx, cy, np.full_like(cx, z)], 1)
        tri = [np.stack([centre, ring[k + 1], ring[k]]) if flip else
               np.stack([centre, ring[k], ring[k + 1]]) for k in range(sides)]
        soup.add(np.array(tri), material, soup.new_surface())


def theatre(n_rays=1_000_000, n_bounces=30, n_receivers=16, seed=3, arc=512,
            col_nv=17, radius=2.0) -> Scene:
    """Procedural open-air theatre, ~436,000 triangles, open sky.

    * cavea: semicircular stepped bleachers, orchestra radius 12 m, outer
      radius 50 m, 30 tiers (riser 0.55 m + tread), `arc` arc segments, each
      tread and riser subdivided 4x across;
    * orchestra half-disc and stage (pulpitum, 1.2 m high, 100 x 12 m);
    * stage wall (scaenae frons) 100 x 35 m, 3 m thick, with 3 arched
      openings (6 m wide, springline 6 m, semicircular heads);
    * 200 columns, 24-sided prisms: 120 on the top tier, 80 in two storeys in
      front of the stage wall (standing on the stage and on a ledge);
    * 6 materials with seeded alpha ~ U[0.02, 0.6]; air at 20 C / 50 % RH;
    * source 1.6 m above the front of the stage; `n_receivers` spheres of
      radius 2 m, 1.2 m above seeded tier treads.
    """
    rng = np.random.default_rng(seed)
    soup = _Soup()
    M_BLEACH, M_ORCH, M_STAGE, M_WALL, M_COL, M_SIDE = range(6)
    R0, R1, NT, rise = 12.0, 50.0, 30, 0.55
    w = (R1 - R0) / NT
    c, s = _arc(arc)
    sub = 4

    def ring_pts(r, z):
        return np.stack([r * c, r * s, np.full_like(c, z)], 1)

    for k in range(NT):
        r_in, r_out = R0 + k * w, R0 + (k + 1) * w
        z_lo, z_hi = k * rise, (k + 1) * rise
        # riser: vertical faceted strip at r_in from z_lo to z_hi; every arc
        # segment is a flat facet, so each is its own surface
        sid = soup.new_surfaces(arc)
        tri, sids = [], []
        for q in range(sub):
            za, zb = z_lo + (z_hi - z_lo) * q / sub, z_lo + (z_hi - z_lo) * (q + 1) / sub
            A, B = ring_pts(r_in, za), ring_pts(r_in, zb)
            tri.append(np.stack([A[:-1], A[1:], B[1:]], 1))
            tri.append(np.stack([A[:-1], B[1:], B[:-1]], 1))
            sids += [sid, sid]
        soup.add(np.concatenate(tri), M_BLEACH, np.concatenate(sids))
        # tread: annulus sector at z_hi from r_in to r_out
        sid = soup.new_surface()
        tri = []
        for q in range(sub):
            ra, rb = r_in + w * q / sub, r_in + w * (q + 1) / sub
            A, B = ring_pts(ra, z_hi), ring_pts(rb, z_hi)
            tri.append(np.stack([A[:-1], B[1:], A[1:]], 1))
            tri.append(np.stack([A[:-1], B[:-1], B[1:]], 1))
        soup.add(np.concatenate(tri), M_BLEACH, sid)
    # cavea side walls in the plane y = 0 (stepped profile), both ends
    for sign in (1.0, -1.0):
        sid = soup.new_surface()
        for k in range(NT):
            x0, x1 = sign * (R0 + k * w), sign * (R0 + (k + 1) * w)
            soup.grid((x0, 0, 0), (x1 - x0, 0, 0), (0, 0, (k + 1) * rise), 1, 1, M_SIDE, sid)
    # orchestra half-disc at z = 0: centre fan + rings
    nr, oseg = 8, 256
    co, so = _arc(oseg)
    sid = soup.new_surface()
    tri = []
    for q in range(nr):
        ra, rb = R0 * q / nr, R0 * (q + 1) / nr
        A = np.stack([ra * co, ra * so, 0 * co], 1)
        B = np.stack([rb * co, rb * so, 0 * co], 1)
        if q == 0:
            tri.append(np.stack([A[:-1], B[:-1], B[1:]], 1))
        else:
            tri.append(np.stack([A[:-1], B[:-1], B[1:]], 1))
            tri.append(np.stack([A[:-1], B[1:], A[1:]], 1))
    soup.add(np.concatenate(tri), M_ORCH, sid)
    # strip of orchestra floor between the stage front (y=-0.5) and y = 0
    soup.grid((-50, -0.5, 0), (100, 0, 0), (0, 0.5, 0), 100, 1, M_ORCH, soup.new_surface())
    # stage: floor at z=1.2 over y in [-12,-0.5], front face at y=-0.5
    SZ, YW, YB = 1.2, -12.0, -15.0
    soup.grid((-50, YW, SZ), (100, 0, 0), (0, 11.5, 0), 100, 23, M_STAGE, soup.new_surface())
    soup.grid((-50, -0.5, 0), (100, 0, 0), (0, 0, SZ), 100, 2, M_STAGE, soup.new_surface())
    # stage wall (front y=-12, back y=-15), x in [-50,50], z in [1.2, 36.2]
    H = 35.0
    openings = [(-26.0, 3.0), (0.0, 3.0), (26.0, 3.0)]   # (x centre, half width)
    spring = SZ + 6.0                                       # springline height

    def in_opening(x, z):
        m = np.zeros_like(x, dtype=bool)
        for xc, a in openings:
            m |= (np.abs(x - xc) < a) & (z < spring + a)
        return m

    keep = lambda i, j: ~in_opening(-50 + i + 0.5, SZ + j + 0.5)
    soup.grid((-50, YW, SZ), (100, 0, 0), (0, 0, H), 100, 35, M_WALL, soup.new_surface(), keep)
    soup.grid((-50, YB, SZ), (100, 0, 0), (0, 0, H), 100, 35, M_WALL, soup.new_surface(), keep)
    soup.grid((-50, YB, SZ + H), (100, 0, 0), (0, 3, 0), 100, 3, M_WALL, soup.new_surface())
    for x in (-50.0, 50.0):
        soup.grid((x, YB, SZ), (0, 3, 0), (0, 0, H), 3, 35, M_WALL, soup.new_surface())
    K = 16
    for xc, a in openings:
        # spandrels: fill between the square head and the semicircular arch, front and back
        phi = math.pi * np.arange(K + 1) / K
        ax, az = xc + a * np.cos(phi), spring + a * np.sin(phi)
        for y in (YW, YB):
            sid = soup.new_surface()
            tri = []
            for k in range(K):
                corner = (xc + a, spring + a) if k < K // 2 else (xc - a, spring + a)
                tri.append([[corner[0], y, corner[1]], [ax[k], y, az[k]], [ax[k + 1], y, az[k + 1]]])
            soup.add(np.array(tri), M_WALL, sid)
        # reveals: jambs and the arch intrados through the wall thickness
        for xj in (xc - a, xc + a):
            soup.grid((xj, YB, SZ), (0, 3, 0), (0, 0, spring - SZ), 3, 6, M_WALL, soup.new_surface())
        sids = soup.new_surfaces(K)
        tri = []
        for k in range(K):
            p, q = (ax[k], az[k]), (ax[k + 1], az[k + 1])
            A0, A1 = [p[0], YW, p[1]], [p[0], YB, p[1]]
            B0, B1 = [q[0], YW, q[1]], [q[0], YB, q[1]]
            tri += [[A0, A1, B1], [A0, B1, B0]]
        soup.add(np.array(tri), M_WALL, np.repeat(sids, 2))
    # ledge for the upper storey of columns: box y in [-12,-10], z in [9.2,10.2]
    _box_faces(soup, (-50, -12, SZ + 8.0), (50, -10, SZ + 9.0), M_SIDE, cells=1.0)
    # columns
    sides, crad, chgt = 24, 0.45, 8.0
    xs = []
    for x in np.linspace(-48, 48, 48):
        if all(abs(x - xc) > a + 1.0 for xc, a in openings):
            xs.append(x)
    xs = np.array(xs[:40])
    for x in xs:
        _column(soup, (x, -11.0, SZ), crad, chgt, sides, col_nv, M_COL)
        _column(soup, (x, -11.0, SZ + 9.0), crad, chgt, sides, col_nv, M_COL)
    th = np.linspace(0.02, math.pi - 0.02, 120) + rng.uniform(-0.004, 0.004, 120)
    rc = R1 - 0.6
    for t in th:
        _column(soup, (rc * math.cos(t), rc * math.sin(t), NT * rise), crad, chgt, sides,
                col_nv, M_COL)
    alpha = seeded_alpha(6, seed)
    beta = iso9613_beta(20.0, 50.0)
    src = (0.0, -2.0, SZ + 1.6)
    rcv = []
    for _ in range(n_receivers):
        k = int(rng.integers(2, NT - 1))
        t = rng.uniform(0.15 * math.pi, 0.85 * math.pi)
        r = R0 + (k + 0.5) * w
        rcv.append((r * math.cos(t), r * math.sin(t), (k + 1) * rise + 1.2))
    return _scene("theatre", soup, alpha, beta, [src], rcv, [radius] * n_receivers,
                  [0] * n_receivers, n_rays, n_bounces)


def icosphere(level=3, n_rays=100_000, n_bounces=6, radius=0.1) -> Scene:
    """100 % reflecting unit sphere from a subdivided icosahedron (20 * 4^level
    facets, each its own surface); source and receiver at the centre
    (paper Sec. 3.1)."""
    t = (1 + 5 ** 0.5) / 2
    V = np.array([[-1, t, 0], [1, t, 0], [-1, -t, 0], [1, -t, 0], [0, -1, t], [0, 1, t],
                  [0, -1, -t], [0, 1, -t], [t, 0, -1], [t, 0, 1], [-t, 0, -1], [-t, 0, 1]], float)
    F = np.array([[0, 11, 5], [0, 5, 1], [0, 1, 7], [0, 7, 10], [0, 10, 11], [1, 5, 9], [5, 11, 4],
                  [11, 10, 2], [10, 7, 6], [7, 1, 8], [3, 9, 4], [3, 4, 2], [3, 2, 6], [3, 6, 8],
                  [3, 8, 9], [4, 9, 5], [2, 4, 11], [6, 2, 10], [8, 6, 7], [9, 8, 1]])
    V /= np.linalg.norm(V, axis=1, keepdims=True)
    for _ in range(level):
        cache, newF, verts = {}, [], list(V)

        def mid(i, j):
            key = (min(i, j), max(i, j))
            if key not in cache:
                m = (verts[i] + verts[j]) / 2
                verts.append(m / np.linalg.norm(m))
                cache[key] = len(verts) - 1
            return cache[key]

        for a, b, c_ in F:
            ab, bc, ca = mid(a, b), mid(b, c_), mid(c_, a)
            newF += [[a, ab, ca], [b, bc, ab], [c_, ca, bc], [ab, bc, ca]]
        V, F = np.array(verts), np.array(newF)
    soup = _Soup()
    tri = V[F]
    soup.coords.append(tri)
    soup.mat.append(np.zeros(len(F), np.int32))
    soup.surf.append(np.arange(len(F), dtype=np.int32))
    soup.n_surf = len(F)
    return _scene("icosphere", soup, np.zeros((1, N_BANDS)), np.zeros(N_BANDS), [(0, 0, 0)],
                  [(0, 0, 0)], [radius], [0], n_rays, n_bounces)


def tetra(level=4, n_rays=None, n_bounces=1) -> Scene:
    """Unit regular tetrahedron (circumradius 1) with each face refined
    `level` times into 4 (4 * 4^level faces); source at the centre
    (paper Sec. 2.2, Table 2: N = M)."""
    V = np.array([[1, 1, 1], [1, -1, -1], [-1, 1, -1], [-1, -1, 1]], float) / math.sqrt(3)
    F = [(0, 1, 2), (0, 3, 1), (0, 2, 3), (1, 3, 2)]
    soup = _Soup()
    n = 2 ** level
    # lattice points (i, j), i + j <= n; per (i, j) an "up" triangle and, away
    # from the far edge, a "down" one, in the same order as a row-by-row loop
    ii, jj = [], []
    for i in range(n):
        jj.append(np.arange(n - i))
        ii.append(np.full(n - i, i))
    ii, jj = np.concatenate(ii), np.concatenate(jj)
    down = jj < n - ii - 1
    for fi, (a, b, c_) in enumerate(F):
        A, B, C = V[a], V[b], V[c_]
        p = lambda u, v: A + (B - A) * (u[:, None] / n) + (C - A) * (v[:, None] / n)
        up_t = np.stack([p(ii, jj), p(ii + 1, jj), p(ii, jj + 1)], axis=1)
        dn_t = np.stack([p(ii + 1, jj), p(ii + 1, jj + 1), p(ii, jj + 1)], axis=1)
        # interleave: up(i, j), down(i, j) where it exists
        order = np.argsort(np.concatenate([2 * np.arange(len(ii)), 2 * np.nonzero(down)[0] + 1]), kind="stable")
        tri = np.concatenate([up_t, dn_t[down]])[order]
        soup.add(tri, 0, soup.new_surface())
    M = 4 * 4 ** level
    return _scene("tetra", soup, np.full((1, N_BANDS), 0.1), np.zeros(N_BANDS), [(0, 0, 0)],
                  [(0.3, 0.1, 0.05)], [0.05], [0], n_rays or M, n_bounces)


def batched_rooms(n_rooms=64, pairs=16, n_rays=262_144, n_bounces=30, seed=4,
                  m_min=12, m_max=200_000, radius=0.5):
    """Rooms of uneven size for one batched launch: shoeboxes (even index) and
    L-rooms (odd index, once the target size allows a grid) whose triangle
    counts are log-uniform on [m_min, m_max] (seeded), 4 materials with
    seeded 8-band absorption, and `pairs` source / receiver pairs each
    (receiver k of a room listens to source k; r = `radius`), placed at seeded
    points at least 0.75 m (or 20 % of the extent) inside the walls and 1 m
    apart.  meta holds the kind and the target size."""
    rng = np.random.default_rng(seed)
    out = []
    for q in range(n_rooms):
        target = math.exp(rng.uniform(math.log(m_min), math.log(m_max)))
        dims = np.round(rng.uniform([4, 3, 2.5], [30, 20, 10]), 1)
        alpha = seeded_alpha(4, int(rng.integers(1 << 31)))
        kind = "shoebox" if (q % 2 == 0) else "lroom"
        S = 2 * (dims[0] * dims[1] + dims[1] * dims[2] + dims[0] * dims[2])
        cell = math.sqrt(2 * S / target) if target > 12 else None
        if kind == "lroom" and target > 400:
            # L-room scaled into dims: grid h from area 800 * scale^2
            sc = dims[0] / 20.0
            h = max(0.05, math.sqrt(2 * 800 * sc * sc / target))
            h = 1.0 / max(1, round(1.0 / h * 1.0)) if h < 1 else round(h * 2) / 2
            soup, ext = _scaled_lroom(sc, dims[2], h, rng)
            inside = lambda p, sc=sc: (p[0] < 10 * sc) or (p[1] < 7.5 * sc)
        else:
            kind = "shoebox"
            soup = _Soup()
            _box_faces(soup, (0, 0, 0), dims, list(rng.integers(0, 4, 6)),
                       cells=None if cell is None else max(0.05, cell))
            ext = dims
            inside = lambda p: True
        margin = np.minimum(0.75, 0.2 * ext)
        src, rcv = [], []
        for _ in range(pairs):
            for _try in range(1000):
                a_ = rng.uniform(margin, ext - margin)
                b_ = rng.uniform(margin, ext - margin)
                if inside(a_) and inside(b_) and np.linalg.norm(a_ - b_) >= 1.0:
                    break
            src.append(a_)
            rcv.append(b_)
        room = _scene(f"batched room {q}", soup, alpha, np.zeros(N_BANDS), src, rcv, [radius] * pairs,
                      np.arange(pairs), n_rays, n_bounces)
        room.meta.update({"kind": kind, "target_tris": target})
        out.append(room)
    return out


def _scaled_lroom(sc, height, h, rng):
    soup = _Soup()
    fp = np.array(LROOM_FOOTPRINT, float) * sc
    X, Y = 20 * sc, 15 * sc
    nx, ny = max(1, int(round(X / h))), max(1, int(round(Y / h)))
    keep = lambda i, j: ((i + 0.5) * X / nx < 10 * sc) | ((j + 0.5) * Y / ny < 7.5 * sc)
    soup.grid((0, 0, 0), (X, 0, 0), (0, Y, 0), nx, ny, 0, soup.new_surface(), keep)
    soup.grid((0, 0, height), (X, 0, 0), (0, Y, 0), nx, ny, 1, soup.new_surface(), keep)
    nz = max(1, int(round(height / h)))
    for k in range(len(fp)):
        p, q = fp[k], fp[(k + 1) % len(fp)]
        na = max(1, int(round(np.linalg.norm(q - p) / h)))
        soup.grid((p[0], p[1], 0), (q[0] - p[0], q[1] - p[1], 0), (0, 0, height), na, nz,
                  2 + (k % 2), soup.new_surface())
    return (soup, np.array([X, Y, height]))


# ----------------------------------------------------------------------------
# rooms for the learned late-reverberation tail
# ----------------------------------------------------------------------------
def surrogate_room(seed: int, v_min=50.0, v_max=20_000.0, radius=0.5, n_rays=65_536, n_bounces=64) -> Scene:
    """One seeded room of the surrogate data set: a shoebox (even seeds) or an
    L-room (odd seeds, a 2.5 m-grid L-room scaled per axis, watertight), with
    volume log-uniform in [v_min, v_max], 3 materials with alpha ~ U[0.02,
    0.6] per band assigned per surface, one source and one receiver sphere
    (radius `radius`) at seeded points at least 1 m (or 20 % of the room)
    inside the walls.  meta holds the analytic volume and surface area."""
    rng = np.random.default_rng(seed)
    V = math.exp(rng.uniform(math.log(v_min), math.log(v_max)))
    alpha = seeded_alpha(3, int(rng.integers(1 << 31)))
    if seed % 2 == 0:
        a = rng.uniform(0.6, 1.6, 3) * np.array([1.4, 1.0, 0.55])
        L = a * (V / np.prod(a)) ** (1.0 / 3.0)
        L = f32(L)
        soup = _Soup()
        _box_faces(soup, (0, 0, 0), L, list(rng.integers(0, 3, 6)))
        Vt = float(np.prod(L))
        St = 2.0 * float(L[0] * L[1] + L[1] * L[2] + L[0] * L[2])
        lo, hi = np.zeros(3), L
        inside = lambda p: True
    else:
        base = lroom(h=2.5, n_rays=1, n_bounces=1, n_receivers=1, seed=seed)
        # L-room area 225 m^2, height 5 m -> volume 1125 m^3; scale per axis
        sxy = rng.uniform(0.7, 1.4)
        k = (V / (1125.0)) ** (1.0 / 3.0)
        sc = np.array([k * sxy, k / sxy, k * rng.uniform(0.5, 1.0)])
        verts = f32(base.vertices * sc)
        mat = rng.integers(0, 3, base.n_surfaces)[base.surface_id].astype(np.int32)
        soup = _Soup()
        soup.coords.append(verts[base.tris])
        soup.mat.append(mat)
        soup.surf.append(base.surface_id.copy())
        soup.n_surf = base.n_surfaces
        Vt = 1125.0 * float(np.prod(sc))
        St = 2 * 225.0 * sc[0] * sc[1] + 5.0 * sc[2] * (2 * 20 * sc[0] + 2 * 15 * sc[1])
        lo, hi = np.zeros(3), np.array([20 * sc[0], 15 * sc[1], 5 * sc[2]])
        inside = lambda p: (p[0] < 10 * sc[0]) or (p[1] < 7.5 * sc[1])
    margin = np.minimum(1.0, 0.2 * (hi - lo))
    pts = []
    while len(pts) < 2:
        p = rng.uniform(lo + margin, hi - margin)
        if inside(p) and inside(p + np.array([margin[0], margin[1], 0])) and \
                inside(p - np.array([0, 0, 0])):
            pts.append(p)
    sc_ = _scene("surrogate_room", soup, alpha, np.zeros(N_BANDS), [pts[0]], [pts[1]], [radius], [0],
                 n_rays, n_bounces)
    sc_.meta.update({"V": Vt, "S": St, "kind": "shoebox" if seed % 2 == 0 else "lroom"})
    return sc_
