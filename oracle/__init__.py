"""FP64 CPU oracle of the ray-propagation path -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA
library (``paper_1811_05784_gb300``) and never imports it; the two meet only
in the seeded input arrays of ``scenes``.

Layout:
  rt_oracle.c   -- ray generation, nearest element (brute force and the
                   paper's median-split tree), measurement spheres,
                   reflection, absorption, eq. 13 range (plain C, FP64)
  this file     -- ctypes loader; image sources by reflection sequence
                   (Sec. 1.4, eq. 19), energy histograms (Sec. 1.4),
                   Schroeder decay, EDT and T30 (plain numpy, FP64)

Citations are to Aussal & Gueguen (2018), arXiv:1811.05784.
"""
from __future__ import annotations

import ctypes as C
import math
import os
import subprocess
import sys
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

N_BANDS = 8


def build(force: bool = False) -> str:
    """Compile rt_oracle.c with gcc (no fused multiply-add contraction)."""
    src = os.path.join(_HERE, "rt_oracle.c")
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(src):
        return _LIB
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-fPIC", "-shared", "-pthread",
           "-ffp-contract=off", "-fno-fast-math", src, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            P = C.c_void_p
            i32, i64, f64 = C.c_int32, C.c_int64, C.c_double
            L.orc_scene_new.restype = P
            L.orc_scene_new.argtypes = [P, i64, P, i64, P, P, P, i32, i32]
            L.orc_scene_free.argtypes = [P]
            L.orc_tree_nodes.restype = i64
            L.orc_tree_nodes.argtypes = [P]
            L.orc_scene_diameter.restype = f64
            L.orc_scene_diameter.argtypes = [P]
            L.orc_fibonacci.argtypes = [i64, i64, P, P]
            L.orc_directions.argtypes = [i64, i64, P, P, f64, P]
            L.orc_nearest.argtypes = [P, i64, P, P, P, i32, f64, i32, P, P, P, P]
            L.orc_crossings.restype = i64
            L.orc_crossings.argtypes = [i64, P, P, P, P, i64, P, P, P, i64, P, P, P]
            L.orc_trace.restype = i64
            L.orc_trace.argtypes = [P, P, P, P, i64, P, P, P, i64, i64, P, P, i32, f64, i32, f64, i32,
                                    P, P, P, P, P, P, i64, P, P, P, P, P, P, P]
            _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


def default_threads() -> int:
    return max(1, os.cpu_count() or 1)


#: default half-width of the near-edge band, relative to the coordinate scale
EPS_EDGE_REL = 2e-6


class OracleScene:
    """Triangles, materials and (optionally) the paper's median-split tree."""

    def __init__(self, scene, tree: bool = True):
        self.scene = scene
        self._V = np.ascontiguousarray(scene.vertices, np.float64)
        self._T = np.ascontiguousarray(scene.tris, np.int32)
        self._mat = np.ascontiguousarray(scene.material_id, np.int32)
        self._surf = np.ascontiguousarray(scene.surface_id, np.int32)
        self._alpha = np.ascontiguousarray(scene.alpha.astype(np.float64))
        L = lib()
        self.h = L.orc_scene_new(_p(self._V), len(self._V), _p(self._T), len(self._T), _p(self._mat),
                                 _p(self._surf), _p(self._alpha), self._alpha.shape[0], int(tree))
        self.has_tree = tree

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            lib().orc_scene_free(h)
            self.h = None

    @property
    def tree_nodes(self) -> int:
        return int(lib().orc_tree_nodes(self.h))

    @property
    def diameter(self) -> float:
        return float(lib().orc_scene_diameter(self.h))

    # -- single queries (lockstep comparison) ------------------------------
    def nearest(self, org, dirs, exclude=None, brute=False, eps_edge_rel=EPS_EDGE_REL, threads=None):
        """Nearest admissible triangle for each (origin, direction) (Sec. 2.1).

        Returns (tri int32 [-1 = none], delta, second delta, ambiguous flag)."""
        org = np.ascontiguousarray(org, np.float64).reshape(-1, 3)
        dirs = np.ascontiguousarray(dirs, np.float64).reshape(-1, 3)
        n = len(org)
        ex = None if exclude is None else np.ascontiguousarray(exclude, np.int32)
        tri = np.empty(n, np.int32)
        d1 = np.empty(n)
        d2 = np.empty(n)
        amb = np.empty(n, np.int32)
        lib().orc_nearest(self.h, n, _p(org), _p(dirs), _p(ex), int(brute or not self.has_tree),
                          eps_edge_rel, threads or default_threads(), _p(tri), _p(d1), _p(d2), _p(amb))
        return tri, d1, d2, amb.astype(bool)


def crossings(scene, org, dirs, seg, ray_src=None):
    """Measurement-sphere crossings of given segments (eq. 22), lockstep use.

    Returns (segment index, receiver, margin (r - dist)/r) arrays."""
    org = np.ascontiguousarray(org, np.float64).reshape(-1, 3)
    dirs = np.ascontiguousarray(dirs, np.float64).reshape(-1, 3)
    seg = np.ascontiguousarray(seg, np.float64).reshape(-1)
    n = len(org)
    rs = np.zeros(n, np.int32) if ray_src is None else np.ascontiguousarray(ray_src, np.int32)
    rc = np.ascontiguousarray(scene.rcv_center, np.float64)
    rr = np.ascontiguousarray(scene.rcv_radius, np.float64)
    rsrc = np.ascontiguousarray(scene.rcv_source, np.int32)
    cap = max(1024, 2 * n)
    while True:
        a, b, c = np.empty(cap, np.int64), np.empty(cap, np.int32), np.empty(cap)
        k = lib().orc_crossings(n, _p(org), _p(dirs), _p(seg), _p(rs), len(rc), _p(rc), _p(rr), _p(rsrc), cap,
                                _p(a), _p(b), _p(c))
        if k <= cap:
            return a[:k], b[:k], c[:k]
        cap = int(k)


def fibonacci(N: int, ids=None) -> np.ndarray:
    """Fibonacci-rule unit sphere sampling (Sec. 1.2), float32-rounded."""
    ids = np.arange(N, dtype=np.int64) if ids is None else np.ascontiguousarray(ids, np.int64)
    out = np.empty((len(ids), 3))
    lib().orc_fibonacci(int(N), len(ids), _p(ids), _p(out))
    return out


def source_directions(N: int, axis, pattern: float, ids=None) -> np.ndarray:
    """Ray directions of a directional source (Sec. 1.2 footnote: non-uniform
    sampling with equal ray energies): density (1 - a + a cos theta) about
    the unit `axis`, a = `pattern` in [0, 1/2]; float32-rounded."""
    ids = np.arange(N, dtype=np.int64) if ids is None else np.ascontiguousarray(ids, np.int64)
    w = np.ascontiguousarray(axis, np.float64).reshape(3)
    out = np.empty((len(ids), 3))
    lib().orc_directions(int(N), len(ids), _p(ids), _p(w), float(pattern), _p(out))
    return out


@dataclass
class TraceResult:
    ray_src: np.ndarray        # int32 [n]
    ray_id: np.ndarray         # int64 [n] index within its source's N rays
    hist: np.ndarray           # int32 [n, B] triangle hit at bounce b, -1 = none
    hist_t: np.ndarray         # float64 [n, B] hit distance
    E: np.ndarray              # float64 [n, 8] band energy after the last hit
    L: np.ndarray              # float64 [n] path length
    first_amb: np.ndarray      # int32 [n] first ambiguous bounce (B = none)
    n_hits: np.ndarray         # int32 [n]
    rec_rcv: np.ndarray        # int32 [k]
    rec_ray: np.ndarray        # int64 [k] index into the ray list
    rec_m: np.ndarray          # int32 [k] reflection order
    rec_L: np.ndarray          # float64 [k] path length at the closest point
    rec_margin: np.ndarray     # float64 [k] (r - dist)/r
    rec_pos: np.ndarray        # float64 [k,3] closest point
    rec_dir: np.ndarray        # float64 [k,3] direction of the crossing segment
    N: int
    B: int

    dmax: float = 0.0

    @property
    def escaped(self) -> np.ndarray:
        """Rays eliminated because their last query met no surface."""
        stopped = (self.L > self.dmax) if self.dmax > 0 else np.zeros(len(self.L), bool)
        return (self.n_hits < self.B) & ~stopped

    @property
    def queries(self) -> int:
        """Nearest-element queries resolved (hits plus escapes)."""
        return int(self.n_hits.sum() + self.escaped.sum())


def trace(osc: OracleScene, ray_ids=None, ray_src=None, brute=False, n_bounces=None,
          max_distance=None, eps_edge_rel=EPS_EDGE_REL, threads=None, rec_cap=None) -> TraceResult:
    """Free-running propagation of the listed rays (Sec. 1.2-1.3, 2.1).

    ``ray_ids`` index each source's N Fibonacci rays (default: all N of every
    source); ``ray_src`` gives the source of each listed ray."""
    sc = osc.scene
    N = sc.n_rays
    S = len(sc.sources)
    if ray_ids is None:
        ray_ids = np.tile(np.arange(N, dtype=np.int64), S)
        ray_src = np.repeat(np.arange(S, dtype=np.int32), N)
    ray_ids = np.ascontiguousarray(ray_ids, np.int64)
    ray_src = (np.zeros(len(ray_ids), np.int32) if ray_src is None
               else np.ascontiguousarray(ray_src, np.int32))
    n = len(ray_ids)
    B = int(sc.n_bounces if n_bounces is None else n_bounces)
    dmax = float(sc.max_distance if max_distance is None else max_distance)
    src = np.ascontiguousarray(sc.sources, np.float64)
    axis = getattr(sc, "src_axis", None)          # directional sources (Sec. 1.2 footnote), else None
    pattern = None
    if axis is not None:
        axis = np.ascontiguousarray(axis, np.float64).reshape(-1, 3)
        pattern = np.ascontiguousarray(sc.src_pattern, np.float64).reshape(-1)
    rc = np.ascontiguousarray(sc.rcv_center, np.float64)
    rr = np.ascontiguousarray(sc.rcv_radius, np.float64)
    rs = np.ascontiguousarray(sc.rcv_source, np.int32)
    hist = np.empty((n, B), np.int32)
    hist_t = np.empty((n, B))
    E = np.empty((n, N_BANDS))
    L = np.empty(n)
    famb = np.empty(n, np.int32)
    nh = np.empty(n, np.int32)
    cap = rec_cap or max(1024, 4 * n)
    while True:
        rr_ = np.empty(cap, np.int32)
        rray = np.empty(cap, np.int64)
        rm = np.empty(cap, np.int32)
        rL = np.empty(cap)
        rmg = np.empty(cap)
        rpos = np.empty((cap, 3))
        rdir = np.empty((cap, 3))
        k = lib().orc_trace(osc.h, _p(src), _p(axis) if axis is not None else None,
                            _p(pattern) if pattern is not None else None, len(rc), _p(rc), _p(rr), _p(rs), N, n,
                            _p(ray_src),
                            _p(ray_ids), B, dmax, int(brute or not osc.has_tree), eps_edge_rel,
                            threads or default_threads(), _p(hist), _p(hist_t), _p(E), _p(L),
                            _p(famb), _p(nh), cap, _p(rr_), _p(rray), _p(rm), _p(rL), _p(rmg),
                            _p(rpos), _p(rdir))
        if k <= cap:
            break
        cap = int(k)
    return TraceResult(ray_src, ray_ids, hist, hist_t, E, L, famb, nh, rr_[:k], rray[:k], rm[:k],
                       rL[:k], rmg[:k], rpos[:k], rdir[:k], N, B, dmax)


# ----------------------------------------------------------------------------
# image sources (Sec. 1.4, Fig. 4, eq. 19)
# ----------------------------------------------------------------------------
def surface_planes(scene) -> np.ndarray:
    """FP64 plane (n, d) with n.x = d for each surface, from the surface's
    lowest-index triangle."""
    S = scene.n_surfaces
    first = np.full(S, -1, np.int64)
    for t in range(scene.n_tris - 1, -1, -1):
        first[scene.surface_id[t]] = t
    P = np.zeros((S, 4))
    for s in range(S):
        if first[s] < 0:
            continue
        a, b, c = scene.vertices[scene.tris[first[s]]]
        n = np.cross(b - a, c - a)
        n = n / math.sqrt(float(n @ n))
        P[s, :3] = n
        P[s, 3] = float(n @ a)
    return P


def surface_material(scene) -> np.ndarray:
    S = scene.n_surfaces
    m = np.zeros(S, np.int32)
    m[scene.surface_id] = scene.material_id
    return m


@dataclass
class ImageSources:
    rcv: np.ndarray            # int32 [K]
    order: np.ndarray          # int32 [K] reflection order m
    n: np.ndarray              # int64 [K] rays in the beam
    rep: np.ndarray            # int64 [K] representative ray (lowest list index)
    seq: list                  # K tuples of surface ids, in hit order
    pos: np.ndarray            # float64 [K,3] image-source position
    d: np.ndarray              # float64 [K] distance to the receiver centre
    t: np.ndarray              # float64 [K] arrival time d / c
    E: np.ndarray              # float64 [K,8] energy (eq. 19)


def image_sources(scene, tr: TraceResult, exclude_rays=None) -> ImageSources:
    """Group measurement-sphere crossings into image sources.

    Rays crossing receiver x_m after the same sequence of surfaces focus on
    one image source (Sec. 1.4); its position is x_s mirrored across the
    sequence's planes in hit order, and its energy follows eq. 19 with
    n = number of rays in the beam."""
    planes = surface_planes(scene)
    smat = surface_material(scene)
    alpha = scene.alpha.astype(np.float64)
    beta = scene.beta.astype(np.float64)
    groups = {}
    skip = set() if exclude_rays is None else set(int(x) for x in exclude_rays)
    for k in range(len(tr.rec_rcv)):
        ray = int(tr.rec_ray[k])
        if ray in skip:
            continue
        m = int(tr.rec_m[k])
        seq = tuple(int(scene.surface_id[t]) for t in tr.hist[ray, :m])
        key = (int(tr.rec_rcv[k]), seq)
        g = groups.get(key)
        if g is None:
            groups[key] = [1, ray]
        else:
            g[0] += 1
            g[1] = min(g[1], ray)
    keys = sorted(groups.keys(), key=lambda kv: (kv[0], len(kv[1]), kv[1]))
    K = len(keys)
    out = ImageSources(np.zeros(K, np.int32), np.zeros(K, np.int32), np.zeros(K, np.int64),
                       np.zeros(K, np.int64), [], np.zeros((K, 3)), np.zeros(K), np.zeros(K),
                       np.zeros((K, N_BANDS)))
    for i, (r, seq) in enumerate(keys):
        n, rep = groups[(r, seq)]
        x = scene.sources[scene.rcv_source[r]].astype(np.float64).copy()
        prod = np.ones(N_BANDS)
        for s in seq:
            nv, dd = planes[s, :3], planes[s, 3]
            x = x - 2.0 * (float(nv @ x) - dd) * nv
            prod = prod * (1.0 - alpha[smat[s]])
        d = float(np.linalg.norm(x - scene.rcv_center[r]))
        out.rcv[i], out.order[i], out.n[i], out.rep[i] = r, len(seq), n, rep
        out.seq.append(seq)
        out.pos[i] = x
        out.d[i] = d
        out.t[i] = d / scene.c
        out.E[i] = (n / tr.N) * prod * np.exp(-beta * d)
    return out


# ----------------------------------------------------------------------------
# energy impulse response (Sec. 1.4): arrival time t = d/c, bin floor(t fs)
# ----------------------------------------------------------------------------
def rir(isrc: ImageSources, n_rcv: int, fs: float, duration: float = 0.0) -> np.ndarray:
    """[n_rcv, 8, n_bins] FP64 band energy histograms."""
    if duration > 0:
        nb = int(math.ceil(duration * fs))
    else:
        nb = int(math.floor(isrc.t.max() * fs)) + 1 if len(isrc.t) else 1
    H = np.zeros((n_rcv, N_BANDS, nb))
    for i in range(len(isrc.t)):
        b = int(math.floor(isrc.t[i] * fs))
        if 0 <= b < nb:
            H[isrc.rcv[i], :, b] += isrc.E[i]
    return H


# ----------------------------------------------------------------------------
# decay metrics from an energy histogram (Sec. 1.4 names T30; ISO 3382 defs)
# ----------------------------------------------------------------------------
def schroeder_db(h: np.ndarray) -> np.ndarray:
    """Backward-integrated energy decay curve in dB re its start."""
    e = np.cumsum(h[::-1])[::-1]
    with np.errstate(divide="ignore"):
        return 10.0 * np.log10(e / e[0])


def _fit_slope(t, y):
    A = np.stack([t, np.ones_like(t)], 1)
    k, _ = np.linalg.lstsq(A, y, rcond=None)[0]
    return k


def decay_time(h: np.ndarray, fs: float, lo_db: float, hi_db: float) -> float:
    """Time for 60 dB of decay extrapolated from a least-squares line through
    the Schroeder curve between lo_db and hi_db (e.g. -5 and -35 for T30)."""
    c = schroeder_db(h)
    t = np.arange(len(h)) / fs
    m = (c <= lo_db) & (c >= hi_db)
    if m.sum() < 2:
        return float("nan")
    k = _fit_slope(t[m], c[m])
    return -60.0 / k


def t30(h, fs):
    return decay_time(h, fs, -5.0, -35.0)


def edt(h, fs):
    return decay_time(h, fs, 0.0, -10.0)
