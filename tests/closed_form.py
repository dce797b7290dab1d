"""Closed forms that pin the oracle (and, through it, the CUDA path).

Nothing here traces rays against triangles.  For a rectangular room the
specular path of a ray is a straight line in the "unfolded" lattice of mirror
copies of the room (McGovern's image-source lattice, paper Sec. 3.2):

* the walls a ray reflects from, in order, are the lattice planes x = j Lx,
  y = j Ly, z = j Lz that the straight line crosses, sorted by distance;
  plane j of axis a is the physical wall at 0 if j is even, at L_a if odd;
* in lattice cell k the receiver's copy sits at k L + x_m (k even) or
  (k+1) L - x_m (k odd), per axis;
* folding cell k back into the room maps the source to its image source:
  x_s - k L (k even) or (k+1) L - x_s (k odd), per axis.

A receiver sphere that lies inside the room is crossed during segment m iff
the straight line passes within r of the receiver copy in the cell the line
occupies during that segment.
"""
from __future__ import annotations

import math

import numpy as np

#: surface ids of the six faces of scenes.shoebox: (x=0, x=L), (y=0, y=L), (z=0, z=L)
FACE_ID = [(0, 1), (2, 3), (4, 5)]


def unfolded_crossings(x_s, u, L, n_segments, dmax=0.0):
    """Plane crossings of the line x_s + t u, in order.

    Returns (times [n], walls [n] surface ids, cells [n+1,3]) for the first
    n_segments segments (n = n_segments - 1 crossings used to bound them)."""
    events = []
    for a in range(3):
        if u[a] == 0:
            continue
        # enough crossings on this axis to cover n_segments of the merged list
        step = L[a] / abs(u[a])
        first = ((L[a] - x_s[a]) / u[a]) if u[a] > 0 else (-x_s[a] / u[a])
        for q in range(n_segments + 1):
            t = first + q * step
            if u[a] > 0:
                j = 1 + q
            else:
                j = -q
            events.append((t, a, j))
    events.sort()
    events = events[:n_segments]
    times = np.array([e[0] for e in events])
    walls = np.array([FACE_ID[e[1]][e[2] % 2] for e in events], np.int32)
    cells = np.zeros((len(events) + 1, 3), np.int64)
    k = np.zeros(3, np.int64)
    cells[0] = k
    for i, (_, a, j) in enumerate(events):
        k = k.copy()
        k[a] += 1 if u[a] > 0 else -1
        cells[i + 1] = k
    return times, walls, cells


def receiver_copy(x_m, L, k):
    x_m, L, k = np.asarray(x_m, float), np.asarray(L, float), np.asarray(k)
    even = (k % 2) == 0
    return np.where(even, k * L + x_m, (k + 1) * L - x_m)


def image_source(x_s, L, k):
    x_s, L, k = np.asarray(x_s, float), np.asarray(L, float), np.asarray(k)
    even = (k % 2) == 0
    return np.where(even, x_s - k * L, (k + 1) * L - x_s)


def shoebox_image_sources(x_s, x_m, r, L, dirs, n_bounces, dmax=0.0, margin_skip=1e-6):
    """Per receiver-copy crossing of every ray (no tracing).

    Returns dict with:
      'crossings': list of (ray, m, seq tuple, cell tuple, margin)
      'groups': {seq: (n, image position, cell)} counting rays per sequence
      'ambiguous_rays': rays with a crossing margin below margin_skip"""
    x_s, x_m, L = (np.asarray(v, float) for v in (x_s, x_m, L))
    crossings, groups, amb = [], {}, set()
    for i, u in enumerate(np.asarray(dirs, float)):
        times, walls, cells = unfolded_crossings(x_s, u, L, n_bounces)
        t_start = np.concatenate([[0.0], times])
        t_end = np.concatenate([times, [math.inf]])
        for m in range(n_bounces):
            if m >= len(t_start):
                break
            if dmax > 0 and t_start[m] > dmax:
                break
            c = receiver_copy(x_m, L, cells[m])
            w = c - x_s
            uu = float(u @ u)
            tc = float(w @ u) / uu
            tc = min(max(tc, t_start[m]), t_end[m])
            dist = float(np.linalg.norm(x_s + tc * u - c))
            margin = (r - dist) / r
            if abs(margin) < margin_skip:
                amb.add(i)
            if dist <= r and (dmax <= 0 or tc <= dmax):
                seq = tuple(int(s) for s in walls[:m])
                crossings.append((i, m, seq, tuple(cells[m]), margin))
    for i, m, seq, cell, margin in crossings:
        g = groups.get(seq)
        if g is None:
            groups[seq] = [1, image_source(x_s, L, np.array(cell)), cell]
        else:
            g[0] += 1
            assert g[2] == cell
    return {"crossings": crossings, "groups": groups, "ambiguous_rays": amb}


def reflections_within(x_s, u, L, length):
    """Number of plane crossings of x_s + t u for 0 < t <= length (per ray)."""
    n = 0
    for a in range(3):
        if u[a] > 0:
            n += int(math.floor((x_s[a] + length * u[a]) / L[a]))
        elif u[a] < 0:
            n += int(math.floor((L[a] - x_s[a] - length * u[a]) / L[a]))
    return n


def cone_fraction(r, d):
    """Solid-angle fraction of a sphere of radius r seen from distance d (eq. 9)."""
    return 0.5 * (1.0 - math.sqrt(1.0 - (r / d) ** 2))
