"""FP64 reference of the specular tail prior -- TEST INFRASTRUCTURE ONLY.

A ray of direction d loses energy at R(d) = sum_k |d_k| rate_k + air (1/s)
when the walls are grouped by the axis of their normal; a measurement
sphere's histogram (Sec. 1.4, eq. 19: an image source found by n of N rays
carries n / N of the source energy times its reflection product) averages
level * exp(-R t) over the ray directions.  This module writes that average
out with plain loops over bands and bins.

Quadrature: R depends on |d_k| only, so the sphere mean is the mean over the
first octant, d = (sin theta cos phi, sin theta sin phi, cos theta) with area
element sin theta dtheta dphi and area pi / 2.  theta and phi are taken on the
Gauss-Legendre nodes of (0, pi / 2) (numpy's leggauss), n nodes each.
"""
from __future__ import annotations

import math

import numpy as np


def octant_rule(n: int):
    """Directions [n*n][3] (theta-major) and weights [n*n] summing to 1."""
    x, w = np.polynomial.legendre.leggauss(n)
    ang = 0.25 * math.pi * (x + 1.0)            # nodes on (0, pi / 2)
    w_ang = 0.25 * math.pi * w                  # their weights
    D, W = [], []
    for i in range(n):
        for j in range(n):
            th, ph = ang[i], ang[j]
            D.append((math.sin(th) * math.cos(ph), math.sin(th) * math.sin(ph), math.cos(th)))
            W.append(w_ang[i] * math.sin(th) * w_ang[j] / (0.5 * math.pi))
    return np.array(D), np.array(W)


def bin_mean_exp(R, t: float, dt: float):
    """(1/dt) * integral_t^{t+dt} exp(-R s) ds, elementwise over R >= 0."""
    R = np.asarray(R, np.float64)
    x = R * dt
    safe = np.where(x > 0.0, x, 1.0)
    avg = np.where(x > 0.0, -np.expm1(-x) / safe, 1.0)
    return np.exp(-R * t) * avg


def tail_prior(rates: np.ndarray, air: np.ndarray, level: np.ndarray, n_nodes: int, t0: float, dt: float,
               n_bins: int) -> np.ndarray:
    """[n][8][n_bins]: level * weighted mean over directions of the bin-averaged exp(-R t)."""
    rates = np.asarray(rates, np.float64).reshape(-1, 3, 8)
    air = np.asarray(air, np.float64).reshape(-1, 8)
    level = np.asarray(level, np.float64).reshape(-1)
    D, W = octant_rule(n_nodes)
    out = np.zeros((len(rates), 8, n_bins))
    for i in range(len(rates)):
        for f in range(8):
            R = D @ rates[i, :, f] + air[i, f]          # one decay rate per direction
            for b in range(n_bins):
                out[i, f, b] = level[i] * np.sum(W * bin_mean_exp(R, t0 + b * dt, dt))
    return out
