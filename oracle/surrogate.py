"""FP64 reference of the surrogate-tail arithmetic -- TEST INFRASTRUCTURE ONLY.

The surrogate-tail mode has no counterpart in the paper: it is the learned
late reverberation of a room, with the method itself as fallback and judge.
This module writes out, with plain numpy loops where they read better, what
the library computes around its networks:
  - room descriptors from the mesh (areas, axis groups, absorption);
  - the tail decay curve of per-bin energies (backward sum in dB) and its
    "target form" (first value, then the decay relative to it, clamped);
  - the network features and the base curve the networks correct;
  - the ensemble's prediction from normalised network outputs;
  - the gate's join and probe gaps and the training-range check;
  - the 10 ms envelope of a room (traced 0-50 ms + a tail).
It imports nothing from the CUDA library.

Layout per room: desc [47], early [8][50] (1 ms bins), probe / *_db [8][195]
(10 ms bins from 50 ms), X [951], env [8][200].
"""
from __future__ import annotations

import math

import numpy as np

N_DESC, N_EARLY, N_TAIL, N_ENV = 47, 50, 195, 200
FIRST_TAIL = N_ENV - N_TAIL
PROBE_BINS = np.r_[np.arange(0, 30), np.arange(30, N_TAIL, 5)]      # 63 per band
X_EARLY = N_DESC
X_PROBE = N_DESC + 8 * N_EARLY
N_FEAT = X_PROBE + 8 * len(PROBE_BINS)                              # 951
REL_FLOOR_DB = 50.0
FLOOR, FLOOR_IN = 1e-30, 1e-10
BASE_PROBE_BINS = 20


def descriptors(vertices, tris, material_id, alpha, volume, radius, beta, c):
    """[log10 V, log10 S, area-weighted mean alpha [8], log10 (axis share +
    1e-6) [3], log10 (c A_k a_kf / (2 V) + 1e-6) [3][8], c beta [8], log10 r,
    log10 (V / bounding-box volume)].

    Each triangle belongs to the axis group of the largest component of its
    normal (the first one on ties); a_kf is the area-weighted -ln(1 - alpha)
    of group k in band f, with 1 - alpha clipped to [1e-6, 1]."""
    V = float(volume)
    S = 0.0
    a_sum = np.zeros(8)
    axis_area = np.zeros(3)
    loss = np.zeros((3, 8))
    for t in range(len(tris)):
        a, b, cc = (np.asarray(vertices[i], np.float64) for i in tris[t])
        n = np.cross(b - a, cc - a)
        area = 0.5 * math.sqrt(float(n @ n))
        k = 0
        for j in (1, 2):
            if abs(n[j]) > abs(n[k]):
                k = j
        al = np.asarray(alpha[material_id[t]], np.float64)
        S += area
        a_sum += area * al
        axis_area[k] += area
        loss[k] += area * -np.log(np.clip(1.0 - al, 1e-6, 1.0))
    ext = np.max(vertices, axis=0).astype(np.float64) - np.min(vertices, axis=0).astype(np.float64)
    out = [math.log10(V), math.log10(S)]
    out += list(a_sum / S)
    out += [math.log10(axis_area[k] / S + 1e-6) for k in range(3)]
    out += [math.log10(c * loss[k, f] / (2.0 * V) + 1e-6) for k in range(3) for f in range(8)]
    out += [c * float(beta[f]) for f in range(8)]
    out += [math.log10(radius), math.log10(V / float(np.prod(ext)))]
    return np.array(out)


def tail_edc_db(e):
    """10 log10 of the energy from each bin to the end (+1e-30), last axis."""
    e = np.asarray(e, np.float64)
    out = np.empty_like(e)
    acc = np.zeros(e.shape[:-1])
    for k in range(e.shape[-1] - 1, -1, -1):
        acc = acc + e[..., k]
        out[..., k] = 10.0 * np.log10(acc + FLOOR)
    return out


def to_targets(d):
    """First value, then the decay relative to it clamped at -50 dB."""
    d = np.asarray(d, np.float64)
    t = np.maximum(d - d[..., :1], -REL_FLOOR_DB)
    t[..., 0] = d[..., 0]
    return t


def from_targets(t):
    """Decay curve of a target-form vector: first value plus the decay clamped to [-50, 0] dB."""
    t = np.asarray(t, np.float64)
    d = t[..., :1] + np.clip(t, -REL_FLOOR_DB, 0.0)
    d[..., 0] = t[..., 0]
    return d


def edc_to_energy(db):
    """Per-bin energies of a decay curve in dB, made non-increasing first."""
    e = 10.0 ** (np.asarray(db, np.float64) / 10.0)
    run = np.minimum.accumulate(e, axis=-1)
    nxt = np.concatenate([run[..., 1:], np.zeros(run.shape[:-1] + (1,))], axis=-1)
    return np.maximum(run - nxt, 0.0)


def features(desc, early, probe, prior_db):
    """Network features [n][951] and base curves [n][8][195].

    The base curve is the probe's curve in target form over the first 20 bins
    of the tail, then the prior's decay shifted to join it without a step,
    clamped and turned back into a decay curve."""
    desc = np.asarray(desc, np.float64)
    n = len(desc)
    a = to_targets(tail_edc_db(probe))
    b = to_targets(np.asarray(prior_db, np.float64))
    X = np.zeros((n, N_FEAT))
    X[:, :N_DESC] = desc
    X[:, X_EARLY:X_PROBE] = (10.0 * np.log10(np.asarray(early, np.float64) + FLOOR_IN)).reshape(n, -1)
    X[:, X_PROBE:] = (a - b)[:, :, PROBE_BINS].reshape(n, -1)
    K = BASE_PROBE_BINS
    t = np.concatenate([a[:, :, :K], b[:, :, K:] - b[:, :, K - 1:K] + a[:, :, K - 1:K]], axis=2)
    return X, from_targets(t)


def predict(Y_members, y_mean, y_std, base_db):
    """Decay curves of the ensemble: the members' mean normalised output,
    de-normalised, plus the base curve in target form.  Y_members [m][n][>=1560]."""
    Y = np.mean([np.asarray(y, np.float64)[:, :8 * N_TAIL] for y in Y_members], axis=0)
    y = Y * np.asarray(y_std, np.float64) + np.asarray(y_mean, np.float64)
    n = len(y)
    t = y.reshape(n, 8, N_TAIL) + to_targets(np.asarray(base_db, np.float64))
    return from_targets(t)


def gate_gaps(desc, X, pred_db, prior_db, lo, hi):
    """(inside the training range with a 2 % margin, join gap dB, probe gap dB) per room.

    Join gap: the largest over the bands with traced energy in 40-50 ms of
    |predicted 50-60 ms energy - traced 40-50 ms energy| in dB (0 when no band
    has traced energy there: nothing to join against).  Probe gap: the largest over bands of the
    RMS of (predicted - prior) - (probe - prior) in target form at PROBE_BINS."""
    desc, X = np.asarray(desc, np.float64), np.asarray(X, np.float64)
    lo, hi = np.asarray(lo, np.float64), np.asarray(hi, np.float64)
    span = hi - lo
    inside = np.all((desc >= lo - 0.02 * span) & (desc <= hi + 0.02 * span), axis=1)
    n = len(X)
    join = np.zeros(n)
    probe = np.zeros(n)
    tp = to_targets(np.asarray(pred_db, np.float64))
    tq = to_targets(np.asarray(prior_db, np.float64))
    for i in range(n):
        best = -1.0
        for f in range(8):
            early = 10.0 ** (X[i, X_EARLY + f * N_EARLY:X_EARLY + (f + 1) * N_EARLY] / 10.0) - FLOOR_IN
            traced = early[40:50].sum()
            if traced > 0.5 * FLOOR_IN:
                pred0 = 10.0 * math.log10(edc_to_energy(pred_db[i, f])[0] + FLOOR_IN)
                best = max(best, abs(pred0 - 10.0 * math.log10(traced)))
            d = (tp[i, f, PROBE_BINS] - tq[i, f, PROBE_BINS]) - X[i, X_PROBE + f * len(PROBE_BINS):
                                                                     X_PROBE + (f + 1) * len(PROBE_BINS)]
            probe[i] = max(probe[i], math.sqrt(float(np.mean(d * d))))
        if best >= 0.0:
            join[i] = best
    return inside, join, probe


def envelope(early, tail, tail_is_db):
    """[n][8][200]: 1 ms early bins summed by ten, then the tail's per-bin energies."""
    early = np.asarray(early, np.float64)
    n = len(early)
    e10 = early.reshape(n, 8, FIRST_TAIL, 10).sum(-1)
    t = edc_to_energy(tail) if tail_is_db else np.asarray(tail, np.float64)
    return np.concatenate([e10, t], axis=2)
