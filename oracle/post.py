"""FP64 reference of the post-processing of energy impulse responses --
TEST INFRASTRUCTURE ONLY.

Sec. 1.4 turns image sources into impulse responses: energies binned at their
arrival times, pressure p = sqrt(E) per image source, FIR filters over the 8
octave bands; Sec. 4 reports "perceptive factors" of the result (EDT, T30,
SPL, C80, D50, Ts).  The paper names these standard metrics without formulas;
this module writes out the usual definitions (ISO 3382-1 style) on a
histogram of energies e[b] per bin [b / fs, (b + 1) / fs):

  E     = sum_b e[b]                           SPL = 10 log10 E (re the emitted energy 1)
  S[b]  = sum_{b' >= b} e[b']  (Schroeder)     L[b] = 10 log10 (S[b] / S[0]) at t = b / fs
  b0    = the first bin with e > 0 (the direct sound), times counted from b0 / fs
  EDT, T20, T30: least-squares line through the (t, L) of the bins b >= b0
        with L in [0, -10], [-5, -25], [-5, -35] dB; the time for -60 dB at
        that slope; NaN when no finite L reaches the lower limit or fewer than
        2 points qualify
  C80   = 10 log10 (sum_{b - b0 < 0.08 fs} e / sum_{b - b0 >= 0.08 fs} e)
  D50   = sum_{b - b0 < 0.05 fs} e / E
  Ts    = sum_b ((b - b0 + 1/2) / fs) e[b] / E
Octave band f = 0..7 has centre 62.5 Hz * 2^f and edges f_c / sqrt 2, f_c sqrt 2.
The band filters are linear-phase windowed sincs of n_taps (odd) taps with a
Hann window:  g_f[n] = w[n] (h(f_hi, n) - h(f_lo, n)), with
h(F, n) = 2 F / fs sinc(2 F (n - D) / fs), D = (n_taps - 1) / 2,
w[n] = 1/2 (1 - cos(2 pi n / (n_taps - 1))).  The pressure response of a
receiver is p[t] = sum_s sum_f sqrt(E_s(f)) g_f[t - floor(t_s fs) + D].
"""
from __future__ import annotations

import math

import numpy as np

PARAMS = ("EDT", "T20", "T30", "C80", "D50", "Ts", "SPL")


def _decay_time(L: np.ndarray, b0: int, fs: float, hi_db: float, lo_db: float) -> float:
    t = np.arange(len(L)) / fs
    L = np.where(np.arange(len(L)) >= b0, L, np.nan)             # from the direct sound on
    if not np.any(np.isfinite(L) & (L <= lo_db)):
        return math.nan
    m = (L <= hi_db) & (L >= lo_db)
    if m.sum() < 2:
        return math.nan
    slope = np.polyfit(t[m], L[m], 1)[0]
    return -60.0 / slope if slope < 0 else math.nan


def room_parameters(H: np.ndarray, fs: float) -> np.ndarray:
    """[n_rcv][8][7] parameters (PARAMS order) of histograms H [n_rcv][8][n_bins]."""
    H = np.asarray(H, np.float64)
    out = np.full(H.shape[:2] + (len(PARAMS),), math.nan)
    for k in range(H.shape[0]):
        for f in range(H.shape[1]):
            e = H[k, f]
            E = e.sum()
            if not E > 0:
                continue
            S = np.cumsum(e[::-1])[::-1]
            with np.errstate(divide="ignore", invalid="ignore"):
                L = 10.0 * np.log10(S / S[0])
            b0 = int(np.argmax(e > 0))
            n80, n50 = int(math.ceil(0.08 * fs)), int(math.ceil(0.05 * fs))
            rel = np.arange(len(e)) - b0
            early80 = e[rel < n80].sum()
            late80 = e[rel >= n80].sum()
            out[k, f, 0] = _decay_time(L, b0, fs, 0.0, -10.0)
            out[k, f, 1] = _decay_time(L, b0, fs, -5.0, -25.0)
            out[k, f, 2] = _decay_time(L, b0, fs, -5.0, -35.0)
            out[k, f, 3] = 10.0 * math.log10(early80 / late80) if late80 > 0 else math.inf
            out[k, f, 4] = e[rel < n50].sum() / E
            out[k, f, 5] = (((rel + 0.5) / fs) * e).sum() / E
            out[k, f, 6] = 10.0 * math.log10(E)
    return out


def octave_filters(fs: float, n_taps: int) -> np.ndarray:
    """[8][n_taps] linear-phase octave band-pass filters (module docstring)."""
    if n_taps % 2 == 0:
        raise ValueError("n_taps must be odd")
    D = (n_taps - 1) / 2.0
    n = np.arange(n_taps)
    w = 0.5 * (1.0 - np.cos(2.0 * math.pi * n / (n_taps - 1)))
    g = np.zeros((8, n_taps))
    for f in range(8):
        fc = 62.5 * 2.0 ** f
        lo, hi = fc / math.sqrt(2.0), fc * math.sqrt(2.0)
        h = lambda F: 2.0 * F / fs * np.sinc(2.0 * F * (n - D) / fs)
        g[f] = w * (h(hi) - h(lo))
    return g


def pressure_rir(rcv: np.ndarray, time: np.ndarray, energy: np.ndarray, n_rcv: int, fs: float, n_out: int,
                 n_taps: int) -> np.ndarray:
    """[n_rcv][n_out] pressure responses of image sources (receiver, arrival
    time, 8-band energy), plain loops over sources."""
    g = octave_filters(fs, n_taps)
    D = (n_taps - 1) // 2
    p = np.zeros((n_rcv, n_out))
    for s in range(len(time)):
        b = int(math.floor(time[s] * fs))
        w = np.sqrt(np.asarray(energy[s], np.float64)) @ g          # this source's combined filter
        lo, hi = b - D, b - D + n_taps                               # output samples it reaches
        a, z = max(lo, 0), min(hi, n_out)
        if a < z:
            p[int(rcv[s]), a:z] += w[a - lo:z - lo]
    return p
