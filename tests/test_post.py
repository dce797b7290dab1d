"""Post-processing reference (room-acoustic parameters, octave filters,
pressure synthesis), pinned to closed forms (CPU)."""
import math

import numpy as np

from oracle import post


def _exp_histogram(k, fs, n, b0=0, E0=1.0):
    """Exact bin energies of E0 k exp(-k (t - t0)) from t0 = b0 / fs (total E0)."""
    b = np.arange(n - b0)
    e = E0 * (np.exp(-k * b / fs) - np.exp(-k * (b + 1) / fs))
    return np.concatenate([np.zeros(b0), e])


def test_parameters_of_an_exponential_decay():
    fs, n = 48_000.0, 48_000 * 3
    for k, b0 in ((6.0, 0), (13.8, 1234), (40.0, 50)):
        H = _exp_histogram(k, fs, n, b0)[None, None, :].repeat(8, axis=1)
        P = post.room_parameters(H, fs)[0, 0]
        T = 6.0 * math.log(10.0) / k                       # 60 dB at energy decay rate k
        tail = math.exp(-k * (n - b0) / fs)
        # T20, T30: the histogram ends after 3 s, which bends the Schroeder curve
        # by tail / exp(-k t) (< 1e-4 at -35 dB): relative slope errors ~1e-5
        assert abs(P[1] / T - 1) < 2e-5 and abs(P[2] / T - 1) < 2e-5
        assert abs(P[0] / T - 1) < 2e-5                    # EDT, fitted from the direct sound on
        c80 = 10 * math.log10((1 - math.exp(-0.08 * k)) / (math.exp(-0.08 * k) - tail))
        assert abs(P[3] - c80) < 1e-6
        assert abs(P[4] - (1 - math.exp(-0.05 * k)) / (1 - tail)) < 1e-9
        ts = 1.0 / k                                         # centre time of the continuous decay
        assert abs(P[5] - ts) < 1e-3 * ts
        assert abs(P[6] - 10 * math.log10(1 - tail)) < 1e-9


def test_decay_times_of_a_double_slope_decay():
    """A Schroeder curve that falls at 60 dB/s down to -30 dB and at 20 dB/s
    after it (the bins' energies are the differences of that curve, so its
    backward integral gives it back): EDT (0 to -10 dB) and T20 (-5 to -25 dB)
    fit the first slope alone and are 1 s; T30 (-5 to -35 dB) takes in the
    second slope, so it lies strictly between the single-slope times 1 s and
    3 s, and apart from T20."""
    fs = 1000.0
    t = np.arange(int(6.0 * fs) + 1) / fs
    L = np.where(t <= 0.5, -60.0 * t, -30.0 - 20.0 * (t - 0.5))
    S = 10.0 ** (L / 10.0)
    e = np.append(S[:-1] - S[1:], S[-1])
    P = post.room_parameters(e[None, None, :].repeat(8, axis=1), fs)[0, 0]
    assert abs(P[0] - 1.0) < 1e-6 and abs(P[1] - 1.0) < 1e-6
    assert 1.1 < P[2] < 3.0


def test_parameters_of_edge_cases():
    fs = 1000.0
    H = np.zeros((2, 8, 100))
    H[1, :, 10] = 2.0                                        # a single arrival
    P = post.room_parameters(H, fs)
    assert np.isnan(P[0]).all()                              # no energy: nothing defined
    assert np.isinf(P[1, :, 3]).all() and np.allclose(P[1, :, 4], 1.0)
    assert np.allclose(P[1, :, 5], 0.5 / fs) and np.allclose(P[1, :, 6], 10 * math.log10(2.0))
    # a decay that never reaches -35 dB has no T30
    e = _exp_histogram(1.0, fs, 100)
    P2 = post.room_parameters(np.tile(e, (1, 8, 1)), fs)
    assert np.isnan(P2[0, :, 2]).all()


def test_octave_filters():
    fs, n = 48_000.0, 8191
    g = post.octave_filters(fs, n)
    assert g.shape == (8, n) and np.allclose(g, g[:, ::-1])          # linear phase
    freqs = np.fft.rfftfreq(1 << 18, 1 / fs)
    G = np.abs(np.fft.rfft(g, 1 << 18, axis=1))
    for f in range(8):
        fc = 62.5 * 2 ** f
        at = lambda x: G[f, int(round(x / (fs / (1 << 18))))]
        assert abs(20 * math.log10(at(fc))) < (1.0 if f < 2 else 0.1)   # pass band
        assert 20 * math.log10(at(fc / 4)) < -20 and 20 * math.log10(at(min(fc * 4, 23_000))) < -20
        assert abs(20 * math.log10(at(fc * math.sqrt(2))) + 6.0) < 1.5   # -6 dB at the band edge
    assert abs(G[:, int(round(1000 / (fs / (1 << 18))))].sum() - 1) < 0.05


def test_pressure_of_single_arrivals():
    fs, n_taps = 48_000.0, 1023
    g = post.octave_filters(fs, n_taps)
    E = np.array([[1, 4, 9, 16, 25, 36, 49, 64]], float)
    t = np.array([(5000 + 0.3) / fs])
    p = post.pressure_rir(np.array([0]), t, E, 1, fs, 12_000, n_taps)[0]
    D = (n_taps - 1) // 2
    ref = (np.sqrt(E[0]) @ g)
    assert np.allclose(p[5000 - D:5000 - D + n_taps], ref) and abs(p).sum() == np.abs(ref).sum()
    # clipping at both ends of the output
    p2 = post.pressure_rir(np.array([0, 0]), np.array([100 / fs, 11_990 / fs]), np.ones((2, 8)), 1, fs,
                           12_000, n_taps)[0]
    w = g.sum(0)
    assert np.allclose(p2[:100 + D + 1], w[D - 100:])
    assert np.allclose(p2[11_990 - D:], w[:12_000 - (11_990 - D)])
