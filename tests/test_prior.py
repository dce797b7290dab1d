"""The specular tail prior's FP64 reference, pinned to closed forms (CPU)."""
import math

import numpy as np

from oracle import prior as P


def test_octant_rule():
    D, W = P.octant_rule(48)
    assert np.allclose(np.linalg.norm(D, axis=1), 1.0, atol=1e-14)
    assert D.min() >= 0.0 and abs(W.sum() - 1) < 1e-14
    # every axis component of a uniform direction is uniform on [0, 1]:
    # mean 1/2, mean square 1/3
    for k in range(3):
        assert abs(W @ D[:, k] - 0.5) < 1e-13
        assert abs(W @ D[:, k] ** 2 - 1.0 / 3.0) < 1e-13
    # E|d_x d_y| = E[1 - u^2] E[sin(2 phi) / 2] = (2/3)(1/pi)
    assert abs(W @ (D[:, 0] * D[:, 1]) - 2.0 / (3.0 * math.pi)) < 1e-12


def _bin_mean_closed_form(r, t, dt):
    """Bin mean over [t, t + dt) of the sphere mean of exp(-r |d_k| s),
    (1 - exp(-r s)) / (r s); its antiderivative is (ln s + E1(r s)) / r."""
    from scipy.special import exp1
    F = lambda s: (math.log(s) + exp1(r * s)) / r
    return (F(t + dt) - F(t)) / dt


def test_one_axis_closed_form():
    for k in range(3):
        rates = np.zeros((1, 3, 8))
        rates[0, k] = np.linspace(5.0, 200.0, 8)
        out = P.tail_prior(rates, np.zeros((1, 8)), np.ones(1), 64, 0.013, 0.2, 5)
        for f in range(8):
            for b in range(5):
                ref = _bin_mean_closed_form(rates[0, k, f], 0.013 + b * 0.2, 0.2)
                assert abs(out[0, f, b] / ref - 1) < 1e-10, (k, f, b, out[0, f, b], ref)


def test_air_only_and_level():
    air = np.array([[0.0, 1.0, 3.0, 10.0, 30.0, 100.0, 300.0, 1000.0]])
    out = P.tail_prior(np.zeros((1, 3, 8)), air, np.array([2.5]), 8, 0.05, 0.01, 20)
    for f in range(8):
        a = air[0, f]
        for b in range(20):
            t = 0.05 + 0.01 * b
            ref = 1.0 if a == 0 else math.exp(-a * t) * (1 - math.exp(-a * 0.01)) / (a * 0.01)
            assert abs(out[0, f, b] / (2.5 * ref) - 1) < 1e-12


def test_initial_slope_is_eyring():
    """For short times the prior decays at the direction-mean rate, i.e.
    sum_k rate_k / 2 (Eyring's rate for these rates)."""
    rates = np.array([[[40.0] * 8, [10.0] * 8, [70.0] * 8]])
    t = 1e-5
    out = P.tail_prior(rates, np.zeros((1, 8)), np.ones(1), 32, t, 1e-9, 1)
    slope = -math.log(out[0, 0, 0]) / t
    assert abs(slope / 60.0 - 1) < 5e-3


def test_against_an_independent_quadrature():
    """A million full-sphere Fibonacci points folded by |d| (another rule) agree."""
    g = np.random.default_rng(3)
    rates = g.uniform(1.0, 150.0, (2, 3, 8))
    air = g.uniform(0.0, 2.0, (2, 8))
    out = P.tail_prior(rates, air, np.ones(2), 64, 0.05, 0.01, 40)
    n = 1_000_000
    i = np.arange(n) + 0.5
    z = 1 - 2 * i / n
    phi = math.pi * (3 - math.sqrt(5)) * i
    r = np.sqrt(1 - z * z)
    D = np.abs(np.stack([r * np.cos(phi), r * np.sin(phi), z], 1))
    for room in range(2):
        for f in (0, 5):
            R = D @ rates[room, :, f] + air[room, f]
            for b in (0, 10, 39):
                t = 0.05 + 0.01 * b
                ref = np.mean(np.exp(-R * t) * -np.expm1(-R * 0.01) / (R * 0.01))
                assert abs(out[room, f, b] / ref - 1) < 3e-3, (room, f, b)
