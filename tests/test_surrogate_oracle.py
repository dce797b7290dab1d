"""Pins of the FP64 surrogate-tail reference (oracle/surrogate.py) against
closed forms: a rectangular room's descriptors, geometric decays, round
trips of the curve forms, a gate fed with a prediction equal to the probe,
and an exponential decay across the 50 ms join."""
import math

import numpy as np

import scenes
from oracle import surrogate as OS

C = 343.2


def test_rectangular_room_descriptors():
    """For a box a x b x h with uniform absorption: S = 2(ab + bh + ah), each
    axis group is the pair of walls normal to it (share 2 bh / S for x), its
    rate is c 2 b h (-ln(1 - alpha)) / (2 V) = c (-ln(1 - alpha)) / a, the
    mean absorption is alpha and the room fills its bounding box."""
    a, b, h = 10.0, 7.0, 3.0
    sc = scenes.shoebox(L=(a, b, h), alpha=0.25)
    alpha = np.asarray(sc.alpha, np.float32)
    d = OS.descriptors(sc.vertices, sc.tris, sc.material_id, alpha, a * b * h, 0.5, np.full(8, 0.01), C)
    al = float(np.float32(0.25))
    S = 2 * (a * b + b * h + a * h)
    assert d[0] == math.log10(a * b * h) and abs(d[1] - math.log10(S)) < 1e-12
    assert np.allclose(d[2:10], al, rtol=1e-12)
    share = [2 * b * h / S, 2 * a * h / S, 2 * a * b / S]
    assert np.allclose(d[10:13], np.log10(np.array(share) + 1e-6), atol=1e-12)
    rate = [C * -math.log(1 - al) / L for L in (a, b, h)]
    assert np.allclose(d[13:37].reshape(3, 8), np.log10(np.array(rate)[:, None] + 1e-6), atol=1e-12)
    assert np.allclose(d[37:45], C * 0.01) and d[45] == math.log10(0.5) and abs(d[46]) < 1e-12


def test_tail_curve_of_a_geometric_decay():
    """e_k = q^k: the energy from bin k on is q^k (1 - q^(N-k)) / (1 - q);
    per-bin energies come back from the curve, and the target form maps back
    to the curve while the decay stays within 50 dB."""
    q = 0.93
    k = np.arange(OS.N_TAIL)
    e = 1e-3 * q ** k
    db = OS.tail_edc_db(e[None])[0]
    ref = 10 * np.log10(1e-3 * q ** k * (1 - q ** (OS.N_TAIL - k)) / (1 - q))
    assert np.allclose(db, ref, atol=1e-9)
    assert np.allclose(OS.edc_to_energy(db[None])[0], e, rtol=1e-9)
    t = OS.to_targets(db[None])[0]
    assert t[0] == db[0] and np.all(t[1:] <= 0)
    within = db - db[0] > -OS.REL_FLOOR_DB
    assert np.allclose(OS.from_targets(t[None])[0][within], db[within], atol=1e-12)
    assert np.all(OS.from_targets(t[None])[0][~within] == db[0] - OS.REL_FLOOR_DB)


def test_rising_curve_energies_are_made_non_negative():
    db = np.array([[-10.0, -12.0, -11.0, -20.0] + [-30.0] * (OS.N_TAIL - 4)])
    e = OS.edc_to_energy(db)[0]
    assert np.all(e >= 0)
    assert e[1] == 0.0                        # -11 dB after -12 dB: held at -12 dB
    assert abs(e.sum() - 0.1) < 1e-12         # the energies add up to the first value


def _decay_room(r, level=1e-2):
    """Early 1 ms bins and 10 ms tail bins of one exponential decay exp(-r t)."""
    t1 = np.arange(OS.N_EARLY) / 1000.0
    early = level * (np.exp(-r * t1) - np.exp(-r * (t1 + 0.001)))
    t10 = 0.05 + np.arange(OS.N_TAIL) / 100.0
    tail = level * (np.exp(-r * t10) - np.exp(-r * (t10 + 0.01)))
    return np.tile(early, (1, 8, 1)), np.tile(tail, (1, 8, 1))


def test_features_base_and_gate_on_an_exponential_decay():
    """A probe and a prior with the same decay: the features' probe part is 0,
    the base curve is the probe's curve, a prediction equal to it has no
    probe gap, and its join gap is the decay over 10 ms: 10 log10 e^(0.01 r)."""
    r = 12.0
    early, probe = _decay_room(r)
    prior_db = OS.tail_edc_db(probe)
    desc = np.zeros((1, OS.N_DESC))
    X, base = OS.features(desc, early, probe, prior_db)
    assert np.allclose(X[0, OS.X_PROBE:], 0.0, atol=1e-12)
    assert np.allclose(X[0, OS.X_EARLY:OS.X_PROBE], 10 * np.log10(early[0].reshape(-1) + 1e-10))
    within = prior_db - prior_db[..., :1] > -OS.REL_FLOOR_DB
    assert np.allclose(base[within], prior_db[within], atol=1e-9)
    assert np.allclose(base[~within], (prior_db[..., :1] - OS.REL_FLOOR_DB + 0 * prior_db)[~within])
    pred = OS.predict([np.zeros((1, 1568))], np.zeros(1560), np.ones(1560), base)
    assert np.allclose(pred, base)
    inside, join, gap = OS.gate_gaps(desc, X, pred, prior_db, np.full(OS.N_DESC, -1.0), np.full(OS.N_DESC, 1.0))
    assert inside[0] and gap[0] < 1e-9
    assert abs(join[0] - 10 * math.log10(math.exp(0.01 * r))) < 1e-6
    # a room with nothing traced in 40-50 ms gives the join no evidence: gap 0
    X2 = X.copy()
    X2[0, OS.X_EARLY:OS.X_PROBE] = 10 * np.log10(1e-10)
    assert OS.gate_gaps(desc, X2, pred, prior_db, np.full(OS.N_DESC, -1.0), np.full(OS.N_DESC, 1.0))[1][0] == 0.0
    # outside the range (2 % margin of the span)
    d2 = desc.copy()
    d2[0, 3] = 1.05
    assert not OS.gate_gaps(d2, X, pred, prior_db, np.full(OS.N_DESC, -1.0), np.full(OS.N_DESC, 1.0))[0][0]


def test_envelope_joins_early_and_tail():
    r = 8.0
    early, tail = _decay_room(r, level=1.0)
    env = OS.envelope(early, tail, False)[0, 0]
    t10 = np.arange(OS.N_ENV) / 100.0
    assert np.allclose(env, np.exp(-r * t10) - np.exp(-r * (t10 + 0.01)), rtol=1e-9)
    env_db = OS.envelope(early, OS.tail_edc_db(tail), True)[0, 0]
    assert np.allclose(env_db[OS.FIRST_TAIL:], tail[0, 0], rtol=1e-9)


def test_base_curve_follows_probe_then_prior():
    """The base curve: the probe's level and decay over its first 20 bins,
    then the prior's decay joined without a step, never below the clamp."""
    g = np.random.default_rng(5)
    n = 3
    t = (np.arange(OS.N_TAIL) + 0.5) / 100.0
    probe = (g.uniform(1e-5, 1e-3, (n, 8, 1)) * np.exp(-g.uniform(5, 40, (n, 8, 1)) * t) *
             g.uniform(0.5, 1.5, (n, 8, OS.N_TAIL)))
    prior = OS.tail_edc_db(g.uniform(1e-5, 1e-3, (n, 8, 1)) * np.exp(-g.uniform(5, 40, (n, 8, 1)) * t))
    _, base = OS.features(np.zeros((n, OS.N_DESC)), np.full((n, 8, OS.N_EARLY), 1e-6), probe, prior)
    base = OS.to_targets(base)
    a = OS.to_targets(OS.tail_edc_db(probe))
    b = OS.to_targets(prior)
    k = OS.BASE_PROBE_BINS
    keep = a[:, :, :k] >= -OS.REL_FLOOR_DB
    assert np.allclose(base[:, :, :k][keep], a[:, :, :k][keep])
    lo = -OS.REL_FLOOR_DB + 1e-6
    free = (base[:, :, k:] > lo) & (base[:, :, k - 1:-1] > lo)
    assert np.allclose(np.diff(base[:, :, k - 1:], axis=2)[free], np.diff(b[:, :, k - 1:], axis=2)[free])
    assert base[:, :, 1:].min() >= -OS.REL_FLOOR_DB - 1e-9
