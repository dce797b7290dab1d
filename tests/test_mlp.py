"""The surrogate MLP: FP64 reference pinned by finite differences (CPU), and
the GPU's tensor-core forward / backward / Adam against it."""
import numpy as np
import pytest

from oracle import mlp as ref


def _params(rng, n_in, h, n_out, scale=0.5):
    return [rng.normal(0, scale / np.sqrt(n_in), (h, n_in)), rng.normal(0, 0.1, h),
            rng.normal(0, scale / np.sqrt(h), (h, h)), rng.normal(0, 0.1, h),
            rng.normal(0, scale / np.sqrt(h), (n_out, h)), rng.normal(0, 0.1, n_out)]


def test_reference_gradients_match_finite_differences():
    rng = np.random.default_rng(0)
    p = _params(rng, 6, 5, 4)
    x = rng.normal(size=(7, 6))
    t = rng.normal(size=(7, 4))
    loss, g = ref.loss_and_grads(p, x, t)
    eps = 1e-6
    for k in range(6):
        flat = p[k].reshape(-1)
        for i in range(0, flat.size, max(1, flat.size // 7)):
            old = flat[i]
            flat[i] = old + eps
            lp, _ = ref.loss_and_grads(p, x, t)
            flat[i] = old - eps
            lm, _ = ref.loss_and_grads(p, x, t)
            flat[i] = old
            fd = (lp - lm) / (2 * eps)
            assert g[k].reshape(-1)[i] == pytest.approx(fd, rel=1e-5, abs=1e-9), (k, i)


def test_bf16_rounding_is_round_to_nearest_even():
    x = np.array([1.0, 1.00390625, 1.005859375, 1.0078125, -3.14159, 0.0, 65504.0])
    y = ref.to_bf16(x)
    assert y[0] == 1.0 and y[1] == 1.0            # tie (1 + 2^-8) rounds to even
    assert y[2] == 1.0078125                      # above the tie rounds up
    assert y[3] == 1.0078125
    assert abs(y[4] + 3.140625) < 1e-12
    assert y[5] == 0.0 and y[6] == 65536.0


@pytest.mark.gpu
def test_gpu_gradients_match_reference():
    torch = pytest.importorskip("torch")
    from paper_1811_05784_gb300 import rt
    I, H, O, B = 96, 64, 160, 37                  # several tiles and a ragged batch
    net = rt.MLP(I, H, O, seed=3)
    rng = np.random.default_rng(1)
    x = rng.normal(size=(B, I)).astype(np.float32)
    t = rng.normal(size=(B, O)).astype(np.float32)
    w = net.copy(0).astype(np.float64)
    p = net.blocks(w)
    xd, td = torch.tensor(x, device="cuda"), torch.tensor(t, device="cuda")
    y = net.forward(xd).cpu().numpy()
    y_ref, _ = ref.forward(p, x, bf16=True)
    assert np.linalg.norm(y - y_ref) / np.linalg.norm(y_ref) < 1e-3
    loss = net.gradients(xd, td)
    g = net.blocks(net.copy(1).astype(np.float64))
    loss_ref, g_ref = ref.loss_and_grads(p, x, t, bf16=True)
    assert loss == pytest.approx(loss_ref, rel=1e-3)
    for k in range(6):
        err = np.linalg.norm(g[k] - g_ref[k]) / np.linalg.norm(g_ref[k])
        assert err < 1e-3, (k, err)


@pytest.mark.gpu
def test_gpu_training_reduces_loss():
    torch = pytest.importorskip("torch")
    from paper_1811_05784_gb300 import rt
    I, H, O, B = 64, 128, 64, 256
    net = rt.MLP(I, H, O, seed=4)
    g = torch.Generator(device="cpu").manual_seed(0)
    A = torch.randn(I, O, generator=g) / I ** 0.5
    x = torch.randn(4096, I, generator=g)
    t = torch.tanh(x @ A) + 0.1 * torch.sin(3 * x[:, :O])
    x, t = x.cuda(), t.cuda()
    first = net.gradients(x[:B], t[:B])
    for step in range(300):
        k = (step * B) % 4096
        loss = net.train_step(x[k:k + B], t[k:k + B], lr=2e-3, want_loss=(step % 50 == 49))
    assert net.step == 300
    final = net.gradients(x[:1024], t[:1024])
    assert final < 0.3 * first, (first, final)


def test_package_decay_metrics_on_exponentials():
    from paper_1811_05784_gb300 import surrogate as S
    fs = 100.0
    n = np.arange(200)
    T = np.array([0.4, 0.9, 1.7])
    env = np.exp(-6 * np.log(10) * n[None, :] / (fs * T[:, None]))   # 60 dB per T seconds
    assert np.allclose(S.edt(env, fs), T, rtol=2e-2)
    got = S.t30(env, fs)
    assert np.allclose(got[:2], T[:2], rtol=2e-2)
    assert np.isnan(got[2]) or abs(got[2] / T[2] - 1) < 2e-2      # 2 s may not reach -35 dB


def test_surrogate_feature_layout():
    from paper_1811_05784_gb300 import surrogate as S
    assert S.N_FEAT == S.N_DESC + 400 + 8 * len(S.PROBE_BINS) and S.N_IN >= S.N_FEAT and S.N_IN % 32 == 0
    assert S.PROBE_BINS.max() < S.N_TAIL and np.all(np.diff(S.PROBE_BINS) > 0)
    assert S.X_EARLY.start == S.N_DESC and S.X_PROBE.start == S.X_EARLY.stop and S.X_PROBE.stop == S.N_FEAT
    assert len(S.BASIC_COLS) == 410 and S.BASIC_COLS[10] == S.N_DESC
    assert S.N_OUT_RAW == 8 * 195 and S.N_OUT >= S.N_OUT_RAW and S.N_OUT % 32 == 0
    import scenes
    d = S.descriptors(scenes.surrogate_room(2))
    assert d.shape == (S.N_DESC,) and 0.02 <= d[2:10].min() and d[2:10].max() <= 0.6


def test_axis_descriptors_closed_form():
    """In a 10 x 7 x 3 m box of uniform absorption 0.1 the walls normal to
    axis k hold 2 V / L_k of area and decay a ray's energy at c a / L_k per
    unit |d_k| (a = -ln 0.9); half their sum is Eyring's rate c S a / (4 V)."""
    from paper_1811_05784_gb300 import surrogate as S
    import scenes
    sc = scenes.shoebox()
    L = np.array([10.0, 7.0, 3.0])
    V, Sa = L.prod(), 2 * (L[0] * L[1] + L[1] * L[2] + L[0] * L[2])
    sc.meta["V"] = V
    d = S.descriptors(sc)
    a = -np.log(0.9)
    assert np.isclose(10 ** d[0], V) and np.isclose(10 ** d[1], Sa)
    assert np.allclose(10 ** d[S.D_AXIS_SHARE], 2 * V / L / Sa, rtol=1e-5)
    rate = (10 ** d[S.D_AXIS_RATE]).reshape(3, 8)
    assert np.allclose(rate, (S.C_SOUND * a / L)[:, None], rtol=1e-5)
    assert np.allclose(rate.sum(0) / 2, S.C_SOUND * Sa * a / (4 * V), rtol=1e-5)
    assert np.all(d[S.D_AIR] == 0)


def test_tail_targets_round_trip():
    from paper_1811_05784_gb300 import surrogate as S
    g = np.random.default_rng(0)
    rate = g.uniform(5, 200, (3, 8, 1))
    t = (np.arange(S.N_TAIL) + 0.5) / S.TAIL_FS
    energy = g.uniform(1e-4, 1e-2, (3, 8, 1)) * np.exp(-rate * t)
    edc = S.tail_edc_db(energy)
    y = S.edc_to_targets(edc)
    back = S.targets_to_edc_db(y).reshape(3, 8, -1)
    e3 = edc.reshape(3, 8, -1)
    keep = e3 >= e3[:, :, :1] - S.REL_FLOOR_DB
    assert np.allclose(back[keep], e3[keep], atol=1e-9)
    assert np.all(back[~keep] >= e3[~keep])                       # clamped, never below the floor
    assert np.allclose(back - back[:, :, :1], np.maximum(e3 - e3[:, :, :1], -S.REL_FLOOR_DB))


def test_base_curve_follows_probe_then_prior():
    from paper_1811_05784_gb300 import surrogate as S
    g = np.random.default_rng(5)
    n = 3
    t = (np.arange(S.N_TAIL) + 0.5) / S.TAIL_FS
    probe = g.uniform(1e-5, 1e-3, (n, 8, 1)) * np.exp(-g.uniform(5, 40, (n, 8, 1)) * t) * g.uniform(0.5, 1.5, (n, 8, S.N_TAIL))
    prior_e = g.uniform(1e-5, 1e-3, (n, 8, 1)) * np.exp(-g.uniform(5, 40, (n, 8, 1)) * t)
    prior = S.tail_edc_db(prior_e)
    base = S.edc_to_targets(S.base_db(probe, prior)).reshape(n, 8, -1)
    a = S.edc_to_targets(S.tail_edc_db(probe)).reshape(n, 8, -1)
    b = S.edc_to_targets(prior).reshape(n, 8, -1)
    k = S.BASE_PROBE_BINS
    keep = a[:, :, :k] >= -S.REL_FLOOR_DB
    assert np.allclose(base[:, :, :k][keep], a[:, :, :k][keep])            # level and first bins: the probe
    step_base = np.diff(base[:, :, k - 1:], axis=2)
    step_prior = np.diff(b[:, :, k - 1:], axis=2)
    lo = -S.REL_FLOOR_DB + 1e-6                                           # off the clamp
    free = (base[:, :, k:] > lo) & (base[:, :, k - 1:-1] > lo)
    assert np.allclose(step_base[free], step_prior[free])                 # then the prior's decay, no step
    assert base[:, :, 1:].min() >= -S.REL_FLOOR_DB - 1e-9
