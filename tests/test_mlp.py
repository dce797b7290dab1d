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
