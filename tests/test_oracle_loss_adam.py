"""Pins of the oracle's loss (Suppl. A: 0.8 L1 + 0.2 D-SSIM) and Adam
(Suppl. A hyper-parameters; Sec. 3.3: matches PyTorch's Adam) against
library routines (P10, P11) and special cases."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")


def _torch_loss(img, tgt, lam):
    """0.8/0.2 loss written with torch.nn.functional.conv2d in float64."""
    x = torch.tensor(img, dtype=torch.float64, requires_grad=True)
    y = torch.tensor(tgt, dtype=torch.float64)
    g = torch.exp(-(torch.arange(11, dtype=torch.float64) - 5) ** 2 / (2 * 1.5 ** 2))
    g = g / g.sum()
    w = (g[:, None] * g[None, :])[None, None].repeat(3, 1, 1, 1)

    def blur(a):
        return torch.nn.functional.conv2d(a[None], w, padding=5, groups=3)[0]

    mx, my = blur(x), blur(y)
    sxx = blur(x * x) - mx * mx
    syy = blur(y * y) - my * my
    sxy = blur(x * y) - mx * my
    C1, C2 = 0.01 ** 2, 0.03 ** 2
    ssim = ((2 * mx * my + C1) * (2 * sxy + C2)) / ((mx * mx + my * my + C1) * (sxx + syy + C2))
    L = (1 - lam) * (x - y).abs().mean() + lam * (1 - ssim.mean())
    L.backward()
    return L.item(), x.grad.numpy()


@pytest.mark.parametrize("H,W,lam", [(16, 16, 0.2), (37, 29, 0.2), (23, 41, 0.0), (12, 20, 1.0)])
def test_p11_loss_matches_torch_conv2d_autograd(oracle_mod, H, W, lam):
    rng = np.random.default_rng(H * W)
    img = rng.uniform(0, 1.2, (3, H, W))
    tgt = rng.uniform(0, 1, (3, H, W))
    L, dL = oracle_mod.loss(img, tgt, lam)
    Lt, dLt = _torch_loss(img, tgt, lam)
    assert L == pytest.approx(Lt, rel=1e-13)
    np.testing.assert_allclose(dL, dLt, rtol=1e-10, atol=1e-16)


def test_p11_ssim_identity(oracle_mod):
    rng = np.random.default_rng(1)
    x = rng.uniform(0, 1, (3, 31, 17))
    L, dL = oracle_mod.loss(x, x, 1.0)          # pure D-SSIM
    assert L == pytest.approx(0.0, abs=1e-14)
    assert np.abs(dL).max() < 1e-14
    L, dL = oracle_mod.loss(x, x, 0.2)          # L1 part has zero subgradient at 0
    assert L == pytest.approx(0.0, abs=1e-14)
    assert np.abs(dL).max() < 1e-14


def test_loss_batch_scaling(oracle_mod):
    rng = np.random.default_rng(2)
    x, y = rng.uniform(0, 1, (2, 3, 9, 13))
    L, dL = oracle_mod.loss(x, y, 0.2)
    L2, dL2 = oracle_mod.loss(x, y, 0.2, grad_scale=0.25)
    assert L2 == L
    np.testing.assert_allclose(dL2, 0.25 * dL, rtol=1e-15)


def test_p10_adam_matches_torch_optim(oracle_mod):
    """Five steps of torch.optim.Adam(foreach=False) in float64."""
    rng = np.random.default_rng(3)
    n = 1000
    p0 = rng.standard_normal(n)
    grads = [rng.standard_normal(n) * 10.0 ** rng.uniform(-8, 1, n) for _ in range(5)]
    grads[2][:100] = 0.0
    for lr in (1.6e-4, 5e-3, 2.5e-2):
        tp = torch.tensor(p0.copy(), dtype=torch.float64, requires_grad=True)
        opt = torch.optim.Adam([tp], lr=lr, betas=(0.9, 0.999), eps=1e-15, foreach=False)
        p, m, v = p0.copy(), np.zeros(n), np.zeros(n)
        for s, g in enumerate(grads, start=1):
            tp.grad = torch.tensor(g, dtype=torch.float64)
            opt.step()
            oracle_mod.adam(p, g.copy(), m, v, lr, s)
            np.testing.assert_allclose(p, tp.detach().numpy(), rtol=1e-13, atol=1e-17)
        # torch forms m with lerp, the oracle as b1 m + (1 - b1) g: the two
        # differ by rounding where m nearly cancels
        st = opt.state[tp]
        np.testing.assert_allclose(m, st["exp_avg"].numpy(), rtol=1e-12, atol=1e-16)
        np.testing.assert_allclose(v, st["exp_avg_sq"].numpy(), rtol=1e-12, atol=1e-300)


def test_adam_first_step_is_signed_lr(oracle_mod):
    """From zero moments the first update is lr * g / (|g| + eps)."""
    g = np.array([1e-3, -2.0, 0.0, 5e-10])
    p, m, v = np.zeros(4), np.zeros(4), np.zeros(4)
    oracle_mod.adam(p, g, m, v, 0.01, 1)
    np.testing.assert_allclose(p, -0.01 * g / (np.abs(g) + 1e-15), rtol=1e-12)
