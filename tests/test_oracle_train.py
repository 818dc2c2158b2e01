"""Pins of the float64 training-step oracle (image loss and Adam step) against
properties the definitions fix (Sec. 4.5 loss; Sec. 5.1 optimiser)."""
import math

import numpy as np
import pytest
import torch

from oracle import train64 as T


def test_window_is_a_normalised_truncated_gaussian():
    g = T.gaussian_window().numpy()
    c = T.SSIM_WINDOW // 2
    assert abs(g.sum() - 1.0) < 1e-15
    assert np.allclose(g, g[::-1], rtol=0, atol=0)
    assert np.argmax(g) == c
    # consecutive taps of a Gaussian: g_{i+1} / g_i = exp(-(2 (i - c) + 1) / (2 sigma^2))
    for i in range(T.SSIM_WINDOW - 1):
        assert math.isclose(g[i + 1] / g[i], math.exp(-(2 * (i - c) + 1) / (2 * T.SSIM_SIGMA ** 2)), rel_tol=1e-13)
    # truncation at +-3.3 sigma leaves the variance just under sigma^2
    var = float(((np.arange(T.SSIM_WINDOW) - c) ** 2 * g).sum())
    assert 2.20 < var < T.SSIM_SIGMA ** 2


def test_ssim_of_an_image_with_itself_is_one_everywhere():
    rng = np.random.default_rng(0)
    x = torch.tensor(rng.random((3, 23, 31)), dtype=torch.float64)
    m = T.ssim_map(x, x)
    assert torch.allclose(m, torch.ones_like(m), rtol=0, atol=1e-12)
    loss, per, grads = T.image_loss([x.numpy()], [x.numpy()])
    assert abs(loss) < 1e-12
    assert np.abs(grads[0]).max() < 1e-9


def test_ssim_of_constant_images_matches_closed_form_away_from_border():
    a, b = 0.3, 0.7
    x = torch.full((3, 20, 24), a, dtype=torch.float64)
    y = torch.full((3, 20, 24), b, dtype=torch.float64)
    m = T.ssim_map(x, y)
    inner = m[:, 5:-5, 5:-5]
    want = (2 * a * b + T.SSIM_C1) / (a * a + b * b + T.SSIM_C1)
    # sigma^2 = G * x^2 - mu^2 cancels to rounding (~1e-15) against C2 = 9e-4
    assert torch.allclose(inner, torch.full_like(inner, want), rtol=1e-11, atol=0)
    # at the border the zero padding lowers both means by the same window mass
    corner = float(m[0, 0, 0])
    assert corner != pytest.approx(want)


def test_ssim_is_symmetric():
    rng = np.random.default_rng(1)
    x = torch.tensor(rng.random((3, 17, 19)), dtype=torch.float64)
    y = torch.tensor(rng.random((3, 17, 19)), dtype=torch.float64)
    assert torch.allclose(T.ssim_map(x, y), T.ssim_map(y, x), rtol=0, atol=1e-14)


def _ssim_at(x, y, ch, i, j):
    """One map value by explicit sums over the zero-padded 11 x 11 window."""
    g = T.gaussian_window().numpy()
    c = T.SSIM_WINDOW // 2
    H, W = x.shape[1:]
    s = dict(x=0.0, y=0.0, xx=0.0, yy=0.0, xy=0.0)
    for di in range(-c, c + 1):
        for dj in range(-c, c + 1):
            ii, jj = i + di, j + dj
            if 0 <= ii < H and 0 <= jj < W:
                w = g[di + c] * g[dj + c]
                a, b = x[ch, ii, jj], y[ch, ii, jj]
                s["x"] += w * a
                s["y"] += w * b
                s["xx"] += w * a * a
                s["yy"] += w * b * b
                s["xy"] += w * a * b
    mx, my = s["x"], s["y"]
    vx, vy, cxy = s["xx"] - mx * mx, s["yy"] - my * my, s["xy"] - mx * my
    return ((2 * mx * my + T.SSIM_C1) * (2 * cxy + T.SSIM_C2)) / ((mx * mx + my * my + T.SSIM_C1) * (vx + vy + T.SSIM_C2))


@pytest.mark.parametrize("ch,i,j", [(0, 0, 0), (1, 7, 9), (2, 15, 3), (1, 16, 18)])
def test_ssim_map_matches_explicit_window_sums(ch, i, j):
    rng = np.random.default_rng(2)
    x = rng.random((3, 17, 19))
    y = np.clip(x + 0.2 * rng.standard_normal(x.shape), 0, 1)
    m = T.ssim_map(torch.tensor(x), torch.tensor(y))
    assert float(m[ch, i, j]) == pytest.approx(_ssim_at(x, y, ch, i, j), rel=1e-12, abs=1e-14)


def test_l1_gradient_is_sign_over_count():
    rng = np.random.default_rng(3)
    x, y = rng.random((3, 9, 11)), rng.random((3, 9, 11))
    loss, per, grads = T.image_loss([x], [y], lam=0.0)
    assert loss == pytest.approx(np.abs(x - y).mean(), rel=1e-14)
    assert np.allclose(grads[0], np.sign(x - y) / x.size, rtol=0, atol=1e-18)


def test_loss_gradient_against_central_differences():
    rng = np.random.default_rng(4)
    views = [(rng.random((3, 13, 15)), rng.random((3, 13, 15))), (rng.random((3, 8, 21)), rng.random((3, 8, 21)))]
    xs, ys = [v[0] for v in views], [v[1] for v in views]
    loss, per, grads = T.image_loss(xs, ys)
    assert loss == pytest.approx(np.mean(per), rel=1e-14)
    h = 1e-6
    for vi, (c, i, j) in [(0, (0, 0, 0)), (0, (1, 6, 7)), (1, (2, 7, 20)), (1, (0, 3, 10))]:
        xp = [x.copy() for x in xs]
        xm = [x.copy() for x in xs]
        xp[vi][c, i, j] += h
        xm[vi][c, i, j] -= h
        fd = (T.image_loss(xp, ys)[0] - T.image_loss(xm, ys)[0]) / (2 * h)
        assert grads[vi][c, i, j] == pytest.approx(fd, rel=1e-5, abs=1e-10)


def test_adam_matches_torch_optim_adam():
    rng = np.random.default_rng(5)
    K, P = 4, 37
    raw = rng.standard_normal((K, P))
    lrs = [1.6e-4, 5e-2, 5e-3, 1e-3]
    planes = [(lr, T.ACT_IDENTITY, 0.0, -1) for lr in lrs]
    tp = [torch.tensor(raw[k], dtype=torch.float64, requires_grad=True) for k in range(K)]
    opt = torch.optim.Adam([{"params": [tp[k]], "lr": lrs[k]} for k in range(K)], betas=(0.9, 0.999), eps=1e-15)
    m = np.zeros((K, P))
    v = np.zeros((K, P))
    r = raw
    for step in range(1, 4):
        g = rng.standard_normal((K, P))
        for k in range(K):
            tp[k].grad = torch.tensor(g[k], dtype=torch.float64)
        opt.step()
        r, act, m, v = T.adam_step(r, g, m, v, step, planes)
        for k in range(K):
            assert np.allclose(r[k], tp[k].detach().numpy(), rtol=1e-13, atol=1e-15)
        assert np.array_equal(act, r)


def test_adam_first_step_closed_form():
    rng = np.random.default_rng(6)
    raw = rng.standard_normal((2, 50))
    g = rng.standard_normal((2, 50))
    planes = [(1e-3, T.ACT_IDENTITY, 0.0, -1), (5e-2, T.ACT_IDENTITY, 0.0, -1)]
    r, _, m, v = T.adam_step(raw, g, np.zeros_like(raw), np.zeros_like(raw), 1, planes, eps=1e-8)
    for k, (lr, *_rest) in enumerate(planes):
        assert np.allclose(r[k] - raw[k], -lr * g[k] / (np.abs(g[k]) + 1e-8), rtol=1e-12, atol=0)


def test_activation_chain_and_regulariser_against_autograd():
    rng = np.random.default_rng(7)
    P = 29
    raw = rng.standard_normal((3, P))
    ga = rng.standard_normal((3, P))
    reg = 0.01
    planes = [(1e-3, T.ACT_SIGMOID, reg, -1), (1e-3, T.ACT_EXP, reg, -1), (1e-3, T.ACT_IDENTITY, 0.0, -1)]
    # with beta1 = 0, beta2 = 0 and eps = 0 the step is lr * sign(g_raw): compare
    # the sign of each raw gradient with autograd of sum(ga * act(raw)) + reg * sum|act(raw)|
    r, act, m, v = T.adam_step(raw, ga, np.zeros_like(raw), np.zeros_like(raw), 1, planes, beta1=0.0, beta2=0.0,
                               eps=0.0)
    t = torch.tensor(raw, dtype=torch.float64, requires_grad=True)
    a = torch.stack([torch.sigmoid(t[0]), torch.exp(t[1]), t[2]])
    f = (torch.tensor(ga) * a).sum() + reg * a[:2].abs().sum()
    f.backward()
    assert np.allclose(m, t.grad.numpy(), rtol=1e-13, atol=1e-16)
    assert np.allclose(r, raw - 1e-3 * np.sign(t.grad.numpy()), rtol=0, atol=1e-15)
    assert np.allclose(act[0], 1 / (1 + np.exp(-r[0])), rtol=1e-15)
    assert np.allclose(act[1], np.exp(r[1]), rtol=1e-15)


def test_noise_is_added_after_the_update():
    rng = np.random.default_rng(8)
    raw = rng.standard_normal((2, 10))
    noise = rng.standard_normal((1, 10))
    planes = [(0.0, T.ACT_IDENTITY, 0.0, 0), (0.0, T.ACT_IDENTITY, 0.0, -1)]
    r, _, _, _ = T.adam_step(raw, rng.standard_normal((2, 10)), np.zeros_like(raw), np.zeros_like(raw), 1, planes,
                             lambda_eps=0.5, noise=noise)
    assert np.allclose(r[0], raw[0] + 0.5 * noise[0], rtol=0, atol=1e-15)
    assert np.array_equal(r[1], raw[1])
