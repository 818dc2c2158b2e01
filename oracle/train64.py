"""Float64 reference of the training step around the rasterizer (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU legs of ``bench.py``
may use this module; the CUDA path never imports it.

Sec. 4.5 (optimisation and implementation), loss:

    L = (1 - lambda_SSIM) L_1 + lambda_SSIM L_SSIM + lambda_o sum_i |o_i|
        + lambda_Sigma sum_i ||s_i||_1

Readings (the paper names the terms but not their definitions):

* L_1 is the mean absolute difference between the rendered and the target
  image over a view's pixels and colour channels.
* L_SSIM = 1 - SSIM, SSIM the mean of the structural-similarity map of Wang,
  Bovik, Sheikh and Simoncelli (2004): per colour channel, local statistics
  under an 11 x 11 Gaussian window of standard deviation 1.5, C1 = 0.01^2,
  C2 = 0.03^2 (unit dynamic range), and a map of the image's own size (the
  window is zero-padded at the border, the 3DGS convention).
* lambda_SSIM is not stated; 0.2, the value of 3DGS, whose loss this one extends.
* Over several views, the image loss is the mean of the views' losses.
* The regularisers act on the activated opacity o in (0, 1) and on the
  spatial scales s_x > 0, so |o| = o and ||s||_1 = sum of the scales; they
  enter the step through their gradients only.

Sec. 5.1 (implementation details): Adam (Kingma and Ba, 2015) with learning
rates 1.6e-4 for positions, 5e-2 for opacity, 5e-3 for scales and 1e-3 for
the other parameters; lambda_o = lambda_Sigma = 0.01, lambda_eps = 1.
Sec. 4.5: spatial noise injection mu_x <- mu_x - lr grad + lambda_eps eps,
read as: after the optimiser's update of the position, lambda_eps eps is
added; eps is drawn by the caller and passed in.

The optimiser works on raw parameters; the rasterizer reads activated ones:
opacity = sigmoid(raw), scales = exp(raw) (the spatial scales and the
diagonal of L_q, which must stay positive), all else the identity.

Parity: pinned (tests/test_oracle_train.py): SSIM(x, x) = 1; the closed form
of SSIM for constant images away from the border; symmetry; the Gaussian
window against its definition; one map value against an explicit double loop
over the zero-padded window; the L1 gradient; autograd against central
differences; Adam against torch.optim.Adam and the first-step closed form
lr * g / (|g| + eps); the activation chain against autograd.
"""
from __future__ import annotations

import math

import numpy as np
import torch

D = torch.float64
SSIM_WINDOW = 11
SSIM_SIGMA = 1.5
SSIM_C1 = 0.01 ** 2
SSIM_C2 = 0.03 ** 2
LAMBDA_SSIM = 0.2

ACT_IDENTITY = 0
ACT_SIGMOID = 1
ACT_EXP = 2


def gaussian_window(size: int = SSIM_WINDOW, sigma: float = SSIM_SIGMA) -> torch.Tensor:
    """1-D Gaussian weights g_i proportional to exp(-(i - c)^2 / (2 sigma^2)),
    c the centre tap, normalised to sum 1 (Wang et al. 2004)."""
    c = size // 2
    g = torch.tensor([math.exp(-((i - c) ** 2) / (2.0 * sigma * sigma)) for i in range(size)], dtype=D)
    return g / g.sum()


def ssim_map(x: torch.Tensor, y: torch.Tensor) -> torch.Tensor:
    """Structural-similarity map of two [3, H, W] images, per channel.

    mu = G * x, sigma_x^2 = G * x^2 - mu_x^2, sigma_xy = G * (x y) - mu_x mu_y,
    SSIM = (2 mu_x mu_y + C1)(2 sigma_xy + C2) / ((mu_x^2 + mu_y^2 + C1)(sigma_x^2 + sigma_y^2 + C2)),
    with G the 2-D window (outer product of the 1-D one) and zero padding."""
    g = gaussian_window()
    w2 = torch.outer(g, g)[None, None].repeat(3, 1, 1, 1)
    pad = SSIM_WINDOW // 2

    def blur(t):
        return torch.nn.functional.conv2d(t[None], w2, padding=pad, groups=3)[0]

    mx, my = blur(x), blur(y)
    sxx = blur(x * x) - mx * mx
    syy = blur(y * y) - my * my
    sxy = blur(x * y) - mx * my
    return ((2 * mx * my + SSIM_C1) * (2 * sxy + SSIM_C2)) / ((mx * mx + my * my + SSIM_C1) * (sxx + syy + SSIM_C2))


def view_loss(x: torch.Tensor, y: torch.Tensor, lam: float = LAMBDA_SSIM) -> torch.Tensor:
    """(1 - lambda) L1 + lambda (1 - SSIM) of one view ([3, H, W] each)."""
    l1 = (x - y).abs().mean()
    return (1.0 - lam) * l1 + lam * (1.0 - ssim_map(x, y).mean())


def image_loss(images, targets, lam: float = LAMBDA_SSIM):
    """Mean over views of the view losses, and its gradient with respect to
    each rendered image (float64 autograd).  images/targets: lists of
    [3, H, W] arrays.  Returns (loss, [per-view loss], [grad per view])."""
    xs = [torch.tensor(np.asarray(im, dtype=np.float64), dtype=D, requires_grad=True) for im in images]
    ys = [torch.tensor(np.asarray(t, dtype=np.float64), dtype=D) for t in targets]
    per = [view_loss(x, y, lam) for x, y in zip(xs, ys)]
    total = torch.stack(per).mean()
    total.backward()
    return float(total.detach()), [float(p.detach()) for p in per], [x.grad.numpy() for x in xs]


# ---------------------------------------------------------------------------
# optimiser step
# ---------------------------------------------------------------------------

def activate(raw: np.ndarray, act: int) -> np.ndarray:
    if act == ACT_SIGMOID:
        return 1.0 / (1.0 + np.exp(-raw))
    if act == ACT_EXP:
        return np.exp(raw)
    return raw.copy()


def adam_step(raw, grad_act, m, v, step, planes, beta1=0.9, beta2=0.999, eps=1e-15, lambda_eps=1.0,
              noise=None):
    """One Adam step (Kingma and Ba 2015, Algorithm 1) on raw parameters, in
    float64, plane by plane.

    raw, grad_act, m, v: [K, P] arrays (grad_act is dL/d(activated value));
    planes: K tuples (lr, act, reg, noise_row): learning rate, activation,
    weight of an L1 penalty on the activated value, and the row of ``noise``
    added after the update (or -1).  Returns (raw', act', m', v').
    For each element:
        a = act(raw);  g = dL/da + reg * sign(a);  g_raw = g * act'(raw)
        m = beta1 m + (1 - beta1) g_raw;  v = beta2 v + (1 - beta2) g_raw^2
        raw = raw - lr * (m / (1 - beta1^t)) / (sqrt(v / (1 - beta2^t)) + eps)
        raw = raw + lambda_eps * noise[row]   (rows with noise)
    """
    raw = np.array(raw, dtype=np.float64)
    m = np.array(m, dtype=np.float64)
    v = np.array(v, dtype=np.float64)
    grad_act = np.asarray(grad_act, dtype=np.float64)
    K = raw.shape[0]
    out_act = np.empty_like(raw)
    for k in range(K):
        lr, act, reg, row = planes[k]
        a = activate(raw[k], act)
        g = grad_act[k] + reg * np.sign(a)
        if act == ACT_SIGMOID:
            g = g * a * (1.0 - a)
        elif act == ACT_EXP:
            g = g * a
        m[k] = beta1 * m[k] + (1.0 - beta1) * g
        v[k] = beta2 * v[k] + (1.0 - beta2) * g * g
        mhat = m[k] / (1.0 - beta1 ** step)
        vhat = v[k] / (1.0 - beta2 ** step)
        raw[k] = raw[k] - lr * mhat / (np.sqrt(vhat) + eps)
        if row >= 0 and noise is not None:
            raw[k] = raw[k] + lambda_eps * np.asarray(noise, dtype=np.float64)[row]
        out_act[k] = activate(raw[k], act)
    return raw, out_act, m, v
