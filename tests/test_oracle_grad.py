"""Pins of the oracle's gradients: autograd of the float64 forward against
central finite differences of the same forward, per parameter group.

Finite differences run with fixed decisions (the float32 lists of the
unperturbed scene) and without thresholds (alpha_min = 0, T_min = 0), on
scenes where every beta_x > 1 so that the kernel is C^1 at the support edge.
"""
import numpy as np
import pytest
import torch

from oracle import render64 as R64
from paper_2510_03312_gb300 import scenes as S

D = torch.float64


def _tiny(N, mode, seed):
    rng = np.random.default_rng(seed)
    sc = S.make_scene(seed, N, 6, means="uniform", extent=0.35, scale_range=(0.08, 0.2),
                      rot_mode=mode, rng=rng)
    sc.plane("b")[0] = rng.uniform(0.0, 0.5, sc.P)
    if N > 3:
        sc.plane("b")[1:] = rng.choice([-1, 1], size=(N - 3, sc.P)) * rng.uniform(0.1, 0.6, (N - 3, sc.P))
    R, t = S.look_at((0.4, 0.6, -2.5))
    v = S.make_view(R, t, 24, 20, fov_x_deg=50.0, time=0.35)
    cfg = S.RasterConfig(alpha_min=0.0, T_min=0.0, tile_w=8, tile_h=8)
    return sc, v, cfg


def _loss(orc, leaves, g):
    img = orc.render(leaves=leaves)["image"][0]
    return float((img * g).sum())


@pytest.mark.parametrize("N,mode", [(3, 0), (3, 1), (6, 0), (7, 1), (4, 0), (3, 2), (6, 3), (3, 4), (7, 4), (3, 5),
                                    (6, 5)])
def test_autograd_matches_central_differences(N, mode):
    sc, v, cfg = _tiny(N, mode, 40 + N + mode)
    orc = R64.Oracle([sc], [v], cfg)
    assert orc.bins["tile"].size > 0
    g = torch.tensor(np.random.default_rng(1).standard_normal((3, v.height, v.width)), dtype=D)
    out = R64.loss_grads(orc, [g.numpy()])
    ana = out["params"][0]
    base = orc.leaves(False)[0]
    for name, t in base.items():
        if t.numel() == 0:
            continue
        num = np.zeros(tuple(t.shape))
        for idx in np.ndindex(*t.shape):
            h = 1e-6 * max(1.0, abs(float(t[idx])))
            lp = {k: x.clone() for k, x in base.items()}
            lm = {k: x.clone() for k, x in base.items()}
            lp[name][idx] += h
            lm[name][idx] -= h
            num[idx] = (_loss(orc, [lp], g) - _loss(orc, [lm], g)) / (2 * h)
        ref = np.abs(num).max()
        if ref == 0:
            assert np.abs(ana[name]).max() == 0
            continue
        err = np.abs(ana[name] - num)
        assert err.max() <= 1e-5 * ref + 1e-9, (name, err.max(), ref)
