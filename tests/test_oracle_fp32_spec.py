"""Pins of the oracle's float32 decision stage.

The float32 stage is pinned against float64 mathematics: its exp and log
against libm in float64, its per-record values against the float64 oracle,
and its integer decisions against per-pixel float64 evaluation (every pixel
the float64 kernel reaches lies inside the float32 tile rectangle; every
culled record is culled in float64 too, up to rounding).
"""
import numpy as np
import pytest
import torch

from oracle import binning, fp32_spec
from oracle import render64 as R64
from paper_2510_03312_gb300 import scenes as S

F = np.float32


def _ulp_err(approx, exact):
    ex32 = exact.astype(F)
    ulp = np.spacing(np.abs(ex32)).astype(np.float64)
    return np.abs(approx.astype(np.float64) - exact) / ulp


def test_exp_spec_within_two_ulp():
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.uniform(-87, 88, 400_000), rng.uniform(-2, 2, 200_000),
                        [0.0, -0.0, 1.0, -1.0, 88.0, -87.0, 0.5]]).astype(F)
    assert _ulp_err(fp32_spec.exp_spec(x), np.exp(x.astype(np.float64))).max() <= 2.0
    assert fp32_spec.exp_spec(np.array([-87.5, -200.0, -np.inf], F)).tolist() == [0.0, 0.0, 0.0]
    assert fp32_spec.exp_spec(np.array([0.0], F))[0] == 1.0


def test_log_spec_within_three_ulp():
    rng = np.random.default_rng(1)
    x = np.exp(rng.uniform(np.log(1e-37), np.log(1e37), 400_000)).astype(F)
    x = np.concatenate([x, rng.uniform(0.5, 2.0, 200_000).astype(F), np.array([1.0, 2.0, 0.5], F)])
    exact = np.log(x.astype(np.float64))
    err = np.abs(fp32_spec.log_spec(x).astype(np.float64) - exact)
    ulp = np.spacing(np.abs(exact.astype(F))).astype(np.float64)
    # relative to the result, or absolute 2^-23 near log x = 0
    assert (err <= np.maximum(3 * ulp, 2.0 ** -23)).all()
    assert fp32_spec.log_spec(np.array([1.0], F))[0] == 0.0
    assert np.isneginf(fp32_spec.log_spec(np.array([0.0, -1.0], F))).all()


def _small_workloads():
    out = [S.workload_static_small(seed=0, P=2048, size=96)]
    for N, seed, P in ((6, 21, 3000), (7, 22, 12000), (4, 23, 3000)):
        rng = np.random.default_rng(seed)
        sc = S.make_scene(seed, N, P, means="clusters", extent=2.0, n_clusters=8, rng=rng)
        views = S.sphere_views(rng, 2, 5.0, 96, 72, hemisphere=True, times=[0.25, 0.8])
        out.append(S.Workload(f"n{N}", [sc], views))
    sk = S.make_scene(24, 3, 1500, means="uniform", extent=1.0, rot_mode=S.ROT_SKEW1)
    out.append(S.Workload("skew", [sk], S.workload_static_small().views))
    for name, mode in (("skew2", S.ROT_SKEW2), ("cayley", S.ROT_CAYLEY), ("chol", S.ROT_CHOL), ("exp", S.ROT_EXP)):
        sk = S.make_scene(25 + mode, 3, 1500, means="uniform", extent=1.0, rot_mode=mode)
        out.append(S.Workload(name, [sk], S.workload_static_small().views))
    return out


@pytest.mark.parametrize("wl", _small_workloads(), ids=lambda w: w.name)
def test_fp32_values_match_float64(wl):
    orc = R64.Oracle(wl.scenes, wl.views, wl.cfg)
    recs = orc.records(orc.leaves())
    for pre, rec in zip(orc.pre32, recs):
        v = pre["valid"]
        assert v.sum() > 100
        with torch.no_grad():
            np.testing.assert_allclose(pre["depth"][v], rec["depth"].numpy()[v], rtol=2e-6)
            np.testing.assert_allclose(pre["mean2d"].T[v], rec["mean2d"].numpy()[v], atol=2e-3)
            cn = rec["conic"].numpy()[v]
            c64 = np.stack([cn[:, 0, 0], cn[:, 0, 1], cn[:, 1, 1]], 1)
            scale = np.abs(c64).max(1, keepdims=True)
            assert (np.abs(pre["conic"].T[v] - c64) / scale).max() < 2e-4
            np.testing.assert_allclose(pre["opacity"][v], rec["opacity"].numpy()[v], rtol=5e-5)
            np.testing.assert_allclose(pre["beta_x"][v], rec["beta_x"].numpy()[v], rtol=1e-6)
            np.testing.assert_allclose(pre["mean3"].T[v], rec["mean3"].numpy()[v], atol=1e-5)


@pytest.mark.parametrize("wl", _small_workloads(), ids=lambda w: w.name)
def test_tile_rectangles_are_conservative(wl):
    """Every pixel whose float64 alpha reaches alpha_min lies in a tile of the
    record's float32 rectangle; culled records cannot reach alpha_min."""
    cfg = wl.cfg
    orc = R64.Oracle(wl.scenes, wl.views, cfg)
    recs = orc.records(orc.leaves())
    amin = float(F(cfg.alpha_min))
    for view, pre, rec in zip(wl.views, orc.pre32, recs):
        with torch.no_grad():
            mu = rec["mean2d"].numpy()
            cn = rec["conic"].numpy()
            oq = rec["opacity"].numpy()
            beta = rec["beta_x"].numpy()
            tz = rec["depth"].numpy()
        ys, xs = np.mgrid[0:view.height, 0:view.width]
        px, py = xs.ravel() + 0.5, ys.ravel() + 0.5
        front = tz > cfg.near * (1 + 1e-6)
        for p in np.nonzero(front)[0]:
            dx, dy = px - mu[p, 0], py - mu[p, 1]
            r = cn[p, 0, 0] * dx * dx + 2 * cn[p, 0, 1] * dx * dy + cn[p, 1, 1] * dy * dy
            a = np.where(r < 1, oq[p] * np.where(r < 1, 1 - r, 1) ** beta[p], 0.0)
            hit = a >= amin * (1 + 1e-4)
            if not hit.any():
                continue
            assert pre["valid"][p], f"record {p} reaches alpha_min but was culled"
            tx, ty = xs.ravel()[hit] // cfg.tile_w, ys.ravel()[hit] // cfg.tile_h
            x0, y0, x1, y1 = pre["rect"][:, p]
            assert (tx >= x0).all() and (tx < x1).all() and (ty >= y0).all() and (ty < y1).all()


def test_near_plane_cull():
    sc = S.make_scene(30, 3, 200, means="uniform", extent=1.0)
    v = S.workload_static_small().views[0]
    v = S.View(v.R, np.array([0, 0, 1.1], F), v.fx, v.fy, v.cx, v.cy, v.width, v.height)
    cfg = S.RasterConfig()
    pre = fp32_spec.preprocess([sc], [v], cfg)[0]
    tz = sc.plane("mean_x")[2].astype(np.float64) + 1.1
    assert not pre["valid"][tz < cfg.near - 1e-6].any()
    assert (pre["tiles_touched"][~pre["valid"]] == 0).all()
