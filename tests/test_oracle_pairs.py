"""Pins of the oracle's pair count, the work unit of the blend kernels: per
pixel, the records with r < 1 (inside the support ellipse of Eq. r) met on
the pixel's front-to-back list before the pixel terminates (Sec. 3
compositing with the skip and stop rules).

Checked against a scalar brute-force loop over every record in depth order,
the closed-form count of pixel centres inside one primitive's disc, and the
equality of the tiled count (lists built without the tight cut) with the
tile-free one."""
from dataclasses import replace

import numpy as np
import torch

from oracle import render64 as R64
from paper_2510_03312_gb300 import scenes as S


def _brute_pairs(orc, recs, vi, x, y):
    """Scalar front-to-back loop over every valid record of view vi in
    (depth bits, record) order: counts r < 1 until the stop rule fires."""
    cfg = orc.cfg
    pre = orc.pre32[vi]
    idx = np.nonzero(pre["valid"] & (pre["tiles_touched"] > 0))[0]
    idx = idx[np.lexsort((idx, pre["depth_bits"][idx]))]
    R = recs[vi]
    amin = float(np.float32(cfg.alpha_min))
    tmin = float(np.float32(cfg.T_min))
    T, n = 1.0, 0
    for p in idx:
        mx, my = (float(u) for u in R["mean2d"][p])
        a, b, c = float(R["conic"][p][0, 0]), float(R["conic"][p][0, 1]), float(R["conic"][p][1, 1])
        dx, dy = x + 0.5 - mx, y + 0.5 - my
        r = a * dx * dx + 2 * b * dx * dy + c * dy * dy
        if r >= 1.0:
            continue
        n += 1
        al = min(cfg.alpha_max, float(R["opacity"][p]) * (1.0 - r) ** float(R["beta_x"][p]))
        if al < amin:
            continue
        if T * (1.0 - al) < tmin:
            break
        T *= 1.0 - al
    return n


def test_pair_count_matches_a_scalar_brute_force_loop():
    wl = S.workload_static_small(seed=5, P=300, size=32)
    cfg = replace(wl.cfg, tight_cut=False)
    orc = R64.Oracle(wl.scenes, wl.views, cfg)
    recs = orc.records(orc.leaves())
    out = orc.render(recs=recs, tile_free=True)
    lo, hi = out["pairs_lo"][0].numpy(), out["pairs_hi"][0].numpy()
    assert hi.max() >= 5
    rng = np.random.default_rng(0)
    for y, x in rng.integers(0, 32, (60, 2)):
        n = _brute_pairs(orc, recs, 0, int(x), int(y))
        assert lo[y, x] <= n <= hi[y, x], (x, y, n, lo[y, x], hi[y, x])
    assert (lo == hi).mean() > 0.95


def test_pair_count_of_one_primitive_is_its_disc():
    """An isotropic primitive on the optical axis: Sigma' = rho^2 I, so the
    count is 1 exactly at the pixel centres with |p - mu'|^2 < rho^2."""
    sc = S.Scene(3, S.ROT_QUAT, np.zeros((S.params_per_primitive(3, S.ROT_QUAT), 1), np.float32))
    sc.plane("rot")[0] = 1.0
    sc.plane("scale_x")[:] = 0.25
    sc.plane("opacity")[:] = 0.8
    v = S.View(R=np.eye(3, dtype=np.float32), t=np.array([0, 0, 3], np.float32), fx=60.0, fy=60.0,
               cx=32.0, cy=24.0, width=64, height=48)
    cfg = S.RasterConfig(tight_cut=False)
    orc = R64.Oracle([sc], [v], cfg)
    out = orc.render(tile_free=True)
    rho2 = (60.0 * float(np.float32(0.25)) / 3.0) ** 2 + float(np.float32(cfg.eps2d))
    ys, xs = np.meshgrid(np.arange(48), np.arange(64), indexing="ij")
    d2 = (xs + 0.5 - 32.0) ** 2 + (ys + 0.5 - 24.0) ** 2
    expect = (d2 < rho2).astype(np.int64)
    assert expect.sum() > 20
    assert np.array_equal(out["pairs_lo"][0].numpy(), expect)
    assert np.array_equal(out["pairs_hi"][0].numpy(), expect)


def test_tiled_pair_count_equals_tile_free_without_the_tight_cut():
    """Without the tight cut every record whose ellipse r < 1 holds a pixel is
    on the pixel's tile list, in the same order, so tiled and tile-free
    counts agree; with the tight cut the tiled count can only be lower."""
    wl = S.workload_static_small(seed=6, P=500, size=64)
    cfg = replace(wl.cfg, tight_cut=False)
    orc = R64.Oracle(wl.scenes, wl.views, cfg)
    tiled = orc.render()
    free = orc.render(tile_free=True)
    for k in ("pairs_lo", "pairs_hi"):
        assert torch.equal(tiled[k][0], free[k][0])
    tight = R64.Oracle(wl.scenes, wl.views, wl.cfg).render()
    assert (tight["pairs_hi"][0] <= free["pairs_hi"][0]).all()
    assert int(free["pairs_hi"][0].sum()) > int(tight["pairs_hi"][0].sum())
