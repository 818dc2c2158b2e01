"""Helpers of the GPU parity tests: run the CUDA path through the C-ABI and
compare it with the oracle on the same seeded inputs."""
from __future__ import annotations

import math

import numpy as np
import torch

from oracle import binning, fp32_spec
from oracle import render64 as R64
from paper_2510_03312_gb300 import raster
from paper_2510_03312_gb300 import ubs as U

IMG_TOL = 1e-4   # maximum absolute image error (float32 image vs float64 oracle)
GRAD_TOL = 1e-3  # relative gradient error: per parameter group, and element by element
GRAD_FLOOR = 1e-6  # element-wise bound |g - g_ref| <= GRAD_TOL |g_ref| + GRAD_FLOOR max|g_ref|


def gpu_forward(scenes, views, cfg, capacity=None):
    dev = [raster.DeviceScene.from_scene(s) for s in scenes]
    r = raster.Rasterizer(dev, views, cfg, capacity=capacity)
    img = r.forward(check=True)
    st = r.status()
    torch.cuda.synchronize()
    out = {"rast": r, "dev": dev, "status": st, "image_flat": img}
    out["images"] = [r.view_image(img, v).cpu().numpy() for v in range(len(views))]
    out["tiles"] = r.export(U.EXPORT_TILES).cpu().numpy().view(np.uint32)
    out["keys"] = r.export(U.EXPORT_KEYS).cpu().numpy().view(np.uint32)
    out["rect"] = r.export(U.EXPORT_RECT).cpu().numpy().view(np.uint32).reshape(-1, 2)
    out["rec"] = r.export(U.EXPORT_RECORDS, torch.float32).cpu().numpy().reshape(-1, 12)
    n = int(st.instances)
    out["instances"] = r.export(U.EXPORT_INSTANCES).cpu().numpy().view(np.uint32)[:n]
    out["tstart"] = r.export(U.EXPORT_TILE_START).cpu().numpy().view(np.uint32)
    out["T"] = r.export(U.EXPORT_FINAL_T, torch.float32).cpu().numpy()
    out["last"] = r.export(U.EXPORT_LAST).cpu().numpy().view(np.uint32)
    return out


def check_preprocess(gpu, orc, views=None):
    """Bit-exact integer outputs and float32 values for every record;
    double-float screen mean against float64 (for ``views`` only, when
    given)."""
    recs = orc.records(orc.leaves(), views=views)
    for vi, (pre, rec64) in enumerate(zip(orc.pre32, recs)):
        o = int(orc.rec_off[vi])
        P = pre["valid"].size
        tiles = gpu["tiles"][o:o + P].astype(np.int64)
        assert np.array_equal(tiles, pre["tiles_touched"]), f"view {vi}: tiles_touched differ"
        v = pre["valid"]
        assert np.array_equal(tiles > 0, v)
        assert np.array_equal(gpu["keys"][o:o + P][v], pre["depth_bits"][v]), f"view {vi}: depth keys differ"
        rc = gpu["rect"][o:o + P][v]
        rect = np.stack([rc[:, 0] & 0xFFFF, rc[:, 0] >> 16, rc[:, 1] & 0xFFFF, rc[:, 1] >> 16]).astype(np.int64)
        assert np.array_equal(rect, pre["rect"][:, v]), f"view {vi}: rectangles differ"
        g = gpu["rec"][o:o + P][v]
        assert np.array_equal(g[:, 4:7].view(np.uint32), pre["conic"].T[v].view(np.uint32)), "conic bits"
        assert np.array_equal(g[:, 8].view(np.uint32), pre["beta_x"][v].view(np.uint32)), "beta bits"
        # the record holds log2 o(q) in float32 (the float32 o(q) itself is
        # the rule set's, bit-exact): within 2 ulps of its float32 value
        with np.errstate(divide="ignore", invalid="ignore"):
            lo = np.log2(pre["opacity"][v].astype(np.float64))  # -inf where o(q) underflowed to 0
            gl = g[:, 7].astype(np.float64)
            ok_lo = (gl == lo) | (np.abs(gl - lo) <= 2.4e-7 * np.maximum(np.abs(lo), 1.0))
        assert ok_lo.all(), f"view {vi}: log2 o(q) off at {np.flatnonzero(~ok_lo)[:5]}"
        if rec64 is None:
            continue
        mu = g[:, 0:2].astype(np.float64) + g[:, 2:4].astype(np.float64)
        mu64 = rec64["mean2d"].detach().numpy()[v]
        tol = 1e-6 if orc.scenes[orc.views[vi].scene_id].N == 3 else 2e-4
        assert np.abs(mu - mu64).max() <= tol, np.abs(mu - mu64).max()
    return recs


def check_bins(gpu, orc):
    b = orc.bins
    n = b["record"].size
    assert int(gpu["status"].instances) == n, (int(gpu["status"].instances), n)
    assert np.array_equal(gpu["instances"].astype(np.int64), b["record"]), "sorted instance lists differ"
    starts = gpu["tstart"].astype(np.int64)
    assert np.array_equal(starts[:-1], b["ranges"][:, 0]) and np.array_equal(starts[1:], b["ranges"][:, 1])


def check_images(gpu, orc, recs=None, tiles=None, tol=IMG_TOL, check_last=True):
    """Every pixel within tol of the float64 value, or of one admissible
    result where the oracle flagged a near-threshold decision.  Returns
    (max error on unflagged pixels, flagged pixel count).  ``check_last``:
    also the last contributor of every unflagged pixel (not in the
    gradient-check mode, where a pair whose r rounds across 1 with alpha
    near 0 counts as composited on one side only and moves the index
    without changing colour or T)."""
    ref = orc.render(tiles=tiles, recs=recs)
    worst, nflag = 0.0, 0
    for vi in range(len(orc.views)):
        a = gpu["images"][vi].astype(np.float64)
        r = ref["image"][vi].detach().numpy()
        m = ~np.isnan(r[0])
        flag = ref["flag"][vi].numpy() & m
        nflag += int(flag.sum())
        err = np.abs(a - r).max(0)
        ok = m & ~flag
        if ok.any():
            worst = max(worst, float(err[ok].max()))
        bad = np.argwhere(ok & (err > tol))
        assert bad.size == 0, f"view {vi}: {len(bad)} unflagged pixels off by up to {err[ok].max():.3e}"
        off = m & flag & (err > tol)
        for y, x in np.argwhere(off):
            alts = orc.admissible(vi, int(x), int(y), recs=recs)
            d = min(np.abs(np.asarray(c) - a[:, y, x]).max() for c, _, _ in alts)
            assert d <= tol, f"view {vi} pixel ({x},{y}): {d:.3e} from every admissible value"
        # transmittance and last contributor on unflagged pixels
        if not ok.any():
            continue
        T = gpu["T"][orc_pix(orc, vi)].reshape(r.shape[1:])
        assert np.abs(T - ref["T"][vi].numpy())[ok].max() <= tol
        if check_last:
            last = gpu["last"][orc_pix(orc, vi)].reshape(r.shape[1:]).astype(np.int64)
            assert np.array_equal(last[ok], ref["last"][vi].numpy()[ok])
    return worst, nflag, ref


def check_pairs(scenes, views, cfg, tiles=None, tile_free=False):
    """Per-pixel pair counts of the forward's counting variant against the
    oracle's: on every pixel of the rendered tiles whose blending decisions
    are not flagged, the GPU count lies in the oracle's interval, which is a
    single value except where some r lies within float32 rounding of 1.
    Returns (pixels compared, pixels with a one-value interval, GPU total
    over compared pixels)."""
    from dataclasses import replace
    dev = [raster.DeviceScene.from_scene(s) for s in scenes]
    cnt = raster.count_pairs(dev, views, cfg)
    torch.cuda.synchronize()
    gp = cnt["pairs"].cpu().numpy()
    orc = R64.Oracle(scenes, views, replace(cfg, tight_cut=False))
    ref = orc.render(tiles=tiles, tile_free=tile_free)
    n_cmp = n_exact = total = 0
    for vi, v in enumerate(views):
        lo, hi = ref["pairs_lo"][vi].numpy(), ref["pairs_hi"][vi].numpy()
        m = (lo >= 0) & ~ref["flag"][vi].numpy()
        g = gp[orc_pix(orc, vi)].reshape(v.height, v.width)
        bad = m & ((g < lo) | (g > hi))
        assert not bad.any(), (f"view {vi}: {int(bad.sum())} pixels' pair counts outside the oracle's "
                               f"interval, e.g. {[(int(x), int(y), int(g[y, x]), int(lo[y, x]), int(hi[y, x])) for y, x in np.argwhere(bad)[:3]]}")
        n_cmp += int(m.sum())
        n_exact += int((m & (lo == hi)).sum())
        total += int(g[m].sum())
    assert int(cnt["visited"].sum()) > 0
    return n_cmp, n_exact, total


def orc_pix(orc, vi):
    off = sum(v.width * v.height for v in orc.views[:vi])
    v = orc.views[vi]
    return slice(off, off + v.width * v.height)


def check_grads(gpu, orc, ref_render, seed=7, tiles=None, tol=GRAD_TOL, views=None, elem_tol=None):
    """GPU backward against the oracle's autograd gradient for the same
    dL/dimage (zero on flagged pixels and outside the rendered tiles): per
    parameter group within ``tol`` of the group's largest gradient, and
    element by element within ``elem_tol`` (default ``tol``) relative plus
    GRAD_FLOOR of the group's largest."""
    elem_tol = tol if elem_tol is None else elem_tol
    rng = np.random.default_rng(seed)
    gl = []
    for vi, v in enumerate(orc.views):
        g = rng.standard_normal((3, v.height, v.width)).astype(np.float32) / (v.height * v.width)
        fl = ref_render["flag"][vi].numpy() | np.isnan(ref_render["image"][vi].detach().numpy()[0])
        g[:, fl] = 0.0
        gl.append(g)
    out = R64.loss_grads(orc, [x.astype(np.float64) for x in gl], tiles=tiles, views=views)
    r = gpu["rast"]
    grads = r.backward(r.pack(gl))
    torch.cuda.synchronize()
    worst = {}
    for si, sc in enumerate(orc.scenes):
        ga = grads[si].cpu().numpy()
        for name, (o, n) in sc.offsets().items():
            if n == 0:
                continue
            a = ga[o:o + n].astype(np.float64)
            ref = out["params"][si][name]
            scale = np.abs(ref).max()
            if scale == 0:
                assert np.abs(a).max() == 0, name
                continue
            e = np.abs(a - ref).max() / scale
            worst[f"{si}:{name}"] = e
            assert e <= tol, f"scene {si} {name}: relative error {e:.2e}"
            # element by element, so that a wrong gradient of a faint
            # primitive is not hidden by a bright one of the same group
            over = np.abs(a - ref) > elem_tol * np.abs(ref) + GRAD_FLOOR * scale
            assert not over.any(), (f"scene {si} {name}: {int(over.sum())} elements beyond "
                                    f"{elem_tol:g} |g| + {GRAD_FLOOR:g} max|g|, e.g. "
                                    f"{[(float(a.flat[i]), float(ref.flat[i])) for i in np.flatnonzero(over)[:3]]}")
    return worst
