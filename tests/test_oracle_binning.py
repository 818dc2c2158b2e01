"""Pins of the oracle's binning: hand-built lists and a per-tile brute force."""
import numpy as np

from oracle import binning, fp32_spec
from paper_2510_03312_gb300 import scenes as S


def _fake(rects, depths):
    rects = np.asarray(rects, np.int64).T
    d = np.asarray(depths, np.float32)
    valid = np.ones(d.size, bool)
    return {"valid": valid, "rect": rects, "depth_bits": d.view(np.uint32),
            "tiles_touched": (rects[2] - rects[0]) * (rects[3] - rects[1])}


def test_hand_built_instances_and_ranges():
    cfg = S.RasterConfig(tile_w=16, tile_h=16)
    v = S.View(np.eye(3, dtype=np.float32), np.zeros(3, np.float32), 1, 1, 0, 0, 48, 32)
    sc = S.make_scene(0, 3, 3)
    # 3x2 tiles; record 0 covers tiles (0,0),(1,0); record 1 covers (1,0),(1,1);
    # record 2 covers (1,0) only and is the nearest; record 0 ties record 1
    pre = [_fake([[0, 0, 2, 1], [1, 0, 2, 2], [1, 0, 2, 1]], [5.0, 5.0, 2.0])]
    out = binning.bin_and_sort([sc], [v], cfg, pre)
    assert out["tile"].tolist() == [0, 1, 1, 1, 4]
    assert out["record"].tolist() == [0, 2, 0, 1, 1]
    assert out["ranges"].tolist() == [[0, 1], [1, 4], [4, 4], [4, 4], [4, 5], [5, 5]]


def test_sorted_lists_equal_per_tile_brute_force():
    wl = S.workload_static_small(seed=5, P=700, size=80)
    cfg = wl.cfg
    pre = fp32_spec.preprocess(wl.scenes, wl.views + wl.views[:1], cfg)
    views = wl.views + wl.views[:1]
    out = binning.bin_and_sort([wl.scenes[0]], views, cfg, pre)
    rec_off, tile_off = out["record_offset"], out["tile_offset"]
    for vi, v in enumerate(views):
        ntx, nty = binning.tile_grid(v, cfg)
        p = pre[vi]
        for ty in range(nty):
            for tx in range(ntx):
                g = tile_off[vi] + ty * ntx + tx
                x0, y0, x1, y1 = p["rect"]
                inside = p["valid"] & (x0 <= tx) & (tx < x1) & (y0 <= ty) & (ty < y1)
                idx = np.nonzero(inside)[0]
                exp = sorted(idx.tolist(), key=lambda i: (float(p["depth"][i]), i))
                s, e = out["ranges"][g]
                got = (out["record"][s:e] - rec_off[vi]).tolist()
                assert got == exp
    assert out["ranges"][:, 1].max() == out["tile"].size
