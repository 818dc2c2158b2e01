"""Tile binning and depth ordering by definition (test infrastructure only).

"Standard splatting" (Sec. 4.5) draws each projected primitive into every
screen tile its footprint rectangle touches and blends each tile's list front
to back (Sec. 3, alpha compositing in sorted order).  The sorted instance list
is defined here without any parallel algorithm: every (tile, record) pair is
listed and the list is sorted lexicographically by

    (global tile id, float32 depth bits, record index)

where global tile id = tile offset of the view + ty * tiles_x + tx and record
index = record offset of the view + primitive index.  Depth bits order
positive floats like the floats themselves; the record index breaks ties.

Parity: pinned by tests against a brute-force per-pixel depth sort and
against hand-built rectangles (tests/test_oracle_binning.py).
"""
from __future__ import annotations

import numpy as np


def tile_grid(view, cfg):
    tx = (view.width + cfg.tile_w - 1) // cfg.tile_w
    ty = (view.height + cfg.tile_h - 1) // cfg.tile_h
    return tx, ty


def offsets(scenes, views, cfg):
    rec_off, tile_off = [0], [0]
    for v in views:
        rec_off.append(rec_off[-1] + scenes[v.scene_id].P)
        tx, ty = tile_grid(v, cfg)
        tile_off.append(tile_off[-1] + tx * ty)
    return np.array(rec_off, np.int64), np.array(tile_off, np.int64)


def bin_and_sort(scenes, views, cfg, pre):
    """``pre`` is the list of per-view dicts from ``fp32_spec.preprocess``.
    Returns the sorted (tile, record) instance list and per-tile ranges."""
    rec_off, tile_off = offsets(scenes, views, cfg)
    tiles_l, depth_l, rec_l = [], [], []
    for v, (view, out) in enumerate(zip(views, pre)):
        ntx, _ = tile_grid(view, cfg)
        idx = np.nonzero(out["valid"] & (out["tiles_touched"] > 0))[0]
        if idx.size == 0:
            continue
        tx0, ty0, tx1, ty1 = (out["rect"][k][idx] for k in range(4))
        w = tx1 - tx0
        cnt = (tx1 - tx0) * (ty1 - ty0)
        rep = np.repeat(np.arange(idx.size), cnt)
        # position of each instance inside its rectangle, row-major
        start = np.repeat(np.cumsum(cnt) - cnt, cnt)
        k = np.arange(rep.size) - start
        tx = tx0[rep] + k % w[rep]
        ty = ty0[rep] + k // w[rep]
        tiles_l.append(tile_off[v] + ty * ntx + tx)
        depth_l.append(out["depth_bits"][idx][rep].astype(np.uint64))
        rec_l.append(rec_off[v] + idx[rep])
    n_tiles = int(tile_off[-1])
    if not tiles_l:
        return {"tile": np.zeros(0, np.int64), "record": np.zeros(0, np.int64),
                "ranges": np.zeros((n_tiles, 2), np.int64), "tile_offset": tile_off,
                "record_offset": rec_off}
    tiles = np.concatenate(tiles_l)
    depth = np.concatenate(depth_l)
    rec = np.concatenate(rec_l)
    order = np.lexsort((rec, depth, tiles))
    tiles, rec = tiles[order], rec[order]
    starts = np.searchsorted(tiles, np.arange(n_tiles), side="left")
    ends = np.searchsorted(tiles, np.arange(n_tiles), side="right")
    return {"tile": tiles, "record": rec, "depth_bits": depth[order].astype(np.uint32),
            "ranges": np.stack([starts, ends], axis=1).astype(np.int64),
            "tile_offset": tile_off, "record_offset": rec_off}
