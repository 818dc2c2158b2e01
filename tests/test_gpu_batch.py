"""Batches of jobs run as several launches or one, eagerly or as a captured
CUDA graph, through the C-ABI: with a fixed tile shape the images are
bit-identical to one launch over all views, and each scene's gradient is
the same sum over its views (up to float summation order)."""
from dataclasses import replace

import numpy as np
import pytest
import torch

from paper_2510_03312_gb300 import autotune as A
from paper_2510_03312_gb300 import raster
from paper_2510_03312_gb300 import scenes as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2510_03312_gb300 import build
    build.build()
    assert torch.cuda.is_available()


def _jobs():
    wl = S.workload_uneven_mix(seed=7, n_scenes=3, n_jobs=7, p_range=(2000, 20000), w_range=(40, 200),
                               h_range=(30, 160))
    ds = [raster.DeviceScene.from_scene(s) for s in wl.scenes]
    return wl, ds


def _reference(ds, views, cfg, dls_per_view):
    r = raster.Rasterizer(ds, views, cfg)
    r.forward(check=True)
    dL = torch.cat([d.reshape(-1) for d in dls_per_view])
    r.forward(check=False)
    g = [x.clone() for x in r.backward(dL)]
    imgs = [r.view_image(r.image, i).clone() for i in range(len(views))]
    return imgs, g


def _dl_per_view(views, seed=0):
    rng = np.random.default_rng(seed)
    return [torch.from_numpy(rng.uniform(-1, 1, (3, v.height, v.width)).astype(np.float32)).cuda() * 1e-3
            for v in views]


def _batch_dls(b, per_view):
    out = b.dL_like()
    for gi, g in enumerate(b.groups):
        r = b.rasterizers[gi]
        for k, i in enumerate(g):
            r.view_image(out[gi], k).copy_(per_view[i])
    return out


def _close(a, b, rel=1e-5):
    scale = max(float(b.abs().max()), 1e-12)
    return float((a - b).abs().max()) <= rel * scale


@pytest.mark.parametrize("name", list(A.SCHEDULES))
@pytest.mark.parametrize("graph", [False, True])
def test_batch_schedules_match_one_launch(name, graph):
    wl, ds = _jobs()
    per_view = _dl_per_view(wl.views)
    ref_img, ref_g = _reference(ds, wl.views, wl.cfg, per_view)
    b = raster.Batch(ds, wl.views, wl.cfg, A.SCHEDULES[name](wl.scenes, wl.views))
    b.size()
    dls = _batch_dls(b, per_view)
    if graph:
        g = b.capture(dls)
        for x in b.grads:
            x.fill_(123.0)  # a replay must re-zero and rebuild them
        g.replay()
    else:
        b.step(dls)
    torch.cuda.synchronize()
    assert all(st.status == 0 for st in b.status())
    for i in range(len(wl.views)):
        assert torch.equal(b.image(i), ref_img[i]), f"view {i} differs"
    for s, (x, y) in enumerate(zip(b.grads, ref_g)):
        assert _close(x, y), f"scene {s}: {float((x - y).abs().max()):.3e}"


@pytest.mark.parametrize("tile", A.TILES)
def test_batch_tile_shapes_agree(tile):
    wl, ds = _jobs()
    per_view = _dl_per_view(wl.views)
    ref_img, ref_g = _reference(ds, wl.views, wl.cfg, per_view)
    cfg = replace(wl.cfg, tile_w=tile[0], tile_h=tile[1])
    b = raster.Batch(ds, wl.views, cfg, A.one_launch(wl.scenes, wl.views))
    b.size()
    b.step(_batch_dls(b, per_view))
    torch.cuda.synchronize()
    for i in range(len(wl.views)):
        # the tile origin enters the staged mean's rounding: 1e-4 is the image bound
        assert float((b.image(i) - ref_img[i]).abs().max()) <= 1e-4
    for x, y in zip(b.grads, ref_g):
        assert _close(x, y, rel=1e-3)


def test_device_autotune_returns_a_valid_plan():
    wl, ds = _jobs()
    meas = A.device_measure(ds, wl.views, wl.cfg, steps=2, warmup=1)
    plan = A.tune(wl.scenes, wl.views, wl.cfg, meas, tiles=((16, 16), (32, 32)),
                  schedules={k: A.SCHEDULES[k] for k in ("one_launch", "per_view")})
    assert plan.tile in ((16, 16), (32, 32)) and plan.ms > 0
    assert len(plan.table) == 4 * len(A.FORMS)


@pytest.mark.parametrize("form", ["persistent", "split"])
@pytest.mark.parametrize("tile", A.TILES)
@pytest.mark.parametrize("graph", [False, True])
def test_launch_forms_match_the_grid(form, tile, graph):
    """The persistent launch form of both blend kernels, and the split-list
    form on lists that need no split, give the grid form's images bit for
    bit and the same gradients (up to float summation order), on three
    steps in a row (the persistent tile counters and the split plan's
    counters reset themselves), eagerly and replayed from a captured graph."""
    wl, ds = _jobs()
    cfg = replace(wl.cfg, tile_w=tile[0], tile_h=tile[1])
    per_view = _dl_per_view(wl.views)
    ref_img, ref_g = _reference(ds, wl.views, cfg, per_view)
    b = raster.Batch(ds, wl.views, replace(cfg, **A.form_fields(form)), A.one_launch(wl.scenes, wl.views))
    b.size()
    dls = _batch_dls(b, per_view)
    graph_obj = b.capture(dls) if graph else None
    for step in range(3):
        if graph:
            graph_obj.replay()
        else:
            b.step(dls)
        torch.cuda.synchronize()
        assert all(st.status == 0 for st in b.status())
        for i in range(len(wl.views)):
            assert torch.equal(b.image(i), ref_img[i]), f"step {step}: view {i} differs"
        for s, (x, y) in enumerate(zip(b.grads, ref_g)):
            assert _close(x, y), f"step {step}, scene {s}: {float((x - y).abs().max()):.3e}"


def test_dense_lists_over_many_tiles_match_views_alone():
    """Three 1600x1060 views of the 1M-primitive scene in one launch (20,100
    tiles, about 250 instances a tile): the blend kernels take the tiles
    longest list first, through the multi-block ordering, and every image is
    bit-identical to its view rendered alone (6,700 tiles, ordered by one
    block) and the gradient is the sum of the views' gradients."""
    rng = np.random.default_rng(5)
    sc = S.make_scene(1, 3, 1_000_000, means="clusters", extent=5.0, rng=rng)
    views = S.sphere_views(rng, 3, 8.0, 1600, 1060)
    cfg = S.RasterConfig()
    ds = [raster.DeviceScene.from_scene(sc)]
    per_view = _dl_per_view(views, seed=3)
    r = raster.Rasterizer(ds, views, cfg)
    r.forward(check=True)
    NT = r.n_tiles()
    st = r.status()
    assert NT > 16384 and st.instances >= 64 * NT and r.capacity >= 64 * NT
    r.forward(check=False)
    g = r.backward(torch.cat([d.reshape(-1) for d in per_view]))[0].clone()
    g_sum = torch.zeros_like(g)
    for i, v in enumerate(views):
        r1 = raster.Rasterizer(ds, [v], cfg)
        r1.forward(check=True)
        assert r1.status().instances >= 64 * r1.n_tiles()
        img1 = r1.forward(check=False)
        assert torch.equal(r.view_image(r.image, i), r1.view_image(img1, 0)), f"view {i} differs"
        g_sum += r1.backward(per_view[i].reshape(-1))[0]
        del r1
    assert _close(g, g_sum)
    # the persistent form takes the same longest-first order from its counter
    rp = raster.Rasterizer(ds, views, replace(cfg, persistent=True))
    rp.forward(check=True)
    for _ in range(2):
        imgp = rp.forward(check=False)
        gp = rp.backward(torch.cat([d.reshape(-1) for d in per_view]))[0]
        torch.cuda.synchronize()
        assert torch.equal(imgp, r.image)
        assert _close(gp, g)
