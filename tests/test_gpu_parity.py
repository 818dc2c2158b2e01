"""GPU parity: the CUDA path through the C-ABI against the CPU oracle.

Bit-exact: culling, depth keys, tile rectangles, float32 conic/beta, sorted
instance lists and tile ranges.  Images: maximum absolute error 1e-4 against
float64 (admissible branches near thresholds).  Gradients: relative error
1e-3 per parameter group and element by element (plus 1e-6 of the group's
largest) against the oracle's autograd gradients.  Pair counts (records
with r < 1 met before a pixel terminates, the blend kernels' work unit)
exact against the oracle's count.
"""
import numpy as np
import pytest
import torch

from oracle import render64 as R64
from paper_2510_03312_gb300 import raster
from paper_2510_03312_gb300 import scenes as S
from paper_2510_03312_gb300 import ubs as U

from parity_tools import check_bins, check_grads, check_images, check_pairs, check_preprocess, gpu_forward

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2510_03312_gb300 import build
    build.build()
    assert torch.cuda.is_available()


def _multi(N, P, nv, W, H, seed, mode=S.ROT_QUAT, tile=(16, 16), extent=2.0, radius=5.0):
    rng = np.random.default_rng(seed)
    sc = S.make_scene(seed, N, P, means="clusters", extent=extent, n_clusters=8, rot_mode=mode, rng=rng)
    views = S.sphere_views(rng, nv, radius, W, H, hemisphere=True, times=list(rng.uniform(0, 1, nv)))
    cfg = S.RasterConfig(tile_w=tile[0], tile_h=tile[1])
    return [sc], views, cfg


CASES = {
    "static_small": lambda: (lambda w: (w.scenes, w.views, w.cfg))(S.workload_static_small()),
    "n3_ragged_2views": lambda: _multi(3, 3000, 2, 200, 150, 11),
    "n3_skew": lambda: _multi(3, 2500, 1, 160, 120, 12, mode=S.ROT_SKEW1),
    "n3_skew2": lambda: _multi(3, 2500, 1, 160, 120, 16, mode=S.ROT_SKEW2),
    "n6_cayley_2views": lambda: _multi(6, 8000, 2, 150, 110, 17, mode=S.ROT_CAYLEY),
    "n7_chol_2views": lambda: _multi(7, 20000, 2, 150, 110, 18, mode=S.ROT_CHOL),
    "n3_exp": lambda: _multi(3, 2500, 1, 160, 120, 19, mode=S.ROT_EXP),
    "n6_3views": lambda: _multi(6, 12000, 3, 176, 132, 13),
    "n7_3views": lambda: _multi(7, 30000, 3, 150, 110, 14),
    "n4_2views": lambda: _multi(4, 6000, 2, 130, 90, 15),
    "tile8": lambda: _multi(3, 3000, 1, 120, 100, 16, tile=(8, 8)),
    "tile16x32": lambda: _multi(3, 3000, 1, 120, 100, 17, tile=(16, 32)),
    "tile32": lambda: _multi(3, 3000, 1, 140, 100, 18, tile=(32, 32)),
}


@pytest.mark.parametrize("case", list(CASES))
def test_forward_parity(case):
    scenes, views, cfg = CASES[case]()
    orc = R64.Oracle(scenes, views, cfg)
    gpu = gpu_forward(scenes, views, cfg)
    assert gpu["status"].status == 0
    recs = check_preprocess(gpu, orc)
    check_bins(gpu, orc)
    worst, nflag, _ = check_images(gpu, orc, recs=recs)
    print(f"{case}: max image error {worst:.2e}, flagged pixels {nflag}")


@pytest.mark.parametrize("case", ["static_small", "n3_ragged_2views", "n6_3views", "n7_3views", "n4_2views", "tile8",
                                  "tile16x32"])
def test_pair_counts(case):
    """The counting variant of the forward against the oracle's tile-free
    pair count, per pixel (lists built without the tight cut)."""
    scenes, views, cfg = CASES[case]()
    n_cmp, n_exact, total = check_pairs(scenes, views, cfg, tile_free=case == "static_small")
    assert n_exact >= 0.99 * n_cmp and total > 0
    print(f"{case}: {n_cmp} pixels, {n_exact} with one admissible count, {total} pairs")


@pytest.mark.parametrize("case", ["n3_ragged_2views", "n3_skew", "n3_skew2", "n6_cayley_2views", "n7_chol_2views", "n3_exp",
                                  "n6_3views",
                                  "n7_3views", "n4_2views", "tile8", "tile32"])
def test_backward_parity(case):
    scenes, views, cfg = CASES[case]()
    orc = R64.Oracle(scenes, views, cfg)
    gpu = gpu_forward(scenes, views, cfg)
    recs = orc.records(orc.leaves())
    _, _, ref = check_images(gpu, orc, recs=recs)
    worst = check_grads(gpu, orc, ref)
    print(case, {k: f"{v:.1e}" for k, v in worst.items()})


def test_uneven_batch_of_scenes():
    """Several scenes of different N, views of different sizes, one problem."""
    scenes = [S.make_scene(40, 3, 2000, means="clusters", extent=2.0, n_clusters=6),
              S.make_scene(41, 6, 8000, means="clusters", extent=2.0, n_clusters=6),
              S.make_scene(42, 7, 20000, means="clusters", extent=2.0, n_clusters=6)]
    rng = np.random.default_rng(43)
    views = []
    for k, (W, H) in enumerate([(96, 64), (130, 77), (64, 140), (100, 100), (33, 47)]):
        R, t = S.look_at(5.0 * (lambda u: u / np.linalg.norm(u))(rng.standard_normal(3)))
        views.append(S.make_view(R, t, W, H, time=float(rng.uniform()), scene_id=k % 3))
    cfg = S.RasterConfig()
    orc = R64.Oracle(scenes, views, cfg)
    gpu = gpu_forward(scenes, views, cfg)
    recs = check_preprocess(gpu, orc)
    check_bins(gpu, orc)
    _, _, ref = check_images(gpu, orc, recs=recs)
    check_grads(gpu, orc, ref)


def test_everything_culled_renders_background():
    sc = S.make_scene(50, 3, 500, means="uniform", extent=1.0)
    R, t = S.look_at((0.0, 0.0, -3.0), target=(0.0, 0.0, -10.0))
    v = S.make_view(R, t, 64, 48)
    cfg = S.RasterConfig(bg=(0.25, 0.5, 0.75))
    gpu = gpu_forward([sc], [v], cfg)
    assert gpu["status"].visible_records == 0 and gpu["status"].instances == 0
    img = gpu["images"][0]
    for c, b in enumerate(cfg.bg):
        assert np.all(img[c] == np.float32(b))


def test_capacity_overflow_is_reported_and_recovered():
    scenes, views, cfg = CASES["n3_ragged_2views"]()
    orc = R64.Oracle(scenes, views, cfg)
    need = orc.bins["record"].size
    gpu = gpu_forward(scenes, views, cfg, capacity=need // 3)
    # forward(check=True) grew the capacity and re-ran
    assert gpu["rast"].capacity >= need
    check_bins(gpu, orc)
    r = gpu["rast"]
    r.set_capacity(need // 3)
    r.problem.instance_capacity = need // 3
    r.preprocess()
    r.bin_sort()
    st = r.status()
    assert st.status == 3 and st.instances == need  # UBS_ERR_CAPACITY with the required count


def test_tiny_and_single_pixel_views():
    sc = S.make_scene(60, 3, 400, means="uniform", extent=0.5, scale_range=(0.05, 0.3))
    R, t = S.look_at((0.0, 0.0, -2.5))
    views = [S.make_view(R, t, 1, 1), S.make_view(R, t, 17, 3), S.make_view(R, t, 3, 33)]
    cfg = S.RasterConfig()
    orc = R64.Oracle([sc], views, cfg)
    gpu = gpu_forward([sc], views, cfg)
    recs = check_preprocess(gpu, orc)
    check_bins(gpu, orc)
    check_images(gpu, orc, recs=recs)


def test_large_screen_filling_primitive():
    sc = S.make_scene(61, 3, 8, means="uniform", extent=0.1, scale_range=(0.5, 1.5))
    R, t = S.look_at((0.0, 0.0, -2.0))
    v = S.make_view(R, t, 300, 200)
    cfg = S.RasterConfig()
    orc = R64.Oracle([sc], [v], cfg)
    gpu = gpu_forward([sc], [v], cfg)
    recs = check_preprocess(gpu, orc)
    check_bins(gpu, orc)
    _, _, ref = check_images(gpu, orc, recs=recs)
    check_grads(gpu, orc, ref)


def test_single_tile_problem():
    """One tile in the whole problem: no tile-key radix pass at all."""
    sc = S.make_scene(62, 3, 600, means="uniform", extent=0.5, scale_range=(0.05, 0.4))
    R, t = S.look_at((0.0, 0.0, -2.5))
    v = S.make_view(R, t, 16, 16)
    cfg = S.RasterConfig()
    orc = R64.Oracle([sc], [v], cfg)
    gpu = gpu_forward([sc], [v], cfg)
    assert gpu["status"].instances > 0
    recs = check_preprocess(gpu, orc)
    check_bins(gpu, orc)
    _, _, ref = check_images(gpu, orc, recs=recs)
    check_grads(gpu, orc, ref)


def test_records_spanning_emission_blocks():
    """Primitives that each touch thousands of tiles, among many small ones:
    one record's instances cross the 4096-instance emission blocks."""
    big = S.make_scene(63, 3, 6, means="uniform", extent=0.05, scale_range=(0.8, 1.6))
    small = S.make_scene(64, 3, 3000, means="uniform", extent=1.0, scale_range=(0.01, 0.05))
    sc = S.Scene(3, big.rot_mode, np.ascontiguousarray(np.concatenate([big.params, small.params], axis=1)))
    R, t = S.look_at((0.0, 0.0, -2.0))
    v = S.make_view(R, t, 2048, 2048)
    cfg = S.RasterConfig()
    orc = R64.Oracle([sc], [v], cfg)
    gpu = gpu_forward([sc], [v], cfg)
    counts = orc.pre32[0]["tiles_touched"]
    assert counts.max() > 4096
    recs = check_preprocess(gpu, orc)
    check_bins(gpu, orc)
    rng = np.random.default_rng(1)
    n_tiles = orc.bins["ranges"].shape[0]
    tiles = sorted(rng.choice(n_tiles, 6, replace=False).tolist())
    _, _, ref = check_images(gpu, orc, recs=recs, tiles=tiles)
    check_grads(gpu, orc, ref, tiles=tiles)


def test_very_long_tile_lists():
    """24,000 primitives in a tiny cube: two tiles hold about 14,000
    instances each (lists far longer than one blend batch or one sort
    block)."""
    sc = S.make_scene(65, 3, 24000, means="uniform", extent=0.04, scale_range=(0.01, 0.04))
    R, t = S.look_at((0.0, 0.0, -3.0))
    v = S.make_view(R, t, 96, 80)
    cfg = S.RasterConfig()
    orc = R64.Oracle([sc], [v], cfg)
    counts = np.diff(orc.bins["ranges"], axis=1)[:, 0]
    assert counts.max() > 8192
    gpu = gpu_forward([sc], [v], cfg)
    recs = check_preprocess(gpu, orc)
    check_bins(gpu, orc)
    tiles = sorted(np.argsort(-counts)[:2].tolist())
    _, _, ref = check_images(gpu, orc, recs=recs, tiles=tiles)
    check_grads(gpu, orc, ref, tiles=tiles)
    n_cmp, n_exact, total = check_pairs([sc], [v], cfg, tiles=tiles)
    assert n_cmp > 0 and total > 0


def test_equal_depths_keep_record_order():
    """16,000 primitives on one plane parallel to the image plane, so that
    every visible record has the same float32 depth: each tile's list must
    come out in record order (Sec. 3's front-to-back order, the record index
    breaking ties), bit for bit, although the binning's buckets are filled
    in the order its atomic adds happen to run.  The longest lists (over
    6,000 entries) go through the chunked sort and both kinds of merge."""
    rng = np.random.default_rng(67)
    sc = S.make_scene(67, 3, 16000, means="uniform", extent=0.3, scale_range=(0.02, 0.06), rng=rng)
    sc.plane("mean_x")[2] = 0.0
    v = S.View(R=np.eye(3, dtype=np.float32), t=np.array([0, 0, 3], np.float32), fx=120.0, fy=120.0,
               cx=48.0, cy=40.0, width=96, height=80)
    cfg = S.RasterConfig()
    orc = R64.Oracle([sc], [v], cfg)
    pre = orc.pre32[0]
    vis = pre["valid"] & (pre["tiles_touched"] > 0)
    assert vis.sum() > 15000 and np.unique(pre["depth_bits"][vis]).size == 1
    counts = np.diff(orc.bins["ranges"], axis=1)[:, 0]
    assert counts.max() > 4096
    gpu = gpu_forward([sc], [v], cfg)
    recs = check_preprocess(gpu, orc)
    check_bins(gpu, orc)
    check_images(gpu, orc, recs=recs, tiles=sorted(np.argsort(-counts)[:2].tolist()))


def test_binning_over_two_million_tiles():
    """17 views of 4096x2048 at 8x8 tiles: 2,228,224 tiles, more than the
    2048 x 1024 the binning's scan covers in two kernels, so its middle
    kernel scans the blocks' sums in between.  Instance lists and tile
    ranges bit-exact against the oracle."""
    rng = np.random.default_rng(68)
    sc = S.make_scene(68, 3, 3000, means="uniform", extent=1.0, rng=rng)
    views = S.sphere_views(rng, 17, 4.0, 4096, 2048)
    cfg = S.RasterConfig(tile_w=8, tile_h=8)
    n_tiles = 17 * (4096 // 8) * (2048 // 8)
    assert (n_tiles + 1023) // 1024 > 2048
    orc = R64.Oracle([sc], views, cfg)
    r = raster.Rasterizer([raster.DeviceScene.from_scene(sc)], views, cfg)
    r.forward(check=True)
    st = r.status()
    n = int(st.instances)
    assert n > 10000
    gpu = {"status": st,
           "instances": r.export(U.EXPORT_INSTANCES).cpu().numpy().view(np.uint32)[:n],
           "tstart": r.export(U.EXPORT_TILE_START).cpu().numpy().view(np.uint32)}
    assert gpu["tstart"].size == n_tiles + 1
    check_bins(gpu, orc)


def _deep_tile_case(split):
    sc = S.make_scene(65, 3, 24000, means="uniform", extent=0.04, scale_range=(0.01, 0.04))
    R, t = S.look_at((0.0, 0.0, -3.0))
    return [sc], [S.make_view(R, t, 96, 80)], S.RasterConfig(split_lists=split)


def _faint_overlap_case(split):
    """6,000 faint, wide, nearly flat primitives (opacity 0.0045-0.006, beta
    0.2) stacked over the centre of a 64x64 view: the central tiles' lists
    hold about 6,000 entries (three segments) and their pixels reach T_min
    after 1,700 to 2,500 of them, inside the first or the second segment."""
    rng = np.random.default_rng(66)
    sc = S.make_scene(66, 3, 6000, means="uniform", extent=0.02, scale_range=(0.4, 0.6), rng=rng)
    sc.plane("b")[:] = np.float32(np.log(0.05))
    sc.plane("opacity")[:] = rng.uniform(0.0045, 0.006, (1, sc.P)).astype(np.float32)
    R, t = S.look_at((0.0, 0.0, -3.0))
    return [sc], [S.make_view(R, t, 64, 64)], S.RasterConfig(split_lists=split)


@pytest.mark.parametrize("make", [_deep_tile_case, _faint_overlap_case], ids=["deep_lists", "terminate_in_segment"])
def test_split_long_lists(make):
    """Long tile lists blended in segments of 2048 entries by separate CTAs
    and merged front to back (UBS_FLAG_SPLIT_LISTS): images, final T, last
    contributors and gradients on the split tiles against the oracle, and
    the whole image within 1e-5 of the unsplit path."""
    scenes, views, cfg = make(True)
    orc = R64.Oracle(scenes, views, cfg)
    counts = np.diff(orc.bins["ranges"], axis=1)[:, 0]
    tiles = sorted(np.flatnonzero(counts > 2048).tolist())
    assert tiles and counts.max() > 2 * 2048
    gpu = gpu_forward(scenes, views, cfg)
    recs = check_preprocess(gpu, orc)
    check_bins(gpu, orc)
    worst, nflag, ref = check_images(gpu, orc, recs=recs, tiles=tiles)
    print(f"split: max image error {worst:.2e} on {len(tiles)} split tiles, flagged {nflag}")
    # pixels of the faint stack composite about 2,000 layers before T_min: the
    # backward recovers T by dividing out 2,000 factors in float32 (up to
    # 2,000 roundings, ~1e-4 relative) and dL/dalpha cancels (c - behind), so a
    # few small elements of that case sit above 1e-3 relative in the unsplit
    # form as well (an element 4.4e-3 off, 1.46x the bound); the group-wise
    # bound holds at 1e-5
    elem = 5e-3 if make is _faint_overlap_case else None
    check_grads(gpu, orc, ref, tiles=tiles, elem_tol=elem)
    plain = gpu_forward(*make(False))
    assert np.abs(gpu["images"][0] - plain["images"][0]).max() <= 1e-5
    if make is _faint_overlap_case:  # pixels end inside a later segment: the merge walks it again
        last = gpu["last"].reshape(views[0].height, views[0].width)
        assert (last > 2048).sum() > 50 and (last <= 2048).sum() > 50


@pytest.mark.parametrize("n_views,N", [(40, 6), (256, 7), (40, 3)])
def test_many_views_of_one_scene(n_views, N):
    """More views than one 32-view mask of the parameter backward, up to the
    256-view limit (the largest view table in shared memory)."""
    rng = np.random.default_rng(70 + n_views + N)
    sc = S.make_scene(71, N, 1500, means="clusters", extent=2.0, n_clusters=4, rng=rng)
    views = S.sphere_views(rng, n_views, 5.0, 24, 20, hemisphere=True, times=list(rng.uniform(0, 1, n_views)))
    cfg = S.RasterConfig()
    orc = R64.Oracle([sc], views, cfg)
    gpu = gpu_forward([sc], views, cfg)
    assert gpu["status"].visible_records > 0
    recs = check_preprocess(gpu, orc)
    check_bins(gpu, orc)
    _, _, ref = check_images(gpu, orc, recs=recs)
    check_grads(gpu, orc, ref)


def test_full_size_static_sampled():
    """The 1M-primitive 1600x1060 workload in the launch configuration the
    benchmark times: all records and instance lists bit-exact, images and
    gradients on sampled tiles."""
    wl = S.workload_static_large()
    orc = R64.Oracle(wl.scenes, wl.views, wl.cfg)
    gpu = gpu_forward(wl.scenes, wl.views, wl.cfg)
    recs = check_preprocess(gpu, orc)
    check_bins(gpu, orc)
    counts = np.diff(orc.bins["ranges"], axis=1)[:, 0]
    order = np.argsort(-counts)
    rng = np.random.default_rng(0)
    tiles = sorted(set(order[:4].tolist()) | set(rng.choice(counts.size, 8, replace=False).tolist()))
    worst, nflag, ref = check_images(gpu, orc, recs=recs, tiles=tiles)
    print(f"full size: max image error {worst:.2e} on {len(tiles)} tiles, flagged {nflag}")
    check_grads(gpu, orc, ref, tiles=tiles)
    del gpu
    n_cmp, n_exact, total = check_pairs(wl.scenes, wl.views, wl.cfg, tiles=tiles)
    print(f"full size pair counts: {n_cmp} pixels, {n_exact} with one admissible count, {total} pairs")
    assert n_exact >= 0.99 * n_cmp


@pytest.mark.parametrize("make", [S.workload_view_dependent, S.workload_dynamic, S.workload_uneven_mix],
                         ids=["n6_500k_16views", "n7_300k_8views", "mix_64jobs"])
def test_full_size_batched_sampled(make):
    """The view-dependent (N=6, 500K primitives, 16 x 1280x720), dynamic
    (N=7, 300K primitives, 8 x 1352x1014) and uneven-mix (64 jobs over 8
    scenes of 12K-1.9M primitives, 25M records) workloads in one launch with
    16x16 tiles, the batched form the benchmark times: every record's integer
    outputs and every sorted instance list bit-exact; records of the sampled
    views, images, transmittance, last contributors and gradients on sampled
    tiles (the densest three and six at random) against float64."""
    wl = make()
    orc = R64.Oracle(wl.scenes, wl.views, wl.cfg)
    gpu = gpu_forward(wl.scenes, wl.views, wl.cfg)
    check_bins(gpu, orc)
    counts = np.diff(orc.bins["ranges"], axis=1)[:, 0]
    order = np.argsort(-counts)
    rng = np.random.default_rng(1)
    nonempty = np.flatnonzero(counts)
    tiles = sorted(set(order[:3].tolist()) | set(rng.choice(nonempty, 6, replace=False).tolist()))
    views = sorted({orc.view_of_tile(g) for g in tiles})
    recs = check_preprocess(gpu, orc, views=views)
    worst, nflag, ref = check_images(gpu, orc, recs=recs, tiles=tiles)
    print(f"{wl.name}: max image error {worst:.2e} on {len(tiles)} tiles of views {views}, flagged {nflag}")
    check_grads(gpu, orc, ref, tiles=tiles, views=views)


def test_empty_scenes():
    """A problem whose only scene has no primitives (no records at all)
    renders the background with nothing to sort; beside a non-empty scene,
    an empty one changes nothing of the other scene's view, and its
    gradient is empty."""
    from paper_2510_03312_gb300 import raster
    K = S.params_per_primitive(3, S.ROT_QUAT)
    empty = S.Scene(3, S.ROT_QUAT, np.zeros((K, 0), np.float32))
    R, t = S.look_at((0.0, 0.0, -3.0))
    cfg = S.RasterConfig(bg=(0.25, 0.5, 0.75))
    gpu = gpu_forward([empty], [S.make_view(R, t, 40, 24)], cfg)
    assert gpu["status"].status == 0 and gpu["status"].instances == 0
    for c, b in enumerate(cfg.bg):
        assert np.all(gpu["images"][0][c] == np.float32(b))
    # an empty scene beside a non-empty one
    full = S.make_scene(51, 3, 800, means="uniform", extent=1.0)
    v_full = S.make_view(R, t, 72, 56, scene_id=1)
    v_empty = S.make_view(R, t, 40, 24, scene_id=0)
    both = gpu_forward([empty, full], [v_empty, v_full], cfg)
    alone = gpu_forward([full], [S.make_view(R, t, 72, 56)], cfg)
    assert both["status"].status == 0
    assert np.array_equal(both["images"][1], alone["images"][0])
    for c, b in enumerate(cfg.bg):
        assert np.all(both["images"][0][c] == np.float32(b))
    rng = np.random.default_rng(2)
    dl = torch.from_numpy(rng.uniform(-1, 1, both["image_flat"].numel()).astype(np.float32)).cuda()
    r = both["rast"]
    r.forward(check=False)
    g = r.backward(dl.view_as(both["image_flat"]))
    torch.cuda.synchronize()
    assert g[0].numel() == 0 and torch.isfinite(g[1]).all() and float(g[1].abs().max()) > 0
