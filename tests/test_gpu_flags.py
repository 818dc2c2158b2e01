"""Configuration flags of the boundary that change no arithmetic of the
path: the gradient-check mode (UBS_FLAG_NO_THRESHOLDS) and the checked mode
(UBS_FLAG_CHECKED), through the C-ABI."""

import numpy as np
import pytest
import torch

from oracle import render64 as R64
from paper_2510_03312_gb300 import raster
from paper_2510_03312_gb300 import scenes as S
from paper_2510_03312_gb300 import ubs as U

from parity_tools import check_grads, check_images, check_preprocess, gpu_forward

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2510_03312_gb300 import build
    build.build()
    assert torch.cuda.is_available()


def _case(N, seed):
    rng = np.random.default_rng(seed)
    sc = S.make_scene(seed, N, 3000, means="clusters", extent=2.0, n_clusters=6, rng=rng)
    views = S.sphere_views(rng, 2, 5.0, 120, 90, hemisphere=True, times=[0.3, 0.8])
    return [sc], views


@pytest.mark.parametrize("N", [3, 6])
def test_no_thresholds_mode_is_the_zero_threshold_configuration(N):
    """With UBS_FLAG_NO_THRESHOLDS the configured alpha_min, alpha_max and
    T_min are replaced by 0, 1 and 0: bit-identical images to a problem that
    configures those values, which matches the oracle under them."""
    scenes, views = _case(N, 80 + N)
    explicit = S.RasterConfig(alpha_min=0.0, alpha_max=1.0, T_min=0.0)
    ref = gpu_forward(scenes, views, explicit)
    dev = [raster.DeviceScene.from_scene(s) for s in scenes]
    r = raster.Rasterizer(dev, views, S.RasterConfig())
    r.problem.cfg.flags |= U.UBS_FLAG_NO_THRESHOLDS
    img = r.forward(check=True)
    torch.cuda.synchronize()
    assert torch.equal(img, ref["image_flat"])
    rng = np.random.default_rng(1)
    dl = torch.from_numpy(rng.uniform(-1, 1, img.numel()).astype(np.float32) * 1e-4).cuda()
    g_flag = r.backward(dl)[0].clone()
    g_ref = ref["rast"].backward(dl)[0]
    torch.cuda.synchronize()
    assert float((g_flag - g_ref).abs().max()) <= 1e-5 * float(g_ref.abs().max())
    # and the zero-threshold configuration against the oracle
    orc = R64.Oracle(scenes, views, explicit)
    recs = check_preprocess(ref, orc)
    _, _, out = check_images(ref, orc, recs=recs, check_last=False)
    check_grads(gpu_forward(scenes, views, explicit), orc, out)


def _instance_offset(r, n):
    """Offset (in int32 words from the workspace start) of the sorted
    instance list, found by its contents."""
    inst = r.export(U.EXPORT_INSTANCES)[:n].cpu().numpy()
    base = (r.ws_ptr - r._ws.data_ptr())
    words = r._ws[base:base + (r.ws_bytes // 4) * 4].view(torch.int32).cpu().numpy()
    k = min(16, n)
    cand = np.flatnonzero(words[: words.size - n + 1] == inst[0])
    for c in cand:
        if np.array_equal(words[c:c + k], inst[:k]) and np.array_equal(words[c:c + n], inst):
            return int(c)
    raise AssertionError("instance list not found in the workspace")


def test_checked_mode_reports_an_out_of_range_record_id():
    """A record id outside the problem in a tile list (planted on the host
    into the workspace) is clamped in every mode; with UBS_FLAG_CHECKED the
    forward also reports it as UBS_ERR_INTERNAL.  On a consistent workspace
    the checked mode renders the same image and reports nothing."""
    scenes, views = _case(3, 90)
    dev = [raster.DeviceScene.from_scene(s) for s in scenes]
    r = raster.Rasterizer(dev, views, S.RasterConfig())
    img = r.forward(check=True).clone()
    st = r.status()
    n = int(st.instances)
    assert st.status == U.UBS_OK and n > 100
    r.problem.cfg.flags |= U.UBS_FLAG_CHECKED
    img_checked = r.forward(check=False).clone()
    assert r.status().status == U.UBS_OK
    assert torch.equal(img_checked, img)
    off = _instance_offset(r, n)
    base = (r.ws_ptr - r._ws.data_ptr()) // 4
    ws32 = r._ws.view(torch.int32)
    ws32[base + off + n // 2] = r.R + 5  # an id past the last record
    r.render_fwd()
    assert r.status().status == U.UBS_ERR_INTERNAL
    # unchecked: clamped, nothing reported
    r.problem.cfg.flags &= ~U.UBS_FLAG_CHECKED
    r.preprocess()
    r.bin_sort()
    ws32[base + off + n // 2] = r.R + 5
    r.render_fwd()
    assert r.status().status == U.UBS_OK


def test_binning_twice_after_one_preprocess():
    """ubs_bin_sort reads what ubs_preprocess wrote and leaves its own
    counters as it found them: a second call on the same workspace gives the
    same lists, ranges, visible records and instances, and the same image."""
    scenes, views = _case(3, 91)
    dev = [raster.DeviceScene.from_scene(s) for s in scenes]
    r = raster.Rasterizer(dev, views, S.RasterConfig())
    img = r.forward(check=True).clone()
    st1 = r.status()
    n = int(st1.instances)
    inst1 = r.export(U.EXPORT_INSTANCES)[:n].clone()
    tstart1 = r.export(U.EXPORT_TILE_START).clone()
    for _ in range(2):
        r.bin_sort()
        st2 = r.status()
        assert st2.status == U.UBS_OK
        assert (st2.visible_records, st2.instances) == (st1.visible_records, st1.instances)
        assert torch.equal(r.export(U.EXPORT_INSTANCES)[:n], inst1)
        assert torch.equal(r.export(U.EXPORT_TILE_START), tstart1)
    assert torch.equal(r.render_fwd().clone(), img)
