"""GPU test of ubs_render_fwd_static, the forward render that allocates
nothing (for callers that cannot allocate device memory while rendering).

It is compared, through the C-ABI, with the regular caller-workspace path
(ubs_preprocess -> ubs_bin_sort -> ubs_render_fwd) on the same problem, on
two calls in a row, so that the second call also shows the shared fixed
scratch is reset between calls.  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2510_03312_gb300 import raster
from paper_2510_03312_gb300 import scenes as S
from paper_2510_03312_gb300 import ubs as U

pytestmark = pytest.mark.gpu

TOL = 1e-4  # the image tolerance of the parity tests


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2510_03312_gb300 import build
    build.build()
    assert torch.cuda.is_available()


def _problem(seed, P, W, H, n_views):
    rng = np.random.default_rng(seed)
    sc = S.make_scene(seed, 6, P, means="clusters", extent=2.0, n_clusters=8, rng=rng)
    views = S.sphere_views(rng, n_views, 5.0, W, H, hemisphere=True, times=list(rng.uniform(0, 1, n_views)))
    ds = raster.DeviceScene.from_scene(sc)
    r = raster.Rasterizer([ds], views, S.RasterConfig())
    r.forward(check=True)  # sizes instance_capacity for this scene
    return r


def _static_render(r):
    img = torch.full_like(r.image, float("nan"))
    st = U.ubs_render_fwd_static(r.problem, img.data_ptr(), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == U.UBS_OK, U.ubs_status_string(st)
    torch.cuda.synchronize()
    return img


def test_static_scratch_matches_workspace_path_twice():
    a = _problem(70, 6000, 120, 90, 2)
    b = _problem(71, 9000, 96, 72, 3)
    ref_a = a.forward(check=False).clone()
    ref_b = b.forward(check=False).clone()
    torch.cuda.synchronize()
    # two calls in a row on different problems, then the first again
    for r, ref in ((a, ref_a), (b, ref_b), (a, ref_a)):
        out = _static_render(r)
        assert torch.isfinite(out).all()
        assert (out - ref).abs().max().item() <= TOL


def test_static_scratch_rejects_problems_larger_than_the_scratch():
    sc = S.make_scene(72, 3, 4000, means="uniform", extent=1.0)
    ds = raster.DeviceScene.from_scene(sc)
    R, t = S.look_at((0.0, 0.0, -3.0))
    r = raster.Rasterizer([ds], [S.make_view(R, t, 4096, 4096)], S.RasterConfig(), capacity=1 << 20)
    img = torch.zeros(3 * 4096 * 4096, dtype=torch.float32, device="cuda")
    st = U.ubs_render_fwd_static(r.problem, img.data_ptr(), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == U.UBS_ERR_WORKSPACE


def test_static_scratch_reports_a_capacity_overflow():
    """With an instance capacity too small for the scene the image is left as
    it was and the overflow, with the count needed, is read back from the
    fixed scratch; with the capacity restored the same call renders again."""
    r = _problem(73, 6000, 120, 90, 2)
    ref = r.forward(check=False).clone()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    need = int(r.status().instances)
    cap = r.problem.instance_capacity
    r.problem.instance_capacity = need // 4
    img = torch.full_like(r.image, float("nan"))
    assert U.ubs_render_fwd_static(r.problem, img.data_ptr(), stream) == U.UBS_OK
    st = U.ubs_read_status_static(r.problem, stream)
    assert st.status == U.UBS_ERR_CAPACITY and st.instances == need
    assert torch.isnan(img).all()
    r.problem.instance_capacity = cap
    out = _static_render(r)
    st = U.ubs_read_status_static(r.problem, stream)
    assert st.status == U.UBS_OK and st.instances == need
    assert (out - ref).abs().max().item() <= TOL
