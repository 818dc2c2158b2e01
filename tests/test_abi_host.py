"""The C-ABI library loads on the host, exports every entry point that
include/ubs.h declares, and validates arguments without touching a GPU."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2510_03312_gb300 import build as B
from paper_2510_03312_gb300 import scenes as S
from paper_2510_03312_gb300 import ubs as U

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return U.load()


def _declared():
    text = open(os.path.join(ROOT, "include", "ubs.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ubs_[a-z_]+)\s*\(", text)))


def test_header_declares_the_path_entry_points():
    names = _declared()
    for n in ("ubs_preprocess", "ubs_bin_sort", "ubs_render_fwd", "ubs_render_bwd"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    names = _declared()
    assert names
    for n in names:
        assert hasattr(lib, n), n
        assert n in U.SIGNATURES, n


def test_status_strings(lib):
    for code in range(8):
        assert U.ubs_status_string(code)
    assert U.ubs_status_string(0) == "ok"


def _problem(scene_N=3, P=100, tile=(16, 16), views=1, cap=1000):
    sc = U.ubs_scene()
    sc.N, sc.rot_mode, sc.P = scene_N, 0, P
    fake = 0x10000  # never dereferenced by host-side validation
    for name in S.PLANE_ORDER:
        setattr(sc, name, fake)
    scs = (U.ubs_scene * 1)(sc)
    vs = (U.ubs_view * views)()
    for i in range(views):
        vs[i].fx = vs[i].fy = 100.0
        vs[i].width, vs[i].height = 130, 70
    pr = U.ubs_problem()
    pr.scenes, pr.n_scenes, pr.views, pr.n_views = scs, 1, vs, views
    pr.cfg.tile_w, pr.cfg.tile_h = tile
    pr.cfg.alpha_min, pr.cfg.alpha_max, pr.cfg.T_min = 1 / 255, 0.99, 1e-4
    pr.cfg.eps2d, pr.cfg.near_plane, pr.cfg.jac_clip = 0.3, 0.2, 1.3
    pr.instance_capacity = cap
    return pr, (scs, vs)


def test_workspace_size_is_host_arithmetic(lib):
    pr, keep = _problem()
    n1 = U.ubs_workspace_size(pr)
    assert n1 > 0 and n1 % 256 == 0
    pr.instance_capacity = 100000
    assert U.ubs_workspace_size(pr) > n1
    pr2, keep2 = _problem(views=3)
    assert U.ubs_workspace_size(pr2) > n1


@pytest.mark.parametrize("bad", ["N", "tile", "views", "cap", "scene_id", "size"])
def test_invalid_problems_are_rejected(lib, bad):
    pr, keep = _problem()
    if bad == "N":
        keep[0][0].N = 5
    elif bad == "tile":
        pr.cfg.tile_w = 12
    elif bad == "views":
        pr.n_views = 0
    elif bad == "cap":
        pr.instance_capacity = -1
    elif bad == "scene_id":
        keep[1][0].scene_id = 3
    elif bad == "size":
        keep[1][0].width = 0
    assert U.ubs_workspace_size(pr) == 0
    # the entry points reject it synchronously, before any CUDA call
    assert U.ubs_preprocess(pr, 0x100000, 1 << 30, None) == U.UBS_ERR_INVALID_ARG


def test_workspace_checks(lib):
    pr, keep = _problem()
    need = U.ubs_workspace_size(pr)
    assert U.ubs_preprocess(pr, None, need, None) == U.UBS_ERR_INVALID_ARG
    assert U.ubs_preprocess(pr, 0x100010, need, None) == U.UBS_ERR_ALIGNMENT
    assert U.ubs_bin_sort(pr, 0x100000, need - 256, None) == U.UBS_ERR_WORKSPACE
    keep[0][0].mean_x = 0x10002
    assert U.ubs_preprocess(pr, 0x100000, need, None) == U.UBS_ERR_ALIGNMENT


def test_loss_workspace_size_arithmetic(lib):
    # three partial planes per pixel and channel, then one float2 per 32x32 block of each channel
    w, h = [1600, 33], [1060, 17]
    pix = sum(a * b for a, b in zip(w, h))
    blocks = sum(3 * ((a + 31) // 32) * ((b + 31) // 32) for a, b in zip(w, h))
    want = ((9 * pix * 4 + 255) // 256) * 256 + ((blocks * 8 + 255) // 256) * 256
    assert U.ubs_loss_workspace_size(w, h) == want
    assert U.ubs_loss_workspace_size([], []) == 0
    assert U.ubs_loss_workspace_size([0], [10]) == 0
    assert U.ubs_loss_workspace_size([10] * 257, [10] * 257) == 0


def test_image_loss_rejects_bad_arguments_before_launching(lib):
    fake = 0x10000
    ws = U.ubs_loss_workspace_size([64], [48])
    ok = dict(widths=[64], heights=[48], image=fake, target=fake, lambda_ssim=0.2, dL_dimage=fake, loss=fake,
              workspace=fake, workspace_bytes=ws, stream=None)

    def call(**kw):
        a = dict(ok)
        a.update(kw)
        return U.ubs_image_loss(**a)

    assert call(image=None) == U.UBS_ERR_INVALID_ARG
    assert call(loss=None) == U.UBS_ERR_INVALID_ARG
    assert call(lambda_ssim=1.5) == U.UBS_ERR_INVALID_ARG
    assert call(widths=[0]) == U.UBS_ERR_INVALID_ARG
    assert call(workspace=fake + 16) == U.UBS_ERR_ALIGNMENT
    assert call(image=fake + 2) == U.UBS_ERR_ALIGNMENT
    assert call(workspace_bytes=ws - 1) == U.UBS_ERR_WORKSPACE


def test_adam_step_rejects_bad_arguments_before_launching(lib):
    fake = 0x10000
    K, P = 3, 40
    planes = (U.ubs_adam_plane * K)()
    for k in range(K):
        planes[k].lr, planes[k].activation, planes[k].noise_row = 1e-3, U.UBS_ACT_IDENTITY, -1
    cfg = U.ubs_adam_config(0.9, 0.999, 1e-15, 1, 1.0)
    bufs = [fake, fake + 0x1000, fake + 0x2000, fake + 0x3000, fake + 0x4000]

    def call(K=K, P=P, planes=planes, cfg=cfg, bufs=bufs, noise=None):
        return U.ubs_adam_step(K, P, planes, cfg, *bufs, noise, None)

    assert call(K=0) == U.UBS_ERR_INVALID_ARG
    assert call(K=65) == U.UBS_ERR_INVALID_ARG
    assert call(P=-1) == U.UBS_ERR_INVALID_ARG
    assert call(P=0) == U.UBS_OK  # nothing to do, nothing launched
    assert call(bufs=[fake, fake] + bufs[2:]) == U.UBS_ERR_INVALID_ARG  # act_out aliases raw
    assert call(bufs=[None] + bufs[1:]) == U.UBS_ERR_INVALID_ARG
    assert call(bufs=[fake + 2] + bufs[1:]) == U.UBS_ERR_ALIGNMENT
    bad = U.ubs_adam_config(0.9, 0.999, 1e-15, 0, 1.0)
    assert call(cfg=bad) == U.UBS_ERR_INVALID_ARG
    planes[1].activation = 7
    assert call() == U.UBS_ERR_INVALID_ARG
    planes[1].activation = U.UBS_ACT_SIGMOID
    planes[0].noise_row = 0
    assert call(noise=None) == U.UBS_ERR_INVALID_ARG


def test_mcmc_workspace_and_argument_checks(lib):
    P = 5000
    nb = (P + 1023) // 1024
    want = 256 + ((P * 8 + 255) // 256) * 256 + ((nb * 8 + 255) // 256) * 256 + 2 * ((P * 4 + 255) // 256) * 256
    assert U.ubs_mcmc_workspace_size(P) == want
    assert U.ubs_mcmc_workspace_size(0) == 0
    fake = 0x10000
    ws = U.ubs_mcmc_workspace_size(P)
    ok = dict(K=15, P=P, opacity_row=13, dead_threshold=0.005, act=fake, raw=fake + 0x1000, m=fake + 0x2000,
              v=fake + 0x3000, rand=fake + 0x4000, sources=None, n_relocated=None, workspace=fake,
              workspace_bytes=ws, stream=None)

    def call(**kw):
        a = dict(ok)
        a.update(kw)
        return U.ubs_mcmc_relocate(**a)

    assert call(K=0) == U.UBS_ERR_INVALID_ARG
    assert call(opacity_row=15) == U.UBS_ERR_INVALID_ARG
    assert call(dead_threshold=1.0) == U.UBS_ERR_INVALID_ARG
    assert call(rand=None) == U.UBS_ERR_INVALID_ARG
    assert call(rand=fake + 4) == U.UBS_ERR_ALIGNMENT
    assert call(workspace=fake + 64) == U.UBS_ERR_ALIGNMENT
    assert call(workspace_bytes=ws - 1) == U.UBS_ERR_WORKSPACE
