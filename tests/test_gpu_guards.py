"""Out-of-bounds writes: every caller-owned device buffer of the C-ABI calls
(workspace, images, dL/dimage, gradients, the loss and relocation
workspaces, the optimiser's raw/m/v planes) is placed between guard regions
of a fixed byte pattern; after the whole path and a training step the guards
must be untouched.  (The device-side sanitizer is not available where these
tests run; this checks every byte the kernels could reach past an end.)"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2510_03312_gb300 import scenes as S

pytestmark = pytest.mark.gpu

PAD = 1 << 16  # bytes of guard on each side
PATTERN = 0xA5


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_03312_gb300 import build as B
    B.build()
    return torch.device("cuda", 0)


class Guarded:
    """A device allocation with PAD guard bytes before and after a 256-byte
    aligned payload of n bytes."""

    def __init__(self, n, dev):
        self.buf = torch.full((n + 2 * PAD + 256,), PATTERN, dtype=torch.uint8, device=dev)
        base = self.buf.data_ptr()
        self.off = ((base + PAD + 255) // 256 * 256) - base
        self.n = n

    def ptr(self):
        return self.buf.data_ptr() + self.off

    def floats(self, shape):
        count = int(np.prod(shape))
        assert count * 4 <= self.n
        t = self.buf[self.off:self.off + 4 * count].view(torch.float32).view(*shape)
        return t

    def intact(self):
        b = self.buf.cpu().numpy()
        return bool((b[:self.off] == PATTERN).all() and (b[self.off + self.n:] == PATTERN).all())


def _run_path(dev, scenes, views, cfg, guards):
    from paper_2510_03312_gb300 import raster
    from paper_2510_03312_gb300 import ubs as U
    ds = [raster.DeviceScene.from_scene(s, device=dev) for s in scenes]
    gr = [Guarded(d.params.numel() * 4, dev) for d in ds]
    guards += gr
    r = raster.Rasterizer(ds, views, cfg, device=dev, grads=[g.floats(tuple(d.params.shape)) for g, d in zip(gr, ds)])
    r.forward(check=True)  # sizes the capacity; then swap in a guarded workspace
    need = U.ubs_workspace_size(r.problem)
    ws = Guarded(need, dev)
    guards.append(ws)
    r._ws, r.ws_ptr, r.ws_bytes = ws.buf, ws.ptr(), need
    img = Guarded(r.n_pix * 3 * 4, dev)
    guards.append(img)
    image = img.floats((r.n_pix * 3,))
    r.preprocess()
    r.bin_sort()
    r.render_fwd(image)
    assert int(r.status().status) == U.UBS_OK
    dl = Guarded(r.n_pix * 3 * 4, dev)
    guards.append(dl)
    dL = dl.floats((r.n_pix * 3,))
    dL.copy_(torch.randn_like(dL) * 1e-6)
    r.render_bwd(dL)
    return r, image, dL


@pytest.mark.parametrize("case", ["static_small", "n6_3views_tile8", "mixed_scenes", "persistent", "split_lists",
                                  "split_lists_tile32"])
def test_rasterizer_writes_stay_in_bounds(dev, case):
    rng = np.random.default_rng(3)
    if case == "static_small":
        wl = S.workload_static_small(P=3000, size=100)
        scenes, views, cfg = wl.scenes, wl.views, wl.cfg
    elif case == "persistent":
        scenes = [S.make_scene(7, 6, 6000, means="clusters", extent=2.0, n_clusters=8, rng=rng)]
        views = S.sphere_views(rng, 3, 5.0, 121, 77, hemisphere=True)
        cfg = S.RasterConfig(persistent=True)
    elif case.startswith("split_lists"):
        # two deep tiles (about 14,000 entries: seven segments each) beside short ones
        scenes = [S.make_scene(65, 3, 24000, means="uniform", extent=0.04, scale_range=(0.01, 0.04))]
        R, t = S.look_at((0.0, 0.0, -3.0))
        views = [S.make_view(R, t, 96, 80)]
        tile = (32, 32) if case.endswith("tile32") else (16, 16)
        cfg = S.RasterConfig(split_lists=True, tile_w=tile[0], tile_h=tile[1])
    elif case == "n6_3views_tile8":
        scenes = [S.make_scene(4, 6, 6000, means="clusters", extent=2.0, n_clusters=8, rng=rng)]
        views = S.sphere_views(rng, 3, 5.0, 121, 77, hemisphere=True)
        cfg = S.RasterConfig(tile_w=8, tile_h=8)
    else:
        scenes = [S.make_scene(5, 3, 4000, means="clusters", extent=2.0, n_clusters=8, rng=rng),
                  S.make_scene(6, 7, 3000, means="clusters", extent=2.0, n_clusters=8, rng=rng)]
        views = S.sphere_views(rng, 2, 5.0, 97, 61, hemisphere=True, times=[0.2, 0.7])
        v2 = S.sphere_views(rng, 2, 5.0, 33, 130, hemisphere=True, times=[0.4, 0.9], scene_id=1)
        views = views + v2
        cfg = S.RasterConfig(tile_w=16, tile_h=32)
    guards = []
    _run_path(dev, scenes, views, cfg, guards)
    torch.cuda.synchronize()
    assert all(g.intact() for g in guards)


def test_training_calls_write_in_bounds(dev):
    from paper_2510_03312_gb300 import train as TR
    from paper_2510_03312_gb300 import ubs as U
    wl = S.workload_static_small(P=2000, size=90)
    guards = []
    r, image, dL = _run_path(dev, wl.scenes, wl.views, wl.cfg, guards)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    # image loss: guarded workspace, gradient and loss outputs
    w, h = [v.width for v in wl.views], [v.height for v in wl.views]
    n = U.ubs_loss_workspace_size(w, h)
    lws, lout, lg = Guarded(n, dev), Guarded(4 * (1 + len(w)), dev), Guarded(image.numel() * 4, dev)
    guards += [lws, lout, lg]
    target = torch.rand_like(image)
    st = U.ubs_image_loss(w, h, image.data_ptr(), target.data_ptr(), 0.2, lg.ptr(), lout.ptr(), lws.ptr(), n, stream)
    assert st == U.UBS_OK
    # Adam on guarded raw/act/grad/m/v planes (P not a multiple of 4: the scalar path)
    sc = S.make_scene(8, 6, 1003)
    K, P = sc.params.shape
    planes = TR.plane_table(6, sc.rot_mode, TR.TrainConfig())
    bufs = [Guarded(K * P * 4, dev) for _ in range(5)]
    guards += bufs
    for b in bufs[:3]:  # raw, act, grad
        b.floats((K, P)).copy_(torch.tensor(sc.params, device=dev))
    for b in bufs[3:]:  # m, v
        b.floats((K, P)).zero_()
    noise = Guarded(3 * P * 4, dev)
    guards.append(noise)
    noise.floats((3, P)).zero_()
    pl = (U.ubs_adam_plane * K)(*[U.ubs_adam_plane(lr, a, l1, row) for lr, a, l1, row in planes])
    cfg = U.ubs_adam_config(0.9, 0.999, 1e-15, 1, 1.0)
    st = U.ubs_adam_step(K, P, pl, cfg, bufs[0].ptr(), bufs[1].ptr(), bufs[2].ptr(), bufs[3].ptr(), bufs[4].ptr(),
                         noise.ptr(), stream)
    assert st == U.UBS_OK
    # relocation with a guarded workspace and outputs
    with torch.no_grad():
        op = bufs[1].floats((K, P))[sc.offsets()["opacity"][0]]
        op[::7] = 0.001
    mws = Guarded(U.ubs_mcmc_workspace_size(P), dev)
    src, nrel, rnd = Guarded(4 * P, dev), Guarded(8, dev), Guarded(8 * P, dev)
    guards += [mws, src, nrel, rnd]
    rnd.buf[rnd.off:rnd.off + 8 * P].view(torch.int64).copy_(torch.randint(0, 2 ** 62, (P,), device=dev))
    st = U.ubs_mcmc_relocate(K, P, sc.offsets()["opacity"][0], 0.005, bufs[1].ptr(), bufs[0].ptr(), bufs[3].ptr(),
                             bufs[4].ptr(), rnd.ptr(), src.ptr(), nrel.ptr(), mws.ptr(), mws.n, stream)
    assert st == U.UBS_OK
    torch.cuda.synchronize()
    assert int(nrel.buf[nrel.off:nrel.off + 8].view(torch.int64).item()) > 0
    assert all(g.intact() for g in guards)
