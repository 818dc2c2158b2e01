"""GPU parity of the training step around the rasterizer (ubs_image_loss,
ubs_adam_step) against the float64 oracle, through the C-ABI."""
import numpy as np
import pytest
import torch

from oracle import train64 as T
from paper_2510_03312_gb300 import scenes as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_03312_gb300 import build as B
    B.build()
    return torch.device("cuda", 0)


class _V:
    def __init__(self, w, h):
        self.width, self.height = w, h


def _pack(ims, dev):
    return torch.cat([torch.as_tensor(a, dtype=torch.float32).reshape(-1) for a in ims]).to(dev)


def _unpack(flat, sizes):
    out, o = [], 0
    for w, h in sizes:
        out.append(flat[o:o + 3 * w * h].reshape(3, h, w))
        o += 3 * w * h
    return out


@pytest.mark.parametrize("sizes,lam", [
    ([(64, 48)], 0.2),
    ([(37, 23), (1, 1), (130, 70), (33, 17)], 0.2),  # ragged tiles, a 1x1 view, several views
    ([(96, 40)], 0.0),
    ([(45, 61)], 1.0),
])
def test_image_loss_matches_oracle(dev, sizes, lam):
    from paper_2510_03312_gb300 import train as TR
    rng = np.random.default_rng(len(sizes) * 10 + int(lam * 10))
    xs = [rng.random((3, h, w)).astype(np.float32) for w, h in sizes]
    ys = [np.clip(x + 0.15 * rng.standard_normal(x.shape), 0, 1).astype(np.float32) for x in xs]
    loss_fn = TR.ImageLoss([_V(w, h) for w, h in sizes], device=dev, lambda_ssim=lam)
    img, tgt = _pack(xs, dev), _pack(ys, dev)
    dL = torch.empty_like(img)
    out = loss_fn(img, tgt, dL).cpu().numpy()
    ref, per, grads = T.image_loss(xs, ys, lam)
    assert out[0] == pytest.approx(ref, rel=2e-5, abs=1e-7)
    assert np.allclose(out[1:], per, rtol=2e-5, atol=1e-7)
    got = _unpack(dL.cpu().numpy(), sizes)
    gmax = max(np.abs(g).max() for g in grads)
    for a, b in zip(got, grads):
        assert np.abs(a - b).max() <= 1e-4 * gmax + 1e-3 * np.abs(b).max()
    # deterministic: a second call gives the same bits
    dL2 = torch.empty_like(img)
    out2 = loss_fn(img, tgt, dL2).cpu().numpy()
    assert np.array_equal(out, out2) and torch.equal(dL, dL2)


def test_image_loss_of_identical_images_is_zero(dev):
    from paper_2510_03312_gb300 import train as TR
    rng = np.random.default_rng(3)
    x = rng.random((3, 50, 70)).astype(np.float32)
    loss_fn = TR.ImageLoss([_V(70, 50)], device=dev)
    img = _pack([x], dev)
    dL = torch.empty_like(img)
    out = loss_fn(img, img.clone(), dL).cpu().numpy()
    assert abs(out[0]) < 1e-6
    assert float(dL.abs().max()) < 1e-7


@pytest.mark.parametrize("P", [1000, 1001])  # the float4 path and the scalar path
def test_adam_step_matches_oracle(dev, P):
    from paper_2510_03312_gb300 import train as TR
    from paper_2510_03312_gb300 import ubs as U
    import ctypes
    rng = np.random.default_rng(P)
    scene = S.make_scene(7, 7, P)
    tc = TR.TrainConfig()
    table = TR.plane_table(7, scene.rot_mode, tc)
    K = len(table)
    raw = rng.standard_normal((K, P)).astype(np.float32) * 0.5
    m = (rng.standard_normal((K, P)) * 1e-3).astype(np.float32)
    v = (rng.random((K, P)) * 1e-5).astype(np.float32)
    noise = rng.standard_normal((3, P)).astype(np.float32) * 1e-3
    d = {k: torch.tensor(a, device=dev).contiguous() for k, a in dict(raw=raw, m=m, v=v, noise=noise).items()}
    act = torch.empty_like(d["raw"])
    planes = (U.ubs_adam_plane * K)()
    for k, (lr, a, l1, row) in enumerate(table):
        planes[k].lr, planes[k].activation, planes[k].l1_weight, planes[k].noise_row = lr, a, l1, row
    r_, m_, v_ = raw.astype(np.float64), m.astype(np.float64), v.astype(np.float64)
    for step in (1, 2, 3):
        g = (rng.standard_normal((K, P)) * 1e-2).astype(np.float32)
        gd = torch.tensor(g, device=dev)
        cfg = U.ubs_adam_config(tc.beta1, tc.beta2, tc.eps, step, tc.lambda_eps)
        st = U.ubs_adam_step(K, P, planes, cfg, d["raw"].data_ptr(), act.data_ptr(), gd.data_ptr(),
                             d["m"].data_ptr(), d["v"].data_ptr(), d["noise"].data_ptr(),
                             ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
        assert st == U.UBS_OK
        r_prev = r_
        r_, a_, m_, v_ = T.adam_step(r_, g, m_, v_, step, table, tc.beta1, tc.beta2, tc.eps, tc.lambda_eps, noise)
        got = d["raw"].cpu().numpy().astype(np.float64)
        # the update (not the raw value) is compared, relative to the plane's learning rate
        for k, (lr, *_rest) in enumerate(table):
            du_g, du_r = got[k] - r_prev[k], r_[k] - r_prev[k]
            assert np.abs(du_g - du_r).max() <= 1e-4 * lr + 2e-6 * np.abs(r_prev[k]).max(), k
        assert np.allclose(act.cpu().numpy(), a_, rtol=2e-5, atol=2e-6)
        assert np.allclose(d["m"].cpu().numpy(), m_, rtol=1e-4, atol=1e-9)
        assert np.allclose(d["v"].cpu().numpy(), v_, rtol=1e-4, atol=1e-12)
        r_ = got  # continue both from the GPU's raw values
        m_ = d["m"].cpu().numpy().astype(np.float64)
        v_ = d["v"].cpu().numpy().astype(np.float64)


def test_training_steps_reduce_the_loss(dev):
    """A few iterations of render -> loss -> backward -> Adam on a small scene
    fitted to a target rendered from the same scene with shifted colours."""
    from paper_2510_03312_gb300 import raster
    from paper_2510_03312_gb300 import train as TR
    wl = S.workload_static_small(P=2048, size=96)
    sc = wl.scenes[0]
    ds = raster.DeviceScene.from_scene(sc, device=dev)
    r = raster.Rasterizer([ds], wl.views, wl.cfg, device=dev)
    target = r.forward(check=True).clone()
    rows = sc.offsets()["rgb"]
    with torch.no_grad():
        ds.params[rows[0]:rows[0] + rows[1]] = torch.rand_like(ds.params[rows[0]:rows[0] + rows[1]])
    loss_fn = TR.ImageLoss(wl.views, device=dev)
    opt = TR.Adam(sc, ds.params, TR.TrainConfig(lr_other=2e-2))
    dL = torch.empty_like(target)
    losses = []
    for _ in range(30):
        losses.append(float(TR.train_step(r, loss_fn, [opt], target, dL)[0]))
    assert np.all(np.isfinite(losses))
    assert losses[-1] < 0.5 * losses[0]


def test_training_resumes_from_a_checkpoint(dev, tmp_path):
    """Three steps, a checkpoint, two more steps; a fresh trainer loaded from
    the checkpoint and run for the same two steps ends in the same state, to
    the rounding left by the backward blend's float atomics (the loaded
    state itself is bit-identical)."""
    from paper_2510_03312_gb300 import raster
    from paper_2510_03312_gb300 import train as TR
    wl = S.workload_static_small(P=1500, size=64)
    sc = wl.scenes[0]

    def trainer():
        ds = raster.DeviceScene.from_scene(sc, device=dev)
        r = raster.Rasterizer([ds], wl.views, wl.cfg, device=dev)
        r.forward(check=True)
        return ds, r, TR.Adam(sc, ds.params), TR.ImageLoss(wl.views, device=dev)

    target = torch.rand(3 * 64 * 64, device=dev)
    noise = torch.randn(3, sc.P, device=dev) * 1e-4
    ds, r, opt, lf = trainer()
    dL = torch.empty_like(target)
    for _ in range(3):
        TR.train_step(r, lf, [opt], target, dL, [noise])
    path = str(tmp_path / "ckpt.npz")
    TR.save_checkpoint(path, [opt], iteration=3)
    for _ in range(2):
        TR.train_step(r, lf, [opt], target, dL, [noise])
    torch.cuda.synchronize()
    ds2, r2, opt2, lf2 = trainer()
    assert TR.load_checkpoint(path, [opt2]) == 3
    with np.load(path) as z:
        assert np.array_equal(opt2.raw.cpu().numpy(), z["raw0"]) and opt2.step_count == 3
    for _ in range(2):
        TR.train_step(r2, lf2, [opt2], target, dL, [noise])
    torch.cuda.synchronize()
    for name in ("raw", "act", "m", "v"):
        a, b = getattr(opt, name), getattr(opt2, name)
        assert torch.allclose(a, b, rtol=1e-4, atol=1e-6), (name, float((a - b).abs().max()))


def test_binding_rejects_bad_tensors_before_launching(dev):
    """Host tensors, short buffers, other dtypes and an aliased gradient are
    refused by the binding; the device keeps working afterwards."""
    from paper_2510_03312_gb300 import raster
    from paper_2510_03312_gb300 import train as TR
    loss_fn = TR.ImageLoss([_V(16, 8)], device=dev)
    img = torch.rand(3 * 16 * 8, device=dev)
    tgt, dL = torch.rand_like(img), torch.empty_like(img)
    for args in ((img.cpu(), tgt, dL), (img[:-1], tgt[:-1], dL[:-1]), (img, tgt, img), (img.double(), tgt, dL)):
        with pytest.raises(ValueError):
            loss_fn(*args)
    wl = S.workload_static_small(P=500, size=32)
    ds = raster.DeviceScene.from_scene(wl.scenes[0], device=dev)
    r = raster.Rasterizer([ds], wl.views, wl.cfg, device=dev)
    r.forward(check=True)
    with pytest.raises(ValueError):
        r.render_fwd(torch.empty(10, device=dev))
    with pytest.raises(ValueError):
        r.render_bwd_blend(torch.empty(3 * r.n_pix))
    with pytest.raises(ValueError):
        r.render_bwd(torch.empty(3 * r.n_pix, device=dev, dtype=torch.float64))
    opt = TR.Adam(wl.scenes[0], ds.params)
    with pytest.raises(ValueError):
        opt.step(torch.zeros(opt.K, opt.P + 1, device=dev))
    out = loss_fn(img, tgt, dL)
    torch.cuda.synchronize()
    assert torch.isfinite(out).all()
    ds.params = ds.params.clone()  # the problem still holds the old pointers
    with pytest.raises(ValueError, match="replaced"):
        r.preprocess()
