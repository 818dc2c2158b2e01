"""The training step around the rasterizer (Sec. 4.5 loss, Sec. 5.1 optimiser,
Sec. 4.5 primitive management), as PyTorch plumbing over the C-ABI calls
``ubs_image_loss``, ``ubs_adam_step`` and ``ubs_mcmc_relocate``: device
buffers, the per-plane optimiser table and the order of the calls.  All
arithmetic runs in libubs.so.

The optimiser keeps raw parameters; the rasterizer reads the activated ones
(``DeviceScene.params``): opacity = sigmoid(raw), spatial scales and the
diagonal of L_q = exp(raw), everything else the identity.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import numpy as np
import torch

from . import scenes as S
from . import ubs as U
from .raster import check_tensor, overlaps

LAMBDA_SSIM = 0.2  # not stated in the paper; the value of 3DGS, whose loss this extends


@dataclass
class TrainConfig:
    """Sec. 5.1 learning rates and Sec. 4.5 weights."""
    lr_position: float = 1.6e-4
    lr_opacity: float = 5e-2
    lr_scale: float = 5e-3
    lr_other: float = 1e-3
    lambda_o: float = 0.01
    lambda_sigma: float = 0.01
    lambda_eps: float = 1.0
    lambda_ssim: float = LAMBDA_SSIM
    beta1: float = 0.9
    beta2: float = 0.999
    eps: float = 1e-15


def plane_table(N: int, rot_mode: int, tc: TrainConfig):
    """(lr, activation, l1 weight, noise row) of every plane of a scene, in
    the plane order of ``scenes.PLANE_ORDER``."""
    rows = S.plane_rows(N, rot_mode)
    C = N - 3
    out = []
    for name in S.PLANE_ORDER:
        for r in range(rows[name]):
            if name == "mean_x":
                out.append((tc.lr_position, U.UBS_ACT_IDENTITY, 0.0, r))
            elif name == "scale_x":
                out.append((tc.lr_scale, U.UBS_ACT_EXP, tc.lambda_sigma, -1))
            elif name == "L_q":
                diag = {i * (i + 1) // 2 + i for i in range(C)}
                if r in diag:  # the query scales s_q
                    out.append((tc.lr_scale, U.UBS_ACT_EXP, 0.0, -1))
                else:
                    out.append((tc.lr_other, U.UBS_ACT_IDENTITY, 0.0, -1))
            elif name == "opacity":
                out.append((tc.lr_opacity, U.UBS_ACT_SIGMOID, tc.lambda_o, -1))
            else:
                out.append((tc.lr_other, U.UBS_ACT_IDENTITY, 0.0, -1))
    return out


def raw_from_activated(act: torch.Tensor, table) -> torch.Tensor:
    """Inverse activations (logit, log) to start the optimiser from a scene."""
    raw = act.clone()
    for k, (_, a, _, _) in enumerate(table):
        if a == U.UBS_ACT_SIGMOID:
            raw[k] = torch.logit(act[k].clamp(1e-6, 1 - 1e-6))
        elif a == U.UBS_ACT_EXP:
            raw[k] = torch.log(act[k])
    return raw


class ImageLoss:
    """ubs_image_loss over the packed images of a list of views."""

    def __init__(self, views, device="cuda", lambda_ssim: float = LAMBDA_SSIM):
        self.widths = [int(v.width) for v in views]
        self.heights = [int(v.height) for v in views]
        self.lam = float(lambda_ssim)
        self.device = torch.device(device)
        if self.device.type != "cuda":
            raise ValueError("ImageLoss runs on a CUDA device")
        n = U.ubs_loss_workspace_size(self.widths, self.heights)
        if n == 0:
            raise ValueError("invalid view sizes for ubs_image_loss")
        self._ws = torch.empty(n + 256, dtype=torch.uint8, device=self.device)
        self.ws_ptr = (self._ws.data_ptr() + 255) // 256 * 256
        self.ws_bytes = n
        self.loss = torch.zeros(1 + len(views), dtype=torch.float32, device=self.device)
        self.numel = 3 * sum(w * h for w, h in zip(self.widths, self.heights))

    def __call__(self, image: torch.Tensor, target: torch.Tensor, dL: torch.Tensor) -> torch.Tensor:
        """Writes dL/dimage into ``dL``; returns the device tensor [total, per view]."""
        for t, name in ((image, "image"), (target, "target"), (dL, "dL")):
            check_tensor(t, name, self.device, numel=self.numel)
        if overlaps(dL, image) or overlaps(dL, target):
            raise ValueError("dL may not alias the image or the target")
        st = U.ubs_image_loss(self.widths, self.heights, image.data_ptr(), target.data_ptr(), self.lam,
                              dL.data_ptr(), self.loss.data_ptr(), self.ws_ptr, self.ws_bytes,
                              ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
        if st != U.UBS_OK:
            raise U.UBSError(st, "ubs_image_loss")
        return self.loss


class Adam:
    """ubs_adam_step over one scene's [K, P] parameter block.  ``act`` is the
    tensor the rasterizer reads (updated in place); raw, m and v are owned
    here."""

    def __init__(self, scene, act: torch.Tensor, tc: TrainConfig | None = None):
        self.tc = tc or TrainConfig()
        self.table = plane_table(scene.N, scene.rot_mode, self.tc)
        if act.dim() != 2:
            raise ValueError("act must be a [K, P] parameter block")
        K, P = act.shape
        check_tensor(act, "act", act.device, shape=(K, P))
        if K != len(self.table):
            raise ValueError("parameter block does not match the scene layout")
        self.K, self.P = K, P
        self.act = act
        self.raw = raw_from_activated(act.detach(), self.table).contiguous()
        self.m = torch.zeros_like(self.raw)
        self.v = torch.zeros_like(self.raw)
        self.step_count = 0
        self._planes = (U.ubs_adam_plane * K)()
        for k, (lr, a, l1, row) in enumerate(self.table):
            self._planes[k].lr, self._planes[k].activation = lr, a
            self._planes[k].l1_weight, self._planes[k].noise_row = l1, row

    def step(self, grad: torch.Tensor, noise: torch.Tensor | None = None):
        """One step with dL/d(activated params) ``grad``; ``noise`` [3, P] is the
        drawn eps of the spatial noise (None: no noise)."""
        if self.act.device.type != "cuda":
            raise ValueError("the optimiser's tensors must be on a CUDA device to step")
        check_tensor(grad, "grad", self.act.device, shape=(self.K, self.P))
        if noise is not None:
            check_tensor(noise, "noise", self.act.device, shape=(3, self.P))
        self.step_count += 1
        cfg = U.ubs_adam_config(self.tc.beta1, self.tc.beta2, self.tc.eps, self.step_count,
                                self.tc.lambda_eps if noise is not None else 0.0)
        planes = self._planes
        if noise is None:
            planes = (U.ubs_adam_plane * self.K)(*self._planes)
            for k in range(self.K):
                planes[k].noise_row = -1
        st = U.ubs_adam_step(self.K, self.P, planes, cfg, self.raw.data_ptr(), self.act.data_ptr(),
                             grad.data_ptr(), self.m.data_ptr(), self.v.data_ptr(),
                             noise.data_ptr() if noise is not None else None,
                             ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
        if st != U.UBS_OK:
            raise U.UBSError(st, "ubs_adam_step")


def save_checkpoint(path: str, opts, iteration: int = 0) -> None:
    """Writes the optimiser state of every scene (raw and activated
    parameters, Adam moments, step count) to one .npz file, from which
    training resumes where it stopped.  (Runs after a resume agree with an
    uninterrupted one to float rounding, not bit for bit: the backward
    blend's per-record sums are float atomics, whose order varies.)"""
    arrays = {"iteration": np.array(iteration, dtype=np.int64), "n_scenes": np.array(len(opts), dtype=np.int64)}
    for i, o in enumerate(opts):
        arrays[f"raw{i}"] = o.raw.detach().cpu().numpy()
        arrays[f"act{i}"] = o.act.detach().cpu().numpy()
        arrays[f"m{i}"] = o.m.detach().cpu().numpy()
        arrays[f"v{i}"] = o.v.detach().cpu().numpy()
        arrays[f"step{i}"] = np.array(o.step_count, dtype=np.int64)
    np.savez(path, **arrays)


def load_checkpoint(path: str, opts) -> int:
    """Restores what save_checkpoint wrote into optimisers of the same scene
    layouts (in place, on their devices); returns the saved iteration."""
    with np.load(path) as z:
        if int(z["n_scenes"]) != len(opts):
            raise ValueError("checkpoint holds a different number of scenes")
        for i, o in enumerate(opts):
            for name in ("raw", "act", "m", "v"):
                a = z[f"{name}{i}"]
                dst = getattr(o, name)
                if tuple(a.shape) != tuple(dst.shape):
                    raise ValueError(f"checkpoint {name}{i} has shape {a.shape}, expected {tuple(dst.shape)}")
                with torch.no_grad():
                    dst.copy_(torch.from_numpy(a))
            o.step_count = int(z[f"step{i}"])
        return int(z["iteration"])


DEAD_THRESHOLD = 0.005  # 3DGS-MCMC's dead opacity, on which the DBS scheme builds


class Relocator:
    """ubs_mcmc_relocate on an ``Adam``'s buffers (Sec. 4.5 primitive
    management): dead primitives move onto live ones drawn by opacity."""

    def __init__(self, opt: "Adam", threshold: float = DEAD_THRESHOLD):
        self.opt = opt
        self.threshold = float(threshold)
        rows = [k for k, (_, a, _, _) in enumerate(opt.table) if a == U.UBS_ACT_SIGMOID]
        if len(rows) != 1:
            raise ValueError("expected exactly one opacity plane")
        self.opacity_row = rows[0]
        n = U.ubs_mcmc_workspace_size(opt.P)
        self._ws = torch.empty(n + 256, dtype=torch.uint8, device=opt.act.device)
        self.ws_ptr = (self._ws.data_ptr() + 255) // 256 * 256
        self.ws_bytes = n
        self.sources = torch.empty(opt.P, dtype=torch.int32, device=opt.act.device)
        self.n_relocated = torch.zeros(1, dtype=torch.int64, device=opt.act.device)

    def __call__(self, rand: torch.Tensor):
        """rand: [P] int64 tensor of random bits (read as uint64)."""
        o = self.opt
        if o.act.device.type != "cuda":
            raise ValueError("the optimiser's tensors must be on a CUDA device to relocate")
        check_tensor(rand, "rand", o.act.device, dtype=torch.int64, shape=(o.P,))
        st = U.ubs_mcmc_relocate(o.K, o.P, self.opacity_row, self.threshold, o.act.data_ptr(), o.raw.data_ptr(),
                                 o.m.data_ptr(), o.v.data_ptr(), rand.data_ptr(), self.sources.data_ptr(),
                                 self.n_relocated.data_ptr(), self.ws_ptr, self.ws_bytes,
                                 ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
        if st != U.UBS_OK:
            raise U.UBSError(st, "ubs_mcmc_relocate")
        return self.sources, self.n_relocated


def train_step(r, loss_fn: ImageLoss, opts, target: torch.Tensor, dL: torch.Tensor, noises=None):
    """One training iteration on rasterizer ``r`` (all scenes): render, image
    loss and its gradient, backward, one Adam step per scene.  Returns the
    device loss tensor (no synchronisation)."""
    r.preprocess()
    r.bin_sort()
    img = r.render_fwd()
    loss = loss_fn(img, target, dL)
    r.render_bwd_blend(dL)
    grads = r.render_bwd_params()
    for i, (opt, g) in enumerate(zip(opts, grads)):
        opt.step(g, None if noises is None else noises[i])
    return loss
