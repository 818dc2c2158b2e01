"""PyTorch plumbing around the C-ABI: device buffers, streams, autograd.

PyTorch supplies device memory and the current CUDA stream; every step of the
rasterizer runs in ``libubs.so`` (see ``ubs.py``).  Nothing here computes any
part of the method.
"""
from __future__ import annotations

import ctypes
from dataclasses import replace

import numpy as np
import torch

from . import ubs as U
from .scenes import PLANE_ORDER, RasterConfig, Scene, View, plane_rows


def check_tensor(t, name: str, device: torch.device, dtype=torch.float32, shape=None, numel=None):
    """Raises unless ``t`` is a contiguous tensor of ``dtype`` on ``device``
    (type, and index when the device names one) with the given shape or
    element count.  The C-ABI takes bare pointers and sizes it cannot check
    against the allocation: a host pointer or a short buffer passed on would
    reach the kernels, so every tensor is checked here before its pointer is."""
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch.Tensor, not {type(t).__name__}")
    if t.device.type != device.type or (device.index is not None and t.device.index != device.index):
        raise ValueError(f"{name} is on {t.device}, expected {device}")
    if t.dtype != dtype:
        raise ValueError(f"{name} has dtype {t.dtype}, expected {dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} has shape {tuple(t.shape)}, expected {tuple(shape)}")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"{name} has {t.numel()} elements, expected {numel}")
    return t


def overlaps(a: torch.Tensor, b: torch.Tensor) -> bool:
    """Whether the memory of two contiguous tensors overlaps."""
    a0, b0 = a.data_ptr(), b.data_ptr()
    return a0 < b0 + b.numel() * b.element_size() and b0 < a0 + a.numel() * a.element_size()


def config_struct(cfg: RasterConfig) -> U.ubs_config:
    c = U.ubs_config()
    c.tile_w, c.tile_h = int(cfg.tile_w), int(cfg.tile_h)
    c.alpha_min, c.alpha_max, c.T_min = cfg.alpha_min, cfg.alpha_max, cfg.T_min
    c.eps2d, c.near_plane, c.jac_clip = cfg.eps2d, cfg.near, cfg.jac_clip
    c.bg[:] = [float(x) for x in cfg.bg]
    c.flags = ((U.UBS_FLAG_TIGHT_CUT if cfg.tight_cut else 0) | (U.UBS_FLAG_PERSISTENT if cfg.persistent else 0) |
               (U.UBS_FLAG_SPLIT_LISTS if cfg.split_lists else 0))
    return c


def view_struct(v: View) -> U.ubs_view:
    s = U.ubs_view()
    s.R[:] = [float(x) for x in np.asarray(v.R, np.float32).ravel()]
    s.t[:] = [float(x) for x in np.asarray(v.t, np.float32).ravel()]
    s.fx, s.fy, s.cx, s.cy = v.fx, v.fy, v.cx, v.cy
    s.width, s.height, s.time, s.scene_id = v.width, v.height, v.time, v.scene_id
    return s


def _plane_ptrs(t: torch.Tensor, N: int, rot_mode: int):
    """Device pointers of the plane blocks of a contiguous [K, P] tensor."""
    P = t.shape[1]
    base = t.data_ptr()
    out, row = {}, 0
    for name, rows in plane_rows(N, rot_mode).items():
        out[name] = base + row * P * 4 if rows > 0 else None
        row += rows
    return out


class DeviceScene:
    """One primitive set on the GPU: ``params`` is a contiguous float32
    [K, P] tensor with the plane order of ``scenes.PLANE_ORDER``."""

    def __init__(self, N: int, rot_mode: int, params: torch.Tensor):
        if params.dtype != torch.float32 or not params.is_cuda or not params.is_contiguous():
            raise ValueError("params must be a contiguous float32 CUDA tensor")
        self.N, self.rot_mode, self.params = N, rot_mode, params

    @classmethod
    def from_scene(cls, sc: Scene, device="cuda") -> "DeviceScene":
        t = torch.from_numpy(np.ascontiguousarray(sc.params)).to(device)
        return cls(sc.N, sc.rot_mode, t)

    @property
    def P(self) -> int:
        return int(self.params.shape[1])

    def struct(self) -> U.ubs_scene:
        p = _plane_ptrs(self.params, self.N, self.rot_mode)
        s = U.ubs_scene()
        s.N, s.rot_mode, s.P = self.N, self.rot_mode, self.P
        for name in PLANE_ORDER:
            setattr(s, name, p[name])
        return s

    def grad_struct(self, g: torch.Tensor) -> U.ubs_scene_grad:
        p = _plane_ptrs(g, self.N, self.rot_mode)
        s = U.ubs_scene_grad()
        for name in PLANE_ORDER:
            setattr(s, name, p[name])
        return s


class Rasterizer:
    """One problem (scenes, views, config) with its workspace and outputs.

    ``forward`` runs preprocess -> bin_sort -> render_fwd on the current
    stream and returns the packed images (views in order, each [3, H, W]);
    ``backward`` runs render_bwd and returns one gradient tensor per scene,
    shaped like the scene's params.
    """

    def __init__(self, scenes, views, cfg: RasterConfig, capacity: int | None = None, device="cuda",
                 grads=None, accumulate: bool = False):
        """``grads``: optional gradient tensors (one per scene, shaped like its
        params) to write into instead of fresh ones; with ``accumulate`` the
        backward adds to them (UBS_FLAG_ACCUMULATE_GRADS)."""
        self.scenes = list(scenes)
        self.views = list(views)
        self.cfg = cfg
        self.device = torch.device(device)
        if self.device.type != "cuda":
            raise ValueError("the rasterizer runs on a CUDA device")
        for s in self.scenes:
            check_tensor(s.params, "scene params", self.device, shape=s.params.shape)
        self._scene_structs = (U.ubs_scene * len(self.scenes))(*[s.struct() for s in self.scenes])
        self._param_ptrs = [s.params.data_ptr() for s in self.scenes]
        self._view_structs = (U.ubs_view * len(self.views))(*[view_struct(v) for v in self.views])
        self.problem = U.ubs_problem()
        self.problem.scenes = self._scene_structs
        self.problem.n_scenes = len(self.scenes)
        self.problem.views = self._view_structs
        self.problem.n_views = len(self.views)
        self.problem.cfg = config_struct(cfg)
        if accumulate:
            self.problem.cfg.flags |= U.UBS_FLAG_ACCUMULATE_GRADS
        self.R = sum(self.scenes[v.scene_id].P for v in self.views)
        self.pix_off = np.cumsum([0] + [v.width * v.height for v in self.views])
        self.n_pix = int(self.pix_off[-1])
        self._ws = None
        self.ws_ptr, self.ws_bytes = None, 0
        self.set_capacity(capacity if capacity is not None else max(4 * self.R, 1 << 16))
        self.image = torch.empty(3 * self.n_pix, dtype=torch.float32, device=self.device)
        if grads is None:
            self.grads = [torch.empty_like(s.params) for s in self.scenes]
        else:
            self.grads = list(grads)
            if len(self.grads) != len(self.scenes):
                raise ValueError("one gradient tensor per scene is required")
            for g, s in zip(self.grads, self.scenes):
                check_tensor(g, "gradient", self.device, shape=s.params.shape)
        self._grad_structs = (U.ubs_scene_grad * len(self.scenes))(
            *[s.grad_struct(g) for s, g in zip(self.scenes, self.grads)])

    # -- workspace
    def set_capacity(self, cap: int):
        cap = int(min(max(cap, 1), 0x7FFFFFFF))
        self.problem.instance_capacity = cap
        need = U.ubs_workspace_size(self.problem)
        if need == 0:
            raise ValueError("invalid problem (ubs_workspace_size returned 0)")
        if self._ws is None or self.ws_bytes < need or 2 * need < self.ws_bytes:  # grown, or far too big
            self._ws = None
            self._ws = torch.empty(need + 256, dtype=torch.uint8, device=self.device)
            base = self._ws.data_ptr()
            self.ws_ptr = (base + 255) // 256 * 256
            self.ws_bytes = need
        self.capacity = cap

    @staticmethod
    def stream():
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)

    def _check(self, st, where):
        if st != U.UBS_OK:
            raise U.UBSError(st, where)

    def status(self):
        return U.ubs_read_status(self.problem, self.ws_ptr, self.ws_bytes, self.stream())

    # -- steps
    def preprocess(self):
        # the problem holds the parameter pointers taken at construction
        if any(s.params.data_ptr() != p for s, p in zip(self.scenes, self._param_ptrs)):
            raise ValueError("a scene's params tensor was replaced after the rasterizer was built "
                             "(update it in place, or build a new Rasterizer)")
        self._check(U.ubs_preprocess(self.problem, self.ws_ptr, self.ws_bytes, self.stream()), "ubs_preprocess")

    def bin_sort(self):
        self._check(U.ubs_bin_sort(self.problem, self.ws_ptr, self.ws_bytes, self.stream()), "ubs_bin_sort")

    def render_fwd(self, image=None):
        if image is None:
            image = self.image
        else:
            check_tensor(image, "image", self.device, numel=3 * self.n_pix)
        self._check(U.ubs_render_fwd(self.problem, self.ws_ptr, self.ws_bytes, image.data_ptr(), self.stream()),
                    "ubs_render_fwd")
        return image

    def render_bwd(self, dL_dimage: torch.Tensor):
        dL = check_tensor(dL_dimage.contiguous(), "dL_dimage", self.device, numel=3 * self.n_pix)
        self._check(U.ubs_render_bwd(self.problem, self.ws_ptr, self.ws_bytes, dL.data_ptr(), self._grad_structs,
                                     self.stream()), "ubs_render_bwd")
        return self.grads

    def render_bwd_blend(self, dL_dimage: torch.Tensor):
        check_tensor(dL_dimage, "dL_dimage", self.device, numel=3 * self.n_pix)
        self._check(U.ubs_render_bwd_blend(self.problem, self.ws_ptr, self.ws_bytes, dL_dimage.data_ptr(),
                                           self.stream()), "ubs_render_bwd_blend")

    def render_bwd_params(self):
        self._check(U.ubs_render_bwd_params(self.problem, self.ws_ptr, self.ws_bytes, self._grad_structs,
                                            self.stream()), "ubs_render_bwd_params")
        return self.grads

    def forward(self, check: bool = True, image=None):
        """Full forward.  With ``check`` the call synchronises once to read the
        device status and fits the instance capacity to the count found: it
        grows it when it was too small, and shrinks it when it is more than
        four times the count (the capacity sizes the instance buffers and the
        per-pass counts), then runs preprocess/bin_sort again.  Later calls
        without ``check`` (and captured graphs) keep the capacity."""
        self.preprocess()
        self.bin_sort()
        if check:
            st = self.status()
            need = int(st.instances)
            refit = st.status == U.UBS_ERR_CAPACITY or (st.status == U.UBS_OK and self.capacity > 4 * need + (1 << 16))
            if refit:
                self.set_capacity(int(need * 1.25) + (1 << 16))
                self.preprocess()
                self.bin_sort()
                st = self.status()
            if st.status != U.UBS_OK:
                raise U.UBSError(st.status, "device status")
        return self.render_fwd(image)

    def backward(self, dL_dimage):
        return self.render_bwd(dL_dimage)

    def capture(self, dL_dimage: torch.Tensor) -> torch.cuda.CUDAGraph:
        """Captures one forward+backward step (preprocess, bin_sort,
        render_fwd, render_bwd) into a CUDA graph; ``graph.replay()`` re-runs
        it on the current tensors (params, dL_dimage, image, grads).  Size the
        instance capacity first (``forward(check=True)``): a replay cannot
        grow it, and an overflow shows up in ``status()``."""
        return capture_steps([(self, dL_dimage)], self.device)

    # -- helpers
    def n_tiles(self) -> int:
        tw, th = int(self.cfg.tile_w), int(self.cfg.tile_h)
        return sum(((v.width + tw - 1) // tw) * ((v.height + th - 1) // th) for v in self.views)

    def view_image(self, flat: torch.Tensor, v: int) -> torch.Tensor:
        w = self.views[v]
        o = int(self.pix_off[v]) * 3
        return flat[o:o + 3 * w.height * w.width].view(3, w.height, w.width)

    def pack(self, images) -> torch.Tensor:
        return torch.cat([torch.as_tensor(im, dtype=torch.float32).reshape(-1) for im in images]).to(self.device)

    def export(self, what: int, dtype=torch.int32, count=None):
        st, need = U.ubs_export(self.problem, self.ws_ptr, self.ws_bytes, what, None, 0, self.stream())
        self._check(st, "ubs_export")
        out = torch.empty(need, dtype=torch.uint8, device=self.device)
        st, _ = U.ubs_export(self.problem, self.ws_ptr, self.ws_bytes, what, out.data_ptr(), need, self.stream())
        self._check(st, "ubs_export")
        return out.view(dtype)


def count_pairs(scenes, views, cfg: RasterConfig, device="cuda"):
    """Per-pixel diagnostic counts of the forward blend, from its counting
    variant (UBS_FLAG_COUNT_PAIRS), as int64 tensors over the packed pixels:

    * ``pairs``: (pixel, record) pairs with r < 1 visited before the pixel
      terminates, counted on lists built without the tight cut, so that
      every record whose support ellipse holds the pixel is on its tile's
      list: the tile-independent pair count;
    * ``visited``: the entries each pixel's warp evaluated in the forward
      with the configuration's own lists (those its support cull keeps,
      walked until the warp's pixels are all done), whether or not the
      pixel was still blending.

    Each count comes from its own problem; neither changes an image."""
    out = {}
    for key, c, what in (("pairs", replace(cfg, tight_cut=False), U.EXPORT_PAIRS),
                         ("visited", cfg, U.EXPORT_VISITED)):
        r = Rasterizer(scenes, views, c, device=device)
        r.problem.cfg.flags |= U.UBS_FLAG_COUNT_PAIRS
        r.forward(check=True)
        out[key] = r.export(what).to(torch.int64)
        del r
    return out


def capture_steps(steps, device) -> torch.cuda.CUDAGraph:
    """One CUDA graph of forward+backward over several (rasterizer, dL)
    pairs, issued in order on one stream."""
    def run():
        for r, dL in steps:
            r.forward(check=False)
            r.backward(dL)

    side = torch.cuda.Stream(device=device)
    side.wait_stream(torch.cuda.current_stream(device))
    with torch.cuda.stream(side):
        run()  # warm-up outside the capture
    torch.cuda.current_stream(device).wait_stream(side)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        run()
    return g


class Batch:
    """A batch of render jobs over several scenes, run as the launches
    (``groups``: lists of view indices) of a schedule.  Each launch is one
    problem over the scenes its views use; every launch adds its gradients
    into one buffer per scene, zeroed at the start of a step, so a scene's
    gradient is the sum over all of its views whichever launch rendered
    them.  Images are returned per view, in the original view order."""

    def __init__(self, scenes, views, cfg: RasterConfig, groups, device="cuda"):
        self.scenes = list(scenes)
        self.views = list(views)
        self.cfg = cfg
        self.device = torch.device(device)
        self.groups = [list(g) for g in groups]
        seen = sorted(i for g in self.groups for i in g)
        if seen != list(range(len(self.views))):
            raise ValueError("groups must partition the views")
        self.grads = [torch.zeros_like(s.params) for s in self.scenes]
        self.rasterizers, self.slot = [], {}
        for gi, g in enumerate(self.groups):
            used = sorted({self.views[i].scene_id for i in g})
            local = {s: k for k, s in enumerate(used)}
            lv = [replace(self.views[i], scene_id=local[self.views[i].scene_id]) for i in g]
            r = Rasterizer([self.scenes[s] for s in used], lv, cfg, device=self.device,
                           grads=[self.grads[s] for s in used], accumulate=True)
            self.rasterizers.append(r)
            for k, i in enumerate(g):
                self.slot[i] = (gi, k)

    @property
    def n_pix(self) -> int:
        return sum(v.width * v.height for v in self.views)

    def size(self):
        """Runs every launch's forward once with the status check, growing
        instance capacities where needed (synchronises)."""
        for r in self.rasterizers:
            r.forward(check=True)

    def dL_like(self, fill=None):
        """One dL/dimage tensor per launch (packed like its images)."""
        return [torch.full_like(r.image, fill) if fill is not None else torch.zeros_like(r.image)
                for r in self.rasterizers]

    def zero_grads(self):
        for g in self.grads:
            g.zero_()

    def step(self, dLs):
        """Forward+backward of every launch (no synchronisation)."""
        self.zero_grads()
        for r, d in zip(self.rasterizers, dLs):
            r.forward(check=False)
            r.backward(d)
        return self.grads

    def capture(self, dLs) -> torch.cuda.CUDAGraph:
        """The whole step (gradient zeroing and every launch) as one CUDA graph."""
        side = torch.cuda.Stream(device=self.device)
        side.wait_stream(torch.cuda.current_stream(self.device))
        with torch.cuda.stream(side):
            self.step(dLs)
        torch.cuda.current_stream(self.device).wait_stream(side)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            self.step(dLs)
        return g

    def image(self, i: int) -> torch.Tensor:
        gi, k = self.slot[i]
        r = self.rasterizers[gi]
        return r.view_image(r.image, k)

    def status(self):
        return [r.status() for r in self.rasterizers]


class UBSRasterize(torch.autograd.Function):
    """Differentiable rendering of one problem.  ``params`` are the scenes'
    [K, P] tensors the rasterizer was built on; the output is the packed
    images.  The backward is the hand-written CUDA backward (render_bwd)."""

    @staticmethod
    def forward(ctx, rasterizer: Rasterizer, *params):
        for p, s in zip(params, rasterizer.scenes):
            if p.data_ptr() != s.params.data_ptr():
                raise ValueError("params must be the tensors the rasterizer was built on")
        ctx.rasterizer = rasterizer
        return rasterizer.forward(image=torch.empty_like(rasterizer.image))

    @staticmethod
    def backward(ctx, dimg):
        grads = ctx.rasterizer.backward(dimg.contiguous())
        return (None, *[g.clone() for g in grads])


def rasterize(rasterizer: Rasterizer, *params):
    return UBSRasterize.apply(rasterizer, *params)
