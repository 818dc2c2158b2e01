"""Seeded synthetic scenes and cameras for the Universal Beta Splatting rasterizer.

This module only draws inputs: primitive parameters (Sec. 4.1-4.3 name them:
spatial mean, query mean, rotation, spatial scales, cross-correlation block
L_qx, query block L_q, Beta parameters b, opacity, RGB) and pinhole cameras.
It holds none of the method's arithmetic (no covariance construction,
conditioning, projection or compositing), so the CUDA path and the CPU oracle
can both consume its arrays without sharing any computation.

Layout (all float32, structure of arrays, one plane per scalar, stride P):

    plane block   rows                  meaning
    mean_x        3                     spatial mean mu_x
    mean_q        C                     query mean mu_q, order q = [t, d] (N=7),
                                        [d] (N=6), [t] (N=4)
    rot           4 (quat) / 3 (skew)   quaternion (w, x, y, z), not normalised,
                                        or omega of the skew matrix A(omega)
                                        (first- or second-order Taylor, Cayley,
                                        matrix exponential),
                                        or the strictly-lower entries
                                        (l10, l20, l21) of a Cholesky factor
    scale_x       3                     spatial scales s_x > 0
    L_qx          3C                    C x 3 block, row-major (k, j) -> 3k + j
    L_q           C(C+1)/2              lower-triangular block, packed row-major
                                        (i, j<=i) -> i(i+1)/2 + j; diagonal s_q > 0
    b             1 + C                 b_x, b_q1 .. b_qC
    opacity       1                     o in (0, 1)
    rgb           3                     colour in [0, 1]

With the skew rotation this is 35 floats for N=6 and 44 for N=7, the counts of
the paper's per-primitive parameter table; the quaternion mode adds one.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

ROT_QUAT = 0
ROT_SKEW1 = 1   # R = I + A(omega), the paper's first-order Taylor
ROT_SKEW2 = 2   # R = I + A + A^2 / 2, second-order Taylor
ROT_CAYLEY = 3  # R = (I - A)^-1 (I + A), the Cayley transform
ROT_CHOL = 4    # no rotation: the spatial block of L is a general lower-triangular
                # factor, rot = its strictly-lower entries (l10, l20, l21),
                # scale_x = its diagonal
ROT_EXP = 5     # R = exp(A), the matrix exponential
ROT_MODES = (ROT_QUAT, ROT_SKEW1, ROT_SKEW2, ROT_CAYLEY, ROT_CHOL, ROT_EXP)

PLANE_ORDER = ("mean_x", "mean_q", "rot", "scale_x", "L_qx", "L_q", "b", "opacity", "rgb")


def plane_rows(N: int, rot_mode: int) -> dict:
    """Rows of each plane block for an N-dimensional primitive."""
    C = N - 3
    return {
        "mean_x": 3,
        "mean_q": C,
        "rot": 4 if rot_mode == ROT_QUAT else 3,
        "scale_x": 3,
        "L_qx": 3 * C,
        "L_q": C * (C + 1) // 2,
        "b": 1 + C,
        "opacity": 1,
        "rgb": 3,
    }


def params_per_primitive(N: int, rot_mode: int) -> int:
    return sum(plane_rows(N, rot_mode).values())


@dataclass
class Scene:
    """One primitive set; ``params`` is the packed [K, P] float32 plane stack."""

    N: int
    rot_mode: int
    params: np.ndarray  # [K, P] float32, planes in PLANE_ORDER

    @property
    def P(self) -> int:
        return int(self.params.shape[1])

    @property
    def C(self) -> int:
        return self.N - 3

    def offsets(self) -> dict:
        out, o = {}, 0
        for name, rows in plane_rows(self.N, self.rot_mode).items():
            out[name] = (o, rows)
            o += rows
        return out

    def plane(self, name: str) -> np.ndarray:
        o, rows = self.offsets()[name]
        return self.params[o:o + rows]

    def subset(self, idx) -> "Scene":
        return Scene(self.N, self.rot_mode, np.ascontiguousarray(self.params[:, idx]))


@dataclass
class View:
    """Pinhole camera: x_cam = R x_world + t (x right, y down, z forward)."""

    R: np.ndarray  # [3, 3] float32, world -> camera
    t: np.ndarray  # [3] float32
    fx: float
    fy: float
    cx: float
    cy: float
    width: int
    height: int
    time: float = 0.0
    scene_id: int = 0


@dataclass
class RasterConfig:
    """Rasterizer constants the paper leaves to "standard splatting" (Sec. 4.5)."""

    tile_w: int = 16
    tile_h: int = 16
    alpha_min: float = 1.0 / 255.0
    alpha_max: float = 0.99
    T_min: float = 1e-4
    eps2d: float = 0.3
    near: float = 0.2
    bg: tuple = (0.0, 0.0, 0.0)
    tight_cut: bool = True
    jac_clip: float = 1.3
    persistent: bool = False   # launch form of the blend kernels (a schedule, not arithmetic)
    split_lists: bool = False  # blend long tile lists in segments (same result up to rounding)


# ----------------------------------------------------------------------------
# Parameter draws
# ----------------------------------------------------------------------------

def _log_uniform(rng, lo, hi, size):
    return np.exp(rng.uniform(math.log(lo), math.log(hi), size=size))


def _unit_vectors(rng, n):
    v = rng.standard_normal((3, n))
    return v / np.linalg.norm(v, axis=0, keepdims=True)


def make_scene(seed: int, N: int, P: int, *, means: str = "uniform", extent: float = 1.0,
               n_clusters: int = 64, cluster_sigma: float = 0.3, rot_mode: int = ROT_QUAT,
               scale_range=(0.01, 0.1), b_std: float = 0.5, ang_scale=(0.2, 2.0),
               time_scale=(0.02, 0.5), lqx_amp: float = 0.5, lq_amp: float = 0.25,
               rng: np.random.Generator | None = None) -> Scene:
    """Draw a seeded scene.  Parameter groups are drawn in a fixed order."""
    rng = np.random.default_rng(seed) if rng is None else rng
    C = N - 3
    if N not in (3, 4, 6, 7):
        raise ValueError("N must be 3, 4, 6 or 7")
    # spatial means
    if means == "uniform":
        mx = rng.uniform(-extent, extent, size=(3, P))
    elif means == "clusters":
        centres = rng.uniform(-extent, extent, size=(3, n_clusters))
        which = rng.integers(0, n_clusters, size=P)
        mx = centres[:, which] + cluster_sigma * rng.standard_normal((3, P))
    else:
        raise ValueError(means)
    sx = _log_uniform(rng, scale_range[0], scale_range[1], (3, P))
    if rot_mode == ROT_QUAT:
        q = rng.standard_normal((4, P))
        rot = q / np.linalg.norm(q, axis=0, keepdims=True)
    elif rot_mode == ROT_CHOL:
        # strictly-lower entries (l10, l20, l21) scaled by their row's diagonal
        rot = sx[[1, 2, 2]] * rng.uniform(-0.5, 0.5, size=(3, P))
    else:
        rot = rng.normal(0.0, 0.3, size=(3, P))
    op = 1.0 / (1.0 + np.exp(-rng.standard_normal(P)))
    b = rng.normal(0.0, b_std, size=(1 + C, P))
    rgb = rng.uniform(0.0, 1.0, size=(3, P))
    # query dimensions: q = [t, d] order
    has_t = C in (1, 4)
    has_d = C >= 3
    mq_rows, sq_rows = [], []
    if has_t:
        mq_rows.append(rng.uniform(0.0, 1.0, size=(1, P)))
        sq_rows.append(_log_uniform(rng, time_scale[0], time_scale[1], (1, P)))
    if has_d:
        mq_rows.append(_unit_vectors(rng, P))
        sq_rows.append(_log_uniform(rng, ang_scale[0], ang_scale[1], (3, P)))
    if C > 0:
        mq = np.concatenate(mq_rows, axis=0)
        sq = np.concatenate(sq_rows, axis=0)
        lqx = (sq[:, None, :] * rng.uniform(-lqx_amp, lqx_amp, size=(C, 3, P))).reshape(3 * C, P)
        lq_rows = []
        for i in range(C):
            for j in range(i + 1):
                if i == j:
                    lq_rows.append(sq[i])
                else:
                    lq_rows.append(sq[i] * rng.uniform(-lq_amp, lq_amp, size=P))
        lq = np.stack(lq_rows, axis=0)
    else:
        mq = np.zeros((0, P))
        lqx = np.zeros((0, P))
        lq = np.zeros((0, P))
    planes = {"mean_x": mx, "mean_q": mq, "rot": rot, "scale_x": sx, "L_qx": lqx, "L_q": lq,
              "b": b, "opacity": op[None], "rgb": rgb}
    params = np.concatenate([np.asarray(planes[k], dtype=np.float64).reshape(-1, P)
                             for k in PLANE_ORDER], axis=0).astype(np.float32)
    return Scene(N, rot_mode, np.ascontiguousarray(params))


# ----------------------------------------------------------------------------
# Cameras
# ----------------------------------------------------------------------------

def look_at(position, target=(0.0, 0.0, 0.0), up=(0.0, 1.0, 0.0)):
    """World->camera rotation and translation of a camera at ``position``
    looking at ``target`` (rows of R: camera x, y, z axes in world frame)."""
    p = np.asarray(position, dtype=np.float64)
    z = np.asarray(target, dtype=np.float64) - p
    z /= np.linalg.norm(z)
    u = np.asarray(up, dtype=np.float64)
    x = np.cross(u, z)
    if np.linalg.norm(x) < 1e-6:
        x = np.cross(np.array([0.0, 0.0, 1.0]), z)
    x /= np.linalg.norm(x)
    y = np.cross(z, x)
    R = np.stack([x, y, z], axis=0)
    t = -R @ p
    return R, t


def make_view(R, t, width, height, fov_x_deg=60.0, time=0.0, scene_id=0) -> View:
    f = (0.5 * width) / math.tan(math.radians(fov_x_deg) * 0.5)
    return View(R=np.asarray(R, np.float32), t=np.asarray(t, np.float32),
                fx=float(np.float32(f)), fy=float(np.float32(f)),
                cx=float(np.float32(0.5 * width)), cy=float(np.float32(0.5 * height)),
                width=int(width), height=int(height), time=float(np.float32(time)),
                scene_id=int(scene_id))


def sphere_views(rng, n, radius, width, height, hemisphere=False, times=None, scene_id=0):
    views = []
    for i in range(n):
        u = rng.standard_normal(3)
        u /= np.linalg.norm(u)
        if hemisphere:
            u[1] = abs(u[1])
        R, t = look_at(radius * u)
        tm = 0.0 if times is None else times[i]
        views.append(make_view(R, t, width, height, time=tm, scene_id=scene_id))
    return views


# ----------------------------------------------------------------------------
# The workloads (static, view-dependent, dynamic, uneven mix)
# ----------------------------------------------------------------------------

@dataclass
class Workload:
    name: str
    scenes: list
    views: list
    cfg: RasterConfig = field(default_factory=RasterConfig)
    forward_only: bool = False


def workload_static_small(seed: int = 0, P: int = 4096, size: int = 128) -> Workload:
    """Static N=3, 4,096 primitives in [-1,1]^3, one 128x128 60-degree camera
    at distance 3 looking at the origin (forward render)."""
    sc = make_scene(seed, 3, P, means="uniform", extent=1.0)
    R = np.eye(3)
    t = np.array([0.0, 0.0, 3.0])
    v = make_view(R, t, size, size)
    return Workload("static_n3_4k_128", [sc], [v], forward_only=True)


def workload_static_large(seed: int = 1, P: int = 1_000_000, width: int = 1600, height: int = 1060):
    """Static N=3, 1M primitives in a 64-cluster Gaussian mixture in [-5,5]^3,
    one 1600x1060 camera on a radius-8 sphere (forward+backward, L1 loss)."""
    rng = np.random.default_rng(seed)
    sc = make_scene(seed, 3, P, means="clusters", extent=5.0, rng=rng)
    views = sphere_views(rng, 1, 8.0, width, height)
    return Workload("static_n3_1m_1600x1060", [sc], views)


def workload_view_dependent(seed: int = 2, P: int = 500_000, n_views: int = 16,
                            width: int = 1280, height: int = 720):
    """View-dependent N=6, 500K primitives, 16 hemisphere cameras at 1280x720."""
    rng = np.random.default_rng(seed)
    sc = make_scene(seed, 6, P, means="clusters", extent=5.0, rng=rng)
    views = sphere_views(rng, n_views, 8.0, width, height, hemisphere=True)
    return Workload(f"viewdep_n6_500k_{n_views}x{width}x{height}", [sc], views)


def workload_dynamic(seed: int = 3, P: int = 300_000, n_views: int = 8,
                     width: int = 1352, height: int = 1014):
    """Dynamic N=7, 300K primitives, 8 (camera, time) queries at 1352x1014."""
    rng = np.random.default_rng(seed)
    sc = make_scene(seed, 7, P, means="clusters", extent=5.0, rng=rng)
    times = rng.uniform(0.0, 1.0, size=n_views)
    views = sphere_views(rng, n_views, 8.0, width, height, hemisphere=True, times=times)
    return Workload(f"dynamic_n7_300k_{n_views}x{width}x{height}", [sc], views)


def workload_uneven_mix(seed: int = 4, n_scenes: int = 8, n_jobs: int = 64,
                        p_range=(10_000, 2_000_000), w_range=(256, 1920), h_range=(256, 1080),
                        scale: float = 1.0):
    """Uneven batch: scenes with N in {3,6,7} and log-uniform primitive counts,
    jobs with log-uniform resolutions, each job a (scene, camera, time) query.
    ``scale`` shrinks primitive counts (for tests)."""
    rng = np.random.default_rng(seed)
    scenes = []
    for k in range(n_scenes):
        srng = np.random.default_rng(100 + k)
        N = int(srng.choice([3, 6, 7]))
        P = int(round(_log_uniform(srng, p_range[0], p_range[1], 1)[0] * scale))
        P = max(P, 1)
        scenes.append(make_scene(100 + k, N, P, means="clusters", extent=5.0, rng=srng))
    views = []
    for j in range(n_jobs):
        s = int(rng.integers(0, n_scenes))
        W = int(round(_log_uniform(rng, w_range[0], w_range[1], 1)[0]))
        H = int(round(_log_uniform(rng, h_range[0], h_range[1], 1)[0]))
        tm = float(rng.uniform(0.0, 1.0))
        u = rng.standard_normal(3)
        u /= np.linalg.norm(u)
        R, t = look_at(8.0 * u)
        views.append(make_view(R, t, W, H, time=tm, scene_id=s))
    return Workload(f"uneven_mix_{n_jobs}jobs_{n_scenes}scenes", scenes, views)


def workload_deep_tile(seed: int = 5, P_sparse: int = 300_000, P_cluster: int = 60_000, width: int = 1600,
                       height: int = 1060):
    """A deep tile in front of a sparse view: N=3, P_sparse primitives
    uniform in [-5,5]^3 and a cluster of P_cluster small, faint primitives
    (scales log-U[0.002, 0.005], opacity sigmoid(N(-3, 0.3))) packed within
    0.01 of a point at depth 4 on the optical axis, seen by one 1600x1060
    camera on a radius-8 sphere: one tile's list holds most of the cluster
    and its pixels do not saturate, so the whole list is walked."""
    rng = np.random.default_rng(seed)
    sp = make_scene(seed, 3, P_sparse, means="uniform", extent=5.0, rng=rng)
    views = sphere_views(rng, 1, 8.0, width, height)
    cl = make_scene(seed + 1, 3, P_cluster, means="uniform", extent=1.0, scale_range=(0.002, 0.005), rng=rng)
    v = views[0]
    centre = -np.asarray(v.R, np.float64).T @ np.asarray(v.t, np.float64)  # camera centre
    ahead = np.asarray(v.R, np.float64)[2]                                  # optical axis
    point = centre + 4.0 * ahead
    cl.plane("mean_x")[:] = (point[:, None] + 0.01 * rng.uniform(-1.0, 1.0, (3, P_cluster))).astype(np.float32)
    cl.plane("opacity")[:] = (1.0 / (1.0 + np.exp(3.0 - 0.3 * rng.standard_normal(P_cluster)))).astype(np.float32)
    params = np.ascontiguousarray(np.concatenate([sp.params, cl.params], axis=1))
    return Workload(f"deep_tile_n3_{P_sparse // 1000}k_{P_cluster // 1000}k_{width}x{height}",
                    [Scene(3, ROT_QUAT, params)], views)


def l1_target(seed: int, views) -> list:
    """Uniform-random target images (one [3, H, W] float32 array per view)."""
    rng = np.random.default_rng(seed + 1000)
    return [rng.uniform(0.0, 1.0, size=(3, v.height, v.width)).astype(np.float32) for v in views]
