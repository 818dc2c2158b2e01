"""ctypes binding of ``include/ubs.h`` (argument marshalling only).

Every function here has the name of the C entry point it calls and passes its
arguments through unchanged; all computation happens in ``libubs.so``.
Loading fails loudly if the library has not been built.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, Structure, c_char_p, c_float, c_int32, c_int64, c_size_t, c_void_p

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libubs.so")

UBS_OK = 0
UBS_ERR_INVALID_ARG = 1
UBS_ERR_ALIGNMENT = 2
UBS_ERR_CAPACITY = 3
UBS_ERR_CUDA = 4
UBS_ERR_TIMEOUT = 5
UBS_ERR_INTERNAL = 6
UBS_ERR_WORKSPACE = 7
UBS_ROT_QUAT = 0
UBS_ROT_SKEW1 = 1
UBS_ROT_SKEW2 = 2
UBS_ROT_CAYLEY = 3
UBS_ROT_CHOL = 4
UBS_ROT_EXP = 5
UBS_FLAG_TIGHT_CUT = 1
UBS_FLAG_COUNT_PAIRS = 2
UBS_FLAG_ACCUMULATE_GRADS = 4
UBS_FLAG_PERSISTENT = 8
UBS_FLAG_SPLIT_LISTS = 16
UBS_FLAG_NO_THRESHOLDS = 32
UBS_FLAG_CHECKED = 64
UBS_ACT_IDENTITY = 0
UBS_ACT_SIGMOID = 1
UBS_ACT_EXP = 2

EXPORT_KEYS, EXPORT_TILES, EXPORT_RECT, EXPORT_RECORDS, EXPORT_INSTANCES = 0, 1, 2, 3, 4
EXPORT_TILE_START, EXPORT_FINAL_T, EXPORT_LAST, EXPORT_SCREEN_GRAD, EXPORT_PAIRS = 5, 6, 7, 8, 9
EXPORT_VISITED = 10


class ubs_scene(Structure):
    _fields_ = [("N", c_int32), ("rot_mode", c_int32), ("P", c_int64),
                ("mean_x", c_void_p), ("mean_q", c_void_p), ("rot", c_void_p), ("scale_x", c_void_p),
                ("L_qx", c_void_p), ("L_q", c_void_p), ("b", c_void_p), ("opacity", c_void_p),
                ("rgb", c_void_p)]


class ubs_scene_grad(Structure):
    _fields_ = [("mean_x", c_void_p), ("mean_q", c_void_p), ("rot", c_void_p), ("scale_x", c_void_p),
                ("L_qx", c_void_p), ("L_q", c_void_p), ("b", c_void_p), ("opacity", c_void_p),
                ("rgb", c_void_p)]


class ubs_view(Structure):
    _fields_ = [("R", c_float * 9), ("t", c_float * 3), ("fx", c_float), ("fy", c_float), ("cx", c_float),
                ("cy", c_float), ("width", c_int32), ("height", c_int32), ("time", c_float),
                ("scene_id", c_int32)]


class ubs_config(Structure):
    _fields_ = [("tile_w", c_int32), ("tile_h", c_int32), ("alpha_min", c_float), ("alpha_max", c_float),
                ("T_min", c_float), ("eps2d", c_float), ("near_plane", c_float), ("jac_clip", c_float),
                ("bg", c_float * 3), ("flags", c_int32)]


class ubs_problem(Structure):
    _fields_ = [("scenes", POINTER(ubs_scene)), ("n_scenes", c_int32), ("views", POINTER(ubs_view)),
                ("n_views", c_int32), ("cfg", ubs_config), ("instance_capacity", c_int64)]


class ubs_device_status(Structure):
    _fields_ = [("status", c_int32), ("reserved", c_int32), ("visible_records", c_int64),
                ("instances", c_int64)]


class ubs_adam_plane(Structure):
    _fields_ = [("lr", c_float), ("activation", c_int32), ("l1_weight", c_float), ("noise_row", c_int32)]


class ubs_adam_config(Structure):
    _fields_ = [("beta1", c_float), ("beta2", c_float), ("eps", c_float), ("step", c_int32),
                ("lambda_eps", c_float)]


# name -> (restype, argtypes), exactly the declarations of include/ubs.h
SIGNATURES = {
    "ubs_workspace_size": (c_size_t, [POINTER(ubs_problem)]),
    "ubs_preprocess": (c_int32, [POINTER(ubs_problem), c_void_p, c_size_t, c_void_p]),
    "ubs_bin_sort": (c_int32, [POINTER(ubs_problem), c_void_p, c_size_t, c_void_p]),
    "ubs_render_fwd": (c_int32, [POINTER(ubs_problem), c_void_p, c_size_t, c_void_p, c_void_p]),
    "ubs_render_bwd": (c_int32, [POINTER(ubs_problem), c_void_p, c_size_t, c_void_p, POINTER(ubs_scene_grad),
                                 c_void_p]),
    "ubs_render_bwd_blend": (c_int32, [POINTER(ubs_problem), c_void_p, c_size_t, c_void_p, c_void_p]),
    "ubs_render_bwd_params": (c_int32, [POINTER(ubs_problem), c_void_p, c_size_t, POINTER(ubs_scene_grad),
                                        c_void_p]),
    "ubs_read_status": (c_int32, [POINTER(ubs_problem), c_void_p, c_size_t, POINTER(ubs_device_status),
                                  c_void_p]),
    "ubs_export": (c_int32, [POINTER(ubs_problem), c_void_p, c_size_t, c_int32, c_void_p, c_size_t,
                             POINTER(c_size_t), c_void_p]),
    "ubs_status_string": (c_char_p, [c_int32]),
    "ubs_render_fwd_static": (c_int32, [POINTER(ubs_problem), c_void_p, c_void_p]),
    "ubs_read_status_static": (c_int32, [POINTER(ubs_problem), POINTER(ubs_device_status), c_void_p]),
    "ubs_loss_workspace_size": (c_size_t, [c_int32, POINTER(c_int32), POINTER(c_int32)]),
    "ubs_image_loss": (c_int32, [c_int32, POINTER(c_int32), POINTER(c_int32), c_void_p, c_void_p, c_float,
                                 c_void_p, c_void_p, c_void_p, c_size_t, c_void_p]),
    "ubs_adam_step": (c_int32, [c_int32, c_int64, POINTER(ubs_adam_plane), POINTER(ubs_adam_config), c_void_p,
                                c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "ubs_mcmc_workspace_size": (c_size_t, [c_int64]),
    "ubs_mcmc_relocate": (c_int32, [c_int32, c_int64, c_int32, c_float, c_void_p, c_void_p, c_void_p, c_void_p,
                                    c_void_p, c_void_p, c_void_p, c_void_p, c_size_t, c_void_p]),
}

_lib = None


def load(path: str = LIB_PATH):
    """Load libubs.so (raises if it is missing: there is no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with paper_2510_03312_gb300.build.build()")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class UBSError(RuntimeError):
    def __init__(self, status, where=""):
        self.status = int(status)
        super().__init__(f"{where}: {ubs_status_string(status)} (status {int(status)})")


def ubs_workspace_size(problem) -> int:
    return int(load().ubs_workspace_size(ctypes.byref(problem)))


def ubs_preprocess(problem, workspace, workspace_bytes, stream) -> int:
    return int(load().ubs_preprocess(ctypes.byref(problem), workspace, workspace_bytes, stream))


def ubs_bin_sort(problem, workspace, workspace_bytes, stream) -> int:
    return int(load().ubs_bin_sort(ctypes.byref(problem), workspace, workspace_bytes, stream))


def ubs_render_fwd(problem, workspace, workspace_bytes, image, stream) -> int:
    return int(load().ubs_render_fwd(ctypes.byref(problem), workspace, workspace_bytes, image, stream))


def ubs_render_bwd(problem, workspace, workspace_bytes, dL_dimage, grads, stream) -> int:
    return int(load().ubs_render_bwd(ctypes.byref(problem), workspace, workspace_bytes, dL_dimage, grads, stream))


def ubs_render_bwd_blend(problem, workspace, workspace_bytes, dL_dimage, stream) -> int:
    return int(load().ubs_render_bwd_blend(ctypes.byref(problem), workspace, workspace_bytes, dL_dimage, stream))


def ubs_render_bwd_params(problem, workspace, workspace_bytes, grads, stream) -> int:
    return int(load().ubs_render_bwd_params(ctypes.byref(problem), workspace, workspace_bytes, grads, stream))


def ubs_read_status(problem, workspace, workspace_bytes, stream) -> ubs_device_status:
    out = ubs_device_status()
    st = load().ubs_read_status(ctypes.byref(problem), workspace, workspace_bytes, ctypes.byref(out), stream)
    if st != UBS_OK:
        raise UBSError(st, "ubs_read_status")
    return out


def ubs_export(problem, workspace, workspace_bytes, what, dst, dst_bytes, stream):
    need = c_size_t(0)
    st = load().ubs_export(ctypes.byref(problem), workspace, workspace_bytes, what, dst, dst_bytes,
                           ctypes.byref(need), stream)
    return int(st), int(need.value)


def ubs_status_string(status) -> str:
    return load().ubs_status_string(int(status)).decode()


def ubs_render_fwd_static(problem, image, stream) -> int:
    return int(load().ubs_render_fwd_static(ctypes.byref(problem), image, stream))


def ubs_read_status_static(problem, stream) -> ubs_device_status:
    out = ubs_device_status()
    st = load().ubs_read_status_static(ctypes.byref(problem), ctypes.byref(out), stream)
    if st != UBS_OK:
        raise UBSError(st, "ubs_read_status_static")
    return out


def _sizes(widths, heights):
    n = len(widths)
    return n, (c_int32 * n)(*[int(w) for w in widths]), (c_int32 * n)(*[int(h) for h in heights])


def ubs_loss_workspace_size(widths, heights) -> int:
    n, w, h = _sizes(widths, heights)
    return int(load().ubs_loss_workspace_size(n, w, h))


def ubs_image_loss(widths, heights, image, target, lambda_ssim, dL_dimage, loss, workspace, workspace_bytes,
                   stream) -> int:
    n, w, h = _sizes(widths, heights)
    return int(load().ubs_image_loss(n, w, h, image, target, float(lambda_ssim), dL_dimage, loss, workspace,
                                     workspace_bytes, stream))


def ubs_adam_step(K, P, planes, cfg, raw, act_out, grad, m, v, noise, stream) -> int:
    return int(load().ubs_adam_step(int(K), int(P), planes, ctypes.byref(cfg), raw, act_out, grad, m, v, noise,
                                    stream))


def ubs_mcmc_workspace_size(P) -> int:
    return int(load().ubs_mcmc_workspace_size(int(P)))


def ubs_mcmc_relocate(K, P, opacity_row, dead_threshold, act, raw, m, v, rand, sources, n_relocated, workspace,
                      workspace_bytes, stream) -> int:
    return int(load().ubs_mcmc_relocate(int(K), int(P), int(opacity_row), float(dead_threshold), act, raw, m, v,
                                        rand, sources, n_relocated, workspace, workspace_bytes, stream))
