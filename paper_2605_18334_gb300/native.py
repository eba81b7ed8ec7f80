"""ctypes binding of ``libskewraster.so`` (include/skewraster.h).

Argument marshalling only: every step of the rasterizer runs in the CUDA
library.  The functions keep the C names (``sr_plan_init``, ``sr_preprocess``,
``sr_bin_sort``, ``sr_render_fwd``, ``sr_render_bwd``, ...).  Loading fails
loudly if the library has not been built; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

from . import build as _build

SR_MAX_VIEWS = 256
SR_ABI_VERSION = 3

SR_OK, SR_ERR_INVALID, SR_ERR_CAPACITY, SR_ERR_CUDA, SR_ERR_TIMEOUT, SR_ERR_UNSUPPORTED = range(6)
SR_F32, SR_BF16, SR_F16 = 0, 1, 2

EXPORTS = ["sr_abi_version", "sr_status_string", "sr_config_default", "sr_camera_from_gl", "sr_plan_init",
           "sr_workspace_size", "sr_preprocess", "sr_bin_sort", "sr_render_fwd", "sr_render_bwd", "sr_read_status",
           "sr_kernel_launches", "sr_frame_counters", "sr_sort_keys_noalloc", "sr_render_bwd_composite",
           "sr_render_bwd_project", "sr_selftest_bounded_wait", "sr_loss_scratch_size", "sr_loss_l1_dssim",
           "sr_adam_step", "sr_densify_stats", "sr_densify_scratch_size", "sr_densify", "sr_densify_remap",
           "sr_measure_alu_peaks"]

SR_ADAM_MAX_GROUPS = 16

# 2D gradients of a render record (dL/d of mean, conic, skew, opacity terms,
# colour) and their slots in the library's 16-float workspace records
D2_NAMES = ["mx", "my", "a", "b", "c", "bx", "by", "m", "h", "ux", "uy", "r", "g", "bl"]
D2_SLOTS = [0, 1, 2, 4, 5, 6, 8, 9, 10, 3, 11, 12, 13, 14]


class sr_adam_group(C.Structure):
    _fields_ = [("param", C.c_void_p), ("grad", C.c_void_p), ("m", C.c_void_p), ("v", C.c_void_p), ("n", C.c_int64),
                ("lr", C.c_float), ("lr_rest", C.c_float), ("period", C.c_int32), ("split_at", C.c_int32)]


class sr_densify_config(C.Structure):
    _fields_ = [("grad_uv", C.c_float), ("grad_z", C.c_float), ("log_scale_split", C.c_float),
                ("logit_prune", C.c_float)]


class sr_scene_arrays(C.Structure):
    _fields_ = [("means", C.c_void_p), ("log_scales", C.c_void_p), ("quats", C.c_void_p),
                ("opacity_logits", C.c_void_p), ("skew", C.c_void_p), ("split_dir", C.c_void_p), ("sh", C.c_void_p)]


class sr_gaussians(C.Structure):
    _fields_ = [("means", C.c_void_p), ("log_scales", C.c_void_p), ("quats", C.c_void_p),
                ("opacity_logits", C.c_void_p), ("skew", C.c_void_p), ("split_dir", C.c_void_p), ("sh", C.c_void_p),
                ("n", C.c_int64), ("sh_degree", C.c_int32), ("two_opacities", C.c_int32), ("dt_sh", C.c_int32),
                ("dt_scale", C.c_int32), ("dt_skew", C.c_int32), ("reserved_", C.c_int32)]


class sr_camera(C.Structure):
    _fields_ = [("w2c", C.c_float * 12), ("fx", C.c_float), ("fy", C.c_float), ("cx", C.c_float), ("cy", C.c_float),
                ("tan_fovx", C.c_float), ("tan_fovy", C.c_float), ("campos", C.c_float * 3), ("width", C.c_int32),
                ("height", C.c_int32)]


class sr_config(C.Structure):
    _fields_ = [("tile_w", C.c_int32), ("tile_h", C.c_int32), ("alpha_min", C.c_float), ("alpha_max", C.c_float),
                ("t_stop", C.c_float), ("dilation", C.c_float), ("fov_clamp", C.c_float), ("near_z", C.c_float),
                ("bg", C.c_float * 3), ("antialias_comp", C.c_int32), ("fwd_batch", C.c_int32),
                ("sort_spin_limit", C.c_int32), ("fwd_pixels_per_thread", C.c_int32),
                ("bwd_pixels_per_thread", C.c_int32), ("forward_only", C.c_int32), ("bwd_batch", C.c_int32),
                ("recompute_keys", C.c_int32), ("persistent", C.c_int32), ("fwd_blocks_per_sm", C.c_int32),
                ("bwd_blocks_per_sm", C.c_int32)]


class sr_grads(C.Structure):
    _fields_ = [(k, C.c_void_p) for k in ("means", "log_scales", "quats", "opacity_logits", "skew", "split_dir", "sh",
                                          "means2d_abs", "depth_grad")]


class sr_plan(C.Structure):
    _fields_ = [("abi_version", C.c_int32), ("n_views", C.c_int32), ("n", C.c_int64), ("sh_degree", C.c_int32),
                ("tile_w", C.c_int32), ("tile_h", C.c_int32), ("sort_passes", C.c_int32), ("sort_bits", C.c_int32),
                ("render_mode", C.c_int32), ("two_opacities", C.c_int32), ("has_split", C.c_int32),
                ("forward_only", C.c_int32), ("recompute_keys", C.c_int32),
                ("key_capacity", C.c_int64), ("total_tiles", C.c_int64), ("total_pixels", C.c_int64),
                ("tile_base", C.c_int64 * (SR_MAX_VIEWS + 1)), ("image_offset", C.c_int64 * (SR_MAX_VIEWS + 1)),
                ("pixel_offset", C.c_int64 * (SR_MAX_VIEWS + 1)), ("width", C.c_int32 * SR_MAX_VIEWS),
                ("height", C.c_int32 * SR_MAX_VIEWS), ("ws_bytes", C.c_size_t), ("off", C.c_size_t * 32)]


class SkewRasterError(RuntimeError):
    def __init__(self, where: str, status: int):
        self.status = status
        super().__init__(f"{where}: {status_string(status)} (status {status})")


_lock = threading.Lock()
_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load the library (building it first if it is missing or stale and a
    compiler is available)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if build_if_missing:
            try:
                path = _build.build()
            except RuntimeError:
                if not os.path.exists(path):
                    raise
        if not os.path.exists(path):
            raise RuntimeError(f"libskewraster is not built ({path}); run __graft_entry__.build()")
        lib = C.CDLL(path)
        P = C.POINTER
        lib.sr_abi_version.restype = C.c_int32
        lib.sr_status_string.restype = C.c_char_p
        lib.sr_status_string.argtypes = [C.c_int]
        lib.sr_config_default.argtypes = [P(sr_config)]
        lib.sr_camera_from_gl.argtypes = [P(C.c_double), C.c_int32, C.c_int32, C.c_double, C.c_double, P(sr_camera)]
        lib.sr_plan_init.argtypes = [P(sr_plan), P(sr_config), P(sr_gaussians), P(sr_camera), C.c_int32, C.c_int64]
        lib.sr_workspace_size.restype = C.c_size_t
        lib.sr_workspace_size.argtypes = [P(sr_plan)]
        lib.sr_preprocess.argtypes = [P(sr_plan), P(sr_gaussians), C.c_void_p, P(sr_config), C.c_void_p, C.c_void_p]
        lib.sr_bin_sort.argtypes = [P(sr_plan), P(sr_config), C.c_void_p, P(C.c_int64), C.c_void_p]
        lib.sr_render_fwd.argtypes = [P(sr_plan), P(sr_config), C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                      C.c_void_p]
        lib.sr_render_bwd.argtypes = [P(sr_plan), P(sr_gaussians), C.c_void_p, P(sr_config), C.c_void_p, C.c_void_p,
                                      C.c_void_p, C.c_void_p, P(sr_grads), C.c_void_p]
        lib.sr_read_status.argtypes = [P(sr_plan), C.c_void_p, P(C.c_int64), C.c_void_p]
        lib.sr_render_bwd_composite.argtypes = [P(sr_plan), P(sr_config), C.c_void_p, C.c_void_p, C.c_void_p,
                                                C.c_void_p, C.c_void_p]
        lib.sr_render_bwd_project.argtypes = [P(sr_plan), P(sr_gaussians), C.c_void_p, P(sr_config), C.c_void_p,
                                              P(sr_grads), C.c_void_p]
        lib.sr_selftest_bounded_wait.argtypes = [P(sr_plan), C.c_void_p, C.c_int32, P(C.c_int64), C.c_void_p]
        lib.sr_selftest_bounded_wait.restype = C.c_int
        lib.sr_kernel_launches.restype = C.c_uint64
        lib.sr_kernel_launches.argtypes = []
        lib.sr_measure_alu_peaks.argtypes = [C.c_void_p, P(sr_alu_peaks), C.c_void_p]
        lib.sr_frame_counters.argtypes = [P(sr_plan), C.c_void_p, P(C.c_uint64), P(C.c_uint64), C.c_void_p]
        lib.sr_frame_counters.restype = C.c_int
        lib.sr_loss_scratch_size.restype = C.c_size_t
        lib.sr_loss_scratch_size.argtypes = [P(sr_plan)]
        lib.sr_loss_l1_dssim.argtypes = [P(sr_plan), C.c_void_p, C.c_void_p, C.c_void_p, C.c_float, C.c_void_p,
                                         C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
        lib.sr_loss_l1_dssim.restype = C.c_int
        lib.sr_adam_step.argtypes = [P(sr_adam_group), C.c_int32, C.c_int64, C.c_float, C.c_float, C.c_float,
                                     C.c_void_p]
        lib.sr_adam_step.restype = C.c_int
        lib.sr_densify_stats.argtypes = [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p,
                                         C.c_void_p]
        lib.sr_densify_stats.restype = C.c_int
        lib.sr_densify_scratch_size.restype = C.c_size_t
        lib.sr_densify_scratch_size.argtypes = [C.c_int64]
        lib.sr_densify.argtypes = [P(sr_gaussians), C.c_void_p, C.c_void_p, C.c_void_p, P(sr_densify_config),
                                   P(sr_scene_arrays), C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
        lib.sr_densify.restype = C.c_int
        lib.sr_densify_remap.argtypes = [C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p,
                                         C.c_void_p]
        lib.sr_densify_remap.restype = C.c_int
        for name in ("sr_config_default", "sr_camera_from_gl", "sr_plan_init", "sr_preprocess", "sr_bin_sort",
                     "sr_render_fwd", "sr_render_bwd", "sr_read_status", "sr_render_bwd_composite",
                     "sr_render_bwd_project"):
            getattr(lib, name).restype = C.c_int
        if lib.sr_abi_version() != SR_ABI_VERSION:
            raise RuntimeError("libskewraster ABI version mismatch")
        _lib = lib
        return lib


def status_string(s: int) -> str:
    try:
        return load(build_if_missing=False).sr_status_string(int(s)).decode()
    except Exception:  # library not loadable: still report the code
        return f"status {s}"


def check(where: str, s: int) -> None:
    if s != SR_OK:
        raise SkewRasterError(where, s)


# --- thin wrappers with the C names -----------------------------------------

def sr_config_default() -> sr_config:
    c = sr_config()
    check("sr_config_default", load().sr_config_default(C.byref(c)))
    return c


def sr_camera_from_gl(c2w_gl, width: int, height: int, fovx: float, fovy: float) -> sr_camera:
    m = (C.c_double * 16)(*[float(x) for x in list(c2w_gl.reshape(16))])
    out = sr_camera()
    check("sr_camera_from_gl", load().sr_camera_from_gl(m, int(width), int(height), float(fovx), float(fovy),
                                                        C.byref(out)))
    return out


def sr_plan_init(cfg: sr_config, g: sr_gaussians, cams: list, key_capacity: int) -> sr_plan:
    arr = (sr_camera * len(cams))(*cams)
    p = sr_plan()
    check("sr_plan_init", load().sr_plan_init(C.byref(p), C.byref(cfg), C.byref(g), arr, len(cams),
                                              int(key_capacity)))
    return p


def sr_preprocess(plan, g, cams_dev_ptr: int, cfg, ws_ptr: int, stream: int) -> None:
    check("sr_preprocess", load().sr_preprocess(C.byref(plan), C.byref(g), C.c_void_p(cams_dev_ptr), C.byref(cfg),
                                                C.c_void_p(ws_ptr), C.c_void_p(stream)))


def sr_bin_sort(plan, cfg, ws_ptr: int, stream: int, sync: bool = True):
    """Returns the key count (sync=True) or None (sync=False, graph-safe).
    Raises SkewRasterError(SR_ERR_CAPACITY) with ``.keys_needed`` set when the
    frame needs more keys than the plan holds."""
    k = C.c_int64(-1)
    s = load().sr_bin_sort(C.byref(plan), C.byref(cfg), C.c_void_p(ws_ptr), C.byref(k) if sync else None,
                           C.c_void_p(stream))
    if s != SR_OK:
        err = SkewRasterError("sr_bin_sort", s)
        err.keys_needed = int(k.value)
        raise err
    return int(k.value) if sync else None


def sr_render_fwd(plan, cfg, ws_ptr: int, images_ptr: int, t_final_ptr: int, n_contrib_ptr: int,
                  stream: int) -> None:
    check("sr_render_fwd", load().sr_render_fwd(C.byref(plan), C.byref(cfg), C.c_void_p(ws_ptr),
                                                C.c_void_p(images_ptr), C.c_void_p(t_final_ptr),
                                                C.c_void_p(n_contrib_ptr), C.c_void_p(stream)))


def sr_render_bwd(plan, g, cams_dev_ptr: int, cfg, ws_ptr: int, d_images_ptr: int, t_final_ptr: int,
                  n_contrib_ptr: int, grads: sr_grads, stream: int) -> None:
    check("sr_render_bwd", load().sr_render_bwd(C.byref(plan), C.byref(g), C.c_void_p(cams_dev_ptr), C.byref(cfg),
                                                C.c_void_p(ws_ptr), C.c_void_p(d_images_ptr),
                                                C.c_void_p(t_final_ptr), C.c_void_p(n_contrib_ptr),
                                                C.byref(grads), C.c_void_p(stream)))


def sr_render_bwd_composite(plan, cfg, ws_ptr: int, d_images_ptr: int, t_final_ptr: int, n_contrib_ptr: int,
                            stream: int) -> None:
    check("sr_render_bwd_composite", load().sr_render_bwd_composite(
        C.byref(plan), C.byref(cfg), C.c_void_p(ws_ptr), C.c_void_p(d_images_ptr), C.c_void_p(t_final_ptr),
        C.c_void_p(n_contrib_ptr), C.c_void_p(stream)))


def sr_render_bwd_project(plan, g, cams_dev_ptr: int, cfg, ws_ptr: int, grads, stream: int) -> None:
    check("sr_render_bwd_project", load().sr_render_bwd_project(
        C.byref(plan), C.byref(g), C.c_void_p(cams_dev_ptr), C.byref(cfg), C.c_void_p(ws_ptr), C.byref(grads),
        C.c_void_p(stream)))


def sr_selftest_bounded_wait(plan, ws_ptr: int, spin_limit: int, stream: int):
    """Returns (status, partition that gave up or -1)."""
    part = C.c_int64(-2)
    s = load().sr_selftest_bounded_wait(C.byref(plan), C.c_void_p(ws_ptr), int(spin_limit), C.byref(part),
                                        C.c_void_p(stream))
    return s, int(part.value)


def sr_kernel_launches() -> int:
    return int(load().sr_kernel_launches())


def sr_frame_counters(plan, ws_ptr: int, stream: int):
    t, b = C.c_uint64(0), C.c_uint64(0)
    check("sr_frame_counters", load().sr_frame_counters(C.byref(plan), C.c_void_p(ws_ptr), C.byref(t), C.byref(b),
                                                        C.c_void_p(stream)))
    return int(t.value), int(b.value)


class sr_alu_peaks(C.Structure):
    _fields_ = [(k, C.c_double) for k in ("fma_lane_ops_per_s", "ffma2_lane_ops_per_s", "minmax_lane_ops_per_s",
                                          "ex2_per_s", "rcp_per_s", "seconds")]


def sr_measure_alu_peaks(scratch_ptr: int, stream: int) -> dict:
    out = sr_alu_peaks()
    check("sr_measure_alu_peaks", load().sr_measure_alu_peaks(C.c_void_p(scratch_ptr), C.byref(out),
                                                               C.c_void_p(stream)))
    return {k: getattr(out, k) for k, _ in sr_alu_peaks._fields_}


def sr_loss_scratch_size(plan) -> int:
    return int(load().sr_loss_scratch_size(C.byref(plan)))


def sr_loss_l1_dssim(plan, ws_ptr: int, images_ptr: int, targets_ptr: int, lam: float, d_images_ptr: int,
                     loss_ptr: int, ssim_l1_ptr: int, scratch_ptr: int, stream: int):
    check("sr_loss_l1_dssim", load().sr_loss_l1_dssim(
        C.byref(plan), C.c_void_p(ws_ptr), C.c_void_p(images_ptr), C.c_void_p(targets_ptr), C.c_float(lam),
        C.c_void_p(d_images_ptr), C.c_void_p(loss_ptr), C.c_void_p(ssim_l1_ptr or None), C.c_void_p(scratch_ptr),
        C.c_void_p(stream)))


def sr_adam_step(groups: list, step: int, beta1: float, beta2: float, eps: float, stream: int):
    """groups: sr_adam_group structures (device pointers as ints)."""
    arr = (sr_adam_group * len(groups))(*groups)
    check("sr_adam_step", load().sr_adam_step(arr, len(groups), C.c_int64(step), C.c_float(beta1), C.c_float(beta2),
                                              C.c_float(eps), C.c_void_p(stream)))


def sr_densify_stats(g_uv_ptr: int, g_z_ptr: int, n: int, uv_sum_ptr: int, seen_ptr: int, z_max_ptr: int,
                     stream: int):
    check("sr_densify_stats", load().sr_densify_stats(C.c_void_p(g_uv_ptr), C.c_void_p(g_z_ptr), C.c_int64(n),
                                                      C.c_void_p(uv_sum_ptr), C.c_void_p(seen_ptr),
                                                      C.c_void_p(z_max_ptr), C.c_void_p(stream)))


def sr_densify_scratch_size(n: int) -> int:
    return int(load().sr_densify_scratch_size(C.c_int64(n)))


def sr_densify(g, uv_sum_ptr: int, seen_ptr: int, z_max_ptr: int, cfg, out, src_map_ptr: int, counts_ptr: int,
               scratch_ptr: int, stream: int) -> None:
    check("sr_densify", load().sr_densify(C.byref(g), C.c_void_p(uv_sum_ptr), C.c_void_p(seen_ptr),
                                          C.c_void_p(z_max_ptr), C.byref(cfg), C.byref(out),
                                          C.c_void_p(src_map_ptr), C.c_void_p(counts_ptr), C.c_void_p(scratch_ptr),
                                          C.c_void_p(stream)))


def sr_densify_remap(in_ptr: int, width: int, src_map_ptr: int, counts_ptr: int, cap: int, out_ptr: int,
                     stream: int) -> None:
    check("sr_densify_remap", load().sr_densify_remap(C.c_void_p(in_ptr), C.c_int32(width), C.c_void_p(src_map_ptr),
                                                      C.c_void_p(counts_ptr), C.c_int64(cap), C.c_void_p(out_ptr),
                                                      C.c_void_p(stream)))


def sr_read_status(plan, ws_ptr: int, stream: int):
    k = C.c_int64(-1)
    s = load().sr_read_status(C.byref(plan), C.c_void_p(ws_ptr), C.byref(k), C.c_void_p(stream))
    return s, int(k.value)
