"""Helpers that run the CUDA path (through the C ABI) and the FP64 oracle on
the same seeded inputs and compare them.  The two sides share only the
input arrays; nothing computed by one is fed to the other."""
from __future__ import annotations

import math

import numpy as np

import oracle

LOG2E = 1.4426950408889634

# Tolerances (documented in the design notes)
IMG_ATOL = 1e-4          # FP32 images, max abs per channel, non-ambiguous pixels
GRAD_RTOL = 1e-3         # gradients: ||g - g_ref|| / ||g_ref|| per tensor


def oracle_config(cfg):
    return oracle.config(tile=cfg.tile, alpha_min=cfg.alpha_min, alpha_max=cfg.alpha_max, t_stop=cfg.t_stop,
                         dilation=cfg.dilation, fov_clamp=cfg.fov_clamp, near_z=cfg.near_z, bg=cfg.bg,
                         antialias_comp=cfg.antialias_comp)


def dequantised(scene, sh_dtype=None, scale_dtype=None, skew_dtype=None):
    """The scene as the GPU sees it after storage rounding (for the oracle)."""
    import copy

    import torch

    s = copy.copy(scene)

    def q(a, dt):
        if dt is None or dt == torch.float32 or a is None:
            return a
        return torch.as_tensor(a).to(dt).float().numpy()

    s.sh = q(scene.sh, sh_dtype)
    s.log_scales = q(scene.log_scales, scale_dtype)
    s.skew = q(scene.skew, skew_dtype)
    s.split_dir = q(scene.split_dir, skew_dtype)
    return s


def gpu_records_to_oracle_layout(rec16: np.ndarray) -> dict:
    """Convert the GPU render records (float32 [m,16]) to natural units."""
    r = rec16.astype(np.float64)
    return dict(mx=r[:, 0], my=r[:, 1], a=-2.0 * r[:, 2] / LOG2E, b=-r[:, 3] / LOG2E, c=-2.0 * r[:, 4] / LOG2E,
                bx=r[:, 5] * math.sqrt(2.0), by=r[:, 6] * math.sqrt(2.0), m=r[:, 7], h=r[:, 8],
                ux=r[:, 9] * math.sqrt(2.0), uy=r[:, 10] * math.sqrt(2.0), rgb=r[:, 12:15], thr=r[:, 15])


def tile_ranges(keys: np.ndarray, total_tiles: int) -> np.ndarray:
    tiles = (keys >> np.uint64(32)).astype(np.int64)
    starts = np.searchsorted(tiles, np.arange(total_tiles), side="left")
    ends = np.searchsorted(tiles, np.arange(total_tiles), side="right")
    return np.stack([starts, ends], 1)


def compare_keys(gpu_keys, gpu_vals, or_keys, or_vals, ambiguous_vals):
    """Bit-exact comparison of sorted key lists after removing Gaussians whose
    tile set is decision-ambiguous; returns the number removed."""
    amb = np.zeros(0, np.int64) if ambiguous_vals is None else np.asarray(ambiguous_vals, np.int64)
    gk, gv = np.asarray(gpu_keys).view(np.uint64), np.asarray(gpu_vals).astype(np.int64)
    ok_g = ~np.isin(gv, amb)
    ok_o = ~np.isin(or_vals, amb)
    np.testing.assert_array_equal(gk[ok_g], or_keys[ok_o])
    np.testing.assert_array_equal(gv[ok_g], or_vals[ok_o])
    return int(amb.size)


def image_error(gpu_img_chw: np.ndarray, or_rgb_hwc: np.ndarray, ambiguous_hw: np.ndarray):
    d = np.abs(np.transpose(gpu_img_chw, (1, 2, 0)).astype(np.float64) - or_rgb_hwc)
    d[ambiguous_hw] = 0.0
    return float(d.max()) if d.size else 0.0


def rel_err(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-12))
