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


def rel_err(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-12))


def gpu_blend_lists(r, v: int, rows_per_block: int = 64):
    """The Gaussians (indices within the view) the GPU forward blended at each
    pixel of view v, in blend order: (offsets int64 [H*W + 1], ids int32)."""
    from paper_2605_18334_gb300.rasterizer import blend_lists

    return blend_lists(r, v, rows_per_block)


def check_key_order(keys: np.ndarray, vals: np.ndarray):
    """The sorted list is ordered by (tile, depth bits) with ties in index
    order, and no (tile, Gaussian) pair repeats."""
    k = np.asarray(keys).view(np.uint64)
    v = np.asarray(vals).astype(np.int64)
    if k.size < 2:
        return
    ok = (k[1:] > k[:-1]) | ((k[1:] == k[:-1]) & (v[1:] > v[:-1]))
    assert ok.all(), int(np.nonzero(~ok)[0][0])


def check_ambiguous_tile_sets(keys, vals, pre, amb_ids, rec64, cam, ocfg, v_base: int, tile_base: int,
                              tol_alpha: float, tol_px: float):
    """For Gaussians whose FP64 tile set is ambiguous (an edge within tol_px
    of a pixel-centre boundary, or a cull within tolerance): the GPU's tiles
    hold every tile with a pixel centre where the FP64 alpha is at least
    alpha_min (1 + tol_alpha), and lie within the FP64 bounding box of the
    footprint widened by tol_px.  Returns the number of Gaussians checked."""
    import oracle as O

    k = np.asarray(keys).view(np.uint64)
    v = np.asarray(vals).astype(np.int64) - v_base
    tiles = (k >> np.uint64(32)).astype(np.int64) - tile_base
    sel = np.isin(v, amb_ids)
    order = np.argsort(v[sel], kind="stable")
    gv, gt = v[sel][order], tiles[sel][order]
    W, H = cam.width, cam.height
    tiles_x = -(-W // 16)
    tau, amax = float(ocfg.alpha_min), float(ocfg.alpha_max)
    checked = 0
    for i in amb_ids:
        got = set(gt[np.searchsorted(gv, i, "left"):np.searchsorted(gv, i, "right")].tolist())
        if not pre["visible"][i]:
            assert not got, i
            continue
        ex, ey = pre["ext"][i, 0], pre["ext"][i, 1]
        mx, my = rec64[i, 0], rec64[i, 1]
        x0 = max(0, int(np.ceil(mx - ex - tol_px - 0.5)))
        x1 = min(W - 1, int(np.floor(mx + ex + tol_px - 0.5)))
        y0 = max(0, int(np.ceil(my - ey - tol_px - 0.5)))
        y1 = min(H - 1, int(np.floor(my + ey + tol_px - 0.5)))
        allowed = set()
        need = set()
        if x0 <= x1 and y0 <= y1:
            ys, xs = np.meshgrid(np.arange(y0, y1 + 1), np.arange(x0, x1 + 1), indexing="ij")
            px = np.stack([xs.reshape(-1), ys.reshape(-1)], 1).astype(np.int32)
            t = (px[:, 1] // 16) * tiles_x + px[:, 0] // 16
            allowed = set(np.unique(t).tolist())
            a = np.minimum(O.alpha_at(pre["rec"][i], px), amax)
            need = set(np.unique(t[a >= tau * (1 + tol_alpha)]).tolist())
        assert need <= got, (i, sorted(need - got))
        assert got <= allowed, (i, sorted(got - allowed))
        checked += 1
    return checked


# per-element gradient bar, relative to the sum of the magnitudes of the terms
# of an element: the FP32 path's projected centres carry up to ~2e-4 px of
# rounding at 1080p, which moves alpha of the smallest splats by up to ~1e-3
# (relative), and T_k compounds the errors of the factors (1 - alpha_j) in
# front of it (up to 3.2e-3 measured); the bar is 1e-2 of the scale
ELEM_RTOL = 1e-2


def compare_grads_elementwise(got: dict, ref: dict, fields, rtol: float = ELEM_RTOL):
    """Element-by-element gradient bar: |g - g_ref| <= rtol * scale + slack,
    where scale is the oracle's sum of the magnitudes of the terms summed into
    the element (the scale a rounding error in any term grows with) and slack
    the magnitude of the terms whose alpha_max or colour clamp decision lies
    within tolerance (either decision is admissible).  Returns, per field,
    (worst ratio |g - g_ref| / (rtol * scale + slack), the share of elements
    within rtol of |g_ref|, the number of elements)."""
    out = {}
    for k in fields:
        a = got[k].detach().cpu().numpy().astype(np.float64).reshape(-1)
        b = np.asarray(ref[k], np.float64).reshape(-1)
        s = np.asarray(ref["scale"][k], np.float64).reshape(-1)
        sl = np.asarray(ref["slack"][k], np.float64).reshape(-1)
        bound = rtol * s + sl + 1e-30
        err = np.abs(a - b)
        ratio = err / bound
        worst = int(np.argmax(ratio)) if ratio.size else 0
        within = float(np.mean(err <= 1e-3 * np.abs(b) + 1e-12 * np.abs(b).max())) if b.size else 1.0
        out[k] = (float(ratio[worst]) if ratio.size else 0.0, within, int(b.size))
        assert ratio.size == 0 or ratio[worst] <= 1.0, (
            k, worst, float(a[worst]), float(b[worst]), float(s[worst]), float(sl[worst]))
    return out
