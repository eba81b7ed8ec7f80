"""Host-side checks of the C ABI (no GPU needed): the library loads and
exports every symbol the header declares, host functions (camera set-up,
planning) are correct, and invalid arguments are rejected before any device
work."""
import ctypes as C
import math
import os
import re

import numpy as np
import pytest

import oracle
from paper_2605_18334_gb300 import native as N
from paper_2605_18334_gb300 import scenes
from paper_2605_18334_gb300.rasterizer import Config

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    return N.load()


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "skewraster.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(sr_[a-z_0-9]+)\s*\(", text)))


def test_library_exports_every_declared_symbol(lib):
    syms = declared_symbols()
    assert set(syms) == set(N.EXPORTS), syms
    for s in syms:
        assert hasattr(lib, s), s
    assert lib.sr_abi_version() == N.SR_ABI_VERSION


def test_status_strings(lib):
    for s in range(6):
        assert N.status_string(s)
    assert N.status_string(2) == "tile-key capacity exceeded"


def test_config_default(lib):
    c = N.sr_config_default()
    assert (c.tile_w, c.tile_h) == (16, 16)
    assert c.alpha_min == np.float32(1 / 255) and c.alpha_max == np.float32(0.99)
    assert c.t_stop == np.float32(1e-4) and c.dilation == np.float32(0.3) and c.near_z == np.float32(0.2)
    assert c.antialias_comp == 1


@pytest.mark.parametrize("which", range(6))
def test_camera_from_gl_matches_oracle_bit_exactly(lib, which):
    """Camera set-up (Alg. 3) gives the same FP32 camera on both sides, so
    both are fed identical inputs."""
    cams = [scenes.identity_camera(64, 64), scenes.orbit_camera(0.0, 1920, 1080),
            scenes.orbit_camera(2.1, 1280, 720)] + scenes.trajectory_cameras(3)
    cam = cams[which]
    a = N.sr_camera_from_gl(cam["c2w_gl"], cam["width"], cam["height"], cam["fovx"], cam["fovy"])
    b = oracle.camera_fields(oracle.camera_from_gl(cam))
    np.testing.assert_array_equal(np.array(a.w2c[:], np.float32), b["w2c"].astype(np.float32))
    for k in ("fx", "fy", "cx", "cy", "tan_fovx", "tan_fovy"):
        assert getattr(a, k) == b[k], k
    np.testing.assert_array_equal(np.array(a.campos[:], np.float32), b["campos"].astype(np.float32))
    assert (a.width, a.height) == (b["width"], b["height"])


def test_camera_from_gl_rejects_bad_input(lib):
    m = (C.c_double * 16)(*np.eye(4).ravel())
    out = N.sr_camera()
    assert lib.sr_camera_from_gl(m, 0, 10, 1.0, 1.0, C.byref(out)) == N.SR_ERR_INVALID
    assert lib.sr_camera_from_gl(m, 10, 10, 0.0, 1.0, C.byref(out)) == N.SR_ERR_INVALID
    assert lib.sr_camera_from_gl(m, 10, 10, 1.0, math.pi, C.byref(out)) == N.SR_ERR_INVALID
    assert lib.sr_camera_from_gl(None, 10, 10, 1.0, 1.0, C.byref(out)) == N.SR_ERR_INVALID
    bad = (C.c_double * 16)(*([float("nan")] + [0.0] * 15))
    assert lib.sr_camera_from_gl(bad, 10, 10, 1.0, 1.0, C.byref(out)) == N.SR_ERR_INVALID


def _desc(n=1000, deg=3, two=0, split=False):
    g = N.sr_gaussians()
    g.n, g.sh_degree, g.two_opacities = n, deg, two
    g.split_dir = 16 if split else None
    return g


def test_plan_layout(lib):
    cams = [N.sr_camera_from_gl(c["c2w_gl"], c["width"], c["height"], c["fovx"], c["fovy"])
            for c in scenes.trajectory_cameras(6)]
    cfg = Config().to_c()
    p = N.sr_plan_init(cfg, _desc(1000), cams, 1 << 20)
    tiles = [(-(-c.width // 16)) * (-(-c.height // 16)) for c in cams]
    assert p.n_views == 6 and p.n == 1000 and p.sh_degree == 3
    assert list(p.tile_base[:7]) == list(np.concatenate([[0], np.cumsum(tiles)]))
    assert p.total_tiles == sum(tiles)
    assert list(p.image_offset[:7]) == list(np.concatenate([[0], np.cumsum([3 * c.width * c.height for c in cams])]))
    assert p.total_pixels == sum(c.width * c.height for c in cams)
    tile_bits = math.ceil(math.log2(sum(tiles)))
    assert p.sort_bits == 32 + tile_bits and p.sort_passes == -(-tile_bits // 8)
    assert p.ws_bytes == lib.sr_workspace_size(C.byref(p)) and p.ws_bytes % 256 == 0
    offs = list(p.off[:22])
    assert offs == sorted(offs) and all(o % 256 == 0 for o in offs)
    assert p.render_mode == 0
    assert N.sr_plan_init(cfg, _desc(10, two=1), cams, 10).render_mode == 1
    assert N.sr_plan_init(cfg, _desc(10, two=1, split=True), cams, 10).render_mode == 2
    # one tile -> the depth bits alone
    one = N.sr_camera_from_gl(np.eye(4), 16, 16, 1.0, 1.0)
    p1 = N.sr_plan_init(cfg, _desc(5), [one], 64)
    assert p1.sort_bits == 32 and p1.sort_passes == 0


@pytest.mark.parametrize("bad", ["n", "deg", "views", "cap", "tile", "size", "dtype", "alpha", "fbatch", "bbatch"])
def test_plan_rejects_invalid(lib, bad):
    cfg = Config().to_c()
    cams = [N.sr_camera_from_gl(np.eye(4), 64, 64, 1.0, 1.0)]
    g = _desc(100)
    n_views, cap = 1, 1000
    if bad == "n":
        g.n = -1
    elif bad == "deg":
        g.sh_degree = 4
    elif bad == "views":
        n_views = 0
    elif bad == "cap":
        cap = 1 << 33
    elif bad == "tile":
        cfg.tile_w = 8
    elif bad == "size":
        cams[0].width = 0
    elif bad == "dtype":
        g.dt_sh = 7
    elif bad == "alpha":
        cfg.alpha_max = 1.5
    elif bad == "fbatch":
        cfg.fwd_batch = 64
    elif bad == "bbatch":
        cfg.bwd_batch = 512
    arr = (N.sr_camera * 1)(*cams)
    p = N.sr_plan()
    s = lib.sr_plan_init(C.byref(p), C.byref(cfg), C.byref(g), arr, n_views, cap)
    assert s in (N.SR_ERR_INVALID, N.SR_ERR_UNSUPPORTED)
    if bad == "tile":
        assert s == N.SR_ERR_UNSUPPORTED


def test_stage_calls_reject_invalid_arguments_without_device_work(lib):
    cfg = Config().to_c()
    cams = [N.sr_camera_from_gl(np.eye(4), 64, 64, 1.0, 1.0)]
    p = N.sr_plan_init(cfg, _desc(100, deg=0), cams, 1000)
    g = _desc(100, deg=0)
    # no workspace
    assert lib.sr_preprocess(C.byref(p), C.byref(g), C.c_void_p(256), C.byref(cfg), None, None) == N.SR_ERR_INVALID
    assert lib.sr_bin_sort(C.byref(p), C.byref(cfg), None, None, None) == N.SR_ERR_INVALID
    # misaligned workspace
    assert lib.sr_render_fwd(C.byref(p), C.byref(cfg), C.c_void_p(4096 + 8), C.c_void_p(256), C.c_void_p(256),
                             C.c_void_p(256), None) == N.SR_ERR_INVALID
    # Gaussians that do not match the plan / missing data pointers
    g2 = _desc(101, deg=0)
    assert lib.sr_preprocess(C.byref(p), C.byref(g2), C.c_void_p(256), C.byref(cfg), C.c_void_p(4096),
                             None) == N.SR_ERR_INVALID
    assert lib.sr_preprocess(C.byref(p), C.byref(g), C.c_void_p(256), C.byref(cfg), C.c_void_p(4096),
                             None) == N.SR_ERR_INVALID
    # missing outputs
    assert lib.sr_render_fwd(C.byref(p), C.byref(cfg), C.c_void_p(4096), None, None, None,
                             None) == N.SR_ERR_INVALID
    gr = N.sr_grads()
    assert lib.sr_render_bwd(C.byref(p), C.byref(g), C.c_void_p(256), C.byref(cfg), C.c_void_p(4096), None, None,
                             None, C.byref(gr), None) == N.SR_ERR_INVALID
    # corrupted plan
    p.abi_version = 99
    assert lib.sr_bin_sort(C.byref(p), C.byref(cfg), C.c_void_p(4096), None, None) == N.SR_ERR_INVALID


def test_training_calls_reject_invalid_arguments_without_device_work(lib):
    cfg = Config().to_c()
    cams = [N.sr_camera_from_gl(np.eye(4), 64, 48, 1.0, 1.0)]
    p = N.sr_plan_init(cfg, _desc(100, deg=0), cams, 1000)
    assert lib.sr_loss_scratch_size(C.byref(p)) >= 9 * 4 * 64 * 48
    ok = C.c_void_p(4096)
    # lambda out of range, NULL buffers, misaligned scratch
    assert lib.sr_loss_l1_dssim(C.byref(p), ok, ok, ok, C.c_float(1.5), ok, ok, None, ok, None) == N.SR_ERR_INVALID
    assert lib.sr_loss_l1_dssim(C.byref(p), ok, None, ok, C.c_float(0.2), ok, ok, None, ok, None) == N.SR_ERR_INVALID
    assert lib.sr_loss_l1_dssim(C.byref(p), ok, ok, ok, C.c_float(0.2), ok, ok, None, C.c_void_p(4096 + 16),
                                None) == N.SR_ERR_INVALID
    g = N.sr_adam_group()
    g.param = g.grad = g.m = g.v = 4096
    g.n, g.lr, g.lr_rest = 10, 1e-3, 1e-3
    arr = (N.sr_adam_group * 1)(g)
    assert lib.sr_adam_step(arr, 0, 1, C.c_float(0.9), C.c_float(0.999), C.c_float(1e-15), None) == N.SR_ERR_INVALID
    assert lib.sr_adam_step(arr, 17, 1, C.c_float(0.9), C.c_float(0.999), C.c_float(1e-15), None) == N.SR_ERR_INVALID
    assert lib.sr_adam_step(arr, 1, 0, C.c_float(0.9), C.c_float(0.999), C.c_float(1e-15), None) == N.SR_ERR_INVALID
    assert lib.sr_adam_step(arr, 1, 1, C.c_float(1.0), C.c_float(0.999), C.c_float(1e-15), None) == N.SR_ERR_INVALID
    assert lib.sr_adam_step(arr, 1, 1, C.c_float(0.9), C.c_float(0.999), C.c_float(0.0), None) == N.SR_ERR_INVALID
    g.grad = None
    arr = (N.sr_adam_group * 1)(g)
    assert lib.sr_adam_step(arr, 1, 1, C.c_float(0.9), C.c_float(0.999), C.c_float(1e-15), None) == N.SR_ERR_INVALID


def test_densify_calls_reject_invalid_arguments_without_device_work(lib):
    g = _desc(100, deg=1)
    for f in ("means", "log_scales", "quats", "opacity_logits", "skew", "sh"):
        setattr(g, f, 4096)
    ok = C.c_void_p(4096)
    cfg = N.sr_densify_config(0.1, 0.1, -3.0, -2.0)
    out = N.sr_scene_arrays()
    for f in ("means", "log_scales", "quats", "opacity_logits", "skew", "sh"):
        setattr(out, f, 8192)
    assert lib.sr_densify_scratch_size(C.c_int64(100)) >= 16
    call = lambda gg, oo, cc=cfg: lib.sr_densify(C.byref(gg), ok, ok, ok, C.byref(cc), C.byref(oo), None, ok, ok, None)
    g.dt_sh = N.SR_BF16  # FP32 attributes only
    assert call(g, out) == N.SR_ERR_INVALID
    g.dt_sh = N.SR_F32
    g.n = 1 << 30  # source indices must fit in 30 bits
    assert call(g, out) == N.SR_ERR_INVALID
    g.n = 100
    out.sh = None
    assert call(g, out) == N.SR_ERR_INVALID
    out.sh = 8192
    out.split_dir = 8192  # an output split direction without an input one
    assert call(g, out) == N.SR_ERR_INVALID
    out.split_dir = None
    out.quats = 8192 + 4  # read and written as float4
    assert call(g, out) == N.SR_ERR_INVALID
    assert lib.sr_densify(C.byref(g), ok, ok, ok, None, C.byref(out), None, ok, ok, None) == N.SR_ERR_INVALID
    assert lib.sr_densify_remap(ok, -1, ok, ok, 10, ok, None) == N.SR_ERR_INVALID
    assert lib.sr_densify_remap(None, 3, ok, ok, 10, ok, None) == N.SR_ERR_INVALID


def test_autotune_keeps_the_default_within_the_margin():
    from paper_2605_18334_gb300.rasterizer import _prefer_default

    # the default stays unless another candidate is more than 2% faster
    assert _prefer_default({128: 0.456, 256: 0.4475}, 128) == 128
    assert _prefer_default({128: 0.456, 256: 0.440}, 128) == 256
    # ties and a faster default
    assert _prefer_default({128: 0.5, 256: 0.5}, 256) == 256
    assert _prefer_default({1: 0.76, 2: 0.58, 4: 0.64}, 2) == 2
    # a default that was not timed: the fastest candidate
    assert _prefer_default({1: 0.76, 4: 0.64}, 2) == 4
    assert _prefer_default({128: 0.456, 256: 0.4475}, 128, margin=0.0) == 256


def test_recompute_keys_plan_keeps_no_blend_masks_and_excludes_forward_only(lib):
    from paper_2605_18334_gb300.rasterizer import Config

    g = N.sr_gaussians()
    g.n, g.sh_degree = 1000, 3
    cam = N.sr_camera()
    cam.width, cam.height = 640, 360
    base = N.sr_plan_init(Config().to_c(), g, [cam], 1 << 16)
    rk = N.sr_plan_init(Config(recompute_keys=True).to_c(), g, [cam], 1 << 16)
    assert rk.recompute_keys == 1 and base.recompute_keys == 0
    assert rk.ws_bytes < base.ws_bytes
    with pytest.raises(N.SkewRasterError) as e:
        N.sr_plan_init(Config(recompute_keys=True, forward_only=True).to_c(), g, [cam], 1 << 16)
    assert e.value.status == N.SR_ERR_INVALID
