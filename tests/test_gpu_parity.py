"""Parity of the CUDA path (called through the C ABI) with the FP64 oracle.

Bars (design notes): depth keys, tile counts and the sorted key list
bit-exact, except for Gaussians whose FP64 tile edge lies within TOL_PX of a
pixel-centre boundary, whose tile sets are counted and checked for validity
instead; every pixel's image within 1e-4 max abs per channel of the oracle
replaying the GPU's own gate and stop decisions, each of which must agree
with FP64's or lie within the stated tolerance of its threshold (no pixel is
excluded); gradients within 1e-3 relative error per tensor and, element by
element, within 1e-2 of the oracle's rounding-error scale (the sum of the
magnitudes of the element's terms) plus the terms whose clamp decision is
within tolerance.
"""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2605_18334_gb300 import native as N
from paper_2605_18334_gb300 import scenes
from paper_2605_18334_gb300.rasterizer import Config, Gaussians, Rasterizer
from tests.parity_util import (ELEM_RTOL, GRAD_RTOL, IMG_ATOL, check_ambiguous_tile_sets, check_key_order, compare_grads_elementwise,
                               compare_keys, dequantised, gpu_blend_lists, gpu_records_to_oracle_layout,
                               oracle_config, rel_err)

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - CPU-only container
    pytest.skip("needs a CUDA GPU", allow_module_level=True)


def gpu_forward(scene, cams, cfg=None, key_capacity=None, **dtypes):
    cfg = cfg or Config()
    g = Gaussians.from_scene(scene, **dtypes)
    r = Rasterizer(g, cams, cfg, key_capacity=key_capacity)
    r.forward(g)
    torch.cuda.synchronize()
    return r, g


def check_view(r, scene, cams, v, cfg, check_keys=True, label=""):
    """Compare view v of the GPU frame with the oracle: every Gaussian's depth
    key, tile count and record, every key of the sorted list, and every pixel.

    Gaussians whose FP64 tile set is ambiguous (an edge within TOL_PX of a
    pixel-centre boundary, or the cull within tolerance) are counted; their
    tile counts and keys are checked for validity (every tile where the FP64
    alpha clears alpha_min (1 + TOL_ALPHA) present, none outside the FP64
    box widened by TOL_PX) and all others bit for bit.  The image, T and the
    blend lists are compared at every pixel against the oracle replaying the
    GPU's own gate and stop decisions (read from its blend masks), each of
    which must agree with FP64's or lie within tolerance of its threshold.
    Returns the counters (also printed)."""
    cam = cams[v]
    oc = oracle.camera_from_gl(cam)
    ocfg = oracle_config(cfg)
    pre = oracle.preprocess(scene, oc, ocfg)
    n = scene.n
    p = r.plan
    stats = {}
    # depth keys and tile counts
    depth = r.depth_bits().cpu().numpy().view(np.uint32)[v * n:(v + 1) * n]
    np.testing.assert_array_equal(depth, pre["depth_bits"])
    cnt = r.tile_counts().cpu().numpy()[v * n:(v + 1) * n]
    or_cnt = np.where(pre["visible"], pre["ntouch"], 0)
    amb = pre["rect_ambig"]
    np.testing.assert_array_equal(cnt[~amb], or_cnt[~amb])
    stats["touching"] = int(((cnt > 0) | (or_cnt > 0)).sum())
    stats["rect_ambiguous"] = int(amb.sum())
    # records of the rendered Gaussians
    sel = np.nonzero((cnt > 0) & ~amb)[0]
    g = gpu_records_to_oracle_layout(r.records().cpu().numpy()[v * n:(v + 1) * n][sel])
    o = pre["rec"][sel]
    if sel.size:
        stats["mu2_max_abs_err_px"] = float(max(np.abs(g["mx"] - o[:, 0]).max(), np.abs(g["my"] - o[:, 1]).max()))
    np.testing.assert_allclose(g["mx"], o[:, 0], atol=2e-3, rtol=1e-6)
    np.testing.assert_allclose(g["my"], o[:, 1], atol=2e-3, rtol=1e-6)
    for k, col in (("a", 2), ("b", 3), ("c", 4)):
        scale = np.maximum(np.abs(o[:, 2]), np.abs(o[:, 4]))
        assert np.all(np.abs(g[k] - o[:, col]) <= 2e-4 * scale + 1e-9), k
    bscale = np.maximum(1.0, np.hypot(o[:, 5], o[:, 6]))
    assert np.all(np.abs(g["bx"] - o[:, 5]) <= 1e-3 * bscale)
    assert np.all(np.abs(g["by"] - o[:, 6]) <= 1e-3 * bscale)
    np.testing.assert_allclose(g["m"], o[:, 7], atol=2e-6, rtol=1e-4)
    np.testing.assert_allclose(g["h"], o[:, 8], atol=2e-6, rtol=1e-4)
    np.testing.assert_allclose(g["rgb"], o[:, 11:14], atol=2e-5, rtol=1e-5)
    # sorted keys: order, bit-exact list of the unambiguous Gaussians, valid
    # tile sets of the ambiguous ones
    keys, vals = r.sorted_keys()
    keys = keys.cpu().numpy().view(np.uint64)
    vals = vals.cpu().numpy().astype(np.int64)
    tb = int(p.tile_base[v]), int(p.tile_base[v + 1])
    sel_k = ((keys >> np.uint64(32)) >= tb[0]) & ((keys >> np.uint64(32)) < tb[1])
    if check_keys:
        check_key_order(keys[sel_k], vals[sel_k])
        ok, ov = oracle.bin_keys(pre, oc, ocfg, tile_base=tb[0], val_base=v * n)
        amb_ids = np.nonzero(amb)[0]
        compare_keys(keys[sel_k], vals[sel_k], ok, ov, amb_ids + v * n)
        stats["keys"] = int(sel_k.sum())
        stats["keys_of_ambiguous"] = int(np.isin(vals[sel_k] - v * n, amb_ids).sum())
        stats["ambiguous_tile_sets_checked"] = check_ambiguous_tile_sets(
            keys[sel_k], vals[sel_k], pre, amb_ids, pre["rec"], oc, ocfg, v * n, tb[0], oracle.TOL_ALPHA,
            oracle.TOL_PX)
        for i in amb_ids:
            assert cnt[i] == int((vals[sel_k] == i + v * n).sum())
    # every pixel, under the GPU's own gate and stop decisions
    lists = gpu_blend_lists(r, v)
    rep = oracle.render_frame(scene, oc, ocfg, pre=pre, gpu_lists=lists)
    st = rep["stats"]
    assert st["inadmissible_pixels"] == 0, (st, np.argwhere(rep["status"] != 0)[:8])
    img = r.view_image(r.images, v).cpu().numpy()
    T = r.view_state(r.t_final, v).cpu().numpy()
    d = np.abs(np.transpose(img, (1, 2, 0)).astype(np.float64) - rep["rgb"])
    stats["img_max_abs"] = float(d.max()) if d.size else 0.0
    dT = np.abs(T.astype(np.float64) - rep["T"])
    stats["T_max_abs"] = float(dT.max()) if dT.size else 0.0
    stats["T_max_rel"] = float((dT / np.maximum(rep["T"], 1e-30)).max()) if dT.size else 0.0
    stats["pixels"] = int(T.size)
    stats["pixels_excluded"] = 0
    for k in ("flipped_pixels", "flipped_gate", "flipped_stop", "max_gate_margin", "max_stop_margin",
              "ambiguous_pixels"):
        stats[k] = st[k]
    stats["blends"] = int(lists[1].size)
    print(f"parity {label or 'view'} v{v}: " + " ".join(f"{k}={val:.3g}" if isinstance(val, float) else f"{k}={val}"
                                                   for k, val in stats.items()))
    assert stats["img_max_abs"] <= IMG_ATOL, stats
    assert stats["T_max_abs"] <= 1e-4, stats
    return stats, pre, rep


# ---------------------------------------------------------------------------
# forward
# ---------------------------------------------------------------------------

def test_cube_1k_64px_full_frame():
    """1,000 skew Gaussians, 64x64 view, SH degree 0 (small workload)."""
    sc = scenes.cube_1k()
    cams = [scenes.identity_camera(64, 64)]
    r, _ = gpu_forward(sc, cams)
    stats, _, _ = check_view(r, sc, cams, 0, Config())
    assert stats["keys"] > 1000


@pytest.mark.parametrize("W,H", [(37, 23), (16, 16), (1, 1), (95, 200)])
def test_ragged_image_sizes(W, H):
    sc = scenes.cube_1k(seed=3, n=600)
    cams = [scenes.identity_camera(W, H)]
    r, _ = gpu_forward(sc, cams)
    check_view(r, sc, cams, 0, Config())


def test_cluster_100k_720p_full_frame():
    """100k Gaussians, SH degree 3, 1280x720: every key and every pixel."""
    sc = scenes.cluster()
    cams = [scenes.identity_camera(1280, 720)]
    r, _ = gpu_forward(sc, cams)
    stats, _, _ = check_view(r, sc, cams, 0, Config(), label="cluster_100k_720p")
    assert stats["keys"] > 100_000


@pytest.mark.parametrize("two,split", [(True, False), (True, True), (False, True)])
def test_enhanced_opacity_modes(two, split):
    sc = scenes.cluster(seed=5, n=3000, sh_degree=2, two_opacities=two, split=split)
    cams = [scenes.identity_camera(160, 120)]
    r, _ = gpu_forward(sc, cams)
    check_view(r, sc, cams, 0, Config())


def test_background_and_config_variants():
    sc = scenes.cube_1k(seed=8, n=800)
    cams = [scenes.identity_camera(80, 60)]
    cfg = Config(bg=(0.2, 0.5, 0.9), antialias_comp=False, dilation=0.2, alpha_max=0.95, t_stop=1e-3)
    r, _ = gpu_forward(sc, cams, cfg)
    check_view(r, sc, cams, 0, cfg)


@pytest.mark.parametrize("dt", [torch.bfloat16, torch.float16])
def test_reduced_precision_storage_arithmetic_error(dt):
    """SH, log-scales and skew stored in BF16/FP16: against the oracle fed the
    dequantised attributes the FP32 bar holds (arithmetic error)."""
    sc = scenes.cluster(seed=6, n=5000)
    cams = [scenes.identity_camera(200, 150)]
    r, _ = gpu_forward(sc, cams, sh_dtype=dt, scale_dtype=dt, skew_dtype=dt)
    check_view(r, dequantised(sc, dt, dt, dt), cams, 0, Config())


def test_multi_view_batched_frame():
    """Several views of mixed resolution in one plan: shared key pool, one
    composite launch over all tiles."""
    sc = scenes.unbounded(seed=7, n=20_000)
    cams = scenes.trajectory_cameras(5, resolutions=((64, 36), (128, 72), (96, 96)))
    r, _ = gpu_forward(sc, cams)
    for v in range(len(cams)):
        check_view(r, sc, cams, v, Config())


def test_zero_skew_binning_equals_symmetric_footprint():
    """Gaussians with skew exactly 0 get kappa = 1, so their tile sets are
    those of the plain 3DGS footprint rho^2 = 2 ln(o comp / tau)(1 + 2^-10)
    (computed here independently in FP64); GPU keys match bit for bit."""
    sc = scenes.unbounded(seed=4, n=20_000, skew_sigma=2.0, zero_skew_fraction=0.5)
    cams = [scenes.orbit_camera(0.4, 320, 180)]
    r, _ = gpu_forward(sc, cams)
    stats, pre, _ = check_view(r, sc, cams, 0, Config())
    zero = np.all(sc.skew == 0, axis=1) & pre["visible"]
    rec = pre["rec"]
    tau = np.float32(1 / 255)
    omax = rec[:, 14] * np.maximum(rec[:, 15], rec[:, 16])
    on = zero & (omax >= tau)
    rho2 = 2 * np.log(omax[on] / tau) * (1 + 2 ** -10)
    np.testing.assert_allclose(pre["ext"][on, 2], rho2, rtol=1e-12)


def test_empty_and_fully_culled_scenes():
    sc = scenes.cube_1k(seed=1, n=50)
    cams = [scenes.identity_camera(48, 32)]
    # all behind the camera
    sc.means[:, 2] = -3.0
    r, _ = gpu_forward(sc, cams, cfg=Config(bg=(0.1, 0.2, 0.3)))
    img = r.view_image(r.images, 0).cpu().numpy()
    assert r.keys == 0
    np.testing.assert_allclose(img, np.broadcast_to(np.float32([0.1, 0.2, 0.3])[:, None, None], img.shape))
    # no Gaussians at all
    sc0 = sc.subset(np.arange(0))
    r0, _ = gpu_forward(sc0, cams)
    assert r0.keys == 0
    assert float(r0.view_image(r0.images, 0).abs().max()) == 0.0


def test_capacity_overflow_reports_and_recovers():
    from paper_2605_18334_gb300 import native as N

    sc = scenes.cube_1k()
    cams = [scenes.identity_camera(64, 64)]
    g = Gaussians.from_scene(sc)
    r = Rasterizer(g, cams, Config(), key_capacity=100)
    r.preprocess(g)
    with pytest.raises(N.SkewRasterError) as e:
        r.bin_sort()
    assert e.value.status == N.SR_ERR_CAPACITY and e.value.keys_needed > 100
    r.forward(g)  # grows the plan and retries
    assert r.key_capacity >= e.value.keys_needed
    check_view(r, sc, cams, 0, Config())


def test_graph_captured_frame_matches_eager():
    """The non-blocking bin/sort (no key-count read-back) inside a CUDA graph
    gives the eager frame's image bit for bit."""
    sc = scenes.cluster(seed=2, n=20_000)
    cams = [scenes.identity_camera(256, 144)]
    g = Gaussians.from_scene(sc)
    r = Rasterizer(g, cams, Config(), key_capacity=1 << 20)
    r.forward(g)
    torch.cuda.synchronize()
    eager = r.images.clone()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        r.preprocess(g, s)
        r.bin_sort(s, sync=False)
        r.render_fwd(s)
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=s):
        r.preprocess(g, s)
        r.bin_sort(s, sync=False)
        r.render_fwd(s)
    r.images.zero_()
    graph.replay()
    torch.cuda.synchronize()
    assert torch.equal(r.images, eager)


def test_graph_captured_mixed_resolution_trajectory_against_oracle():
    """A five-view trajectory of three image sizes in one plan, captured as a
    CUDA graph (non-blocking bin/sort) and replayed: every view's keys and
    every pixel against the oracle."""
    sc = scenes.unbounded(seed=23, n=30_000)
    cams = scenes.trajectory_cameras(5, resolutions=((160, 90), (320, 180), (240, 240)))
    g = Gaussians.from_scene(sc)
    r = Rasterizer(g, cams, Config())
    r.forward(g)  # sizes the key pool
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        r.preprocess(g, s)
        r.bin_sort(s, sync=False)
        r.render_fwd(s)
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=s):
        r.preprocess(g, s)
        r.bin_sort(s, sync=False)
        r.render_fwd(s)
    r.images.zero_()
    graph.replay()
    torch.cuda.synchronize()
    r.keys = r.check()
    sizes = set()
    for v, cam in enumerate(cams):
        check_view(r, sc, cams, v, Config(), label="graph_trajectory")
        sizes.add((cam["width"], cam["height"]))
    assert len(sizes) == 3


# ---------------------------------------------------------------------------
# backward
# ---------------------------------------------------------------------------

GRAD_FIELDS = ["means", "log_scales", "quats", "opacity_logits", "skew", "sh"]


def compare_grads(gr, og, fields, rtol=GRAD_RTOL, label=""):
    """Per tensor: ||g - g_ref|| / ||g_ref|| <= rtol; with the oracle's
    bounds (``scale``/``slack``), also element by element (see
    compare_grads_elementwise).  Prints both."""
    errs = {k: rel_err(gr[k].detach().cpu().numpy().astype(np.float64), og[k]) for k in fields}
    msg = " ".join(f"{k}={e:.2e}" for k, e in errs.items())
    if "scale" in og:
        el = compare_grads_elementwise(gr, og, fields)
        msg += " | per element (worst bound ratio, share within 1e-3 rel): " + " ".join(
            f"{k}=({w:.2f},{s:.4f})" for k, (w, s, _) in el.items())
    print(f"grads {label}: {msg}")
    assert all(e <= rtol for e in errs.values()), errs
    return errs


def oracle_grads(r, sc, cams, cfg, ups):
    """The oracle's gradients of sum_v <ups[v], image_v>, replaying the GPU's
    gate and stop decisions in every view, with element-wise bounds."""
    tot = None
    for v, c in enumerate(cams):
        og = oracle.render_backward(sc, oracle.camera_from_gl(c), oracle_config(cfg), ups[v], frame=True,
                                    gpu_lists=gpu_blend_lists(r, v), bounds=True)
        assert og["inadmissible_pixels"] == 0
        if tot is None:
            tot = og
            continue
        for k, val in og.items():
            if isinstance(val, dict):
                for kk, vv in val.items():
                    if vv is not None:
                        tot[k][kk] = tot[k][kk] + vv
            elif isinstance(val, np.ndarray):
                tot[k] = tot[k] + val
    return tot


def test_backward_fd_crop_2k():
    """2k Gaussians projecting near a 32x32 crop of the 1280x720 view, full
    upstream gradient N(0,1): every attribute gradient within 1e-3."""
    sc, cam = scenes.fd_crop_scene()
    cams = [cam]
    r, g = gpu_forward(sc, cams)
    up = scenes.upstream_grad(3, 32, 32)
    gr = r.backward(g, torch.as_tensor(up).cuda().reshape(-1).contiguous())
    og = oracle_grads(r, sc, cams, Config(), [up])
    compare_grads(gr, og, GRAD_FIELDS, label="fd_crop_2k")
    # 2D gradients of the records too, per column and element by element
    d2 = r.d2().cpu().numpy()
    cnt = r.tile_counts().cpu().numpy() > 0
    o2, s2, l2 = og["d2"], og["scale"]["d2"], og["slack"]["d2"]
    for col in (0, 1, 2, 3, 4, 5, 6, 7, 11, 12, 13):
        assert rel_err(d2[cnt, col], o2[cnt, col]) <= GRAD_RTOL, col
        assert np.all(np.abs(d2[cnt, col] - o2[cnt, col]) <= ELEM_RTOL * s2[cnt, col] + l2[cnt, col] + 1e-30), col


@pytest.mark.parametrize("two,split,deg", [(True, False, 1), (True, True, 3), (False, False, 0)])
def test_backward_modes(two, split, deg):
    sc = scenes.cluster(seed=9, n=1500, sh_degree=deg, two_opacities=two, split=split)
    cams = [scenes.identity_camera(96, 72)]
    cfg = Config(bg=(0.3, 0.2, 0.1))
    r, g = gpu_forward(sc, cams, cfg=cfg)
    up = scenes.upstream_grad(9, 72, 96)
    gr = r.backward(g, torch.as_tensor(up).cuda().reshape(-1).contiguous())
    og = oracle_grads(r, sc, cams, cfg, [up])
    compare_grads(gr, og, GRAD_FIELDS + (["split_dir"] if split else []), label=f"modes {two} {split} {deg}")


def test_backward_cluster_100k_dense_upstream():
    """Full 100k / 720p frame with an upstream gradient N(0,1) at every pixel
    and channel: every gradient element within its bound."""
    sc = scenes.cluster()
    cams = [scenes.identity_camera(1280, 720)]
    r, g = gpu_forward(sc, cams)
    up = scenes.upstream_grad(1, 720, 1280)
    gr = r.backward(g, torch.as_tensor(up).cuda().reshape(-1).contiguous())
    og = oracle_grads(r, sc, cams, Config(), [up])
    compare_grads(gr, og, GRAD_FIELDS, label="cluster_100k_720p")


def test_4k_view_of_the_mixed_scene_law_full_frame_and_backward():
    """One 3840x2160 view (32,400 tiles: two tile-id passes and the
    many-tile composite order) of 200k Gaussians of the 5M scene's law (half
    the skew vectors exactly zero): every key and every pixel against the
    oracle, then an upstream gradient at every pixel and channel with every
    gradient element within its bound."""
    sc = scenes.unbounded(seed=5, n=200_000, skew_sigma=2.0, zero_skew_fraction=0.5)
    cams = scenes.trajectory_cameras(32, resolutions=((3840, 2160),))[:1]
    r, g = gpu_forward(sc, cams)
    assert int(r.plan.total_tiles) == 240 * 135
    check_tile_order(r)
    check_view(r, sc, cams, 0, Config(), label="mixed_law_200k_4k")
    up = scenes.upstream_grad(9, 2160, 3840)
    gr = r.backward(g, torch.as_tensor(up).cuda().reshape(-1).contiguous())
    og = oracle_grads(r, sc, cams, Config(), [up])
    compare_grads(gr, og, GRAD_FIELDS, label="mixed_law_200k_4k")


def test_backward_batched_views_sum():
    """Gradients of a multi-view plan are the sum over views."""
    sc = scenes.cluster(seed=12, n=3000, sh_degree=1)
    cams = [scenes.identity_camera(64, 48), scenes.camera(scenes.look_at_c2w_cv((0.5, -0.2, 0.5), (0, 0, 4)), 80, 40)]
    r, g = gpu_forward(sc, cams)
    ups = [scenes.upstream_grad(20 + v, c["height"], c["width"]) for v, c in enumerate(cams)]
    flat = torch.as_tensor(np.concatenate([u.reshape(-1) for u in ups])).cuda().contiguous()
    gr = r.backward(g, flat)
    compare_grads(gr, oracle_grads(r, sc, cams, Config(), ups), GRAD_FIELDS, label="two views")


@pytest.mark.parametrize("px,fb,bb,pers", [(1, 128, 128, 0), (2, 256, 256, 0), (4, 512, 128, 3), (2, 512, 128, 0),
                                           (1, 0, 0, 0), (2, 256, 128, 3), (1, 128, 256, 1), (4, 256, 256, 2)])
def test_pixels_per_thread_launch_shapes(px, fb, bb, pers):
    """Every launch shape of the composites (pixels per thread, records per
    staged batch, one block per tile or a persistent grid) gives the oracle's
    image and gradients (the autotuner only changes speed)."""
    sc = scenes.cluster(seed=31, n=4000, sh_degree=1, two_opacities=True)
    cams = [scenes.identity_camera(100, 70)]
    cfg = Config(fwd_pixels_per_thread=px, bwd_pixels_per_thread=px, fwd_batch=fb, bwd_batch=bb,
                 bg=(0.1, 0.0, 0.2), persistent=pers)
    r, g = gpu_forward(sc, cams, cfg)
    check_view(r, sc, cams, 0, cfg, label=f"shape {px} {fb} {bb} {pers}")
    up = scenes.upstream_grad(31, 70, 100)
    gr = r.backward(g, torch.as_tensor(up).cuda().reshape(-1).contiguous())
    compare_grads(gr, oracle_grads(r, sc, cams, cfg, [up]), GRAD_FIELDS, label=f"shape {px} {fb} {bb} {pers}")


def test_autotune_picks_a_shape_and_keeps_results():
    sc = scenes.cluster(seed=32, n=20_000)
    cams = [scenes.identity_camera(256, 192)]
    r, g = gpu_forward(sc, cams)
    ref = r.images.clone()
    up = torch.as_tensor(scenes.upstream_grad(32, 192, 256)).cuda().reshape(-1).contiguous()
    ref_g = r.backward(g, up)["means"].clone()
    res = r.autotune(g, up)
    assert res["fwd_pixels_per_thread"] in (1, 2, 4) and res["bwd_pixels_per_thread"] in (1, 2, 4)
    assert res["fwd_batch"] in (128, 256, 512) and res["bwd_batch"] in (128, 256)
    assert res["fwd_persistent"] in (False, True) and res["bwd_persistent"] in (False, True)
    r.forward(g)
    assert torch.equal(r.images, ref)
    gm = r.backward(g, up)["means"]
    assert rel_err(gm.cpu().numpy(), ref_g.cpu().numpy()) < 1e-5


def test_densification_statistics_match_oracle():
    """Per-Gaussian |dL/dmu_2| (the 2D positional statistic g^(uv)) and the
    depth gradient dL/dz of the centre along the camera axis (Eq. depth_grad,
    one iteration), against the oracle's 2D and world-space gradients."""
    sc = scenes.cluster(seed=33, n=3000, sh_degree=2)
    cams = [scenes.camera(scenes.look_at_c2w_cv((0.3, -0.2, -0.5), (0, 0, 4)), 120, 90)]
    r, g = gpu_forward(sc, cams)
    up = scenes.upstream_grad(33, 90, 120)
    gr = r.backward(g, torch.as_tensor(up).cuda().reshape(-1).contiguous(), want_stats=True)
    oc = oracle.camera_from_gl(cams[0])
    og = oracle_grads(r, sc, cams, Config(), [up])
    uv = np.hypot(og["d2"][:, 0], og["d2"][:, 1])
    assert rel_err(gr["means2d_abs"].cpu().numpy(), uv) <= GRAD_RTOL
    W = oracle.camera_fields(oc)["w2c"].reshape(3, 4)[:, :3]
    dz = og["means"] @ W[2]
    assert rel_err(gr["depth_grad"].cpu().numpy(), dz) <= GRAD_RTOL


@pytest.mark.parametrize("dt,bound", [(torch.bfloat16, 0.03), (torch.float16, 0.02)])
def test_reduced_precision_storage_error_against_fp32_originals(dt, bound):
    """Storage error: the GPU renders from BF16/FP16 SH, log-scales and skew,
    the oracle from the FP32 originals (its own decisions, every pixel).  The
    stated bound is a max abs error per channel of 0.03 (BF16) / 0.02 (FP16),
    the bound of the full-size workloads (tests/test_gpu_precision.py)."""
    sc = scenes.cluster(seed=6, n=5000)
    cams = [scenes.identity_camera(200, 150)]
    r, _ = gpu_forward(sc, cams, sh_dtype=dt, scale_dtype=dt, skew_dtype=dt)
    out = oracle.render_frame(sc, oracle.camera_from_gl(cams[0]), oracle_config(Config()))
    img = r.view_image(r.images, 0).cpu().numpy()
    d = np.abs(np.transpose(img, (1, 2, 0)) - out["rgb"])
    print(f"storage error {dt}: max {d.max():.3e} mean {d.mean():.3e}")
    assert d.max() <= bound


def test_forward_only_plan_renders_the_same_and_refuses_backward():
    from paper_2605_18334_gb300 import native as N

    sc = scenes.cluster(seed=34, n=8000)
    cams = [scenes.identity_camera(160, 96), scenes.identity_camera(64, 64)]
    r, g = gpu_forward(sc, cams)
    r_fo, _ = gpu_forward(sc, cams, Config(forward_only=True))
    assert r_fo.plan.ws_bytes < r.plan.ws_bytes
    assert torch.equal(r.images, r_fo.images)
    up = torch.zeros_like(r_fo.images)
    with pytest.raises(N.SkewRasterError) as e:
        r_fo.backward(g, up)
    assert e.value.status == N.SR_ERR_UNSUPPORTED


def test_autograd_function():
    from paper_2605_18334_gb300.rasterizer import render

    sc = scenes.cube_1k(seed=2, n=500)
    cams = [scenes.identity_camera(48, 48)]
    g = Gaussians.from_scene(sc)
    r = Rasterizer(g, cams, Config())
    leaves = [t.clone().requires_grad_(True) for t in (g.means, g.log_scales, g.quats, g.opacity_logits, g.skew, g.sh)]
    img = render(r, *leaves[:5], leaves[5], sh_degree=0)
    up = torch.as_tensor(scenes.upstream_grad(4, 48, 48)).cuda().reshape(-1)
    (img * up).sum().backward()
    og = oracle_grads(r, sc, cams, Config(), [scenes.upstream_grad(4, 48, 48)])
    compare_grads({k: t.grad for t, k in zip(leaves, GRAD_FIELDS)}, og, GRAD_FIELDS, label="autograd")


def test_recompute_keys_matches_batched_plan():
    """Several views rendered with the tile key lists rebuilt for the
    backward (one workspace per image size) give the batched plan's images
    and gradients."""
    from paper_2605_18334_gb300.rasterizer import render_views_recompute

    sc = scenes.cluster(seed=35, n=6000, sh_degree=1)
    cams = scenes.trajectory_cameras(4, resolutions=((96, 64), (64, 48)))
    cams = [dict(c, c2w_gl=scenes.camera(scenes.look_at_c2w_cv(e, (0, 0, 4)), c["width"], c["height"])["c2w_gl"])
            for c, e in zip(cams, [(0.3, -0.1, 0.0), (-0.4, 0.2, 0.5), (0.1, 0.3, -0.3), (0.0, 0.0, 0.2)])]
    r, g = gpu_forward(sc, cams)
    ups = [torch.as_tensor(scenes.upstream_grad(50 + v, c["height"], c["width"])).cuda() for v, c in enumerate(cams)]
    flat = torch.cat([u.reshape(-1) for u in ups]).contiguous()
    ref = r.backward(g, flat)
    imgs, tot = render_views_recompute(g, cams, ups)
    for v in range(len(cams)):
        assert torch.equal(imgs[v], r.view_image(r.images, v))
    for k in GRAD_FIELDS:
        assert rel_err(tot[k].cpu().numpy(), ref[k].cpu().numpy()) < 1e-5, k


def test_recompute_keys_plan_matches_mask_plan_and_oracle():
    """A recompute_keys plan (no blend masks; sr_render_bwd rebuilds the
    records and key lists and replays with the alpha gate) gives the mask
    plan's images and, within FP32 atomics' reordering, its gradients; both
    against the oracle replaying the same decisions."""
    sc = scenes.cluster(seed=36, n=6000, sh_degree=2, two_opacities=True, split=True)
    cams = [scenes.identity_camera(96, 64), scenes.camera(scenes.look_at_c2w_cv((0.4, -0.2, 0.3), (0, 0, 4)), 80, 72)]
    cfg = Config(bg=(0.1, 0.2, 0.0))
    r, g = gpu_forward(sc, cams, cfg)
    rr, _ = gpu_forward(sc, cams, Config(bg=(0.1, 0.2, 0.0), recompute_keys=True))
    assert rr.plan.ws_bytes < r.plan.ws_bytes
    assert torch.equal(rr.images, r.images)
    ups = [scenes.upstream_grad(70 + v, c["height"], c["width"]) for v, c in enumerate(cams)]
    flat = torch.as_tensor(np.concatenate([u.reshape(-1) for u in ups])).cuda().contiguous()
    ref = r.backward(g, flat)
    got = rr.backward(g, flat)
    fields = GRAD_FIELDS + ["split_dir"]
    for k in fields:
        assert rel_err(got[k].cpu().numpy(), ref[k].cpu().numpy()) < 1e-5, k
    compare_grads(got, oracle_grads(r, sc, cams, cfg, ups), fields, label="recompute_keys")


def test_recompute_keys_backward_after_the_workspace_served_another_frame():
    """Render view A, keep its frame state, render view B through the same
    recompute_keys workspace, then differentiate view A: the gradients are
    those of A's own backward right after its forward."""
    sc = scenes.cluster(seed=38, n=5000, sh_degree=1)
    cam_a = scenes.identity_camera(96, 72)
    cam_b = scenes.camera(scenes.look_at_c2w_cv((0.5, 0.2, 0.4), (0, 0, 4)), 96, 72)
    g = Gaussians.from_scene(sc)
    r = Rasterizer(g, [cam_a], Config(recompute_keys=True))
    up = torch.as_tensor(scenes.upstream_grad(38, 72, 96)).cuda().reshape(-1).contiguous()
    r.forward(g)
    direct = {k: v.clone() for k, v in r.backward(g, up).items() if v is not None}
    r.forward(g)
    st = r.frame_state()
    r.set_cameras([cam_b])
    r.forward(g)
    late = r.backward(g, up, state=st)
    for k in GRAD_FIELDS:
        assert rel_err(late[k].cpu().numpy(), direct[k].cpu().numpy()) < 1e-6, k


def test_autograd_with_recompute_keys_and_two_renders_before_backward():
    """Two differentiable renders of different views through one
    recompute_keys rasterizer, one backward of their summed loss: each leaf's
    gradient is the sum of the two views' gradients from mask plans."""
    from paper_2605_18334_gb300.rasterizer import render

    sc = scenes.cluster(seed=39, n=3000, sh_degree=1)
    cams = [scenes.identity_camera(64, 48), scenes.camera(scenes.look_at_c2w_cv((-0.4, 0.1, 0.3), (0, 0, 4)), 64, 48)]
    g = Gaussians.from_scene(sc)
    r = Rasterizer(g, [cams[0]], Config(recompute_keys=True))
    leaves = [t.clone().requires_grad_(True) for t in (g.means, g.log_scales, g.quats, g.opacity_logits, g.skew, g.sh)]
    ups = [torch.as_tensor(scenes.upstream_grad(80 + v, 48, 64)).cuda().reshape(-1) for v in range(2)]
    img0 = render(r, *leaves[:5], leaves[5], sh_degree=1)
    r.set_cameras([cams[1]])
    img1 = render(r, *leaves[:5], leaves[5], sh_degree=1)
    ((img0 * ups[0]).sum() + (img1 * ups[1]).sum()).backward()
    ref = None
    for v in range(2):
        rv, gv = gpu_forward(sc, [cams[v]])
        gr = rv.backward(gv, ups[v].contiguous())
        ref = gr if ref is None else {k: (ref[k] + gr[k] if gr[k] is not None else None) for k in gr}
    for t, k in zip(leaves, GRAD_FIELDS):
        assert rel_err(t.grad.cpu().numpy(), ref[k].cpu().numpy()) < 1e-5, k


def test_unbounded_1m_1080p_in_the_bench_launch_configuration():
    """The timed workload at full size (1M skew Gaussians, SH 3, 1920x1080,
    key capacity 12 N, the autotuned launch shapes): depth keys, tile counts
    and records of all 1M Gaussians, the whole sorted key list, every pixel
    of the image and every gradient element of an upstream gradient N(0,1)
    at every pixel, all against the oracle (mode B)."""
    sc = scenes.unbounded(seed=2, n=1_000_000)
    cam = scenes.orbit_camera(0.0, 1920, 1080)
    g = Gaussians.from_scene(sc)
    r = Rasterizer(g, [cam], Config(), key_capacity=12 * sc.n)
    up = scenes.upstream_grad(2, 1080, 1920)
    up_dev = torch.as_tensor(up).cuda().reshape(-1).contiguous()
    r.autotune(g, up_dev)
    r.forward(g)
    torch.cuda.synchronize()
    stats, _, _ = check_view(r, sc, [cam], 0, Config(), label="unbounded_1m_1080p")
    assert stats["keys"] > 5_000_000
    assert stats["rect_ambiguous"] <= 4e-3 * stats["touching"]
    gr = r.backward(g, up_dev)
    compare_grads(gr, oracle_grads(r, sc, [cam], Config(), [up]), GRAD_FIELDS, label="unbounded_1m_1080p")


def order_bucket(length: np.ndarray) -> np.ndarray:
    """Bucket of a key-list length in the composites' tile order: 16 buckets
    per power of two, heaviest first, empty lists last (the rule the order
    kernels implement)."""
    length = np.asarray(length, np.int64)
    e = np.floor(np.log2(np.maximum(length, 1))).astype(np.int64)
    frac = np.where(e >= 4, (length >> np.maximum(e - 4, 0)) & 15, (length << np.maximum(4 - e, 0)) & 15)
    return np.where(length > 0, 16 * (31 - e) + 15 - frac, 16 * 32)


def check_tile_order(r):
    """The composites' tile order is a permutation of every tile, with bucket
    numbers that never decrease along it (heaviest key lists first)."""
    order = r.tile_order().cpu().numpy()
    t = int(r.plan.total_tiles)
    assert np.array_equal(np.sort(order), np.arange(t))
    rng = r.ranges().cpu().numpy()
    b = order_bucket(rng[:, 1] - rng[:, 0])[order]
    assert np.all(np.diff(b) >= 0)
    return b


def test_composite_order_is_a_bucketed_permutation_of_the_tiles():
    """One 1280x720 view (3,600 tiles, the one-block ordering): the order
    holds every tile once, heaviest key lists first; the bucket rule itself
    is checked at the edges of its ranges."""
    assert list(order_bucket([0, 1, 2, 3, 15, 16, 17, 31, 32, 1 << 20])) == [
        512, 16 * 31 + 15, 16 * 30 + 15, 16 * 30 + 7, 16 * 28 + 1, 16 * 27 + 15, 16 * 27 + 14, 16 * 27, 16 * 26 + 15,
        16 * 11 + 15]
    sc = scenes.cluster()
    r, _ = gpu_forward(sc, [scenes.identity_camera(1280, 720)])
    b = check_tile_order(r)
    assert len(np.unique(b)) > 16  # the frame spreads over many buckets


def test_composite_order_over_many_tiles():
    """Nine 1080p views (73,440 tiles, past the one-block ordering of the
    composites' tile order): every view's keys and pixels against the
    oracle, and the order a bucketed permutation of every tile."""
    sc = scenes.unbounded(seed=21, n=3000)
    cams = scenes.trajectory_cameras(9, resolutions=((1920, 1080),))
    r, _ = gpu_forward(sc, cams)
    assert int(r.plan.total_tiles) > 65536
    check_tile_order(r)
    for v in range(len(cams)):
        check_view(r, sc, cams, v, Config(), label="nine_1080p")


def test_persistent_composites_over_many_views_equal_the_block_per_tile_grid():
    """Persistent forward and backward composites over a 12-view plan of
    mixed sizes (far more tiles than resident blocks) give the block-per-tile
    grid's images bit for bit and its gradients within FP32 atomics'
    reordering."""
    sc = scenes.unbounded(seed=24, n=40_000)
    cams = scenes.trajectory_cameras(12, resolutions=((320, 180), (640, 360), (200, 200)))
    r, g = gpu_forward(sc, cams)
    rp, _ = gpu_forward(sc, cams, Config(persistent=3))
    assert torch.equal(rp.images, r.images)
    assert torch.equal(rp.n_contrib, r.n_contrib)
    up = torch.as_tensor(np.concatenate([scenes.upstream_grad(90 + v, c["height"], c["width"]).reshape(-1)
                                         for v, c in enumerate(cams)])).cuda().contiguous()
    ref = r.backward(g, up)
    got = rp.backward(g, up)
    for k in GRAD_FIELDS:
        assert rel_err(got[k].cpu().numpy(), ref[k].cpu().numpy()) < 1e-5, k


@pytest.mark.parametrize("fb,bb", [(3, 5), (1, 1), (8, 9)])
def test_blocks_per_sm_caps_leave_results_unchanged(fb, bb):
    """Capping the composites' resident blocks per SM (shared-memory
    reservation) changes speed only: images bit for bit, gradients within
    FP32 atomics' reordering."""
    sc = scenes.cluster(seed=44, n=6000, sh_degree=1)
    cams = [scenes.identity_camera(160, 120)]
    r, g = gpu_forward(sc, cams)
    rc, _ = gpu_forward(sc, cams, Config(fwd_blocks_per_sm=fb, bwd_blocks_per_sm=bb, persistent=3 if fb == 3 else 0))
    assert torch.equal(rc.images, r.images)
    up = torch.as_tensor(scenes.upstream_grad(44, 120, 160)).cuda().reshape(-1).contiguous()
    ref, got = r.backward(g, up), rc.backward(g, up)
    for k in GRAD_FIELDS:
        assert rel_err(got[k].cpu().numpy(), ref[k].cpu().numpy()) < 1e-5, k


def test_repeated_backward_calls_restart_from_zero():
    """The 2D-gradient records are zeroed by the projection for its frame and
    again by the backward itself when a backward composite has used them
    since: a second backward after one forward, a composite-only call
    followed by a full backward, and a re-render without a new projection
    all give the first backward's gradients."""
    sc = scenes.cluster(seed=35, n=3000, sh_degree=1)
    cams = [scenes.identity_camera(96, 72)]
    r, g = gpu_forward(sc, cams)
    up = torch.as_tensor(scenes.upstream_grad(35, 72, 96)).cuda().reshape(-1).contiguous()
    ref = {k: v.clone() for k, v in r.backward(g, up).items() if v is not None}
    again = r.backward(g, up)
    r.backward_composite(up)
    after_composite = r.backward(g, up)
    r.render_fwd()  # same frame rendered again, no new projection
    rerender = r.backward(g, up)
    for got in (again, after_composite, rerender):
        for k in ("means", "skew", "sh", "opacity_logits"):
            assert rel_err(got[k].cpu().numpy(), ref[k].cpu().numpy()) < 1e-5, k


def test_non_blocking_forward_matches_and_reports_overflow():
    """forward(sync=False) renders the same image without a host round trip,
    and an overflow of the key capacity is reported by check()."""
    sc = scenes.cluster(seed=37, n=4000, sh_degree=1)
    cams = [scenes.identity_camera(96, 72)]
    r, g = gpu_forward(sc, cams)
    ref = r.images.clone()
    keys = r.keys
    r.forward(g, sync=False)
    assert torch.equal(r.images, ref) and r.check() == keys
    small = Rasterizer(g, cams, Config(), key_capacity=max(1, keys // 2))
    small.forward(g, sync=False)
    with pytest.raises(N.SkewRasterError) as e:
        small.check()
    assert e.value.status == N.SR_ERR_CAPACITY and e.value.keys_needed == keys


def test_near_degenerate_splats():
    """Needle- and disc-like Gaussians (one or two axes 10^-4 of the others),
    extreme skew (|eta| up to 40) and centres just beyond the near plane or
    far outside the view: FP32 projection, binning and compositing still
    match the FP64 oracle (binning exactly, images within 1e-4, gradients
    within 1e-3)."""
    rng = np.random.default_rng(41)
    sc = scenes.cluster(seed=41, n=3000, sh_degree=1)
    n = sc.n
    thin = rng.random(n) < 0.4
    axis = rng.integers(0, 3, n)
    ls = sc.log_scales.astype(np.float64)
    ls[thin, axis[thin]] = ls[thin, axis[thin]] - 9.0          # needles / discs
    two = thin & (rng.random(n) < 0.3)
    ls[two, (axis[two] + 1) % 3] -= 9.0
    sc.log_scales[:] = ls.astype(np.float32)
    big = rng.random(n) < 0.05
    sc.skew[big] = (rng.normal(0, 1, (int(big.sum()), 3)) * 20.0).astype(np.float32)
    near = rng.random(n) < 0.02
    sc.means[near, 2] = rng.uniform(0.19, 0.3, int(near.sum())).astype(np.float32)
    cams = [scenes.identity_camera(96, 80)]
    r, g = gpu_forward(sc, cams)
    check_view(r, sc, cams, 0, Config(), label="near_degenerate")
    up = scenes.upstream_grad(41, 80, 96)
    gr = r.backward(g, torch.as_tensor(up).cuda().reshape(-1).contiguous())
    compare_grads(gr, oracle_grads(r, sc, cams, Config(), [up]), GRAD_FIELDS, label="near_degenerate")


def test_maximum_view_count():
    """A plan with the maximum number of views (SR_MAX_VIEWS) of mixed small
    sizes renders every view as its own frame would: spot-checked views
    against the oracle, and all views against single-view plans."""
    sc = scenes.cluster(seed=43, n=2000, sh_degree=0)
    sizes = ((16, 16), (24, 8), (17, 31))
    cams = scenes.trajectory_cameras(N.SR_MAX_VIEWS, radius=4.0, resolutions=sizes)
    r, g = gpu_forward(sc, cams)
    assert r.plan.n_views == N.SR_MAX_VIEWS
    for v in (0, 1, 2, 127, N.SR_MAX_VIEWS - 1):
        check_view(r, sc, cams, v, Config())
    for v in range(0, N.SR_MAX_VIEWS, 17):
        r1, g1 = gpu_forward(sc, [cams[v]])
        assert torch.equal(r.view_image(r.images, v), r1.view_image(r1.images, 0)), v
