"""Error of reduced-precision attribute storage against the FP64 oracle, per
workload, on every pixel (the precision pattern: SH coefficients, log-scales
and skew stored in BF16 or FP16, unpacked to FP32 in registers, FP32
transmittance and colour accumulation).

Two figures per form:
  * arithmetic error: the oracle is fed the dequantised attributes and
    replays the GPU's own gate and stop decisions; the FP32 image bar of
    1e-4 holds;
  * storage error: the oracle is fed the FP32 originals and takes its own
    decisions; max and mean absolute error per channel are printed and held
    to the stated bounds.

Workloads: the 1M-Gaussian 1920x1080 frame (SH 3; BF16 and FP16 storage of
SH, log-scales and skew) and the 5M mixed scene (half the skew vectors
exactly zero, SH 3 stored in BF16) in a batched 8-view 1920x1080 plan.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2605_18334_gb300 import scenes
from paper_2605_18334_gb300.rasterizer import Config, Gaussians, Rasterizer
from tests.parity_util import IMG_ATOL, dequantised, gpu_blend_lists, oracle_config

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - CPU-only container
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

# stated storage-error bounds (max abs per channel, every pixel): the
# largest figures these tests measured (BF16 0.020 and FP16 0.0142 on the 1M
# frame, BF16 SH alone 0.010 on the 5M views) times 1.5, rounded up
STORAGE_BOUND = {torch.bfloat16: 0.03, torch.float16: 0.02}


def _errors(r, v, scene, deq, cam, cfg, ref_fp32=None):
    """(arithmetic max abs, storage max abs per channel, storage mean abs per
    channel, pixels with a decision that differs from the FP32-original
    oracle's) of view v."""
    oc = oracle.camera_from_gl(cam)
    ocfg = oracle_config(cfg)
    img = np.transpose(r.view_image(r.images, v).cpu().numpy(), (1, 2, 0)).astype(np.float64)
    rep = oracle.render_frame(deq, oc, ocfg, gpu_lists=gpu_blend_lists(r, v))
    assert rep["stats"]["inadmissible_pixels"] == 0, rep["stats"]
    arith = float(np.abs(img - rep["rgb"]).max())
    ref = ref_fp32 if ref_fp32 is not None else oracle.render_frame(scene, oc, ocfg)
    d = np.abs(img - ref["rgb"])
    return arith, d.reshape(-1, 3).max(0), d.reshape(-1, 3).mean(0), ref


def test_storage_error_1m_1080p_bf16_and_fp16():
    sc = scenes.unbounded(seed=2, n=1_000_000)
    cam = scenes.orbit_camera(0.0, 1920, 1080)
    cfg = Config()
    ref = None
    for dt in (torch.bfloat16, torch.float16):
        g = Gaussians.from_scene(sc, sh_dtype=dt, scale_dtype=dt, skew_dtype=dt)
        r = Rasterizer(g, [cam], cfg, key_capacity=12 * sc.n)
        r.forward(g)
        torch.cuda.synchronize()
        arith, smax, smean, ref = _errors(r, 0, sc, dequantised(sc, dt, dt, dt), cam, cfg, ref)
        print(f"precision unbounded_1m_1080p {str(dt).split('.')[-1]} (SH, log-scales, skew): arithmetic max abs "
              f"{arith:.3e}; storage max abs per channel {np.array2string(smax, precision=4)} mean "
              f"{np.array2string(smean, formatter={'float_kind': lambda x: f'{x:.2e}'})}")
        assert arith <= IMG_ATOL
        assert smax.max() <= STORAGE_BOUND[dt]
        del r, g
        torch.cuda.empty_cache()


def test_storage_error_5m_mixed_bf16_sh_8_views_1080p():
    sc = scenes.mixed_5m()
    cams = scenes.trajectory_cameras(8, resolutions=((1920, 1080),))
    cfg = Config()
    dt = torch.bfloat16
    g = Gaussians.from_scene(sc, sh_dtype=dt)
    r = Rasterizer(g, cams, cfg, key_capacity=1 << 27)
    r.forward(g)
    torch.cuda.synchronize()
    deq = dequantised(sc, sh_dtype=dt)
    worst_a, worst_s, means = 0.0, np.zeros(3), []
    for v, cam in enumerate(cams):
        arith, smax, smean, _ = _errors(r, v, sc, deq, cam, cfg)
        worst_a = max(worst_a, arith)
        worst_s = np.maximum(worst_s, smax)
        means.append(smean)
    mean = np.mean(means, 0)
    print(f"precision mixed_5m 8x1080p bf16 (SH): arithmetic max abs {worst_a:.3e}; storage max abs per channel "
          f"{np.array2string(worst_s, precision=4)} mean "
          f"{np.array2string(mean, formatter={'float_kind': lambda x: f'{x:.2e}'})}")
    assert worst_a <= IMG_ATOL
    assert worst_s.max() <= STORAGE_BOUND[dt]
