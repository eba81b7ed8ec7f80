"""Seeded synthetic scenes, cameras and upstream gradients.

This module only draws inputs.  It holds none of the rasterizer's arithmetic
(no projection, no skew kernel, no compositing); both the CUDA path and the
FP64 CPU oracle consume the arrays it returns, byte for byte.

The datasets of the paper (Mip-NeRF 360, Tanks & Temples, Deep Blending) are
not available, so the workloads are synthetic stand-ins with the primitive
counts, resolutions and attribute distributions of the paper's setting
(Sec. "Experiment", Table 2: 2.4-3.2M kernels per scene):

* ``cube_1k``      1,000 Gaussians in a 1x1x2 box 3-5 units ahead, 64x64 view,
                   SH degree 0, skew ~ N(0, 1).
* ``cluster_100k`` 100k Gaussians around (0,0,4), 1280x720 view, SH degree 3,
                   skew ~ N(0, 1.5^2), upstream image gradient ~ N(0, 1).
* ``unbounded_1m`` 1M Gaussians: 60% in a ball of radius 2, 40% on a shell of
                   radius 20-50, camera on a radius-6 orbit, 1920x1080.
* ``trajectory``   64 cameras on a closed centripetal Catmull-Rom spline,
                   resolutions cycling 640x360 / 1280x720 / 1920x1080.
* ``mixed_5m``     5M Gaussians, half of them with skew exactly zero.

Conventions of the arrays (all float32 unless stated):
  means [N,3]; log_scales [N,3]; quats [N,4] as (w,x,y,z), not normalised;
  opacity_logits [N] or [N,2]; skew [N,3] (dimensionless, local frame);
  split_dir [N,3] or None; sh [N,(deg+1)^2,3].
Cameras are dicts with ``c2w_gl`` (float64 4x4, OpenGL/Blender convention:
camera looks down -Z, +Y up), ``width``, ``height``, ``fovx``, ``fovy``
(radians, float64).  World "up" is -Y, so an OpenCV camera (+Y down) with an
identity pose sees the world upright.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# Only used to write degree-0 colours as SH DC coefficients (input encoding).
_Y00 = 0.5 / math.sqrt(math.pi)
_CV_TO_GL = np.diag([1.0, -1.0, -1.0, 1.0])


@dataclass
class Scene:
    means: np.ndarray
    log_scales: np.ndarray
    quats: np.ndarray
    opacity_logits: np.ndarray
    skew: np.ndarray
    sh: np.ndarray
    sh_degree: int
    split_dir: np.ndarray | None = None
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.means.shape[0])

    @property
    def two_opacities(self) -> bool:
        return self.opacity_logits.ndim == 2

    def subset(self, idx) -> "Scene":
        return Scene(
            self.means[idx], self.log_scales[idx], self.quats[idx],
            self.opacity_logits[idx], self.skew[idx], self.sh[idx],
            self.sh_degree,
            None if self.split_dir is None else self.split_dir[idx],
            dict(self.meta),
        )


def _f32(x):
    return np.ascontiguousarray(np.asarray(x, dtype=np.float64).astype(np.float32))


def uniform_quats(rng: np.random.Generator, n: int) -> np.ndarray:
    """Uniformly distributed rotations: normalised 4-D standard normals (w,x,y,z)."""
    q = rng.standard_normal((n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    return q


def opacity_logits_uniform(rng, n, lo=0.05, hi=0.99, two=False):
    """Opacity drawn uniform in (lo, hi) and stored as its logit."""
    p = rng.uniform(lo, hi, size=(n, 2) if two else (n,))
    return np.log(p) - np.log1p(-p)


def sh_from_rgb(rgb: np.ndarray) -> np.ndarray:
    """Degree-0 SH coefficients whose DC term reproduces ``rgb`` (FP64, then FP32)."""
    return ((rgb - 0.5) / _Y00)[:, None, :]


def look_at_c2w_cv(eye, target, up=(0.0, -1.0, 0.0)) -> np.ndarray:
    """OpenCV camera-to-world pose (x right, y down, z forward) looking at ``target``."""
    eye = np.asarray(eye, np.float64)
    z = np.asarray(target, np.float64) - eye
    z /= np.linalg.norm(z)
    x = np.cross(z, np.asarray(up, np.float64))
    x /= np.linalg.norm(x)
    y = np.cross(z, x)
    m = np.eye(4)
    m[:3, 0], m[:3, 1], m[:3, 2], m[:3, 3] = x, y, z, eye
    return m


def camera(c2w_cv: np.ndarray, width: int, height: int, fovx_deg: float = 60.0) -> dict:
    """A camera as a Blender-style frontend would hand it over: a C2W pose in
    the OpenGL convention, the viewport size and the horizontal FoV.  The
    vertical FoV keeps square pixels: tan(fovy/2) = tan(fovx/2) * H / W."""
    fovx = math.radians(fovx_deg)
    fovy = 2.0 * math.atan(math.tan(fovx / 2.0) * height / width)
    return dict(c2w_gl=np.asarray(c2w_cv, np.float64) @ _CV_TO_GL,
                width=int(width), height=int(height), fovx=fovx, fovy=fovy)


def identity_camera(width: int, height: int, fovx_deg: float = 60.0) -> dict:
    return camera(np.eye(4), width, height, fovx_deg)


def orbit_camera(angle: float, width: int, height: int, radius=6.0, height_off=0.5) -> dict:
    """Camera on a circle of ``radius`` around the origin, ``height_off`` above
    the equator (world up is -Y), looking at the origin."""
    eye = (radius * math.sin(angle), -height_off, -radius * math.cos(angle))
    return camera(look_at_c2w_cv(eye, (0.0, 0.0, 0.0)), width, height)


def catmull_rom_closed(ctrl: np.ndarray, n_samples: int, alpha: float = 0.5) -> np.ndarray:
    """Closed centripetal Catmull-Rom spline (Barry-Goldman pyramid form),
    sampled uniformly in the segment parameter."""
    k = len(ctrl)
    out = []
    for s in range(n_samples):
        u = s * k / n_samples
        seg = int(math.floor(u))
        f = u - seg
        p0, p1, p2, p3 = (ctrl[(seg + j - 1) % k] for j in range(4))
        t0 = 0.0
        t1 = t0 + np.linalg.norm(p1 - p0) ** alpha
        t2 = t1 + np.linalg.norm(p2 - p1) ** alpha
        t3 = t2 + np.linalg.norm(p3 - p2) ** alpha
        t = t1 + f * (t2 - t1)
        a1 = (t1 - t) / (t1 - t0) * p0 + (t - t0) / (t1 - t0) * p1
        a2 = (t2 - t) / (t2 - t1) * p1 + (t - t1) / (t2 - t1) * p2
        a3 = (t3 - t) / (t3 - t2) * p2 + (t - t2) / (t3 - t2) * p3
        b1 = (t2 - t) / (t2 - t0) * a1 + (t - t0) / (t2 - t0) * a2
        b2 = (t3 - t) / (t3 - t1) * a2 + (t - t1) / (t3 - t1) * a3
        out.append((t2 - t) / (t2 - t1) * b1 + (t - t1) / (t2 - t1) * b2)
    return np.array(out)


TRAJ_RESOLUTIONS = ((640, 360), (1280, 720), (1920, 1080))


def trajectory_cameras(n_views=64, radius=6.0, resolutions=TRAJ_RESOLUTIONS) -> list:
    """Closed orbit through 8 control points on the radius-6 circle with
    heights alternating +-0.75; view i gets resolution i mod len(resolutions)."""
    ctrl = []
    for j in range(8):
        a = 2 * math.pi * j / 8
        ctrl.append([radius * math.sin(a), 0.75 if j % 2 else -0.75, -radius * math.cos(a)])
    eyes = catmull_rom_closed(np.array(ctrl), n_views)
    cams = []
    for i, eye in enumerate(eyes):
        w, h = resolutions[i % len(resolutions)]
        cams.append(camera(look_at_c2w_cv(eye, (0.0, 0.0, 0.0)), w, h))
    return cams


# ----------------------------------------------------------------------------
# Workloads
# ----------------------------------------------------------------------------

def cube_1k(seed: int = 0, n: int = 1000, skew_sigma: float = 1.0) -> Scene:
    """1k Gaussians, x,y ~ U[-0.5,0.5], z ~ U[3,5], log-scales U[-4,-2],
    skew ~ N(0,1), opacity U(0.05,0.99), SH degree 0 from RGB ~ U[0,1]."""
    rng = np.random.default_rng(seed)
    means = np.stack([rng.uniform(-0.5, 0.5, n), rng.uniform(-0.5, 0.5, n),
                      rng.uniform(3.0, 5.0, n)], axis=1)
    return Scene(
        means=_f32(means),
        log_scales=_f32(rng.uniform(-4.0, -2.0, (n, 3))),
        quats=_f32(uniform_quats(rng, n)),
        opacity_logits=_f32(opacity_logits_uniform(rng, n)),
        skew=_f32(rng.standard_normal((n, 3)) * skew_sigma),
        sh=_f32(sh_from_rgb(rng.uniform(0.0, 1.0, (n, 3)))),
        sh_degree=0,
        meta=dict(name="cube_1k", seed=seed),
    )


def cluster(seed: int = 1, n: int = 100_000, sh_degree: int = 3, skew_sigma: float = 1.5,
            two_opacities: bool = False, split: bool = False) -> Scene:
    """Gaussian cluster (sigma 1) around (0,0,4); log-scales ~ N(-4, 0.5);
    skew ~ N(0, 1.5^2); SH coefficients ~ N(0, 0.3^2)."""
    rng = np.random.default_rng(seed)
    k = (sh_degree + 1) ** 2
    means = rng.standard_normal((n, 3)) + np.array([0.0, 0.0, 4.0])
    return Scene(
        means=_f32(means),
        log_scales=_f32(rng.normal(-4.0, 0.5, (n, 3))),
        quats=_f32(uniform_quats(rng, n)),
        opacity_logits=_f32(opacity_logits_uniform(rng, n, two=two_opacities)),
        skew=_f32(rng.standard_normal((n, 3)) * skew_sigma),
        sh=_f32(rng.normal(0.0, 0.3, (n, k, 3))),
        sh_degree=sh_degree,
        split_dir=_f32(rng.standard_normal((n, 3))) if split else None,
        meta=dict(name="cluster", seed=seed),
    )


def unbounded(seed: int = 2, n: int = 1_000_000, sh_degree: int = 3, skew_sigma: float = 1.5,
              zero_skew_fraction: float = 0.0, cluster_fraction: float = 0.6) -> Scene:
    """Unbounded-scene stand-in: ``cluster_fraction`` uniform in a ball of
    radius 2, the rest on a shell (uniform direction, r ~ U[20,50]) with
    log-scales grown by ln(r/4) so far splats keep a similar pixel size."""
    rng = np.random.default_rng(seed)
    k = (sh_degree + 1) ** 2
    nc = int(round(n * cluster_fraction))
    ns = n - nc
    d = rng.standard_normal((nc, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    ball = d * (2.0 * rng.uniform(0.0, 1.0, (nc, 1)) ** (1.0 / 3.0))
    d = rng.standard_normal((ns, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    r = rng.uniform(20.0, 50.0, (ns, 1))
    shell = d * r
    ls = rng.normal(-4.0, 0.5, (n, 3))
    ls[nc:] += np.log(r / 4.0)
    skew = rng.standard_normal((n, 3)) * skew_sigma
    if zero_skew_fraction > 0:
        zero = rng.uniform(0.0, 1.0, n) < zero_skew_fraction
        skew[zero] = 0.0
    return Scene(
        means=_f32(np.concatenate([ball, shell])),
        log_scales=_f32(ls),
        quats=_f32(uniform_quats(rng, n)),
        opacity_logits=_f32(opacity_logits_uniform(rng, n)),
        skew=_f32(skew),
        sh=_f32(rng.normal(0.0, 0.3, (n, k, 3))),
        sh_degree=sh_degree,
        meta=dict(name="unbounded", seed=seed, n_cluster=nc),
    )


def mixed_5m(seed: int = 4, n: int = 5_000_000) -> Scene:
    """5M Gaussians, config-3 geometry; 50% skew exactly 0, 50% ~ N(0, 2^2)."""
    return unbounded(seed=seed, n=n, skew_sigma=2.0, zero_skew_fraction=0.5)


def upstream_grad(seed: int, height: int, width: int, channels: int = 3) -> np.ndarray:
    """dL/dC ~ N(0,1) per pixel and channel, planar [3,H,W]."""
    rng = np.random.default_rng(seed + 1000)
    return _f32(rng.standard_normal((channels, height, width)))


def sparse_upstream_grad(seed: int, height: int, width: int, n_pixels: int):
    """dL/dC that is N(0,1) on ``n_pixels`` random pixels and zero elsewhere,
    so per-Gaussian gradients of a full-size frame are sums over a few pixels."""
    rng = np.random.default_rng(seed + 2000)
    flat = rng.choice(height * width, size=min(n_pixels, height * width), replace=False)
    g = np.zeros((3, height * width), np.float32)
    g[:, flat] = rng.standard_normal((3, flat.size)).astype(np.float32)
    return g.reshape(3, height, width), np.sort(flat)


def fd_crop_scene(seed: int = 3, n: int = 2000, crop=32):
    """Finite-difference set: Gaussians drawn from the cluster law,
    rejection-sampled to project within 32 px of the crop [624,656)x[344,376)
    of the 1280x720 view, rendered as a 32x32 camera with the same focal
    length and the principal point moved to the crop centre.

    Returns (scene, camera dict).  The camera dict carries explicit
    ``fx, fy, cx, cy`` overrides in addition to the pose."""
    rng = np.random.default_rng(seed)
    W, H = 1280, 720
    fx = W / (2.0 * math.tan(math.radians(60.0) / 2.0))
    keep = []
    batch = 0
    while sum(len(k) for k in keep) < n:
        m = rng.standard_normal((200_000, 3)) + np.array([0.0, 0.0, 4.0])
        u = fx * m[:, 0] / m[:, 2] + W / 2
        v = fx * m[:, 1] / m[:, 2] + H / 2
        ok = (m[:, 2] > 0.5) & (u > 624 - 32) & (u < 656 + 32) & (v > 344 - 32) & (v < 376 + 32)
        keep.append(m[ok])
        batch += 1
    means = np.concatenate(keep)[:n]
    base = cluster(seed=seed + 17, n=n)
    base.means = _f32(means)
    base.meta = dict(name="fd_crop", seed=seed)
    cam = identity_camera(crop, crop)
    t = math.tan(math.radians(60.0) / 2.0)
    cam.update(fx=fx, fy=fx, cx=W / 2.0 - 624.0, cy=H / 2.0 - 344.0,
               tan_fovx=t, tan_fovy=t * H / W)
    return base, cam


WORKLOADS = {
    "cube_1k": dict(scene=lambda: cube_1k(), cams=lambda: [identity_camera(64, 64)]),
    "cluster_100k": dict(scene=lambda: cluster(), cams=lambda: [identity_camera(1280, 720)]),
    "unbounded_1m": dict(scene=lambda: unbounded(), cams=lambda: [orbit_camera(0.0, 1920, 1080)]),
    "trajectory_64": dict(scene=lambda: unbounded(), cams=lambda: trajectory_cameras(64)),
}
