"""FP64 CPU oracle of the skew-Gaussian rasterizer (ctypes wrapper).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may use it.  The product path (the CUDA library
and its Python binding) never imports it, and it imports nothing from the
product.  The arithmetic lives in ``skew_oracle.cpp``; this module only
marshals numpy arrays.

Every function follows the paper as cited in ``skew_oracle.cpp``:
camera set-up (Alg. 3, Eq. coord_transform, the K matrix), projection
(Preliminaries, Eq. 1; Appendix "Forward Pass"), the skew kernel and
compositing (Alg. 1, Eq. 2, Eq. color, Eq. alpha) and gradients (Appendix
"Backward Pass"; Alg. 2 computes the same derivatives).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "skew_oracle.cpp")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libskew_oracle.so")
_lock = threading.Lock()
_lib = None

# Parity tolerances for decisions taken in floating point (documented in the
# design notes): a pair whose alpha lies within TOL_ALPHA of alpha_min, or
# whose T' lies within TOL_T (relative) of T_stop, makes its pixel
# "decision-ambiguous"; a rectangle edge within TOL_PX of a pixel-centre
# boundary makes a Gaussian's tile set ambiguous.
TOL_ALPHA = 2e-6
TOL_T = 1e-3
TOL_PX = 2e-3


def build(force: bool = False) -> str:
    """Compile the oracle with g++ (FP64, OpenMP, no FP contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        cmd = ["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
               "-fno-fast-math", _SRC, "-o", tmp]
        subprocess.check_call(cmd)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class Camera(C.Structure):
    _fields_ = [("w2c", C.c_double * 12), ("fx", C.c_double), ("fy", C.c_double), ("cx", C.c_double),
                ("cy", C.c_double), ("tan_fovx", C.c_double), ("tan_fovy", C.c_double),
                ("campos", C.c_double * 3), ("width", C.c_int32), ("height", C.c_int32)]


class Config(C.Structure):
    _fields_ = [("tile_w", C.c_int32), ("tile_h", C.c_int32), ("alpha_min", C.c_double),
                ("alpha_max", C.c_double), ("t_stop", C.c_double), ("dilation", C.c_double),
                ("fov_clamp", C.c_double), ("near_z", C.c_double), ("bg", C.c_double * 3),
                ("antialias_comp", C.c_int32), ("pad_", C.c_int32)]


class _Scene(C.Structure):
    _fields_ = [("n", C.c_int64), ("means", C.c_void_p), ("log_scales", C.c_void_p), ("quats", C.c_void_p),
                ("opac", C.c_void_p), ("skew", C.c_void_p), ("split", C.c_void_p), ("sh", C.c_void_p),
                ("two_opac", C.c_int32), ("sh_degree", C.c_int32)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = C.CDLL(build())
            _lib.or_nrec.restype = C.c_int
            _lib.or_ndiff.restype = C.c_int
            _lib.or_bin.restype = C.c_int64
            _lib.or_num_threads.restype = C.c_int
    return _lib


def _p(a):
    return C.c_void_p(a.ctypes.data) if a is not None else C.c_void_p(0)


def _d(a):
    return None if a is None else np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def num_threads() -> int:
    return int(lib().or_num_threads())


def config(tile=16, alpha_min=1.0 / 255.0, alpha_max=0.99, t_stop=1e-4, dilation=0.3, fov_clamp=1.3,
           near_z=0.2, bg=(0.0, 0.0, 0.0), antialias_comp=True) -> Config:
    """The rasterizer's constants, each rounded to FP32 as the CUDA side holds them."""
    f = lambda v: float(np.float32(v))
    c = Config()
    c.tile_w = c.tile_h = int(tile)
    c.alpha_min, c.alpha_max, c.t_stop = f(alpha_min), f(alpha_max), f(t_stop)
    c.dilation, c.fov_clamp, c.near_z = f(dilation), f(fov_clamp), f(near_z)
    for k in range(3):
        c.bg[k] = f(bg[k])
    c.antialias_comp = 1 if antialias_comp else 0
    return c


def camera_from_gl(cam: dict) -> Camera:
    """Alg. 3 camera set-up (FP64, rounded once to FP32), then any explicit
    intrinsics overrides in ``cam`` (fx, fy, cx, cy, tan_fovx, tan_fovy)."""
    out = Camera()
    m = np.ascontiguousarray(np.asarray(cam["c2w_gl"], np.float64).reshape(16))
    lib().or_camera_from_gl(_p(m), C.c_int32(cam["width"]), C.c_int32(cam["height"]),
                            C.c_double(cam["fovx"]), C.c_double(cam["fovy"]), C.byref(out))
    for k in ("fx", "fy", "cx", "cy", "tan_fovx", "tan_fovy"):
        if k in cam:
            setattr(out, k, float(np.float32(cam[k])))
    return out


def camera_fields(c: Camera) -> dict:
    return dict(w2c=np.array(c.w2c[:]), fx=c.fx, fy=c.fy, cx=c.cx, cy=c.cy, tan_fovx=c.tan_fovx,
                tan_fovy=c.tan_fovy, campos=np.array(c.campos[:]), width=c.width, height=c.height)


class _Arrays:
    """Keeps the FP64 copies of a scene alive while C reads them."""

    def __init__(self, scene):
        self.means = _d(scene.means)
        self.log_scales = _d(scene.log_scales)
        self.quats = _d(scene.quats)
        self.opac = _d(scene.opacity_logits)
        self.skew = _d(scene.skew)
        self.split = _d(scene.split_dir)
        self.sh = _d(scene.sh)
        self.s = _Scene(int(scene.n), _p(self.means).value, _p(self.log_scales).value, _p(self.quats).value,
                        _p(self.opac).value, _p(self.skew).value,
                        _p(self.split).value if self.split is not None else None,
                        _p(self.sh).value, 1 if self.opac.ndim == 2 else 0, int(scene.sh_degree))


# names of the record columns (first NDIFF are the differentiable 2D quantities)
REC_NAMES = ["mx", "my", "a", "b", "c", "bx", "by", "m", "h", "ux", "uy", "r", "g", "bl",
             "comp", "o1", "o2", "tz", "dxx", "dxy", "dyy"]
NDIFF = 14


def preprocess(scene, cam: Camera, cfg: Config, tol_px: float = TOL_PX) -> dict:
    L = lib()
    nrec = L.or_nrec()
    assert nrec == len(REC_NAMES)
    n = scene.n
    a = _Arrays(scene)
    rec = np.zeros((n, nrec))
    bits = np.zeros(n, np.uint32)
    vis = np.zeros(n, np.int32)
    rect = np.zeros((n, 4), np.int32)
    ext = np.zeros((n, 3))
    amb = np.zeros(n, np.int32)
    cnt = np.zeros(n, np.int32)
    L.or_preprocess(C.byref(a.s), C.byref(cam), C.byref(cfg), C.c_double(tol_px), _p(rec), _p(bits), _p(vis),
                    _p(rect), _p(ext), _p(amb), _p(cnt))
    return dict(rec=rec, depth_bits=bits, visible=vis.astype(bool), rect=rect, ext=ext, rect_ambig=amb.astype(bool),
                ntouch=cnt, _vis32=vis)


def all_pixels(cam: Camera) -> np.ndarray:
    ys, xs = np.meshgrid(np.arange(cam.height, dtype=np.int32), np.arange(cam.width, dtype=np.int32), indexing="ij")
    return np.ascontiguousarray(np.stack([xs.ravel(), ys.ravel()], axis=1))


def render(scene, cam: Camera, cfg: Config, pixels=None, pre=None, tol_alpha=TOL_ALPHA, tol_t=TOL_T) -> dict:
    """Brute-force render: every visible Gaussian, in (depth key, index) order,
    at each listed pixel (default: all pixels, row-major).  With the default
    pixel list, ``rgb`` is [H,W,3] and the other outputs [H,W]."""
    pre = pre or preprocess(scene, cam, cfg)
    full = pixels is None
    pix = all_pixels(cam) if full else np.ascontiguousarray(np.asarray(pixels, np.int32).reshape(-1, 2))
    m = pix.shape[0]
    rgb = np.zeros((m, 3))
    T = np.zeros(m)
    last = np.zeros(m, np.int64)
    cnt = np.zeros(m, np.int32)
    amb = np.zeros(m, np.int32)
    sig = np.zeros(m, np.uint64)
    lib().or_render_pixels(C.byref(cam), C.byref(cfg), C.c_int64(scene.n), _p(pre["rec"]), _p(pre["depth_bits"]),
                           _p(pre["_vis32"]), C.c_int64(m), _p(pix), C.c_double(tol_alpha), C.c_double(tol_t),
                           _p(rgb), _p(T), _p(last), _p(cnt), _p(amb), _p(sig))
    out = dict(rgb=rgb, T=T, last=last, count=cnt, ambiguous=amb.astype(bool), pixels=pix, signature=sig)
    if full:
        H, W = cam.height, cam.width
        out.update(rgb=rgb.reshape(H, W, 3), T=T.reshape(H, W), last=last.reshape(H, W), count=cnt.reshape(H, W),
                   ambiguous=out["ambiguous"].reshape(H, W), signature=sig.reshape(H, W))
    return out


def render_backward(scene, cam: Camera, cfg: Config, dL_dC, pixels=None, pre=None) -> dict:
    """Gradients of L = sum(dL_dC * C).  ``dL_dC`` is planar [3,H,W] when
    ``pixels`` is None, else [n_pix,3] aligned with ``pixels``."""
    pre = pre or preprocess(scene, cam, cfg)
    n = scene.n
    if pixels is None:
        pix = all_pixels(cam)
        g = np.ascontiguousarray(np.asarray(dL_dC, np.float64).reshape(3, -1).T)
    else:
        pix = np.ascontiguousarray(np.asarray(pixels, np.int32).reshape(-1, 2))
        g = np.ascontiguousarray(np.asarray(dL_dC, np.float64).reshape(-1, 3))
    a = _Arrays(scene)
    K = (scene.sh_degree + 1) ** 2
    nop = 2 if a.opac.ndim == 2 else 1
    d2 = np.zeros((n, NDIFF))
    gm, gl, gs = np.zeros((n, 3)), np.zeros((n, 3)), np.zeros((n, 3))
    gq = np.zeros((n, 4))
    go = np.zeros((n, nop))
    gd = np.zeros((n, 3)) if a.split is not None else None
    gsh = np.zeros((n, K, 3))
    lib().or_render_backward(C.byref(a.s), C.byref(cam), C.byref(cfg), _p(pre["rec"]), _p(pre["depth_bits"]),
                             _p(pre["_vis32"]), C.c_int64(pix.shape[0]), _p(pix), _p(g), _p(d2), _p(gm), _p(gl),
                             _p(gq), _p(go), _p(gs), _p(gd), _p(gsh))
    return dict(d2=d2, means=gm, log_scales=gl, quats=gq, opacity_logits=go.reshape(n) if nop == 1 else go,
                skew=gs, split_dir=gd, sh=gsh)


def bin_keys(pre: dict, cam: Camera, cfg: Config, tile_base: int = 0, val_base: int = 0):
    """Sorted (tile << 32 | depth bits) keys and Gaussian ids of one view."""
    n = pre["rec"].shape[0]
    L = lib()
    args = [C.c_int64(n), _p(pre["rec"]), _p(pre["ext"]), _p(pre["depth_bits"]), _p(pre["_vis32"]), _p(pre["rect"]),
            C.c_int32(cam.width), C.c_int32(cam.height), C.c_int32(cfg.tile_w), C.c_double(cfg.alpha_min),
            C.c_int64(tile_base), C.c_int64(val_base)]
    cnt = L.or_bin(*args, C.c_int64(0), None, None)
    keys = np.zeros(max(cnt, 1), np.uint64)
    vals = np.zeros(max(cnt, 1), np.int64)
    L.or_bin(*args, C.c_int64(cnt), _p(keys), _p(vals))
    return keys[:cnt], vals[:cnt]


def kernel_at(abc, beta, dxy) -> np.ndarray:
    """exp(-1/2 d^T A d) (1 + erf(beta^T d / sqrt 2)) at offsets d (o = 1)."""
    abc = _d(abc)
    beta = _d(beta)
    dxy = np.ascontiguousarray(np.asarray(dxy, np.float64).reshape(-1, 2))
    out = np.zeros(dxy.shape[0])
    lib().or_kernel_at(_p(abc), _p(beta), C.c_int64(dxy.shape[0]), _p(dxy), _p(out))
    return out


def alpha_at(rec_row, pixels) -> np.ndarray:
    r = _d(rec_row)
    pix = np.ascontiguousarray(np.asarray(pixels, np.int32).reshape(-1, 2))
    out = np.zeros(pix.shape[0])
    lib().or_alpha_at(_p(r), C.c_int64(pix.shape[0]), _p(pix), _p(out))
    return out


def sh_basis(deg: int, dirs) -> np.ndarray:
    dirs = np.ascontiguousarray(np.asarray(dirs, np.float64).reshape(-1, 3))
    K = (deg + 1) ** 2
    out = np.zeros((dirs.shape[0], K))
    lib().or_sh_basis(C.c_int(deg), C.c_int64(dirs.shape[0]), _p(dirs), _p(out))
    return out
