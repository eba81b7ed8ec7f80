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

# Parity tolerances for decisions taken in floating point (the measured FP32
# errors they cover are stated in the design notes): a pair whose alpha lies
# within TOL_ALPHA (relative) of alpha_min or of alpha_max, or whose T' lies
# within TOL_T (relative) of T_stop, is "decision-ambiguous"; a tile edge
# within TOL_PX of a pixel-centre boundary makes a Gaussian's tile set
# ambiguous.
TOL_ALPHA = 5e-4
TOL_T = 1e-2
TOL_PX = 1e-3


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


def set_num_threads(n: int) -> None:
    """Threads of the oracle's parallel loops from now on (timing runs)."""
    lib().or_set_num_threads(C.c_int(int(n)))


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
    """Brute-force render (mode A): every visible Gaussian, in (depth key,
    index) order, at each listed pixel (default: all pixels, row-major).  With
    the default pixel list, ``rgb`` is [H,W,3] and the other outputs [H,W].
    ``tol_alpha`` is relative to alpha_min, ``tol_t`` to t_stop."""
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


class _GradsOut(C.Structure):
    _fields_ = [(k, C.c_void_p) for k in ("means", "log_scales", "quats", "opac", "skew", "split", "sh")]


def _grad_arrays(scene, with_split):
    n = scene.n
    K = (scene.sh_degree + 1) ** 2
    nop = 2 if np.asarray(scene.opacity_logits).ndim == 2 else 1
    d = dict(means=np.zeros((n, 3)), log_scales=np.zeros((n, 3)), quats=np.zeros((n, 4)),
             opacity_logits=np.zeros((n, nop)), skew=np.zeros((n, 3)),
             split_dir=np.zeros((n, 3)) if with_split else None, sh=np.zeros((n, K, 3)))
    s = _GradsOut(*[_p(d[k]).value if d[k] is not None else None
                    for k in ("means", "log_scales", "quats", "opacity_logits", "skew", "split_dir", "sh")])
    return d, s


def _flat_opac(d, nop):
    if nop == 1:
        d["opacity_logits"] = d["opacity_logits"].reshape(-1)
    return d


def render_frame(scene, cam: Camera, cfg: Config, pre=None, gpu_lists=None, tol_alpha=TOL_ALPHA,
                 tol_t=TOL_T, want_lists: bool = False) -> dict:
    """Whole frame by mode B (per-pixel lists of the Gaussians whose footprint
    reaches the pixel, in depth order; equal to mode A bit for bit).  With
    ``gpu_lists`` = (offsets [H*W+1] int64, ids int32), the gate and stop
    decisions of another renderer (which blended ids[off[p]:off[p+1]] at pixel
    p, row-major) are replayed: ``status`` is nonzero at pixels where one of
    them is not admissible, ``rgb``/``T`` are the FP64 results under them.
    ``stats``: flipped-decision counts and the largest margins.
    ``want_lists``: also return ``lists`` = (offsets, ids) of the Gaussians
    each pixel blended (a second pass)."""
    assert tol_alpha < 1e-2 or gpu_lists is None, "mode B's lists hold only pairs with alpha >= alpha_min (1 - 1e-2)"
    pre = pre or preprocess(scene, cam, cfg)
    H, W = cam.height, cam.width
    m = H * W
    rgb = np.zeros((m, 3))
    T = np.zeros(m)
    last = np.zeros(m, np.int64)
    cnt = np.zeros(m, np.int32)
    amb = np.zeros(m, np.int32)
    status = np.zeros(m, np.int32)
    st = np.zeros(8)
    if gpu_lists is not None:
        off = np.ascontiguousarray(gpu_lists[0], np.int64)
        ids = np.ascontiguousarray(gpu_lists[1], np.int32)
        assert off.shape == (m + 1,)
    else:
        off = ids = None
    lib().or_render_frame(C.byref(cam), C.byref(cfg), C.c_int64(scene.n), _p(pre["rec"]), _p(pre["depth_bits"]),
                          _p(pre["_vis32"]), C.c_double(tol_alpha), C.c_double(tol_t), _p(off), _p(ids), _p(rgb),
                          _p(T), _p(last), _p(cnt), _p(amb), _p(status), _p(st), None, None)
    lists = None
    if want_lists:
        loff = np.zeros(m + 1, np.int64)
        np.cumsum(cnt, out=loff[1:])
        lids = np.zeros(max(1, int(loff[-1])), np.int32)
        t2 = [np.zeros_like(a) for a in (rgb, T, last, cnt, amb, status)]
        lib().or_render_frame(C.byref(cam), C.byref(cfg), C.c_int64(scene.n), _p(pre["rec"]),
                              _p(pre["depth_bits"]), _p(pre["_vis32"]), C.c_double(tol_alpha), C.c_double(tol_t),
                              _p(off), _p(ids), *[_p(a) for a in t2], None, _p(loff), _p(lids))
        lists = (loff, lids[:int(loff[-1])])
    names = ["flipped_pixels", "flipped_gate", "flipped_stop", "max_gate_margin", "max_stop_margin",
             "inadmissible_pixels", "candidate_pairs", "ambiguous_pixels"]
    stats = {k: (float(v) if "margin" in k else int(v)) for k, v in zip(names, st)}
    return dict(rgb=rgb.reshape(H, W, 3), T=T.reshape(H, W), last=last.reshape(H, W), count=cnt.reshape(H, W),
                ambiguous=amb.astype(bool).reshape(H, W), status=status.reshape(H, W), stats=stats, lists=lists)


def render_backward(scene, cam: Camera, cfg: Config, dL_dC, pixels=None, pre=None, frame: bool = False,
                    gpu_lists=None, bounds: bool = False, tol_alpha=TOL_ALPHA, tol_t=TOL_T) -> dict:
    """Gradients of L = sum(dL_dC * C).  ``dL_dC`` is planar [3,H,W] when
    ``pixels`` is None, else [n_pix,3] aligned with ``pixels``.  ``frame``:
    every pixel through mode B (else mode A over the pixel list, default all
    pixels).  ``gpu_lists`` (indexed like the pixels): replay another
    renderer's gate and stop decisions.  ``bounds``: also return, per
    element, ``scale`` (the rounding-error scale: sum of the magnitudes of
    the terms) and ``slack`` (the terms whose alpha_max or colour clamp lies
    within tolerance), as dicts of the same layouts."""
    assert tol_alpha < 1e-2 or not frame or gpu_lists is None, "mode B's lists hold only pairs with alpha >= alpha_min (1 - 1e-2)"
    pre = pre or preprocess(scene, cam, cfg)
    n = scene.n
    if pixels is None:
        g = np.ascontiguousarray(np.asarray(dL_dC, np.float64).reshape(3, -1).T)
        pix = None if frame else all_pixels(cam)
    else:
        assert not frame
        pix = np.ascontiguousarray(np.asarray(pixels, np.int32).reshape(-1, 2))
        g = np.ascontiguousarray(np.asarray(dL_dC, np.float64).reshape(-1, 3))
    a = _Arrays(scene)
    nop = 2 if a.opac.ndim == 2 else 1
    d2 = np.zeros((n, NDIFF))
    d2s = np.zeros((n, NDIFF)) if bounds else None
    d2l = np.zeros((n, NDIFF)) if bounds else None
    G, Gs = _grad_arrays(scene, a.split is not None)
    S, Ss = _grad_arrays(scene, a.split is not None) if bounds else (None, None)
    L, Ls = _grad_arrays(scene, a.split is not None) if bounds else (None, None)
    if gpu_lists is not None:
        off = np.ascontiguousarray(gpu_lists[0], np.int64)
        ids = np.ascontiguousarray(gpu_lists[1], np.int32)
        assert off.shape == (g.shape[0] + 1,)
    else:
        off = ids = None
    bad = C.c_int64(0)
    lib().or_render_backward(C.byref(a.s), C.byref(cam), C.byref(cfg), _p(pre["rec"]), _p(pre["depth_bits"]),
                             _p(pre["_vis32"]), C.c_int64(0 if pix is None else pix.shape[0]), _p(pix), _p(g),
                             _p(off), _p(ids), C.c_double(tol_alpha), C.c_double(tol_t), _p(d2), _p(d2s), _p(d2l),
                             C.byref(Gs), C.byref(Ss) if bounds else None, C.byref(Ls) if bounds else None,
                             C.byref(bad))
    out = _flat_opac(G, nop)
    out["d2"] = d2
    out["inadmissible_pixels"] = int(bad.value)
    if bounds:
        out["scale"] = _flat_opac(S, nop)
        out["scale"]["d2"] = d2s
        out["slack"] = _flat_opac(L, nop)
        out["slack"]["d2"] = d2l
    return out


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
