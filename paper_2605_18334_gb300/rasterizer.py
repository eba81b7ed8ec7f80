"""Torch-facing API of the skew-Gaussian rasterizer.

PyTorch supplies device memory, streams and autograd plumbing only; every
stage runs in ``libskewraster.so`` through the C ABI (``native``):

    rast = Rasterizer(GaussianDesc.of(g), cameras, Config())
    out = rast.forward(g)                    # sr_preprocess, sr_bin_sort, sr_render_fwd
    grads = rast.backward(g, d_images)       # sr_render_bwd

``render(...)`` wraps the same calls in a ``torch.autograd.Function``.
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass, field

import numpy as np
import torch

from . import native as N

_TAG = {torch.float32: N.SR_F32, torch.bfloat16: N.SR_BF16, torch.float16: N.SR_F16}


@dataclass
class Config:
    """Rasterizer constants (sr_config)."""
    tile: int = 16
    alpha_min: float = 1.0 / 255.0
    alpha_max: float = 0.99
    t_stop: float = 1e-4
    dilation: float = 0.3
    fov_clamp: float = 1.3
    near_z: float = 0.2
    bg: tuple = (0.0, 0.0, 0.0)
    antialias_comp: bool = True
    sort_spin_limit: int = 0
    fwd_pixels_per_thread: int = 0   # 0: library default (2)
    bwd_pixels_per_thread: int = 0
    forward_only: bool = False       # plan without backward state (blend masks)
    fwd_batch: int = 0               # records staged per batch by the forward composite (0: 256)
    bwd_batch: int = 0               # ... by the backward composite (0: 128)
    recompute_keys: bool = False     # plan without blend masks: the backward rebuilds the key lists
    persistent: int = 0              # bit 0 forward, bit 1 backward composite: persistent launches
    fwd_blocks_per_sm: int = 0       # cap on resident forward-composite blocks per SM (0: as many as fit)
    bwd_blocks_per_sm: int = 0       # ... backward composite

    def to_c(self) -> N.sr_config:
        c = N.sr_config()
        c.tile_w = c.tile_h = int(self.tile)
        c.alpha_min, c.alpha_max, c.t_stop = self.alpha_min, self.alpha_max, self.t_stop
        c.dilation, c.fov_clamp, c.near_z = self.dilation, self.fov_clamp, self.near_z
        for k in range(3):
            c.bg[k] = float(self.bg[k])
        c.antialias_comp = 1 if self.antialias_comp else 0
        c.sort_spin_limit = int(self.sort_spin_limit)
        c.fwd_pixels_per_thread = int(self.fwd_pixels_per_thread)
        c.bwd_pixels_per_thread = int(self.bwd_pixels_per_thread)
        c.forward_only = 1 if self.forward_only else 0
        c.fwd_batch = int(self.fwd_batch)
        c.bwd_batch = int(self.bwd_batch)
        c.recompute_keys = 1 if self.recompute_keys else 0
        c.persistent = int(self.persistent)
        c.fwd_blocks_per_sm = int(self.fwd_blocks_per_sm)
        c.bwd_blocks_per_sm = int(self.bwd_blocks_per_sm)
        return c


def camera_from_dict(cam: dict) -> N.sr_camera:
    """sr_camera_from_gl on a camera dict (c2w_gl, width, height, fovx, fovy),
    then explicit intrinsics overrides (fx, fy, cx, cy, tan_fovx, tan_fovy)."""
    c = N.sr_camera_from_gl(np.asarray(cam["c2w_gl"], np.float64), cam["width"], cam["height"], cam["fovx"],
                            cam["fovy"])
    for k in ("fx", "fy", "cx", "cy", "tan_fovx", "tan_fovy"):
        if k in cam:
            setattr(c, k, float(np.float32(cam[k])))
    return c


@dataclass
class Gaussians:
    """Device tensors of one scene (layouts of sr_gaussians)."""
    means: torch.Tensor
    log_scales: torch.Tensor
    quats: torch.Tensor
    opacity_logits: torch.Tensor
    skew: torch.Tensor
    sh: torch.Tensor
    sh_degree: int
    split_dir: torch.Tensor | None = None

    @property
    def n(self) -> int:
        return int(self.means.shape[0])

    @staticmethod
    def from_scene(scene, device="cuda", sh_dtype=torch.float32, scale_dtype=torch.float32,
                   skew_dtype=torch.float32) -> "Gaussians":
        t = lambda a, dt=torch.float32: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float32).to(
            device=device, dtype=dt).contiguous()
        return Gaussians(t(scene.means), t(scene.log_scales, scale_dtype), t(scene.quats), t(scene.opacity_logits),
                         t(scene.skew, skew_dtype), t(scene.sh, sh_dtype), int(scene.sh_degree),
                         None if scene.split_dir is None else t(scene.split_dir, skew_dtype))

    def to_c(self) -> N.sr_gaussians:
        for name in ("means", "quats", "opacity_logits"):
            if getattr(self, name).dtype != torch.float32:
                raise TypeError(f"{name} must be float32")
        g = N.sr_gaussians()
        g.means = self.means.data_ptr()
        g.log_scales = self.log_scales.data_ptr()
        g.quats = self.quats.data_ptr()
        g.opacity_logits = self.opacity_logits.data_ptr()
        g.skew = self.skew.data_ptr()
        g.split_dir = self.split_dir.data_ptr() if self.split_dir is not None else None
        g.sh = self.sh.data_ptr()
        g.n = self.n
        g.sh_degree = int(self.sh_degree)
        g.two_opacities = 1 if self.opacity_logits.dim() == 2 else 0
        g.dt_sh = _TAG[self.sh.dtype]
        g.dt_scale = _TAG[self.log_scales.dtype]
        g.dt_skew = _TAG[self.skew.dtype]
        for t in (self.means, self.log_scales, self.quats, self.opacity_logits, self.skew, self.sh):
            if not t.is_contiguous() or not t.is_cuda:
                raise ValueError("Gaussian attributes must be contiguous CUDA tensors")
        return g


def _stream_ptr(stream=None) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


def _prefer_default(times: dict, default, margin: float = 0.02):
    """The fastest candidate, unless the default is within ``margin`` of it
    (timing noise should not flip a launch parameter between frames)."""
    best = min(times, key=times.get)
    if default in times and times[default] <= times[best] * (1.0 + margin):
        return default
    return best


class Rasterizer:
    """One plan (Gaussian count, SH degree, cameras) and its device buffers."""

    def __init__(self, gaussians: Gaussians, cameras: list, config: Config | None = None,
                 key_capacity: int | None = None, device=None):
        self.config = config or Config()
        self.cfg_c = self.config.to_c()
        self.cams = [c if isinstance(c, N.sr_camera) else camera_from_dict(c) for c in cameras]
        self.device = torch.device(device) if device is not None else gaussians.means.device
        self.n_views = len(self.cams)
        self._g_desc = gaussians.to_c()
        raw = b"".join(bytes(c) for c in self.cams)
        self.cams_dev = torch.frombuffer(bytearray(raw), dtype=torch.uint8).to(self.device)
        if key_capacity is None:
            key_capacity = max(1 << 16, 8 * gaussians.n * self.n_views)
        self._make_plan(int(key_capacity))

    def _make_plan(self, key_capacity: int):
        key_capacity = min(key_capacity, 0xFFFFFFFF)
        self.plan = N.sr_plan_init(self.cfg_c, self._g_desc, self.cams, key_capacity)
        self.ws = torch.empty(int(self.plan.ws_bytes), dtype=torch.uint8, device=self.device)
        p = self.plan
        self.images = torch.empty(int(p.image_offset[self.n_views]), dtype=torch.float32, device=self.device)
        self.t_final = torch.empty(int(p.total_pixels), dtype=torch.float32, device=self.device)
        self.n_contrib = torch.empty(int(p.total_pixels), dtype=torch.int32, device=self.device)

    @property
    def key_capacity(self) -> int:
        return int(self.plan.key_capacity)

    def set_cameras(self, cameras: list):
        """Replace the cameras of the plan with views of the same sizes."""
        cams = [c if isinstance(c, N.sr_camera) else camera_from_dict(c) for c in cameras]
        if len(cams) != self.n_views or any((c.width, c.height) != (o.width, o.height) for c, o in zip(cams, self.cams)):
            raise ValueError("set_cameras needs the same number of views with the same sizes")
        self.cams = cams
        raw = b"".join(bytes(c) for c in cams)
        self.cams_dev.copy_(torch.frombuffer(bytearray(raw), dtype=torch.uint8))

    def view_image(self, flat: torch.Tensor, v: int) -> torch.Tensor:
        p = self.plan
        return flat[p.image_offset[v]:p.image_offset[v + 1]].view(3, p.height[v], p.width[v])

    def view_state(self, flat: torch.Tensor, v: int) -> torch.Tensor:
        p = self.plan
        return flat[p.pixel_offset[v]:p.pixel_offset[v + 1]].view(p.height[v], p.width[v])

    # -- stages ------------------------------------------------------------
    def preprocess(self, g: Gaussians, stream=None):
        N.sr_preprocess(self.plan, g.to_c(), self.cams_dev.data_ptr(), self.cfg_c, self.ws.data_ptr(),
                        _stream_ptr(stream))

    def bin_sort(self, stream=None, sync: bool = True):
        return N.sr_bin_sort(self.plan, self.cfg_c, self.ws.data_ptr(), _stream_ptr(stream), sync=sync)

    def render_fwd(self, stream=None, out: torch.Tensor | None = None):
        img = self.images if out is None else out
        if out is not None and (out.dtype != torch.float32 or not out.is_contiguous() or
                                out.numel() != self.images.numel() or out.device != self.images.device):
            raise ValueError("out must be a contiguous float32 tensor shaped like the image buffer")
        N.sr_render_fwd(self.plan, self.cfg_c, self.ws.data_ptr(), img.data_ptr(), self.t_final.data_ptr(),
                        self.n_contrib.data_ptr(), _stream_ptr(stream))
        return img

    def forward(self, g: Gaussians, stream=None, grow: bool = True, out: torch.Tensor | None = None,
                sync: bool = True) -> torch.Tensor:
        """Preprocess, bin and sort (growing the key capacity if the frame
        needs more), composite.  Returns the flat image buffer (``out`` if
        given, else the rasterizer's own).  With ``sync=False`` nothing
        blocks the host (the key count is not read back): a frame that
        overflows the key capacity is then reported by ``check()``."""
        self.preprocess(g, stream)
        if not sync:
            self.bin_sort(stream, sync=False)
            return self.render_fwd(stream, out)
        try:
            self.keys = self.bin_sort(stream)
        except N.SkewRasterError as e:
            if e.status != N.SR_ERR_CAPACITY or not grow:
                raise
            self._make_plan(int(e.keys_needed * 1.25) + 1024)
            self.preprocess(g, stream)
            self.keys = self.bin_sort(stream)
        return self.render_fwd(stream, out)

    def check(self, stream=None) -> int:
        """Synchronise and read the last frame's status word: raises
        SkewRasterError on a key-capacity overflow or a bounded wait that gave
        up; returns the frame's key count."""
        s, keys = N.sr_read_status(self.plan, self.ws.data_ptr(), _stream_ptr(stream))
        if s != N.SR_OK:
            err = N.SkewRasterError("sr_read_status", s)
            err.keys_needed = keys
            raise err
        return keys

    def backward_composite(self, d_images: torch.Tensor, stream=None):
        """Reverse replay of the last forward (2D gradients stay in the workspace)."""
        if d_images.dtype != torch.float32 or not d_images.is_contiguous() or d_images.numel() != self.images.numel():
            raise ValueError("d_images must be a contiguous float32 tensor shaped like the image buffer")
        N.sr_render_bwd_composite(self.plan, self.cfg_c, self.ws.data_ptr(), d_images.data_ptr(),
                                  self.t_final.data_ptr(), self.n_contrib.data_ptr(), _stream_ptr(stream))

    def backward_project(self, g: Gaussians, stream=None, want_stats: bool = False) -> dict:
        """Chain rule from the workspace's 2D gradients to every attribute (FP32)."""
        dev = self.device
        n = g.n
        out = dict(means=torch.empty(n, 3, device=dev), log_scales=torch.empty(n, 3, device=dev),
                   quats=torch.empty(n, 4, device=dev),
                   opacity_logits=torch.empty(g.opacity_logits.shape, device=dev),
                   skew=torch.empty(n, 3, device=dev), sh=torch.empty(g.sh.shape, device=dev),
                   split_dir=torch.empty(n, 3, device=dev) if g.split_dir is not None else None)
        if want_stats:
            out["means2d_abs"] = torch.empty(n, device=dev)
            out["depth_grad"] = torch.empty(n, device=dev)
        gr = N.sr_grads()
        for k in ("means", "log_scales", "quats", "opacity_logits", "skew", "sh", "split_dir", "means2d_abs",
                  "depth_grad"):
            t = out.get(k)
            setattr(gr, k, t.data_ptr() if t is not None else None)
        N.sr_render_bwd_project(self.plan, g.to_c(), self.cams_dev.data_ptr(), self.cfg_c, self.ws.data_ptr(), gr,
                                _stream_ptr(stream))
        return out

    def frame_state(self) -> dict:
        """Copies of what a backward of the last forward needs besides the
        workspace (per-pixel T and n_contrib, the cameras): with a
        recompute_keys plan, ``backward(..., state=...)`` can run after the
        rasterizer has rendered other frames."""
        return {"t_final": self.t_final.clone(), "n_contrib": self.n_contrib.clone(),
                "cams_dev": self.cams_dev.clone()}

    def backward(self, g: Gaussians, d_images: torch.Tensor, stream=None, want_stats: bool = False,
                 out: dict | None = None, state: dict | None = None) -> dict:
        """Gradients of sum(d_images * images) w.r.t. every attribute (FP32),
        through sr_render_bwd (into ``out``'s tensors when given, e.g. the
        previous call's result).  ``state`` (from frame_state(), recompute_keys
        plans only): the frame to differentiate, if not the last one."""
        if d_images.dtype != torch.float32 or not d_images.is_contiguous() or d_images.numel() != self.images.numel():
            raise ValueError("d_images must be a contiguous float32 tensor shaped like the image buffer")
        if state is not None and not self.config.recompute_keys:
            raise ValueError("a saved frame state can be replayed only by a recompute_keys plan")
        st = state or {"t_final": self.t_final, "n_contrib": self.n_contrib, "cams_dev": self.cams_dev}
        dev = self.device
        n = g.n
        if out is not None and out["means"].shape[0] == n and (out.get("means2d_abs") is not None) == want_stats:
            return self._backward_into(g, d_images, stream, out, st)
        out = dict(means=torch.empty(n, 3, device=dev), log_scales=torch.empty(n, 3, device=dev),
                   quats=torch.empty(n, 4, device=dev),
                   opacity_logits=torch.empty(g.opacity_logits.shape, device=dev),
                   skew=torch.empty(n, 3, device=dev), sh=torch.empty(g.sh.shape, device=dev),
                   split_dir=torch.empty(n, 3, device=dev) if g.split_dir is not None else None)
        if want_stats:
            out["means2d_abs"] = torch.empty(n, device=dev)
            out["depth_grad"] = torch.empty(n, device=dev)
        gr = N.sr_grads()
        for k in ("means", "log_scales", "quats", "opacity_logits", "skew", "sh", "split_dir", "means2d_abs",
                  "depth_grad"):
            t = out.get(k)
            setattr(gr, k, t.data_ptr() if t is not None else None)
        N.sr_render_bwd(self.plan, g.to_c(), st["cams_dev"].data_ptr(), self.cfg_c, self.ws.data_ptr(),
                        d_images.data_ptr(), st["t_final"].data_ptr(), st["n_contrib"].data_ptr(), gr,
                        _stream_ptr(stream))
        return out

    def _backward_into(self, g: Gaussians, d_images: torch.Tensor, stream, out: dict, st: dict) -> dict:
        gr = N.sr_grads()
        for k in ("means", "log_scales", "quats", "opacity_logits", "skew", "sh", "split_dir", "means2d_abs",
                  "depth_grad"):
            t = out.get(k)
            setattr(gr, k, t.data_ptr() if t is not None else None)
        N.sr_render_bwd(self.plan, g.to_c(), st["cams_dev"].data_ptr(), self.cfg_c, self.ws.data_ptr(),
                        d_images.data_ptr(), st["t_final"].data_ptr(), st["n_contrib"].data_ptr(), gr,
                        _stream_ptr(stream))
        return out

    # -- launch-shape autotuning --------------------------------------------
    def set_pixels_per_thread(self, fwd: int | None = None, bwd: int | None = None):
        if fwd is not None:
            self.config.fwd_pixels_per_thread = int(fwd)
        if bwd is not None:
            self.config.bwd_pixels_per_thread = int(bwd)
        self.cfg_c = self.config.to_c()

    def set_batch(self, fwd: int | None = None, bwd: int | None = None):
        """Records the composites stage in shared memory per batch."""
        if fwd is not None:
            self.config.fwd_batch = int(fwd)
        if bwd is not None:
            self.config.bwd_batch = int(bwd)
        self.cfg_c = self.config.to_c()

    def set_persistent(self, fwd: bool | None = None, bwd: bool | None = None):
        """Persistent composite launches (blocks take tiles from a counter)."""
        bits = int(self.config.persistent)
        if fwd is not None:
            bits = (bits | 1) if fwd else (bits & ~1)
        if bwd is not None:
            bits = (bits | 2) if bwd else (bits & ~2)
        self.config.persistent = bits
        self.cfg_c = self.config.to_c()

    def set_blocks_per_sm(self, fwd: int | None = None, bwd: int | None = None):
        """Caps on the composites' resident blocks per SM (0: as many as fit)."""
        if fwd is not None:
            self.config.fwd_blocks_per_sm = int(fwd)
        if bwd is not None:
            self.config.bwd_blocks_per_sm = int(bwd)
        self.cfg_c = self.config.to_c()

    def autotune(self, g: Gaussians, d_images: torch.Tensor | None = None, candidates=(1, 2, 4), reps: int = 3,
                 stream=None, batches=((128, 256, 512), (128, 256)), blocks=(0, 8, 6, 4)) -> dict:
        """Choose the launch shape of the forward and backward composites by
        timing candidates on this frame (CUDA events on the launching stream,
        best of ``reps``): first how many pixels each thread owns, then how
        many Gaussian records a block stages in shared memory per batch
        (``batches`` = forward and backward candidates), then a cap on the
        resident blocks per SM (``blocks``, 0 = none), then one block per tile
        or a persistent grid; keeps the fastest (a non-default choice only
        when it is more than 2% faster).  The results do not depend on the
        choice."""
        s = stream if stream is not None else torch.cuda.current_stream()
        self.forward(g, stream)

        def best_of(fn):
            ts = []
            for _ in range(reps):
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(s)
                fn()
                b.record(s)
                b.synchronize()
                ts.append(a.elapsed_time(b))
            return min(ts)

        fwd = {}
        for px in candidates:
            self.set_pixels_per_thread(fwd=px)
            self.render_fwd(stream)  # warm
            fwd[px] = best_of(lambda: self.render_fwd(stream))
        pf = min(fwd, key=fwd.get)
        self.set_pixels_per_thread(fwd=pf)
        fb = {}
        for bt in batches[0]:
            self.set_batch(fwd=bt)
            self.render_fwd(stream)  # warm
            fb[bt] = best_of(lambda: self.render_fwd(stream))
        bf = _prefer_default(fb, 256)
        self.set_batch(fwd=bf)
        fo = {}
        for nb in blocks:
            self.set_blocks_per_sm(fwd=nb)
            self.render_fwd(stream)  # warm
            fo[nb] = best_of(lambda: self.render_fwd(stream))
        ofwd = _prefer_default(fo, 0)
        self.set_blocks_per_sm(fwd=ofwd)
        fp = {}
        for on in (False, True):
            self.set_persistent(fwd=on)
            self.render_fwd(stream)  # warm
            fp[on] = best_of(lambda: self.render_fwd(stream))
        pfwd = _prefer_default(fp, False)
        self.set_persistent(fwd=pfwd)
        out = {"fwd_ms": fwd, "fwd_pixels_per_thread": pf, "fwd_batch_ms": fb, "fwd_batch": bf,
               "fwd_blocks_per_sm_ms": fo, "fwd_blocks_per_sm": ofwd, "fwd_persistent_ms": fp,
               "fwd_persistent": pfwd}
        if d_images is not None:
            self.render_fwd(stream)
            bwd = {}
            for px in candidates:
                self.set_pixels_per_thread(bwd=px)
                self.backward(g, d_images, stream)  # warm
                bwd[px] = best_of(lambda: self.backward(g, d_images, stream))
            pb = min(bwd, key=bwd.get)
            self.set_pixels_per_thread(bwd=pb)
            bb = {}
            for bt in batches[1]:
                self.set_batch(bwd=bt)
                self.backward(g, d_images, stream)  # warm
                bb[bt] = best_of(lambda: self.backward(g, d_images, stream))
            bbest = _prefer_default(bb, 128)
            self.set_batch(bwd=bbest)
            bo = {}
            for nb in blocks:
                self.set_blocks_per_sm(bwd=nb)
                self.backward(g, d_images, stream)  # warm
                bo[nb] = best_of(lambda: self.backward(g, d_images, stream))
            obwd = _prefer_default(bo, 0)
            self.set_blocks_per_sm(bwd=obwd)
            bp = {}
            for on in (False, True):
                self.set_persistent(bwd=on)
                self.backward(g, d_images, stream)  # warm
                bp[on] = best_of(lambda: self.backward(g, d_images, stream))
            pbwd = _prefer_default(bp, False)
            self.set_persistent(bwd=pbwd)
            out.update(bwd_ms=bwd, bwd_pixels_per_thread=pb, bwd_batch_ms=bb, bwd_batch=bbest,
                       bwd_blocks_per_sm_ms=bo, bwd_blocks_per_sm=obwd, bwd_persistent_ms=bp, bwd_persistent=pbwd)
        return out

    # -- read-only views of the workspace (tests and diagnostics) ---------
    # slot numbers of the workspace layout (csrc/common.cuh, enum WsSlot)
    _S_STATUS, _S_REC, _S_DEPTH, _S_RECT, _S_NTOUCH = 0, 2, 3, 8, 9
    _S_KEYS0, _S_VALS0, _S_RANGES, _S_D2, _S_MASK, _S_TILE_ORDER = 12, 14, 19, 20, 22, 23

    def _slot(self, k: int, nbytes: int) -> torch.Tensor:
        off = int(self.plan.off[k])
        return self.ws[off:off + nbytes]

    def sorted_keys(self):
        """The last frame's sorted list as (tile << 32 | FP32 depth bits) keys
        (int64 tensor holding the uint64 bits) and record indices (int32)."""
        kn = int(self.keys)
        st = self._slot(self._S_STATUS, 16).clone().cpu().numpy()
        buf = int(st[4:8].view(np.uint32)[0])
        tiles = self._slot(self._S_KEYS0 + buf, 4 * kn).view(torch.int32).to(torch.int64) & 0xFFFFFFFF
        vals = self._slot(self._S_VALS0 + buf, 4 * kn).view(torch.int32)
        depth = self.depth_bits().to(torch.int64) & 0xFFFFFFFF
        keys = (tiles << 32) | depth[vals.to(torch.int64)] if kn else tiles
        return keys, vals

    def records(self) -> torch.Tensor:
        m = self.plan.n * self.n_views
        return self._slot(self._S_REC, 64 * m).view(torch.float32).view(m, 16)

    def depth_bits(self) -> torch.Tensor:
        m = self.plan.n * self.n_views
        return self._slot(self._S_DEPTH, 4 * m).view(torch.int32)

    def tile_counts(self) -> torch.Tensor:
        m = self.plan.n * self.n_views
        return self._slot(self._S_NTOUCH, 4 * m).view(torch.int32)

    def rects(self) -> torch.Tensor:
        m = self.plan.n * self.n_views
        return self._slot(self._S_RECT, 8 * m).view(torch.int32).view(m, 2)

    def ranges(self) -> torch.Tensor:
        """[total_tiles, 2] int64: [start, end) of each tile's run in the
        sorted key list of the last frame (empty tiles [0, 0))."""
        t = int(self.plan.total_tiles)
        raw = self._slot(self._S_RANGES, 8 * t).view(torch.int32).view(t, 2).to(torch.int64) & 0xFFFFFFFF
        start = torch.where(raw[:, 1] > 0, (~raw[:, 0]) & 0xFFFFFFFF, torch.zeros_like(raw[:, 0]))
        return torch.stack([start, raw[:, 1]], 1)

    def tile_order(self) -> torch.Tensor:
        """[total_tiles] int64: the order in which the last frame's composites
        take the tiles (heaviest key lists first)."""
        t = int(self.plan.total_tiles)
        return self._slot(self._S_TILE_ORDER, 4 * t).view(torch.int32).to(torch.int64) & 0xFFFFFFFF

    def blend_masks(self) -> torch.Tensor:
        """The last forward's per-pixel blend masks (int32 words; layout in
        render.cu: tile t's word for pixel i of the tile and positions
        start + 32c .. start + 32c + 31 of its range at ((start >> 5) + t + c)
        * 256 + i, valid up to the word holding the pixel's last blend)."""
        if self.plan.forward_only or self.plan.recompute_keys:
            raise ValueError("forward-only and recompute-keys plans keep no blend masks")
        words = (int(self.plan.key_capacity) // 32 + int(self.plan.total_tiles) + 1) * 256
        return self._slot(self._S_MASK, 4 * words).view(torch.int32)

    def blend_lists(self, v: int = 0):
        """Per pixel of view v, the Gaussians the last forward blended (see
        the module-level blend_lists)."""
        return blend_lists(self, v)

    def d2(self) -> torch.Tensor:
        """The 2D gradients of every (view, Gaussian) record after a backward
        composite, [M, 14] in the order of ``native.D2_NAMES``."""
        m = self.plan.n * self.n_views
        raw = self._slot(self._S_D2, 64 * m).view(torch.float32).view(m, 16)
        return raw[:, torch.as_tensor(N.D2_SLOTS, device=raw.device)]


def blend_lists(r, v: int, rows_per_block: int = 64):
    """The Gaussians (indices within the view) the last forward of rasterizer
    ``r`` blended at each pixel of view v, in blend order, read from its blend
    masks, tile ranges, sorted values and n_contrib: (offsets int64 [H*W + 1],
    ids int32), pixels row-major (a diagnostic of the workspace; host-side
    decoding only)."""
    p = r.plan
    n = int(p.n)
    H, W = int(p.height[v]), int(p.width[v])
    tiles_x = -(-W // 16)
    tb = int(p.tile_base[v])
    ranges = r.ranges().cpu().numpy()
    mask = r.blend_masks().cpu().numpy().view(np.uint32)
    _, vals = r.sorted_keys()
    vals = vals.cpu().numpy().astype(np.int64) - v * n
    nc_all = r.view_state(r.n_contrib, v).cpu().numpy().astype(np.int64).reshape(-1)
    counts = np.zeros(H * W, np.int64)
    chunks = []
    for y0 in range(0, H, rows_per_block):
        y1 = min(H, y0 + rows_per_block)
        ys, xs = np.meshgrid(np.arange(y0, y1), np.arange(W), indexing="ij")
        ys, xs = ys.reshape(-1), xs.reshape(-1)
        pix = ys * W + xs
        nc = nc_all[pix]
        tile = tb + (ys // 16) * tiles_x + xs // 16
        start = ranges[tile, 0]
        assert np.all(nc <= ranges[tile, 1] - start)
        pi = (ys % 16) * 16 + xs % 16
        nch = (nc + 31) // 32
        tot = int(nch.sum())
        if tot == 0:
            continue
        owner = np.repeat(np.arange(len(pix)), nch)
        first = np.repeat(np.cumsum(nch) - nch, nch)
        c = np.arange(tot) - first
        words = mask[((start[owner] >> 5) + tile[owner] + c) * 256 + pi[owner]]
        bits = np.unpackbits(words.view(np.uint8).reshape(-1, 4), axis=1, bitorder="little").astype(bool)
        bits &= (np.arange(32)[None, :] + 32 * c[:, None]) < nc[owner][:, None]
        wr, b = np.nonzero(bits)                      # row-major: by pixel, then chunk, then bit
        pos = 32 * c[wr] + b
        own = owner[wr]
        ids = vals[start[own] + pos]
        counts[pix] = np.bincount(own, minlength=len(pix))
        chunks.append(ids.astype(np.int32))
    off = np.zeros(H * W + 1, np.int64)
    np.cumsum(counts, out=off[1:])
    ids = np.concatenate(chunks) if chunks else np.zeros(0, np.int32)
    assert ids.size == off[-1]
    return off, ids


def shard_views(cameras: list, rank: int, world: int) -> list:
    """Indices of the views rank ``rank`` of ``world`` renders: views are
    independent, so they are dealt out largest first (by pixel count) to the
    rank with the least work so far (ties to the lowest rank).  No data moves
    between ranks; each renders its share with its own plan."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank / world")
    size = [int(c["width"]) * int(c["height"]) if isinstance(c, dict) else int(c.width) * int(c.height)
            for c in cameras]
    load = [0] * world
    owner = [0] * len(cameras)
    for i in sorted(range(len(cameras)), key=lambda k: (-size[k], k)):
        r = min(range(world), key=lambda q: (load[q], q))
        owner[i] = r
        load[r] += size[i]
    return [i for i in range(len(cameras)) if owner[i] == rank]


def render_views_recompute(g: Gaussians, cameras: list, d_images: list, config: Config | None = None,
                           rasterizers: dict | None = None):
    """Forward and backward of several views through one single-view
    recompute_keys workspace per image size: every view is rendered first
    (keeping only its image, per-pixel T and n_contrib), then each view's
    backward rebuilds its records and tile key lists inside sr_render_bwd and
    replays with the alpha gate (no blend masks, no key list kept between
    the passes).  Returns the images (list of [3,H,W] tensors) and the
    attribute gradients summed over views.  ``rasterizers`` may carry plans
    from an earlier call (keyed by size)."""
    config = Config(**{**config.__dict__, "recompute_keys": True}) if config else Config(recompute_keys=True)
    rasterizers = {} if rasterizers is None else rasterizers

    def plan_for(cam):
        c = cam if isinstance(cam, N.sr_camera) else camera_from_dict(cam)
        key = (c.width, c.height)
        if key not in rasterizers:
            rasterizers[key] = Rasterizer(g, [c], config)
        r = rasterizers[key]
        r.set_cameras([c])
        return r

    images, states = [], []
    for cam in cameras:  # forward: keep the images and the per-pixel state
        r = plan_for(cam)
        images.append(r.forward(g).view(3, r.plan.height[0], r.plan.width[0]).clone())
        states.append(r.frame_state())
    total = None
    for cam, dimg, st in zip(cameras, d_images, states):  # backward: the keys are rebuilt by sr_render_bwd
        r = plan_for(cam)
        gr = r.backward(g, dimg.reshape(-1).contiguous(), state=st)
        if total is None:
            total = gr
        else:
            for k, t in gr.items():
                if t is not None:
                    total[k] += t
    return images, total


class _RasterizeFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, rast, sh_degree, means, log_scales, quats, opacity_logits, skew, sh, split_dir):
        g = Gaussians(means.detach(), log_scales.detach(), quats.detach(), opacity_logits.detach(), skew.detach(),
                      sh.detach(), sh_degree, None if split_dir is None else split_dir.detach())
        images = rast.forward(g).clone()
        ctx.rast = rast
        ctx.g = g
        # a recompute_keys plan may render other frames before this backward
        ctx.state = rast.frame_state() if rast.config.recompute_keys else None
        ctx.mark_non_differentiable()
        return images

    @staticmethod
    def backward(ctx, d_images):
        g = ctx.g
        gr = ctx.rast.backward(g, d_images.contiguous().float(), state=ctx.state)
        cast = lambda t, like: None if t is None else t.to(like.dtype)
        return (None, None, gr["means"], cast(gr["log_scales"], g.log_scales), gr["quats"], gr["opacity_logits"],
                cast(gr["skew"], g.skew), cast(gr["sh"], g.sh),
                None if g.split_dir is None else cast(gr["split_dir"], g.split_dir))


def render(rast: Rasterizer, means, log_scales, quats, opacity_logits, skew, sh, sh_degree: int, split_dir=None):
    """Differentiable render of every view of ``rast``: the flat image buffer
    (views at rast.plan.image_offset[v], each [3,H,W])."""
    return _RasterizeFn.apply(rast, sh_degree, means, log_scales, quats, opacity_logits, skew, sh, split_dir)
