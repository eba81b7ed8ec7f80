"""The training step around the rasterizer: photometric loss and Adam.

The paper optimises its skew Gaussians inside the 3DGS framework
(Preliminaries: gradient descent driven by a photometric loss; Appendix
"Implementation": the 3DGS protocol, learning rate 1e-4 for the skew
parameters).  A step is render (forward) -> loss and dL/dC
(``sr_loss_l1_dssim``) -> backward to every attribute (``sr_render_bwd``) ->
one Adam update of every attribute (``sr_adam_step``); every step runs in the
CUDA library, this module only holds buffers and calls it.
"""
from __future__ import annotations

import torch

from . import native as N
from .rasterizer import Config, Gaussians, Rasterizer, _stream_ptr

# Learning rates: 3DGS's for positions, SH features (the degree-0 coefficients
# and, 20x smaller, the rest), opacity, scales and rotations; the paper's 1e-4
# for the skew vector (and its split direction).
DEFAULT_LR = dict(means=1.6e-4, sh=2.5e-3, sh_rest=2.5e-3 / 20, opacity_logits=5e-2, log_scales=5e-3,
                  quats=1e-3, skew=1e-4, split_dir=1e-4)


class PhotometricLoss:
    """L = (1 - lam) mean|C - T| + lam (1 - mean SSIM(C, T)) over all views of a
    rasterizer's plan, and dL/dC in the image layout."""

    def __init__(self, rast: Rasterizer, lam: float = 0.2):
        self.rast = rast
        self.lam = float(lam)
        dev = rast.device
        self.scratch = torch.empty(N.sr_loss_scratch_size(rast.plan), dtype=torch.uint8, device=dev)
        self.loss = torch.zeros(1, device=dev)
        self.stats = torch.zeros(2, device=dev)  # mean SSIM, mean |C - T|
        self.d_images = torch.empty_like(rast.images)

    def __call__(self, targets: torch.Tensor, stream=None) -> torch.Tensor:
        if targets.dtype != torch.float32 or not targets.is_contiguous() or targets.numel() != self.rast.images.numel():
            raise ValueError("targets must be a contiguous float32 tensor shaped like the image buffer")
        if self.scratch.numel() != N.sr_loss_scratch_size(self.rast.plan):
            self.scratch = torch.empty(N.sr_loss_scratch_size(self.rast.plan), dtype=torch.uint8,
                                       device=self.rast.device)
        N.sr_loss_l1_dssim(self.rast.plan, self.rast.ws.data_ptr(), self.rast.images.data_ptr(), targets.data_ptr(),
                           self.lam, self.d_images.data_ptr(), self.loss.data_ptr(), self.stats.data_ptr(),
                           self.scratch.data_ptr(), _stream_ptr(stream))
        return self.loss


_FIELDS = ("means", "log_scales", "quats", "opacity_logits", "skew", "sh", "split_dir")


class Adam:
    """Adam moments for every attribute of a (FP32) scene and the fused update."""

    def __init__(self, g: Gaussians, lr: dict | None = None, betas=(0.9, 0.999), eps: float = 1e-15):
        self.g = g
        self.lr = dict(DEFAULT_LR, **(lr or {}))
        self.betas = betas
        self.eps = float(eps)
        self.step_count = 0
        self.state = {}
        for k in _FIELDS:
            p = getattr(g, k)
            if p is None:
                continue
            if p.dtype != torch.float32:
                raise TypeError(f"{k}: training updates FP32 attributes")
            self.state[k] = (torch.zeros_like(p), torch.zeros_like(p))

    def step(self, grads: dict, stream=None):
        self.step_count += 1
        groups = []
        k3 = 3 * (self.g.sh_degree + 1) ** 2
        for k, (m, v) in self.state.items():
            p = getattr(self.g, k)
            gr = grads[k]
            grp = N.sr_adam_group()
            grp.param, grp.grad, grp.m, grp.v = p.data_ptr(), gr.data_ptr(), m.data_ptr(), v.data_ptr()
            grp.n = p.numel()
            grp.lr = self.lr[k]
            if k == "sh":  # degree-0 coefficients: the first 3 of each Gaussian's 3K
                grp.lr_rest, grp.period, grp.split_at = self.lr["sh_rest"], k3, 3
            else:
                grp.lr_rest, grp.period, grp.split_at = self.lr[k], 0, 0
            groups.append(grp)
        N.sr_adam_step(groups, self.step_count, self.betas[0], self.betas[1], self.eps, _stream_ptr(stream))


class Trainer:
    """Fits a scene's attributes to target images of its cameras."""

    def __init__(self, g: Gaussians, cameras: list, targets: torch.Tensor, config: Config | None = None,
                 lr: dict | None = None, lam: float = 0.2, key_capacity: int | None = None,
                 densify_stats: bool = False):
        self.g = g
        self.rast = Rasterizer(g, cameras, config, key_capacity=key_capacity)
        self.targets = targets
        self.loss = PhotometricLoss(self.rast, lam)
        self.adam = Adam(g, lr)
        self.grads = None
        # densification statistics over the steps (Sec. "Depth-Aware
        # Densification Strategy"): g^(uv) summed with its step count, g^(z) max
        self.densify_stats = densify_stats
        if densify_stats:
            dev = g.means.device
            self.uv_sum = torch.zeros(g.n, device=dev)
            self.seen = torch.zeros(g.n, dtype=torch.int32, device=dev)
            self.z_max = torch.zeros(g.n, device=dev)

    def densify(self, grad_uv: float, grad_z: float, log_scale_split: float, logit_prune: float,
                stream=None) -> dict:
        """One densification (``sr_densify``) from the statistics collected
        since the last one: the scene is replaced by the densified one, the
        Adam moments follow their Gaussians (new ones start at zero), the
        statistics restart from zero and the rasterizer is re-planned for the
        new size.  Returns the counts (kept, cloned, split, total)."""
        if not self.densify_stats:
            raise RuntimeError("the trainer was made without densify_stats=True")
        from .densify import densify, remap_state
        res = densify(self.g, self.uv_sum, self.seen, self.z_max, grad_uv, grad_z, log_scale_split, logit_prune,
                      stream)
        ng = res.gaussians
        for k, (m, v) in list(self.adam.state.items()):
            self.adam.state[k] = (remap_state(m, res, stream), remap_state(v, res, stream))
        self.g = ng
        self.adam.g = ng
        cams, cfg = self.rast.cams, self.rast.config
        cap = max(1 << 16, int(self.rast.key_capacity * max(1.0, ng.n / max(1, res.src_map.numel() // 2))))
        self.rast = Rasterizer(ng, cams, cfg, key_capacity=cap)
        self.loss = PhotometricLoss(self.rast, self.loss.lam)
        self.grads = None
        dev = ng.means.device
        self.uv_sum = torch.zeros(ng.n, device=dev)
        self.seen = torch.zeros(ng.n, dtype=torch.int32, device=dev)
        self.z_max = torch.zeros(ng.n, device=dev)
        self.last_densify = res  # source and kind of every new Gaussian
        return res.counts

    def step(self, stream=None) -> torch.Tensor:
        """One training step; returns the device loss of the rendered frame."""
        self.rast.forward(self.g, stream)
        if self.loss.d_images.numel() != self.rast.images.numel():  # the plan grew: new image buffer sizes
            self.loss = PhotometricLoss(self.rast, self.loss.lam)
        loss = self.loss(self.targets, stream)
        self.grads = self.rast.backward(self.g, self.loss.d_images, stream, want_stats=self.densify_stats,
                                        out=self.grads)
        if self.densify_stats:
            N.sr_densify_stats(self.grads["means2d_abs"].data_ptr(), self.grads["depth_grad"].data_ptr(), self.g.n,
                               self.uv_sum.data_ptr(), self.seen.data_ptr(), self.z_max.data_ptr(),
                               _stream_ptr(stream))
        self.adam.step(self.grads, stream)
        return loss
