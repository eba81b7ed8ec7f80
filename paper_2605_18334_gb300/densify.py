"""Densification of a scene (Sec. "Depth-Aware Densification Strategy"; the
split of Fig. "split") through ``sr_densify``: remove, keep, clone or split
every Gaussian from the statistics ``sr_densify_stats`` collected, and carry
per-Gaussian state (the Adam moments) over with ``sr_densify_remap``.  The
work runs in the CUDA library; this module allocates the outputs and reads
back the new size."""
from __future__ import annotations

from dataclasses import dataclass

import torch

from . import native as N
from .rasterizer import Gaussians, _stream_ptr


@dataclass
class DensifyResult:
    gaussians: Gaussians
    src: torch.Tensor       # [n_out] int64: source Gaussian of each output
    kind: torch.Tensor      # [n_out] int32: 0 kept, 1 clone copy, 2 child (+ side), 3 child (- side)
    src_map: torch.Tensor   # [capacity] the library's packed map (source | kind << 30)
    counts_dev: torch.Tensor  # [4] int64 on the device: kept, cloned, split, total
    counts: dict


def densify(g: Gaussians, uv_sum: torch.Tensor, seen: torch.Tensor, z_max: torch.Tensor, grad_uv: float,
            grad_z: float, log_scale_split: float, logit_prune: float, stream=None) -> DensifyResult:
    """New scene (FP32) after one densification step; reads the output count
    back (one synchronisation)."""
    for name in ("means", "log_scales", "quats", "opacity_logits", "skew", "sh"):
        if getattr(g, name).dtype != torch.float32:
            raise TypeError(f"densification works on FP32 attributes ({name} is {getattr(g, name).dtype})")
    n, dev = g.n, g.means.device
    cap = 2 * n
    k = (g.sh_degree + 1) ** 2
    out = Gaussians(torch.empty(cap, 3, device=dev), torch.empty(cap, 3, device=dev), torch.empty(cap, 4, device=dev),
                    torch.empty((cap,) + tuple(g.opacity_logits.shape[1:]), device=dev),
                    torch.empty(cap, 3, device=dev), torch.empty(cap, k, 3, device=dev), g.sh_degree,
                    torch.empty(cap, 3, device=dev) if g.split_dir is not None else None)
    arrays = N.sr_scene_arrays()
    for f in ("means", "log_scales", "quats", "opacity_logits", "skew", "sh"):
        setattr(arrays, f, getattr(out, f).data_ptr())
    arrays.split_dir = out.split_dir.data_ptr() if out.split_dir is not None else None
    src_map = torch.empty(max(cap, 1), dtype=torch.int32, device=dev)
    counts = torch.zeros(4, dtype=torch.int64, device=dev)
    scratch = torch.empty(N.sr_densify_scratch_size(n), dtype=torch.uint8, device=dev)
    cfg = N.sr_densify_config(float(grad_uv), float(grad_z), float(log_scale_split), float(logit_prune))
    for t, dt in ((uv_sum, torch.float32), (seen, torch.int32), (z_max, torch.float32)):
        if t.dtype != dt or t.numel() != n or not t.is_contiguous():
            raise ValueError("statistics must be contiguous [n] tensors (uv_sum, z_max float32; seen int32)")
    N.sr_densify(g.to_c(), uv_sum.data_ptr(), seen.data_ptr(), z_max.data_ptr(), cfg, arrays, src_map.data_ptr(),
                 counts.data_ptr(), scratch.data_ptr(), _stream_ptr(stream))
    kept, cloned, split, total = (int(v) for v in counts.cpu().tolist())
    m = src_map[:total].to(torch.int64) & 0xFFFFFFFF
    cut = lambda t: None if t is None else t[:total]
    ng = Gaussians(cut(out.means), cut(out.log_scales), cut(out.quats), cut(out.opacity_logits), cut(out.skew),
                   cut(out.sh), g.sh_degree, cut(out.split_dir))
    return DensifyResult(ng, m & 0x3FFFFFFF, (m >> 30).to(torch.int32), src_map, counts,
                         dict(kept=kept, cloned=cloned, split=split, total=total))


def remap_state(t: torch.Tensor, res: DensifyResult, stream=None) -> torch.Tensor:
    """Per-Gaussian state [n, ...] (FP32) for the densified scene: kept
    Gaussians keep theirs, new ones start at zero."""
    if t.dtype != torch.float32 or not t.is_contiguous():
        raise ValueError("state must be a contiguous float32 tensor")
    width = t[0].numel() if t.shape[0] else 0
    total = res.counts["total"]
    out = torch.empty((total,) + tuple(t.shape[1:]), dtype=torch.float32, device=t.device)
    N.sr_densify_remap(t.data_ptr(), width, res.src_map.data_ptr(), res.counts_dev.data_ptr(), total,
                       out.data_ptr(), _stream_ptr(stream))
    return out
