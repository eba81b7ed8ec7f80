"""FP64 oracle of the training step around the rasterizer (test infrastructure).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU baseline
use this module; the product path never imports it.  Plain numpy, slow and
literal:

* the photometric loss of the 3DGS protocol the paper trains with
  (Preliminaries: "driven by photometric loss"; Appendix "Implementation"):
  L = (1 - lam) mean|C - T| + lam (1 - mean SSIM(C, T)), SSIM per channel
  with an 11 x 11 Gaussian window (sigma 1.5, normalised, zero padding),
  C1 = 0.01^2, C2 = 0.03^2 (Wang et al. 2004, the index's definition);
* its gradient dL/dC by the chain rule through the windowed moments;
* one Adam step (Kingma & Ba 2015), in torch.optim.Adam's form.

Pins (tests/test_train.py): SSIM(x, x) = 1; the windowed moments against
scipy.ndimage's correlation; the gradient against central differences of the
FP64 loss; Adam against torch.optim.Adam in FP64.
"""
from __future__ import annotations

import numpy as np

C1, C2 = 0.01 ** 2, 0.03 ** 2


def gaussian_window(size: int = 11, sigma: float = 1.5) -> np.ndarray:
    k = np.arange(size) - size // 2
    w = np.exp(-(k * k) / (2.0 * sigma * sigma))
    return w / w.sum()


def window_filter(img: np.ndarray, w: np.ndarray | None = None) -> np.ndarray:
    """Correlation of a 2-D array with the separable window w (x) w, zero
    outside the array, same size as the input."""
    w = gaussian_window() if w is None else w
    r = len(w) // 2
    H, W = img.shape
    pad = np.zeros((H + 2 * r, W + 2 * r))
    pad[r:r + H, r:r + W] = img
    rows = sum(w[k] * pad[:, k:k + W] for k in range(len(w)))
    return sum(w[k] * rows[k:k + H, :] for k in range(len(w)))


def ssim_map(x: np.ndarray, y: np.ndarray) -> np.ndarray:
    """SSIM index at every pixel of one channel."""
    mx, my = window_filter(x), window_filter(y)
    sx = window_filter(x * x) - mx * mx
    sy = window_filter(y * y) - my * my
    sxy = window_filter(x * y) - mx * my
    return ((2 * mx * my + C1) * (2 * sxy + C2)) / ((mx * mx + my * my + C1) * (sx + sy + C2))


def photometric_loss(images: list, targets: list, lam: float = 0.2) -> dict:
    """images, targets: per view [3][H][W].  Returns L, the mean SSIM and the
    mean |C - T| over all channels and pixels of all views."""
    n = sum(im.size for im in images)
    s = sum(ssim_map(np.asarray(im[c], np.float64), np.asarray(tg[c], np.float64)).sum()
            for im, tg in zip(images, targets) for c in range(3))
    l1 = sum(np.abs(np.asarray(im, np.float64) - np.asarray(tg, np.float64)).sum() for im, tg in zip(images, targets))
    return dict(loss=(1 - lam) * l1 / n + lam * (1 - s / n), ssim=s / n, l1=l1 / n)


def photometric_loss_grad(images: list, targets: list, lam: float = 0.2) -> list:
    """dL/dC per view, by the chain rule through the windowed moments of each
    pixel q (SSIM(q) as a function of mu_x, s_x, s_xy) down to every pixel p
    inside q's window; the window is symmetric, so the adjoint of the
    correlation is the same correlation."""
    n = sum(im.size for im in images)
    out = []
    for im, tg in zip(images, targets):
        g = np.zeros(im.shape)
        for c in range(3):
            x = np.asarray(im[c], np.float64)
            y = np.asarray(tg[c], np.float64)
            mx, my = window_filter(x), window_filter(y)
            sx = window_filter(x * x) - mx * mx
            sy = window_filter(y * y) - my * my
            sxy = window_filter(x * y) - mx * my
            a1, a2 = 2 * mx * my + C1, 2 * sxy + C2
            b1, b2 = mx * mx + my * my + C1, sx + sy + C2
            d_mx = (2 * my * a2 * b1 * b2 - a1 * a2 * b2 * 2 * mx) / (b1 * b2) ** 2  # dS/dmu_x
            d_sx = -a1 * a2 * b1 / (b1 * b2) ** 2                                    # dS/ds_x
            d_sxy = 2 * a1 / (b1 * b2)                                               # dS/ds_xy
            gs = -lam / n  # dL/dS(q)
            # S(q) depends on x_p through mu_x (w), s_x (2 w (x_p - mu_x)) and s_xy (w (y_p - mu_y))
            g[c] = (window_filter(gs * (d_mx - 2 * mx * d_sx - my * d_sxy)) + 2 * x * window_filter(gs * d_sx)
                    + y * window_filter(gs * d_sxy) + (1 - lam) * np.sign(x - y) / n)
        out.append(g)
    return out


def adam_step(p, g, m, v, step: int, lr, beta1=0.9, beta2=0.999, eps=1e-15):
    """One Adam step on FP64 copies (the update of torch.optim.Adam); lr may
    be an array of per-element learning rates.  Returns (p, m, v)."""
    p, g, m, v = (np.asarray(a, np.float64).copy() for a in (p, g, m, v))
    m = beta1 * m + (1 - beta1) * g
    v = beta2 * v + (1 - beta2) * g * g
    bc1, bc2 = 1 - beta1 ** step, 1 - beta2 ** step
    p = p - (np.asarray(lr, np.float64) / bc1) * m / (np.sqrt(v) / np.sqrt(bc2) + eps)
    return p, m, v
