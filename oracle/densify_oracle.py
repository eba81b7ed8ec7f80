"""FP64 oracle of densification (test infrastructure).

Only ``tests/`` and ``bench.py``'s CPU baseline use this module; the product
path never imports it.  Plain numpy, one Gaussian at a time where that reads
more easily.

What it computes (Sec. "Depth-Aware Densification Strategy"; the split of
Fig. "split"), with the readings the paper leaves open:

* Decision per Gaussian, from the statistics collected over the iterations:
  g^(uv) = uv_sum / seen (the mean 2D positional gradient norm, 3DGS's
  criterion) and g^(z) = z_max (Eq. depth_grad).  A Gaussian whose largest
  opacity logit is below ``logit_prune`` is removed; otherwise it is
  densified when g^(uv) >= grad_uv or g^(z) >= grad_z: split when its largest
  log-scale exceeds ``log_scale_split``, cloned otherwise (3DGS's size rule).
  These decisions are taken in FP32, as the kernel takes them.
* Split along the largest axis k (the paper: "split the skew kernel on the
  max axis and adjust the scale of new kernels ... with the skew
  parameters").  In the Gaussian's standardised frame Z = S^-1 R^T (X - mu)
  the skew normal is Z ~ SN_3(0, I, eta), whose marginal along axis k is
  SN(0, 1, alpha_k) with delta_k = eta_k / sqrt(1 + |eta|^2) (closure of the
  skew-normal family under linear maps, Azzalini & Capitanio 1999).  The
  parent is cut at Z_k = 0; child + stands for the half Z_k >= 0, child - for
  Z_k < 0, and each matches the mean and variance of its half along axis k
  (``half_moments``): its centre moves by s_k m_+- along the axis and its
  scale on that axis becomes s_k sqrt(v_+-).  The asymmetry along axis k is
  carried by the unequal pair, so the children take eta_k = 0; on the other
  axes each child keeps the parent's marginal skew exactly:
  eta'_j = delta_j / sqrt(1 - sum_{i != k} delta_i^2).  Rotation, SH,
  opacities and the split direction are copied (as 3DGS copies them).
* Output order: the kept Gaussians in index order (a cloned one included),
  then the clones' copies in index order, then for each split Gaussian in
  index order its children (+, -).  Kinds: 0 kept, 1 clone copy, 2 child +,
  3 child -; the source index of every output.

Pins (tests/test_densify.py): the half moments against numerical quadrature
of the skew-normal density (scipy) and against Monte Carlo samples of the 3D
skew normal built from its stochastic representation; eta = 0 against the
half-normal; the children's mixture against the parent's mean and variance
along the axis; the kept marginal skew against the parent's.
"""
from __future__ import annotations

import math

import numpy as np

KEPT, CLONE, CHILD_POS, CHILD_NEG = 0, 1, 2, 3


def half_moments(delta: float):
    """Mass, mean and variance of each half of Z ~ SN(0, 1, alpha) with
    delta = alpha / sqrt(1 + alpha^2): returns (w+, m+, v+, w-, m-, v-).

    P(Z > 0) = 1/2 + asin(delta) / pi;
    E[Z 1{Z > 0}] = (1 + delta) / sqrt(2 pi);
    E[Z^2 1{Z > 0}] = 1/2 + asin(delta) / pi + delta sqrt(1 - delta^2) / pi;
    the negative half is the positive half of -Z ~ SN(0, 1, -alpha)."""
    d = float(delta)
    a = math.asin(d) / math.pi
    c = d * math.sqrt(max(0.0, 1.0 - d * d)) / math.pi
    wp, wn = 0.5 + a, 0.5 - a
    e1p, e1n = (1.0 + d) / math.sqrt(2.0 * math.pi), -(1.0 - d) / math.sqrt(2.0 * math.pi)
    e2p, e2n = 0.5 + a + c, 0.5 - a - c
    mp, mn = e1p / wp, e1n / wn
    return wp, mp, e2p / wp - mp * mp, wn, mn, e2n / wn - mn * mn


def rotation(q) -> np.ndarray:
    """Rotation matrix of the normalised quaternion (w, x, y, z)."""
    q = np.asarray(q, np.float64)
    w, x, y, z = q / np.linalg.norm(q)
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def split_children(mean, log_scale, quat, skew):
    """The two children of one Gaussian: [(mean, log_scale, skew)] for +, -."""
    mean = np.asarray(mean, np.float64)
    ls = np.asarray(log_scale, np.float64)
    eta = np.asarray(skew, np.float64)
    k = int(np.argmax(ls))  # first of equal maxima
    s_k = math.exp(ls[k])
    axis = rotation(quat)[:, k]
    delta = eta / math.sqrt(1.0 + float(eta @ eta))
    wp, mp, vp, wn, mn, vn = half_moments(delta[k])
    rest = 1.0 - sum(delta[j] ** 2 for j in range(3) if j != k)
    eta_c = np.array([0.0 if j == k else delta[j] / math.sqrt(rest) for j in range(3)])
    out = []
    for m, v in ((mp, vp), (mn, vn)):
        ls_c = ls.copy()
        ls_c[k] = ls[k] + 0.5 * math.log(v)
        out.append((mean + s_k * m * axis, ls_c, eta_c.copy()))
    return out


def classify(log_scales, opacity_logits, uv_sum, seen, z_max, grad_uv, grad_z, log_scale_split, logit_prune):
    """Per-Gaussian action, decided in FP32: 0 remove, 1 keep, 2 keep and
    clone, 3 split."""
    ls = np.asarray(log_scales, np.float32).reshape(-1, 3)
    op = np.asarray(opacity_logits, np.float32)
    op = op.reshape(len(ls), -1).max(axis=1)
    uv = np.asarray(uv_sum, np.float32)
    cnt = np.asarray(seen, np.int32)
    zm = np.asarray(z_max, np.float32)
    act = np.ones(len(ls), np.int32)
    for i in range(len(ls)):
        if op[i] < np.float32(logit_prune):
            act[i] = 0
            continue
        g_uv = np.float32(uv[i] / np.float32(cnt[i])) if cnt[i] > 0 else np.float32(0.0)
        if g_uv >= np.float32(grad_uv) or zm[i] >= np.float32(grad_z):
            act[i] = 3 if ls[i].max() > np.float32(log_scale_split) else 2
    return act


def densify(scene: dict, uv_sum, seen, z_max, grad_uv, grad_z, log_scale_split, logit_prune):
    """New attribute arrays (FP64), source index and kind per output."""
    n = len(scene["means"])
    act = classify(scene["log_scales"], scene["opacity_logits"], uv_sum, seen, z_max, grad_uv, grad_z,
                   log_scale_split, logit_prune)
    fields = [f for f in ("means", "log_scales", "quats", "opacity_logits", "skew", "sh", "split_dir")
              if scene.get(f) is not None]
    src, kind = [], []
    for i in range(n):
        if act[i] in (1, 2):
            src.append(i)
            kind.append(KEPT)
    for i in range(n):
        if act[i] == 2:
            src.append(i)
            kind.append(CLONE)
    for i in range(n):
        if act[i] == 3:
            src += [i, i]
            kind += [CHILD_POS, CHILD_NEG]
    src = np.asarray(src, np.int64)
    kind = np.asarray(kind, np.int32)
    out = {f: np.asarray(scene[f], np.float64)[src].copy() for f in fields}
    for j in np.nonzero(kind >= CHILD_POS)[0]:
        i = src[j]
        ch = split_children(scene["means"][i], scene["log_scales"][i], scene["quats"][i], scene["skew"][i])
        mu, ls, eta = ch[kind[j] - CHILD_POS]
        out["means"][j], out["log_scales"][j], out["skew"][j] = mu, ls, eta
    counts = dict(kept=int(np.sum((act == 1) | (act == 2))), cloned=int(np.sum(act == 2)),
                  split=int(np.sum(act == 3)), total=len(src))
    return out, src, kind, counts
