"""Densification: oracle pins (CPU) and the CUDA path against the oracle (GPU).

The split follows the reading in ``oracle/densify_oracle.py``: a skew
Gaussian is cut at its centre across its largest axis and each child matches
the mass-normalised mean and variance of its half.  The oracle's closed forms
are pinned here by numerical quadrature and by Monte Carlo samples of the 3D
skew normal, not by re-deriving them."""
from __future__ import annotations

import math

import numpy as np
import pytest

from oracle import densify_oracle as D


def _sn_pdf(z, alpha):
    return 2.0 * np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi) * 0.5 * (1.0 + _erf(alpha * z / math.sqrt(2.0)))


def _erf(x):
    return np.vectorize(math.erf)(x) if np.ndim(x) else math.erf(x)


@pytest.mark.parametrize("alpha", [0.0, 0.7, -1.3, 4.0, -12.0])
def test_half_moments_against_quadrature(alpha):
    integrate = pytest.importorskip("scipy.integrate")
    delta = alpha / math.sqrt(1.0 + alpha * alpha)
    wp, mp, vp, wn, mn, vn = D.half_moments(delta)
    for lo, hi, w, m, v in ((0.0, np.inf, wp, mp, vp), (-np.inf, 0.0, wn, mn, vn)):
        mom = [integrate.quad(lambda z, p=p: z ** p * _sn_pdf(z, alpha), lo, hi, epsabs=1e-13, epsrel=1e-12)[0]
               for p in range(3)]
        assert abs(mom[0] - w) < 1e-10
        assert abs(mom[1] / mom[0] - m) < 1e-9
        assert abs(mom[2] / mom[0] - (mom[1] / mom[0]) ** 2 - v) < 1e-8


def test_half_moments_zero_skew_is_the_half_normal():
    wp, mp, vp, wn, mn, vn = D.half_moments(0.0)
    assert wp == wn == 0.5
    assert abs(mp - math.sqrt(2.0 / math.pi)) < 1e-15 and abs(mn + math.sqrt(2.0 / math.pi)) < 1e-15
    assert abs(vp - (1.0 - 2.0 / math.pi)) < 1e-15 and abs(vn - vp) < 1e-15


@pytest.mark.parametrize("delta", [0.0, 0.3, -0.8, 0.999])
def test_children_mixture_matches_the_parent_along_the_axis(delta):
    wp, mp, vp, wn, mn, vn = D.half_moments(delta)
    assert abs(wp + wn - 1.0) < 1e-15
    # mean and second moment of SN(0, 1, alpha): sqrt(2/pi) delta and 1
    assert abs(wp * mp + wn * mn - math.sqrt(2.0 / math.pi) * delta) < 1e-14
    assert abs(wp * (vp + mp * mp) + wn * (vn + mn * mn) - 1.0) < 1e-14
    assert vp > 0.0 and vn > 0.0


def _sample_sn3(eta, n, rng):
    """Stochastic representation of SN_3(0, I, eta): Z = delta |U0| + (I -
    delta delta^T)^(1/2) U with delta = eta / sqrt(1 + |eta|^2)."""
    eta = np.asarray(eta, np.float64)
    delta = eta / math.sqrt(1.0 + eta @ eta)
    cov = np.eye(3) - np.outer(delta, delta)
    ev, evec = np.linalg.eigh(cov)
    root = evec @ np.diag(np.sqrt(ev)) @ evec.T
    return np.abs(rng.standard_normal(n))[:, None] * delta[None, :] + rng.standard_normal((n, 3)) @ root


def test_children_against_monte_carlo_of_the_3d_skew_normal():
    rng = np.random.default_rng(5)
    eta = np.array([0.4, -1.7, 0.9])
    ls = np.log(np.array([0.05, 0.2, 0.1]))  # largest axis k = 1
    mu = np.array([0.3, -0.2, 4.0])
    q = np.array([0.9, 0.1, -0.3, 0.2])
    R = D.rotation(q)
    n = 2_000_000
    z = _sample_sn3(eta, n, rng)
    x = mu[None, :] + (z * np.exp(ls)[None, :]) @ R.T  # X = mu + R S Z
    (mu_p, ls_p, eta_p), (mu_n, ls_n, eta_n) = D.split_children(mu, ls, q, eta)
    k = 1
    for sel, mu_c, ls_c in ((z[:, k] >= 0, mu_p, ls_p), (z[:, k] < 0, mu_n, ls_n)):
        half = x[sel]
        u = (half - mu[None, :]) @ R[:, k]  # coordinate along the world axis of the split
        se = u.std() / math.sqrt(len(u))
        assert abs(u.mean() - (mu_c - mu) @ R[:, k]) < 5 * se
        assert abs(u.var() - math.exp(2 * ls_c[k])) < 5 * math.sqrt(2.0 / len(u)) * u.var()
        # the child moves along the split axis only
        off = mu_c - mu
        assert np.linalg.norm(off - (off @ R[:, k]) * R[:, k]) < 1e-12
        assert np.allclose(np.delete(ls_c, k), np.delete(ls, k), rtol=0, atol=0)
    # mass of each half
    wp = D.half_moments(eta[k] / math.sqrt(1 + eta @ eta))[0]
    assert abs((z[:, k] >= 0).mean() - wp) < 5 * math.sqrt(wp * (1 - wp) / n)
    # on the other axes a child keeps the parent's marginal skew: the mean of
    # the parent's Z_j is sqrt(2/pi) delta_j, and the child's delta'_j equals it
    for eta_c in (eta_p, eta_n):
        assert eta_c[k] == 0.0
        d_c = eta_c / math.sqrt(1.0 + eta_c @ eta_c)
        for j in (0, 2):
            assert abs(z[:, j].mean() - math.sqrt(2.0 / math.pi) * d_c[j]) < 5 * z[:, j].std() / math.sqrt(n)


def test_split_axis_follows_the_rotation():
    # 90 degrees about z: local x -> world y, local y -> world -x
    q = np.array([math.cos(math.pi / 4), 0.0, 0.0, math.sin(math.pi / 4)])
    ls = np.log(np.array([0.3, 0.1, 0.1]))
    (mu_p, ls_p, _), (mu_n, _, _) = D.split_children(np.zeros(3), ls, q, np.zeros(3))
    h = 0.3 * math.sqrt(2.0 / math.pi)
    assert np.allclose(mu_p, [0.0, h, 0.0], atol=1e-15) and np.allclose(mu_n, [0.0, -h, 0.0], atol=1e-15)
    assert abs(math.exp(ls_p[0]) - 0.3 * math.sqrt(1 - 2 / math.pi)) < 1e-15


def test_classify_every_branch():
    # Gaussians: removed, kept, cloned (uv), cloned (depth statistic only),
    # split, never seen (uv) but z above threshold and large -> split
    ls = np.log(np.array([[0.01] * 3, [0.01] * 3, [0.01] * 3, [0.01] * 3, [0.5, 0.01, 0.01], [0.02, 0.3, 0.02]]))
    op = np.array([-6.0, 1.0, 1.0, 1.0, 1.0, 0.5])
    uv = np.array([9.0, 0.1, 0.9, 0.1, 0.9, 0.0])
    seen = np.array([3, 2, 3, 2, 3, 0])
    zm = np.array([9.0, 0.0, 0.0, 0.7, 0.0, 0.7])
    act = D.classify(ls, op, uv, seen, zm, grad_uv=0.2, grad_z=0.5, log_scale_split=math.log(0.1),
                     logit_prune=-5.0)
    assert act.tolist() == [0, 1, 2, 2, 3, 3]
    scene = dict(means=np.arange(18, dtype=float).reshape(6, 3), log_scales=ls, quats=np.tile([1.0, 0, 0, 0], (6, 1)),
                 opacity_logits=op, skew=np.zeros((6, 3)), sh=np.arange(18, dtype=float).reshape(6, 1, 3))
    out, src, kind, counts = D.densify(scene, uv, seen, zm, 0.2, 0.5, math.log(0.1), -5.0)
    assert src.tolist() == [1, 2, 3, 2, 3, 4, 4, 5, 5]
    assert kind.tolist() == [0, 0, 0, 1, 1, 2, 3, 2, 3]
    assert counts == dict(kept=3, cloned=2, split=2, total=9)
    assert np.array_equal(out["sh"][3], scene["sh"][2])


# ---------------------------------------------------------------------------
# CUDA path
# ---------------------------------------------------------------------------
def _scene_with_stats(n, seed, two=False, split=False, deg=1):
    from paper_2605_18334_gb300 import scenes
    sc = scenes.cluster(seed=seed, n=n, sh_degree=deg, two_opacities=two, split=split)
    rng = np.random.default_rng(seed + 100)
    # log-scales spread across the split threshold, logits across the prune threshold
    sc.log_scales[:] = rng.normal(-3.0, 0.8, size=sc.log_scales.shape).astype(np.float32)
    stats = dict(uv_sum=(rng.exponential(0.2, n) * (rng.random(n) < 0.8)).astype(np.float32),
                 seen=rng.integers(0, 6, n).astype(np.int32),
                 z_max=rng.exponential(0.1, n).astype(np.float32))
    return sc, stats


def _cfg():
    return dict(grad_uv=0.06, grad_z=0.25, log_scale_split=-3.0, logit_prune=-2.0)


@pytest.mark.gpu
@pytest.mark.parametrize("two,split,deg", [(False, False, 3), (True, True, 1), (False, False, 0)])
def test_densify_matches_oracle(two, split, deg):
    import torch
    from paper_2605_18334_gb300.densify import densify
    from paper_2605_18334_gb300.rasterizer import Gaussians
    n = 20_000 + 77  # several blocks and a ragged tail
    sc, st = _scene_with_stats(n, 41, two, split, deg)
    g = Gaussians.from_scene(sc)
    cfg = _cfg()
    res = densify(g, torch.as_tensor(st["uv_sum"]).cuda(), torch.as_tensor(st["seen"]).cuda(),
                  torch.as_tensor(st["z_max"]).cuda(), **cfg)
    scene = dict(means=sc.means, log_scales=sc.log_scales, quats=sc.quats, opacity_logits=sc.opacity_logits,
                 skew=sc.skew, sh=np.asarray(sc.sh).reshape(n, -1, 3), split_dir=sc.split_dir)
    out, src, kind, counts = D.densify(scene, st["uv_sum"], st["seen"], st["z_max"], **cfg)
    assert res.counts == counts
    assert counts["cloned"] > 100 and counts["split"] > 100 and counts["kept"] < n  # every branch taken
    assert np.array_equal(res.src.cpu().numpy(), src) and np.array_equal(res.kind.cpu().numpy(), kind)
    ng = res.gaussians
    for f in ("means", "log_scales", "quats", "opacity_logits", "skew", "sh", "split_dir"):
        a = getattr(ng, f)
        if a is None:
            assert out.get(f) is None
            continue
        a = a.cpu().numpy().reshape(len(src), -1)
        b = np.asarray(out[f]).reshape(len(src), -1)
        copy = kind < D.CHILD_POS
        # copies are bit-exact; split children within FP32 rounding of the oracle's FP64
        assert np.array_equal(a[copy], b[copy].astype(np.float32)), f
        if f in ("means", "log_scales", "skew"):
            err = np.abs(a[~copy] - b[~copy]).max()
            assert err < 2e-5 * max(1.0, np.abs(b[~copy]).max()), (f, err)
        else:
            assert np.array_equal(a[~copy], b[~copy].astype(np.float32)), f


@pytest.mark.gpu
def test_densify_remaps_optimizer_state_and_handles_edge_cases():
    import torch
    from paper_2605_18334_gb300.densify import densify, remap_state
    from paper_2605_18334_gb300.rasterizer import Gaussians
    n = 5000
    sc, st = _scene_with_stats(n, 43)
    g = Gaussians.from_scene(sc)
    cfg = _cfg()
    args = [torch.as_tensor(st[k]).cuda() for k in ("uv_sum", "seen", "z_max")]
    res = densify(g, *args, **cfg)
    m = torch.randn(n, 3, device="cuda")
    mo = remap_state(m, res)
    src, kind = res.src.cpu().numpy(), res.kind.cpu().numpy()
    ref = np.where((kind == D.KEPT)[:, None], m.cpu().numpy()[src], 0.0)
    assert np.array_equal(mo.cpu().numpy(), ref.astype(np.float32))
    # nothing densified, nothing removed: the identity
    res0 = densify(g, *args, grad_uv=1e30, grad_z=1e30, log_scale_split=0.0, logit_prune=-1e30)
    assert res0.counts == dict(kept=n, cloned=0, split=0, total=n)
    assert torch.equal(res0.gaussians.sh, g.sh) and torch.equal(res0.gaussians.means, g.means)
    # everything removed, and an empty scene
    res1 = densify(g, *args, grad_uv=0.0, grad_z=0.0, log_scale_split=0.0, logit_prune=1e30)
    assert res1.counts["total"] == 0 and res1.gaussians.n == 0
