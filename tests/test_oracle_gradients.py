"""Pin of the oracle's gradients: FP64 central finite differences of the
oracle's own forward (Alg. 1 / Eq. color) against its analytic derivatives
(Appendix "Backward Pass" for dL/dalpha; dual numbers through the
projection).  Stencils that change a discrete decision (gate, clamp, stop,
order) are detected by the per-pixel decision signature and skipped."""
import math

import numpy as np
import pytest

import oracle
from paper_2605_18334_gb300 import scenes


def _scene(seed, n=30, two=True, split=True, deg=3):
    rng = np.random.default_rng(seed)
    K = (deg + 1) ** 2
    means = np.stack([rng.uniform(-0.25, 0.25, n), rng.uniform(-0.25, 0.25, n), rng.uniform(3.0, 4.0, n)], 1)
    sh = rng.normal(0, 0.1, (n, K, 3))
    sh[:, 0, :] = rng.uniform(0.5, 1.5, (n, 3))  # keeps colours well above the clamp at 0
    op = rng.uniform(-1.5, 1.5, (n, 2) if two else (n,))
    return scenes.Scene(means=means, log_scales=rng.uniform(-3.2, -2.4, (n, 3)),
                        quats=rng.normal(size=(n, 4)), opacity_logits=op, skew=rng.normal(0, 1.0, (n, 3)),
                        sh=sh, sh_degree=deg, split_dir=rng.normal(0, 0.7, (n, 3)) if split else None)


def _loss(sc, cam, cfg, g):
    out = oracle.render(sc, cam, cfg)
    return float(np.einsum("chw,hwc->", g, out["rgb"])), out["signature"]


@pytest.mark.parametrize("two,split,deg,bg", [(True, True, 3, (0.2, 0.4, 0.6)), (False, False, 0, (0, 0, 0)),
                                              (False, False, 3, (1, 1, 1))])
def test_gradients_match_central_differences(two, split, deg, bg):
    sc = _scene(seed=11 + deg + 2 * two, two=two, split=split, deg=deg)
    cam = oracle.camera_from_gl(scenes.identity_camera(24, 24))
    cfg = oracle.config(bg=bg)
    g = np.random.default_rng(5).normal(size=(3, 24, 24))
    grads = oracle.render_backward(sc, cam, cfg, g)
    L0, sig0 = _loss(sc, cam, cfg, g)
    fields = ["means", "log_scales", "quats", "opacity_logits", "skew", "sh"] + (["split_dir"] if split else [])
    contributing = np.nonzero(np.abs(grads["d2"]).sum(1) > 0)[0]
    assert contributing.size >= 8
    pick = contributing[:8]
    skipped = 0
    for name in fields:
        arr = getattr(sc, name)
        an_all, fd_all = [], []
        for i in pick:
            for idx in np.ndindex(arr.shape[1:]):
                full = (i,) + idx
                base = arr[full]
                h = 1e-6 * max(1.0, abs(base))
                arr[full] = base + h
                Lp, sp = _loss(sc, cam, cfg, g)
                arr[full] = base - h
                Lm, sm = _loss(sc, cam, cfg, g)
                arr[full] = base
                if not (np.array_equal(sp, sig0) and np.array_equal(sm, sig0)):
                    skipped += 1
                    continue
                fd_all.append((Lp - Lm) / (2 * h))
                an_all.append(grads[name][full])
        an, fd = np.array(an_all), np.array(fd_all)
        assert an.size > 0, name
        rel = np.linalg.norm(an - fd) / max(np.linalg.norm(fd), 1e-12)
        assert rel < 1e-5, (name, rel)
        np.testing.assert_allclose(an, fd, rtol=1e-4, atol=1e-7 * max(1.0, np.abs(fd).max()), err_msg=name)
    assert skipped < 0.1 * sum(getattr(sc, f)[pick].size for f in fields)


def test_dalpha_matches_alg2_recursion_on_a_stack():
    """Alg. 2's dL/dalpha_k = T_k sum_i g_i (c_k[i] - R_{k+1}[i]) with the bg term
    (read as R_{k+1} = colour behind k normalised by T_{k+1}, including T_N bg):
    checked on splats stacked on one pixel centre, where dalpha/dm = 1."""
    cam = oracle.camera_from_gl(scenes.identity_camera(65, 65))
    cfg = oracle.config(bg=(0.3, 0.1, 0.7))
    bg = np.array(cfg.bg[:])  # the FP32-rounded background
    depths = [2.0, 2.7, 3.1, 4.4]
    logits = [-0.5, 0.4, -1.2, 0.9]
    rgbs = np.array([[0.9, 0.1, 0.2], [0.2, 0.8, 0.3], [0.1, 0.2, 0.7], [0.5, 0.6, 0.4]])
    n = 4
    sh = ((rgbs - 0.5) / (0.5 / math.sqrt(math.pi)))[:, None, :]
    sc = scenes.Scene(np.array([[0.0, 0.0, z] for z in depths]), np.full((n, 3), math.log(0.5)),
                      np.tile([1.0, 0.0, 0.0, 0.0], (n, 1)), np.array(logits), np.zeros((n, 3)), sh, 0)
    gC = np.array([0.7, -1.1, 0.4])
    gr = oracle.render_backward(sc, cam, cfg, gC[None, :], pixels=[[32, 32]])
    pre = oracle.preprocess(sc, cam, cfg)
    alphas = pre["rec"][:, 7]  # delta = 0: alpha = m
    T = np.cumprod(np.concatenate([[1.0], 1 - alphas]))
    R = bg.copy()  # R_{N+1}: only the background behind the last splat
    dlda = np.zeros(n)
    for k in range(n - 1, -1, -1):
        dlda[k] = T[k] * np.dot(gC, rgbs[k] - R)
        R = alphas[k] * rgbs[k] + (1 - alphas[k]) * R
    np.testing.assert_allclose(gr["d2"][:, 7], dlda, rtol=1e-12)
