"""Mode B of the oracle (per-pixel footprint lists) against mode A (brute
force over every Gaussian), and the replay of another renderer's gate and
stop decisions.

Mode B leaves out of a pixel's list only Gaussians whose alpha there is
below alpha_min (1 - 1e-2), which the conservative footprint bounds for any
threshold (the reading of the footprint, Alg. 1 gate); mode A skips those
pairs without changing any state, so the two must agree bit for bit.  The
replay accepts a decision that differs from FP64's only within the stated
tolerance of its threshold; the planted mistakes below must be rejected.
"""
import numpy as np
import pytest

import oracle
from paper_2605_18334_gb300 import scenes


def _frames(sc, cam_dict, cfg=None, **kw):
    cam = oracle.camera_from_gl(cam_dict)
    cfg = cfg or oracle.config(**kw)
    pre = oracle.preprocess(sc, cam, cfg)
    a = oracle.render(sc, cam, cfg, pre=pre)
    b = oracle.render_frame(sc, cam, cfg, pre=pre, want_lists=True)
    return cam, cfg, pre, a, b


def _skewed_scene(seed=7, n=1500):
    sc = scenes.cluster(seed=seed, n=n, sh_degree=2, two_opacities=True, split=True)
    rng = np.random.default_rng(seed)
    big = rng.random(n) < 0.2
    sc.skew[big] = (rng.normal(0, 1, (int(big.sum()), 3)) * 8.0).astype(np.float32)
    return sc


CASES = {
    "cube_1k_64px": lambda: (scenes.cube_1k(), scenes.identity_camera(64, 64), {}),
    "fd_crop_2k_32px": lambda: scenes.fd_crop_scene() + ({},),
    "two_opacities_split_big_skew": lambda: (_skewed_scene(), scenes.identity_camera(120, 90), {}),
    "background_variants": lambda: (scenes.cube_1k(seed=8, n=800), scenes.identity_camera(80, 60),
                                    dict(bg=(0.2, 0.5, 0.9), antialias_comp=False, dilation=0.2, alpha_max=0.95,
                                         t_stop=1e-3)),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_mode_b_equals_mode_a_bit_for_bit(case):
    sc, cam_dict, kw = CASES[case]()
    _, _, _, a, b = _frames(sc, cam_dict, **kw)
    for k in ("rgb", "T", "last", "count", "ambiguous"):
        np.testing.assert_array_equal(a[k], b[k], err_msg=k)
    assert b["stats"]["inadmissible_pixels"] == 0 and b["stats"]["flipped_pixels"] == 0
    assert a["count"].sum() > 0


def test_mode_b_backward_equals_mode_a():
    sc, cam_dict = scenes.fd_crop_scene()
    cam = oracle.camera_from_gl(cam_dict)
    cfg = oracle.config()
    g = scenes.upstream_grad(3, 32, 32)
    a = oracle.render_backward(sc, cam, cfg, g)
    b = oracle.render_backward(sc, cam, cfg, g, frame=True)
    for k in ("d2", "means", "log_scales", "quats", "opacity_logits", "skew", "sh"):
        np.testing.assert_allclose(b[k], a[k], rtol=1e-12, atol=1e-14 * np.abs(a[k]).max(), err_msg=k)


@pytest.mark.parametrize("case", sorted(CASES))
def test_replay_of_own_decisions_is_admissible_and_identical(case):
    sc, cam_dict, kw = CASES[case]()
    cam, cfg, pre, _, b = _frames(sc, cam_dict, **kw)
    r = oracle.render_frame(sc, cam, cfg, pre=pre, gpu_lists=b["lists"])
    assert r["stats"]["inadmissible_pixels"] == 0
    assert r["stats"]["flipped_pixels"] == 0
    for k in ("rgb", "T", "last", "count"):
        np.testing.assert_array_equal(r[k], b[k], err_msg=k)


def _pixel_alphas(pre, ids, x, y):
    return np.array([oracle.alpha_at(pre["rec"][i], [[x, y]])[0] for i in ids])


def _edit(lists, p, new_ids):
    off, ids = lists
    per = [list(ids[off[q]:off[q + 1]]) for q in range(len(off) - 1)]
    per[p] = list(new_ids)
    cnt = np.array([len(v) for v in per], np.int64)
    o = np.zeros(len(per) + 1, np.int64)
    np.cumsum(cnt, out=o[1:])
    return o, np.array([i for v in per for i in v], np.int32)


def test_replay_rejects_planted_mistakes():
    """A renderer that drops a pair well above the gate, blends one far below
    it, blends in the wrong order, or stops while T is far above t_stop is
    caught at exactly that pixel."""
    sc, cam_dict = scenes.cube_1k(), scenes.identity_camera(64, 64)
    cam, cfg, pre, _, b = _frames(sc, cam_dict)
    off, ids = b["lists"]
    W = 64
    cnt = np.diff(off)
    # a pixel with several blends, all well clear of the gate
    tau = float(cfg.alpha_min)
    p = None
    for q in np.argsort(-cnt):
        lst = ids[off[q]:off[q + 1]]
        al = _pixel_alphas(pre, lst, q % W, q // W)
        if len(lst) >= 3 and np.all(np.minimum(al, cfg.alpha_max) > 1.5 * tau) and b["T"].reshape(-1)[q] > 10 * cfg.t_stop:
            p = int(q)
            break
    assert p is not None
    lst = list(ids[off[p]:off[p + 1]])
    # dropped pair in the middle: FP64 blends it, the replay cannot skip it
    r = oracle.render_frame(sc, cam, cfg, pre=pre, gpu_lists=_edit(b["lists"], p, lst[:1] + lst[2:]))
    st = r["status"].reshape(-1)
    assert st[p] == 4 and np.count_nonzero(st) == 1
    # stopped early (the last two dropped) while T is far above t_stop
    r = oracle.render_frame(sc, cam, cfg, pre=pre, gpu_lists=_edit(b["lists"], p, lst[:-2]))
    st = r["status"].reshape(-1)
    assert st[p] == 4 and np.count_nonzero(st) == 1
    # order swapped
    r = oracle.render_frame(sc, cam, cfg, pre=pre, gpu_lists=_edit(b["lists"], p, [lst[1], lst[0]] + lst[2:]))
    st = r["status"].reshape(-1)
    assert st[p] != 0 and np.count_nonzero(st) == 1
    # a Gaussian blended where its alpha is far below the gate
    x, y = p % W, p // W
    vis = np.nonzero(pre["visible"])[0]
    far = [int(i) for i in vis if oracle.alpha_at(pre["rec"][i], [[x, y]])[0] < 0.1 * tau and i not in lst][:1]
    assert far
    order = sorted(lst + far, key=lambda i: (int(pre["depth_bits"][i]), i))
    r = oracle.render_frame(sc, cam, cfg, pre=pre, gpu_lists=_edit(b["lists"], p, order))
    st = r["status"].reshape(-1)
    assert st[p] in (1, 5) and np.count_nonzero(st) == 1


def test_replay_accepts_a_flip_within_tolerance_only():
    """One Gaussian whose opacity puts its alpha at one pixel a relative
    distance r = 3e-3 below the gate: blending it there is admissible with a
    tolerance of 2r, not with r / 2."""
    def scene(logit):
        return scenes.Scene(means=np.array([[0.0, 0.0, 4.0]]), log_scales=np.full((1, 3), -1.5),
                            quats=np.array([[1.0, 0.0, 0.0, 0.0]]), opacity_logits=np.array([logit]),
                            skew=np.zeros((1, 3)), sh=np.full((1, 1, 3), 0.5), sh_degree=0)

    cam = oracle.camera_from_gl(scenes.identity_camera(48, 48))
    cfg = oracle.config()
    tau = float(cfg.alpha_min)
    x, y = 30, 24
    a0 = oracle.alpha_at(oracle.preprocess(scene(0.0), cam, cfg)["rec"][0], [[x, y]])[0]  # opacity 1/2
    o = 0.5 * tau * (1 - 3e-3) / a0                     # alpha is proportional to the opacity
    sc = scene(float(np.log(o / (1 - o))))
    pre = oracle.preprocess(sc, cam, cfg)
    rel = (tau - oracle.alpha_at(pre["rec"][0], [[x, y]])[0]) / tau
    assert 2.9e-3 < rel < 3.1e-3
    p = y * 48 + x
    base = oracle.render_frame(sc, cam, cfg, pre=pre, want_lists=True)["lists"]
    assert base[0][p + 1] == base[0][p]                  # FP64 skips the pair
    lists = _edit(base, p, [0])
    ok = oracle.render_frame(sc, cam, cfg, pre=pre, gpu_lists=lists, tol_alpha=2 * rel)
    assert ok["stats"]["inadmissible_pixels"] == 0 and ok["stats"]["flipped_gate"] == 1
    assert ok["stats"]["max_gate_margin"] == pytest.approx(rel, rel=1e-9)
    assert ok["count"].reshape(-1)[p] == 1
    bad = oracle.render_frame(sc, cam, cfg, pre=pre, gpu_lists=lists, tol_alpha=0.5 * rel)
    st = bad["status"].reshape(-1)
    assert st[p] == 1 and np.count_nonzero(st) == 1


def test_backward_scale_bounds_every_gradient_and_slack_marks_only_clamp_decisions():
    """|gradient| <= scale element by element (a sum is bounded by the sum of
    its terms' magnitudes); slack is zero with a tolerance of zero and
    nonzero only on Gaussians whose alpha reaches alpha_max."""
    sc = _skewed_scene(seed=9, n=800)
    rng = np.random.default_rng(9)
    dense = rng.random(sc.n) < 0.3           # opaque, larger splats whose alpha crosses alpha_max
    sc.opacity_logits[dense] = 4.0
    sc.log_scales[dense] += 1.0
    cam = oracle.camera_from_gl(scenes.identity_camera(64, 48))
    cfg = oracle.config()
    g = scenes.upstream_grad(9, 48, 64)
    out = oracle.render_backward(sc, cam, cfg, g, frame=True, bounds=True)
    for k in ("d2", "means", "log_scales", "quats", "opacity_logits", "skew", "split_dir", "sh"):
        assert np.all(np.abs(out[k]) <= out["scale"][k] * (1 + 1e-9) + 1e-300), k
    zero = oracle.render_backward(sc, cam, cfg, g, frame=True, bounds=True, tol_alpha=0.0)
    assert np.abs(zero["slack"]["d2"]).max() == 0.0
    wide = oracle.render_backward(sc, cam, cfg, g, frame=True, bounds=True, tol_alpha=0.05)
    has = np.abs(wide["slack"]["d2"]).max(axis=1) > 0
    assert has.any()
    pre = oracle.preprocess(sc, cam, cfg)
    peak = pre["rec"][:, 14] * np.maximum(pre["rec"][:, 15], pre["rec"][:, 16]) * 2.0  # o comp (1 + erf) <= 2 o comp
    assert np.all(peak[has] >= cfg.alpha_max * 0.95)


def test_config1_frame_pairs_within_the_survey_tolerances():
    """The 1,000-Gaussian 64x64 frame at the tolerances of 1e-5 (relative) of
    the gate and of the stop: no pair is that close to the stop, and one pair
    (Gaussian 578 at pixel (22, 31), 9.6e-6 below the gate) is that
    close to the gate.  The GPU parity test compares every pixel, this one
    included, against the oracle under the GPU's own decision there."""
    sc, cam_dict = scenes.cube_1k(), scenes.identity_camera(64, 64)
    cam = oracle.camera_from_gl(cam_dict)
    cfg = oracle.config()
    pre = oracle.preprocess(sc, cam, cfg)
    stop = oracle.render_frame(sc, cam, cfg, pre=pre, tol_alpha=0.0, tol_t=1e-5)
    assert stop["stats"]["ambiguous_pixels"] == 0
    gate = oracle.render_frame(sc, cam, cfg, pre=pre, tol_alpha=1e-5, tol_t=0.0)
    assert gate["stats"]["ambiguous_pixels"] == 1
    ys, xs = np.nonzero(gate["ambiguous"])
    assert (int(xs[0]), int(ys[0])) == (22, 31)
    a = oracle.alpha_at(pre["rec"][578], [[22, 31]])[0]
    assert -1e-5 < (a - cfg.alpha_min) / cfg.alpha_min < 0
