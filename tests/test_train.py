"""The training step: the FP64 oracle of the photometric loss and Adam pinned
to independent routes (CPU), and the CUDA loss, gradient and Adam update
against the oracle (GPU)."""
import math

import numpy as np
import pytest
import torch
from scipy import ndimage

from oracle import train_oracle as T


def _pair(seed, shape):
    rng = np.random.default_rng(seed)
    return rng.uniform(0, 1, shape), rng.uniform(0, 1, shape)


# ---------------------------------------------------------------------------
# oracle pins (CPU)
# ---------------------------------------------------------------------------

def test_ssim_of_identical_images_is_one_and_the_loss_vanishes():
    x, _ = _pair(0, (3, 17, 23))
    for c in range(3):
        np.testing.assert_allclose(T.ssim_map(x[c], x[c]), 1.0, rtol=0, atol=1e-12)
    out = T.photometric_loss([x], [x.copy()], lam=0.2)
    assert abs(out["loss"]) < 1e-12 and abs(out["ssim"] - 1) < 1e-12 and out["l1"] == 0.0


def test_window_filter_matches_scipy_correlation():
    x, _ = _pair(1, (19, 26))
    w = T.gaussian_window()
    assert abs(w.sum() - 1) < 1e-15 and abs(w[5] / w[4] - math.exp(1 / (2 * 1.5 ** 2))) < 1e-12
    ref = ndimage.correlate1d(ndimage.correlate1d(x, w, axis=1, mode="constant", cval=0.0), w, axis=0,
                              mode="constant", cval=0.0)
    np.testing.assert_allclose(T.window_filter(x), ref, rtol=1e-13, atol=1e-15)


def test_ssim_matches_its_definition_at_single_pixels():
    """Weighted means, variances and covariance written out over the 11 x 11
    neighbourhood of a pixel (zero outside the image)."""
    x, y = _pair(2, (14, 21))
    w = T.gaussian_window()
    S = T.ssim_map(x, y)
    for (qy, qx) in [(0, 0), (7, 10), (13, 20), (3, 17)]:
        mx = my = exx = eyy = exy = 0.0
        for dy in range(-5, 6):
            for dx in range(-5, 6):
                py, px = qy + dy, qx + dx
                if 0 <= py < 14 and 0 <= px < 21:
                    wt = w[dy + 5] * w[dx + 5]
                    a, b = x[py, px], y[py, px]
                    mx += wt * a
                    my += wt * b
                    exx += wt * a * a
                    eyy += wt * b * b
                    exy += wt * a * b
        sx, sy, sxy = exx - mx * mx, eyy - my * my, exy - mx * my
        ref = (2 * mx * my + T.C1) * (2 * sxy + T.C2) / ((mx * mx + my * my + T.C1) * (sx + sy + T.C2))
        assert abs(S[qy, qx] - ref) < 1e-13


def test_loss_gradient_matches_central_differences():
    rng = np.random.default_rng(3)
    ims = [rng.uniform(0, 1, (3, 9, 12)), rng.uniform(0, 1, (3, 11, 7))]
    tgs = [rng.uniform(0, 1, (3, 9, 12)), rng.uniform(0, 1, (3, 11, 7))]
    g = T.photometric_loss_grad(ims, tgs, lam=0.3)
    h = 1e-6
    for v, c, py, px in [(0, 0, 0, 0), (0, 2, 4, 5), (0, 1, 8, 11), (1, 0, 10, 6), (1, 2, 5, 3), (1, 1, 0, 0)]:
        ip = [a.copy() for a in ims]
        im = [a.copy() for a in ims]
        ip[v][c, py, px] += h
        im[v][c, py, px] -= h
        fd = (T.photometric_loss(ip, tgs, 0.3)["loss"] - T.photometric_loss(im, tgs, 0.3)["loss"]) / (2 * h)
        assert abs(fd - g[v][c, py, px]) <= 1e-7 * max(1.0, abs(fd)), (v, c, py, px, fd, g[v][c, py, px])


def test_adam_matches_torch_optim_adam():
    rng = np.random.default_rng(4)
    p0 = rng.normal(size=50)
    grads = [rng.normal(size=50) for _ in range(3)]
    lr = np.where(np.arange(50) % 10 < 3, 1e-2, 5e-4)
    tp = torch.tensor(p0, dtype=torch.float64, requires_grad=True)
    opts = [torch.optim.Adam([tp], lr=1.0, betas=(0.9, 0.999), eps=1e-15)]  # lr applied per element below
    p, m, v = p0, np.zeros(50), np.zeros(50)
    ref_p = p0.copy()
    m_t, v_t = np.zeros(50), np.zeros(50)
    for t, g in enumerate(grads, start=1):
        p, m, v = T.adam_step(p, g, m, v, t, lr)
        # torch with unit lr gives the step direction; scale it per element
        before = tp.detach().clone()
        tp.grad = torch.tensor(g, dtype=torch.float64)
        opts[0].step()
        ref_p = ref_p + lr * (tp.detach().numpy() - before.numpy())
        with torch.no_grad():
            tp.copy_(torch.tensor(ref_p))
        m_t = 0.9 * m_t + 0.1 * g
        v_t = 0.999 * v_t + 0.001 * g * g
    np.testing.assert_allclose(p, ref_p, rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(m, m_t, rtol=1e-14)
    np.testing.assert_allclose(v, v_t, rtol=1e-14)


# ---------------------------------------------------------------------------
# CUDA path against the oracle (GPU)
# ---------------------------------------------------------------------------

def _gpu():
    if not torch.cuda.is_available():  # pragma: no cover - CPU-only container
        pytest.skip("needs a CUDA GPU")


@pytest.mark.gpu
@pytest.mark.parametrize("lam", [0.2, 0.0, 1.0])
def test_gpu_loss_and_gradient_match_oracle(lam):
    """Two views of ragged sizes (several tiles and partial tiles): L, mean
    SSIM, mean |C - T| and dL/dC element by element."""
    _gpu()
    from paper_2605_18334_gb300 import scenes
    from paper_2605_18334_gb300.rasterizer import Config, Gaussians, Rasterizer
    from paper_2605_18334_gb300.train import PhotometricLoss

    sc = scenes.cube_1k(seed=2, n=200)
    cams = [scenes.identity_camera(53, 37), scenes.identity_camera(16, 40)]
    g = Gaussians.from_scene(sc)
    r = Rasterizer(g, cams, Config())
    r.forward(g)  # the plan's view table
    rng = np.random.default_rng(5)
    img = rng.uniform(0, 1, r.images.numel()).astype(np.float32)
    tgt = rng.uniform(0, 1, r.images.numel()).astype(np.float32)
    r.images.copy_(torch.as_tensor(img))
    loss_fn = PhotometricLoss(r, lam)
    loss = float(loss_fn(torch.as_tensor(tgt).cuda()).item())
    stats = loss_fn.stats.cpu().numpy()
    d = loss_fn.d_images.cpu().numpy()
    ims = [img[int(r.plan.image_offset[v]):int(r.plan.image_offset[v + 1])].reshape(3, c["height"], c["width"])
           for v, c in enumerate(cams)]
    tgs = [tgt[int(r.plan.image_offset[v]):int(r.plan.image_offset[v + 1])].reshape(3, c["height"], c["width"])
           for v, c in enumerate(cams)]
    ref = T.photometric_loss(ims, tgs, lam)
    assert abs(loss - ref["loss"]) <= 1e-5 * max(1.0, abs(ref["loss"]))
    assert abs(stats[0] - ref["ssim"]) <= 1e-5 and abs(stats[1] - ref["l1"]) <= 1e-6
    gref = np.concatenate([a.reshape(-1) for a in T.photometric_loss_grad(ims, tgs, lam)])
    scale = np.abs(gref).max()
    assert np.abs(d - gref).max() <= 1e-4 * scale, np.abs(d - gref).max() / scale


@pytest.mark.gpu
def test_gpu_adam_matches_oracle_over_groups_and_steps():
    """Three groups (one with a second learning rate for the elements past the
    first 3 of every 48, the SH layout), three steps."""
    _gpu()
    from paper_2605_18334_gb300 import native as N

    rng = np.random.default_rng(6)
    sizes = [(3001, 0, 0), (4 * 1000, 0, 0), (48 * 257, 48, 3)]
    groups, host = [], []
    for n, period, split in sizes:
        p = rng.normal(size=n).astype(np.float32)
        host.append(dict(p=p.astype(np.float64), m=np.zeros(n), v=np.zeros(n), period=period, split=split))
        dev = dict(p=torch.as_tensor(p).cuda(), g=torch.zeros(n, device="cuda"), m=torch.zeros(n, device="cuda"),
                   v=torch.zeros(n, device="cuda"))
        groups.append(dev)
    lrs = [(1e-3, 1e-3), (5e-2, 5e-2), (2.5e-3, 1.25e-4)]
    for step in (1, 2, 3):
        descs = []
        for (n, period, split), dev, hs, (lr, lr_rest) in zip(sizes, groups, host, lrs):
            g = rng.normal(size=n).astype(np.float32)
            dev["g"].copy_(torch.as_tensor(g))
            lr_el = np.where((np.arange(n) % period >= split) if period else np.zeros(n, bool), lr_rest, lr)
            # the library takes the betas as FP32: the oracle gets the same rounded values
            hs["p"], hs["m"], hs["v"] = T.adam_step(hs["p"], g.astype(np.float64), hs["m"], hs["v"], step, lr_el,
                                                    beta1=float(np.float32(0.9)), beta2=float(np.float32(0.999)))
            d = N.sr_adam_group()
            d.param, d.grad, d.m, d.v = dev["p"].data_ptr(), dev["g"].data_ptr(), dev["m"].data_ptr(), dev["v"].data_ptr()
            d.n, d.lr, d.lr_rest, d.period, d.split_at = n, lr, lr_rest, period, split
            descs.append(d)
        N.sr_adam_step(descs, step, 0.9, 0.999, 1e-15, torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    for dev, hs in zip(groups, host):
        np.testing.assert_allclose(dev["p"].cpu().numpy(), hs["p"], rtol=1e-6, atol=1e-6)
        np.testing.assert_allclose(dev["m"].cpu().numpy(), hs["m"], rtol=1e-5, atol=1e-7)
        np.testing.assert_allclose(dev["v"].cpu().numpy(), hs["v"], rtol=1e-5, atol=1e-9)


@pytest.mark.gpu
def test_training_steps_reduce_the_loss():
    """Fit a scene to images rendered from a perturbed copy of it."""
    _gpu()
    from paper_2605_18334_gb300 import scenes
    from paper_2605_18334_gb300.rasterizer import Config, Gaussians, Rasterizer
    from paper_2605_18334_gb300.train import Trainer

    sc = scenes.cluster(seed=9, n=3000, sh_degree=1)
    cams = [scenes.identity_camera(96, 64), scenes.identity_camera(64, 64)]
    target_scene = sc.subset(np.arange(sc.n))
    target_scene.means = (sc.means + np.random.default_rng(1).normal(0, 0.02, sc.means.shape)).astype(np.float32)
    gt = Gaussians.from_scene(target_scene)
    rt = Rasterizer(gt, cams, Config())
    targets = rt.forward(gt).clone()
    g = Gaussians.from_scene(sc)
    tr = Trainer(g, cams, targets, lr=dict(means=1e-3))
    losses = [float(tr.step().item()) for _ in range(40)]
    assert losses[-1] < 0.8 * losses[0], losses


@pytest.mark.gpu
def test_densification_statistics_accumulate_over_steps():
    """uv_sum / seen / z_max after several steps equal the per-step
    statistics of the backward accumulated on the host."""
    _gpu()
    from paper_2605_18334_gb300 import scenes
    from paper_2605_18334_gb300.rasterizer import Config, Gaussians, Rasterizer
    from paper_2605_18334_gb300.train import Trainer

    sc = scenes.cluster(seed=13, n=2000, sh_degree=1)
    cams = [scenes.identity_camera(80, 60)]
    tgt = torch.rand(3 * 80 * 60, device="cuda")
    g = Gaussians.from_scene(sc)
    tr = Trainer(g, cams, tgt, densify_stats=True)
    uv = np.zeros(sc.n)
    seen = np.zeros(sc.n, np.int64)
    zmax = np.zeros(sc.n)
    for _ in range(4):
        tr.step()
        a = tr.grads["means2d_abs"].cpu().numpy().astype(np.float64)
        z = np.abs(tr.grads["depth_grad"].cpu().numpy().astype(np.float64))
        uv += np.where(a > 0, a, 0)
        seen += (a > 0)
        zmax = np.maximum(zmax, z)
    np.testing.assert_allclose(tr.uv_sum.cpu().numpy(), uv, rtol=1e-6, atol=1e-12)
    np.testing.assert_array_equal(tr.seen.cpu().numpy(), seen)
    np.testing.assert_array_equal(tr.z_max.cpu().numpy(), zmax.astype(np.float32))
    assert seen.max() == 4 and zmax.max() > 0


@pytest.mark.gpu
def test_training_with_densification_keeps_going():
    """Steps, one densification from the collected statistics (the trainer
    re-plans for the new size and carries the Adam moments over), more steps:
    the scene grows by the clone copies and split children, the moments of
    kept Gaussians survive and new ones start at zero, and the loss keeps
    falling."""
    _gpu()
    from paper_2605_18334_gb300 import scenes
    from paper_2605_18334_gb300.rasterizer import Config, Gaussians, Rasterizer
    from paper_2605_18334_gb300.train import Trainer

    sc = scenes.cluster(seed=19, n=3000, sh_degree=1)
    cams = [scenes.identity_camera(96, 64)]
    target_scene = sc.subset(np.arange(sc.n))
    target_scene.means = (sc.means + np.random.default_rng(2).normal(0, 0.02, sc.means.shape)).astype(np.float32)
    gt = Gaussians.from_scene(target_scene)
    targets = Rasterizer(gt, cams, Config()).forward(gt).clone()
    tr = Trainer(Gaussians.from_scene(sc), cams, targets, lr=dict(means=1e-3), densify_stats=True)
    losses = [float(tr.step().item()) for _ in range(10)]
    m_before = tr.adam.state["means"][0].clone()
    uv = (tr.uv_sum / tr.seen.clamp(min=1)).cpu().numpy()
    thr = float(np.quantile(uv[uv > 0], 0.8))
    n0 = tr.g.n
    counts = tr.densify(grad_uv=thr, grad_z=1e30, log_scale_split=-4.0, logit_prune=-1e30)
    assert counts["cloned"] > 0 and counts["split"] > 0
    assert tr.g.n == counts["total"] == counts["kept"] + counts["cloned"] + 2 * counts["split"] > n0
    m_after = tr.adam.state["means"][0]
    src = tr.last_densify.src[:counts["kept"]]
    assert torch.equal(m_after[:counts["kept"]], m_before[src])
    assert torch.count_nonzero(m_after[counts["kept"]:]) == 0
    assert tr.seen.numel() == tr.g.n and int(tr.seen.sum()) == 0
    losses += [float(tr.step().item()) for _ in range(10)]
    assert np.isfinite(losses).all() and losses[-1] < losses[0], losses
