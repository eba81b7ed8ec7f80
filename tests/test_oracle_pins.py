"""Pins of the FP64 oracle against what the paper and mathematics fix.

None of these re-types an oracle formula: each compares the oracle with an
independent route (a library routine, a closed form, quadrature, Monte Carlo
sampling of the 3D skew normal, brute force, finite differences), chosen so
that a dropped term, a wrong sign or index or a transposed operand in the
oracle fails at least one of them.
"""
import json
import math
import os

import numpy as np
import pytest
from scipy import special
from scipy.spatial.transform import Rotation

import oracle
from paper_2605_18334_gb300 import scenes

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")))


@pytest.fixture(scope="module", autouse=True)
def _build():
    oracle.build()


# ---------------------------------------------------------------------------
# independent helpers (numpy / scipy; none of them calls the oracle)
# ---------------------------------------------------------------------------

def rot_scipy(q_wxyz):
    q = np.asarray(q_wxyz, np.float64)
    return Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()


def cam_arrays(cam):
    f = oracle.camera_fields(cam)
    W2C = f["w2c"].reshape(3, 4)
    return W2C, f


def pinhole(f, t):
    return np.array([f["fx"] * t[0] / t[2] + f["cx"], f["fy"] * t[1] / t[2] + f["cy"]])


def pinhole_jacobian_fd(f, t, h=1e-6):
    """Jacobian of the pinhole projection by central differences."""
    J = np.zeros((2, 3))
    for k in range(3):
        e = np.zeros(3)
        e[k] = h * max(1.0, abs(t[k]))
        J[:, k] = (pinhole(f, t + e) - pinhole(f, t - e)) / (2 * e[k])
    return J


def independent_projection(mu, log_s, q, eta, W2C, f, s_dil=float(np.float32(0.3))):
    """mu_2, Sigma_d, comp and delta_2 by a separate route: scipy rotation,
    numerical Jacobian, explicit matrix products and inverses."""
    t = W2C[:, :3] @ mu + W2C[:, 3]
    R = rot_scipy(q)
    S = np.diag(np.exp(log_s))
    Sigma = R @ S @ S @ R.T
    A = pinhole_jacobian_fd(f, t) @ W2C[:, :3]
    Sp = A @ Sigma @ A.T
    Sd = Sp + s_dil * np.eye(2)
    comp = math.sqrt(np.linalg.det(Sp) / np.linalg.det(Sd))
    de = eta / math.sqrt(1.0 + eta @ eta)
    delta2 = A @ R @ S @ de
    return dict(t=t, mu2=pinhole(f, t), Sd=Sd, Sp=Sp, comp=comp, A=A, R=R, S=S, delta2=delta2)


def one_gaussian_scene(mu, log_s, q, eta, logit=2.0, sh_deg=0, rgb=(0.6, 0.4, 0.2), logit2=None, split=None):
    sh = ((np.asarray(rgb) - 0.5) / (0.5 / math.sqrt(math.pi)))[None, None, :]
    if sh_deg > 0:
        sh = np.concatenate([sh, np.zeros((1, (sh_deg + 1) ** 2 - 1, 3))], axis=1)
    op = np.array([logit]) if logit2 is None else np.array([[logit, logit2]])
    return scenes.Scene(np.array([mu], np.float64), np.array([log_s], np.float64), np.array([q], np.float64),
                        op, np.array([eta], np.float64), sh.astype(np.float64), sh_deg,
                        None if split is None else np.array([split], np.float64))


# ---------------------------------------------------------------------------
# erf, the factor 2 and the sqrt 2 (Appendix "Forward Pass"; Alg. 1)
# ---------------------------------------------------------------------------

def test_erf_matches_paper_taylor_series_small_z():
    """Kernel with A = I, beta = (sqrt 2, 0) at (z, 0): k = exp(-z^2/2)(1 + erf z).
    erf recovered from the oracle must match the paper's Taylor series."""
    z = np.linspace(-0.5, 0.5, 101)
    k = oracle.kernel_at([1.0, 0.0, 1.0], [math.sqrt(2.0), 0.0], np.stack([z, 0 * z], 1))
    erf_or = k / np.exp(-0.5 * z * z) - 1.0
    coef = GOLDEN["erf_taylor"]["coefficients_of_z^(2n+1)"]
    # the printed terms, then the series continued: (-1)^n / (n! (2n+1))
    series = sum(c * z ** (2 * n + 1) for n, c in enumerate(coef))
    series += sum((-1) ** n / (math.factorial(n) * (2 * n + 1)) * z ** (2 * n + 1) for n in range(len(coef), 30))
    series *= 2.0 / math.sqrt(math.pi)
    np.testing.assert_allclose(erf_or, series, rtol=0, atol=1e-14)


def test_erf_matches_library_wide_range():
    z = np.linspace(-4.0, 4.0, 801)
    k = oracle.kernel_at([1.0, 0.0, 1.0], [math.sqrt(2.0), 0.0], np.stack([z, 0 * z], 1))
    np.testing.assert_allclose(k, np.exp(-0.5 * z * z) * (1.0 + special.erf(z)), rtol=1e-13, atol=1e-16)


@pytest.mark.parametrize("beta", [(0.0, 0.0), (1.0, -2.0), (5.0, 3.0), (-0.3, 0.1)])
def test_skew_kernel_integrates_to_gaussian_mass(beta):
    """2 phi(d; Sigma) Phi(beta^T d) is a density (Sec. '3D Skew Gaussian
    Kernel'): the unnormalised kernel integrates to 2 pi sqrt(det Sigma) for
    every beta.  Tensor trapezoid quadrature in whitened coordinates."""
    Sigma = np.array([[2.0, 0.7], [0.7, 1.1]])
    A = np.linalg.inv(Sigma)
    L = np.linalg.cholesky(Sigma)
    u = np.arange(-12.0, 12.0 + 1e-9, 0.02)
    U, V = np.meshgrid(u, u, indexing="ij")
    d = np.stack([U.ravel(), V.ravel()], 1) @ L.T
    k = oracle.kernel_at([A[0, 0], A[0, 1], A[1, 1]], beta, d)
    integral = k.sum() * 0.02 * 0.02 * np.linalg.det(L)
    assert abs(integral / (2 * math.pi * math.sqrt(np.linalg.det(Sigma))) - 1.0) < 1e-10


def test_beta_zero_gives_phi_half():
    """beta = 0: Phi(0) = 1/2, so 2 G Phi = G (the 3DGS kernel)."""
    phi0 = GOLDEN["beta_zero"]["phi_at_zero"]
    d = np.random.default_rng(0).normal(size=(50, 2))
    k = oracle.kernel_at([0.7, 0.2, 1.3], [0.0, 0.0], d)
    g = np.exp(-0.5 * (0.7 * d[:, 0] ** 2 + 2 * 0.2 * d[:, 0] * d[:, 1] + 1.3 * d[:, 1] ** 2))
    np.testing.assert_allclose(k, 2.0 * g * phi0, rtol=1e-15)


# ---------------------------------------------------------------------------
# projection: beta = 0 reduces to 3DGS (Sec. '3D Skew Gaussian Kernel')
# ---------------------------------------------------------------------------

def test_zero_skew_projection_matches_independent_3dgs():
    sc = scenes.cube_1k(seed=5, n=200)
    sc.skew[:] = 0.0
    cam = oracle.camera_from_gl(scenes.identity_camera(64, 64))
    cfg = oracle.config()
    pre = oracle.preprocess(sc, cam, cfg)
    W2C, f = cam_arrays(cam)
    rec = pre["rec"]
    for i in range(sc.n):
        ind = independent_projection(sc.means[i].astype(np.float64), sc.log_scales[i].astype(np.float64),
                                     sc.quats[i].astype(np.float64), np.zeros(3), W2C, f)
        conic = np.linalg.inv(ind["Sd"])
        np.testing.assert_allclose(rec[i, 0:2], ind["mu2"], rtol=1e-12)
        np.testing.assert_allclose(rec[i, 2:5], [conic[0, 0], conic[0, 1], conic[1, 1]], rtol=2e-6, atol=1e-9)
        assert abs(rec[i, 14] - ind["comp"]) < 1e-6 * ind["comp"]
        assert rec[i, 5] == 0.0 and rec[i, 6] == 0.0  # beta_2 is exactly zero
        o = 1.0 / (1.0 + math.exp(-float(sc.opacity_logits[i])))
        assert abs(rec[i, 7] - ind["comp"] * o) < 1e-6 * ind["comp"] * o
        assert rec[i, 8] == 0.0
    # alpha at pixels equals o' exp(-1/2 d^T (Sigma'+sI)^-1 d) (Appendix alpha expansion with beta = 0)
    i = int(np.argmax(rec[:, 7]))
    pix = np.stack(np.meshgrid(np.arange(64), np.arange(64), indexing="xy"), -1).reshape(-1, 2).astype(np.int32)
    al = oracle.alpha_at(rec[i], pix)
    d = pix + 0.5 - rec[i, 0:2]
    A = np.array([[rec[i, 2], rec[i, 3]], [rec[i, 3], rec[i, 4]]])
    ref = rec[i, 7] * np.exp(-0.5 * np.einsum("ni,ij,nj->n", d, A, d))
    np.testing.assert_allclose(al, ref, rtol=1e-12, atol=1e-300)


def test_rotation_and_scale_enter_as_R_S():
    """A quaternion for 90 deg about the camera z axis swaps the footprint axes."""
    cam = oracle.camera_from_gl(scenes.identity_camera(128, 128))
    cfg = oracle.config(dilation=0.0, antialias_comp=False)
    base = dict(mu=[0.0, 0.0, 4.0], log_s=[math.log(0.2), math.log(0.05), math.log(0.1)], eta=[0.0, 0.0, 0.0])
    q0 = [1.0, 0.0, 0.0, 0.0]
    qz = [math.cos(math.pi / 4), 0.0, 0.0, math.sin(math.pi / 4)]
    r0 = oracle.preprocess(one_gaussian_scene(q=q0, **base), cam, cfg)["rec"][0]
    r1 = oracle.preprocess(one_gaussian_scene(q=qz, **base), cam, cfg)["rec"][0]
    f = cam.fx / 4.0
    # conic of diag((f sx)^2, (f sy)^2) and of the swapped one
    np.testing.assert_allclose([r0[2], r0[4]], [1 / (f * 0.2) ** 2, 1 / (f * 0.05) ** 2], rtol=1e-12)
    np.testing.assert_allclose([r1[2], r1[4]], [1 / (f * 0.05) ** 2, 1 / (f * 0.2) ** 2], rtol=1e-12)
    assert abs(r0[3]) < 1e-15 and abs(r1[3]) < 1e-9


# ---------------------------------------------------------------------------
# skew projection: Monte Carlo of the 3D skew normal (reading of Alg. 1 inputs)
# ---------------------------------------------------------------------------

def _mc_case():
    cam = oracle.camera_from_gl(scenes.identity_camera(256, 256))
    cfg = oracle.config()
    mu = np.array([0.3, -0.2, 4.0])
    log_s = np.log([0.05, 0.02, 0.08])
    q = np.array([0.8, 0.3, -0.4, 0.33])
    eta = np.array([1.2, -0.7, 2.0])
    sc = one_gaussian_scene(mu, log_s, q, eta)
    rec = oracle.preprocess(sc, cam, cfg)["rec"][0]
    W2C, f = cam_arrays(cam)
    ind = independent_projection(mu, log_s, q, eta, W2C, f, s_dil=cfg.dilation)
    return cam, cfg, rec, ind


def _oracle_density_grid(rec, ind, h=0.05, span=8.0):
    sd = np.sqrt(np.diag(ind["Sd"]))
    xs = np.arange(-span * sd[0], span * sd[0] + 1e-9, h)
    ys = np.arange(-span * sd[1], span * sd[1] + 1e-9, h)
    X, Y = np.meshgrid(xs, ys, indexing="ij")
    d = np.stack([X.ravel(), Y.ravel()], 1)
    k = oracle.kernel_at(rec[2:5], rec[5:7], d)
    dens = k / (2 * math.pi * math.sqrt(np.linalg.det(ind["Sd"])))
    return d, dens, h * h


def test_skew_projection_moments_closed_form():
    """The projected skew normal has mean mu_2 + sqrt(2/pi) delta_2 and
    covariance Sigma_d - (2/pi) delta_2 delta_2^T, with delta_2 = A R S eta /
    sqrt(1+|eta|^2) computed here independently.  Moments of the oracle's
    2D density (its conic and beta_2) by quadrature must agree."""
    cam, cfg, rec, ind = _mc_case()
    np.testing.assert_allclose(rec[0:2], ind["mu2"], rtol=1e-12)
    d, dens, dA = _oracle_density_grid(rec, ind)
    mass = dens.sum() * dA
    mean = (d * dens[:, None]).sum(0) * dA
    cov = ((d - mean)[:, :, None] * (d - mean)[:, None, :] * dens[:, None, None]).sum(0) * dA
    assert abs(mass - 1.0) < 1e-9
    np.testing.assert_allclose(mean, math.sqrt(2 / math.pi) * ind["delta2"], rtol=1e-6, atol=1e-8)
    ref_cov = ind["Sd"] - (2 / math.pi) * np.outer(ind["delta2"], ind["delta2"])
    np.testing.assert_allclose(cov, ref_cov, rtol=1e-5, atol=1e-7)


def test_skew_projection_monte_carlo_histogram():
    """Sample X = mu + R S (delta |U0| + U), U ~ N(0, I - delta delta^T)
    (stochastic representation of the skew normal, Azzalini & Dalla Valle
    1996), map by the local-affine camera, add N(0, sI); a chi-square test
    against the oracle's normalised 2D skew density."""
    cam, cfg, rec, ind = _mc_case()
    rng = np.random.default_rng(123)
    n = 2_000_000
    eta = np.array([1.2, -0.7, 2.0])
    de = eta / math.sqrt(1 + eta @ eta)
    U0 = np.abs(rng.standard_normal(n))
    cov = np.eye(3) - np.outer(de, de)
    U = rng.multivariate_normal(np.zeros(3), cov, size=n, method="eigh")
    Z = de[None, :] * U0[:, None] + U
    X3 = Z @ (ind["R"] @ ind["S"]).T
    x2 = X3 @ ind["A"].T + math.sqrt(cfg.dilation) * rng.standard_normal((n, 2))
    # sample mean against the closed form (checks the sampler itself)
    se = np.sqrt(np.diag(ind["Sd"]) / n)
    assert np.all(np.abs(x2.mean(0) - math.sqrt(2 / math.pi) * ind["delta2"]) < 5 * se)
    # chi-square on a 16x16 grid of cells over +-3 sd
    sd = np.sqrt(np.diag(ind["Sd"]))
    ex = np.linspace(-3 * sd[0], 3 * sd[0], 17)
    ey = np.linspace(-3 * sd[1], 3 * sd[1], 17)
    H, _, _ = np.histogram2d(x2[:, 0], x2[:, 1], bins=[ex, ey])
    # expected cell masses from the oracle density on a 12x12 sub-grid per cell
    sub = 12
    cx = (ex[:-1, None] + (np.arange(sub)[None, :] + 0.5) / sub * np.diff(ex)[:, None]).ravel()
    cy = (ey[:-1, None] + (np.arange(sub)[None, :] + 0.5) / sub * np.diff(ey)[:, None]).ravel()
    X, Y = np.meshgrid(cx, cy, indexing="ij")
    k = oracle.kernel_at(rec[2:5], rec[5:7], np.stack([X.ravel(), Y.ravel()], 1)).reshape(X.shape)
    dens = k / (2 * math.pi * math.sqrt(np.linalg.det(ind["Sd"])))
    cell = (ex[1] - ex[0]) * (ey[1] - ey[0]) / sub ** 2
    E = dens.reshape(16, sub, 16, sub).sum(axis=(1, 3)) * cell * n
    ok = E > 20
    chi2 = (((H - E) ** 2) / E)[ok].sum()
    dof = ok.sum() - 1
    p = special.chdtrc(dof, chi2)
    assert p > 1e-4, (chi2, dof, p)
    # a wrong sign of beta_2 or a missing sqrt 2 in z would be far off
    k_bad = oracle.kernel_at(rec[2:5], -rec[5:7], np.stack([X.ravel(), Y.ravel()], 1)).reshape(X.shape)
    E_bad = (k_bad / (2 * math.pi * math.sqrt(np.linalg.det(ind["Sd"])))).reshape(16, sub, 16, sub).sum(
        axis=(1, 3)) * cell * n
    assert (((H - E_bad) ** 2) / E_bad)[ok].sum() > 50 * dof


# ---------------------------------------------------------------------------
# compositing (Eq. 2, Eq. color, Alg. 1 blend loop)
# ---------------------------------------------------------------------------

def _stack_scene(depths, logits, rgbs, etas, log_s=math.log(0.5)):
    n = len(depths)
    sh = ((np.asarray(rgbs, np.float64) - 0.5) / (0.5 / math.sqrt(math.pi)))[:, None, :]
    return scenes.Scene(np.array([[0.0, 0.0, z] for z in depths]), np.full((n, 3), log_s),
                        np.tile([1.0, 0.0, 0.0, 0.0], (n, 1)), np.asarray(logits, np.float64),
                        np.asarray(etas, np.float64), sh, 0)


def _comp_indep(z, cam, s_dil, log_s=math.log(0.5)):
    W2C, f = cam_arrays(cam)
    ind = independent_projection(np.array([0.0, 0.0, z]), np.full(3, log_s), [1, 0, 0, 0], np.zeros(3), W2C, f,
                                 s_dil=s_dil)
    return ind["comp"]


# ---------------------------------------------------------------------------
# Enhanced opacity (the alpha equation with two opacities and a split direction)
# ---------------------------------------------------------------------------

def test_enhanced_opacity_equal_logits_is_one_opacity():
    """alpha_1 = alpha_2 makes h = 0: the image equals the one-opacity image,
    whatever the split direction."""
    sc = scenes.cluster(seed=71, n=300, sh_degree=1, two_opacities=True, split=True)
    sc.opacity_logits[:, 1] = sc.opacity_logits[:, 0]
    one = scenes.Scene(sc.means, sc.log_scales, sc.quats, np.ascontiguousarray(sc.opacity_logits[:, 0]), sc.skew,
                       sc.sh, sc.sh_degree, None)
    cam = oracle.camera_from_gl(scenes.identity_camera(48, 40))
    cfg = oracle.config()
    a, b = oracle.render(sc, cam, cfg), oracle.render(one, cam, cfg)
    np.testing.assert_allclose(a["rgb"], b["rgb"], rtol=0, atol=1e-13)


def test_enhanced_opacity_split_direction_and_limits():
    """With zero skew the projected split direction is the skew projection of
    d itself, u_2 = Sigma_d^-1 delta_2(d) / sqrt(1 - delta_2^T Sigma_d^-1 delta_2)
    with delta_2(d) = A R S d / sqrt(1 + |d|^2) (computed here independently),
    and the opacity factor m + h erf(u_2^T delta / sqrt 2) tends to comp
    sigmoid(l_1) far along +u_2 and comp sigmoid(l_2) far along -u_2: the
    ratio alpha(delta) / alpha(-delta) (equal kernels, zero skew) approaches
    sigmoid(l_1) / sigmoid(l_2), and is 1 across u_2."""
    cam = oracle.camera_from_gl(scenes.identity_camera(257, 257))
    cfg = oracle.config()
    mu, log_s, q = [0.0, 0.0, 5.0], np.log([0.4, 0.3, 0.2]), [0.9, 0.2, -0.1, 0.3]
    d = np.array([1.5, -0.7, 0.4])
    l1, l2 = 2.0, -1.0
    sc = one_gaussian_scene(mu, log_s, q, [0.0, 0.0, 0.0], logit=l1, logit2=l2, split=d)
    rec = oracle.preprocess(sc, cam, cfg)["rec"][0]
    W2C, f = cam_arrays(cam)
    ind = independent_projection(np.array(mu), log_s, np.array(q), np.zeros(3), W2C, f)
    d2 = ind["A"] @ ind["R"] @ ind["S"] @ (d / math.sqrt(1.0 + d @ d))
    Si = np.linalg.inv(ind["Sd"])
    u = Si @ d2 / math.sqrt(1.0 - d2 @ Si @ d2)
    np.testing.assert_allclose(rec[9:11], u, rtol=1e-6)
    assert rec[5] == 0.0 and rec[6] == 0.0
    assert np.allclose(rec[0:2], [128.5, 128.5])  # the centre is the centre of pixel (128, 128)
    pc = np.array([128, 128])
    s1, s2 = 1 / (1 + math.exp(-l1)), 1 / (1 + math.exp(-l2))
    # o(e) + o(-e) = 2 m = comp (s1 + s2) for any offset e, with the independent Sigma_d and comp
    rng = np.random.default_rng(3)
    offs = rng.integers(-20, 21, size=(64, 2))
    al_p = oracle.alpha_at(rec, (pc + offs).astype(np.int32))
    al_n = oracle.alpha_at(rec, (pc - offs).astype(np.int32))
    G = np.exp(-0.5 * np.einsum("ni,ij,nj->n", offs, Si, offs))
    np.testing.assert_allclose(al_p + al_n, ind["comp"] * (s1 + s2) * G, rtol=1e-6, atol=1e-300)
    # far along +u_2 / -u_2 the ratio tends to s1 / s2
    ud = u / np.linalg.norm(u)
    errs = []
    for t in (2.0, 4.0, 6.0):  # u^T e / sqrt 2 = t
        off = np.round(t * math.sqrt(2.0) / np.linalg.norm(u) * ud)
        al = oracle.alpha_at(rec, np.array([pc + off, pc - off]).astype(np.int32))
        errs.append(abs(al[0] / al[1] / (s1 / s2) - 1.0))
    assert errs[-1] < 1e-3 and errs[0] > errs[-1]


def test_compositing_closed_form_at_splat_centres():
    """Splats on the optical axis of a 65x65 view land exactly on the centre of
    pixel (32, 32), where delta = 0: alpha = min(alpha_max, comp sigmoid(l))
    whatever the skew; colour c_1 a_1 + c_2 a_2 (1-a_1) + ... + T bg."""
    cam = oracle.camera_from_gl(scenes.identity_camera(65, 65))
    bg = (0.25, 0.5, 0.75)
    cfg = oracle.config(bg=bg)
    depths = [2.0, 3.0, 4.0, 5.0]
    logits = [0.3, -1.0, 1.5, 0.0]
    rgbs = [[0.9, 0.1, 0.2], [0.2, 0.8, 0.3], [0.1, 0.2, 0.7], [0.5, 0.5, 0.5]]
    etas = [[3.0, -2.0, 1.0], [0.0, 0.0, 0.0], [-1.0, 4.0, 0.5], [0.2, 0.2, 0.2]]
    sc = _stack_scene(depths, logits, rgbs, etas)
    out = oracle.render(sc, cam, cfg, pixels=[[32, 32]])
    T, C = 1.0, np.zeros(3)
    for z, l, c in zip(depths, logits, rgbs):
        a = min(cfg.alpha_max, _comp_indep(z, cam, cfg.dilation) / (1 + math.exp(-l)))
        C += np.array(c) * a * T
        T *= 1 - a
    C += T * np.array(bg)
    np.testing.assert_allclose(out["rgb"][0], C, rtol=1e-9)
    assert abs(out["T"][0] - T) < 1e-9 * T
    assert out["count"][0] == 4 and out["last"][0] == 3


def test_compositing_gate_clamp_and_stop():
    """alpha_max clamp, alpha_min gate and the T_stop rule (stop before the
    splat that would take T below T_stop), read as in the design notes."""
    cam = oracle.camera_from_gl(scenes.identity_camera(65, 65))
    cfg = oracle.config(bg=(1.0, 1.0, 1.0))
    # 1: opaque -> clamped to 0.99; 2: tiny opacity -> gated out;
    # 3: 0.98 -> T = 0.01*0.02 = 2e-4 >= 1e-4, blended; 4: 0.9 -> T' = 2e-5 < 1e-4, stop
    s = _comp_indep(2.0, cam, cfg.dilation)
    comps = [_comp_indep(z, cam, cfg.dilation) for z in (2.0, 2.5, 3.0, 3.5, 4.0)]
    target = [0.999999, 0.003, 0.98, 0.9, 0.5]
    logits = [math.log(a / c / (1 - a / c)) if a / c < 1 else 30.0 for a, c in zip(target, comps)]
    rgbs = [[1.0, 0.0, 0.0], [0.0, 1.0, 0.0], [0.0, 0.0, 1.0], [0.5, 0.5, 0.5], [0.3, 0.3, 0.3]]
    sc = _stack_scene([2.0, 2.5, 3.0, 3.5, 4.0], logits, rgbs, np.zeros((5, 3)))
    out = oracle.render(sc, cam, cfg, pixels=[[32, 32]])
    a = [min(cfg.alpha_max, c / (1 + math.exp(-l))) for c, l in zip(comps, logits)]
    assert a[0] == cfg.alpha_max and a[1] < cfg.alpha_min
    T1 = 1 - a[0]
    C = np.array(rgbs[0]) * a[0] + np.array(rgbs[2]) * a[2] * T1
    T = T1 * (1 - a[2])
    assert T >= cfg.t_stop and T * (1 - a[3]) < cfg.t_stop
    C += T * 1.0
    np.testing.assert_allclose(out["rgb"][0], C, rtol=1e-9)
    assert out["count"][0] == 2 and out["last"][0] == 2
    del s


# ---------------------------------------------------------------------------
# camera set-up (Alg. 3, Eq. coord_transform, the K matrix)
# ---------------------------------------------------------------------------

def test_camera_alignment_and_intrinsics():
    g = GOLDEN["intrinsics"]["example"]
    Talign = np.array(GOLDEN["t_align"]["matrix"], np.float64)
    # Blender camera at (0,0,5), identity rotation: looks down -Z at the origin, +Y up
    c2w_gl = np.eye(4)
    c2w_gl[2, 3] = 5.0
    cam = oracle.camera_from_gl(dict(c2w_gl=c2w_gl, width=g["W"], height=g["H"], fovx=math.radians(g["fovx_deg"]),
                                     fovy=2 * math.atan(math.tan(math.radians(30)) * g["H"] / g["W"])))
    W2C, f = cam_arrays(cam)
    assert f["fx"] == float(np.float32(g["fx"])) and f["cx"] == g["cx"] and f["cy"] == g["cy"]
    assert f["fy"] == float(np.float32(g["fx"]))  # square pixels
    t0 = W2C[:, :3] @ np.zeros(3) + W2C[:, 3]
    assert np.allclose(t0, [0, 0, 5]) and np.allclose(pinhole(f, t0), [g["cx"], g["cy"]])
    up = W2C[:, :3] @ np.array([0.0, 1.0, 0.0]) + W2C[:, 3]   # world +Y (up in Blender)
    right = W2C[:, :3] @ np.array([1.0, 0.0, 0.0]) + W2C[:, 3]
    assert pinhole(f, up)[1] < g["cy"] and pinhole(f, right)[0] > g["cx"]
    # a general pose: W2C is the inverse of M_gl T_align (rounded to FP32)
    rng = np.random.default_rng(7)
    Rg = Rotation.random(random_state=11).as_matrix()
    c2w = np.eye(4)
    c2w[:3, :3], c2w[:3, 3] = Rg, rng.normal(size=3)
    cam = oracle.camera_from_gl(dict(c2w_gl=c2w, width=640, height=480, fovx=1.0, fovy=0.8))
    W2C, f = cam_arrays(cam)
    M = np.vstack([W2C, [0, 0, 0, 1]]) @ (c2w @ Talign)
    np.testing.assert_allclose(M, np.eye(4), atol=1e-6)
    np.testing.assert_allclose(f["campos"], c2w[:3, 3], rtol=1e-6)
    assert f["fx"] == float(np.float32(640 / (2 * math.tan(0.5))))
    assert f["fy"] == float(np.float32(480 / (2 * math.tan(0.4))))


# ---------------------------------------------------------------------------
# SH colour basis against scipy's complex spherical harmonics
# ---------------------------------------------------------------------------

def test_sh_basis_matches_scipy_real_harmonics():
    rng = np.random.default_rng(3)
    d = rng.normal(size=(200, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    Y = oracle.sh_basis(3, d)
    theta = np.arccos(np.clip(d[:, 2], -1, 1))
    phi = np.arctan2(d[:, 1], d[:, 0])
    k = 0
    for l in range(4):
        for m in range(-l, l + 1):
            c = special.sph_harm_y(l, abs(m), theta, phi)  # includes the Condon-Shortley phase
            if m < 0:
                ref = math.sqrt(2) * c.imag
            elif m == 0:
                ref = c.real
            else:
                ref = math.sqrt(2) * c.real
            np.testing.assert_allclose(Y[:, k], ref, atol=1e-13, err_msg=f"l={l} m={m}")
            k += 1


def test_sh_colour_uses_the_direction_from_the_camera_to_the_centre():
    """The view direction of the SH colour points from the camera centre to
    the Gaussian (the convention the library states).  Cameras on the +x,
    -x, +z and -z sides of a Gaussian carrying only degree-1 coefficients see
    the colours that scipy's harmonics give for that direction, and the
    opposite colours for the reversed one (odd degree: a flipped direction
    flips the sign of the degree-1 term, which these expected values fail)."""
    mu = np.array([0.3, -0.2, 4.0])
    sh = np.zeros((1, 4, 3))
    sh[0, 1:, 0] = [0.11, -0.07, 0.05]   # red: all three degree-1 coefficients
    sh[0, 3, 1] = 0.2                    # green: the x-aligned one only
    sc = scenes.Scene(means=mu[None], log_scales=np.full((1, 3), -3.0), quats=np.array([[1.0, 0, 0, 0]]),
                      opacity_logits=np.array([2.0]), skew=np.zeros((1, 3)), sh=sh, sh_degree=1)
    cfg = oracle.config()

    def basis_deg1(d):
        # real SH of degree 1 from scipy (Condon-Shortley phase included), order m = -1, 0, 1
        theta, phi = math.acos(d[2]), math.atan2(d[1], d[0])
        c = special.sph_harm_y(1, 1, theta, phi)
        return np.array([math.sqrt(2) * c.imag, special.sph_harm_y(1, 0, theta, phi).real, math.sqrt(2) * c.real])

    seen = 0
    for eye in ([3.0, -0.2, 4.0], [-2.4, -0.2, 4.0], [0.3, -0.2, 1.0], [0.3, -0.2, 7.5]):
        cam = oracle.camera_from_gl(scenes.camera(scenes.look_at_c2w_cv(eye, mu), 32, 32))
        pre = oracle.preprocess(sc, cam, cfg)
        assert pre["visible"][0]
        campos = np.array(oracle.camera_fields(cam)["campos"])
        d = (mu - campos) / np.linalg.norm(mu - campos)
        Y = basis_deg1(d)
        want = 0.5 + np.array([Y @ sh[0, 1:, 0], Y @ sh[0, 1:, 1], 0.0]) + sh[0, 0] * 0.28209479177387814
        flipped = 0.5 + np.array([-(Y @ sh[0, 1:, 0]), -(Y @ sh[0, 1:, 1]), 0.0])
        got = pre["rec"][0, 11:14]
        np.testing.assert_allclose(got, np.maximum(want, 0.0), atol=1e-6)
        assert np.abs(got - np.maximum(flipped, 0.0)).max() > 1e-3
        seen += 1
    assert seen == 4


# ---------------------------------------------------------------------------
# depth key and binning (tile-based, depth sorted: Preliminaries)
# ---------------------------------------------------------------------------

def test_depth_key_is_the_specified_fp32_sequence():
    sc = scenes.unbounded(seed=9, n=5000)
    cam = oracle.camera_from_gl(scenes.orbit_camera(0.7, 320, 240))
    pre = oracle.preprocess(sc, cam, oracle.config())
    W2C, _ = cam_arrays(cam)
    w = W2C[2].astype(np.float32)
    m = sc.means.astype(np.float32)
    z = ((w[0] * m[:, 0] + w[1] * m[:, 1]) + w[2] * m[:, 2]) + w[3]
    assert z.dtype == np.float32
    np.testing.assert_array_equal(pre["depth_bits"], z.view(np.uint32))
    np.testing.assert_array_equal(pre["visible"], z > np.float32(0.2))


def _footprint_scene(seed=4, n=300):
    sc = scenes.cluster(seed=seed, n=n, sh_degree=1, skew_sigma=3.0, two_opacities=True, split=True)
    sc.log_scales[:] = np.random.default_rng(seed).uniform(-4.5, -2.0, (n, 3)).astype(np.float32)
    return sc


def test_footprint_is_conservative_dense_sampling():
    """No pixel centre outside a Gaussian's box [mu +- e] has alpha >= alpha_min,
    and a culled Gaussian reaches alpha_min nowhere (grid wider than the image)."""
    sc = _footprint_scene()
    cam = oracle.camera_from_gl(scenes.identity_camera(96, 72))
    cfg = oracle.config()
    pre = oracle.preprocess(sc, cam, cfg)
    n_checked = 0
    for i in np.nonzero(pre["visible"])[0]:
        r = pre["rec"][i]
        lo = np.floor(r[0:2] - 80).astype(int)
        xs, ys = np.arange(lo[0], lo[0] + 160), np.arange(lo[1], lo[1] + 160)
        pix = np.stack(np.meshgrid(xs, ys, indexing="xy"), -1).reshape(-1, 2).astype(np.int32)
        al = np.minimum(oracle.alpha_at(r, pix), cfg.alpha_max)
        hit = al >= cfg.alpha_min
        ex, ey, _ = pre["ext"][i]
        if ex == 0.0:
            assert not hit.any(), i
            continue
        c = pix[hit] + 0.5
        assert np.all(np.abs(c[:, 0] - r[0]) <= ex) and np.all(np.abs(c[:, 1] - r[1]) <= ey), i
        n_checked += 1
    assert n_checked > 100


def ellipse_meets_rect(mx, my, A, rho2, x0, x1, y0, y1):
    """Independent test: does {p : (p-m)^T A (p-m) <= rho2} meet the
    rectangle [x0,x1] x [y0,y1]?  Yes if the centre is inside; otherwise the
    minimum of the convex quadratic over the rectangle lies on an edge, where
    it is a 1-D quadratic minimised in closed form."""
    if x0 <= mx <= x1 and y0 <= my <= y1:
        return True
    m = np.array([mx, my])
    corners = [np.array(c, float) for c in ((x0, y0), (x1, y0), (x1, y1), (x0, y1))]
    best = np.inf
    for k in range(4):
        p0, p1 = corners[k], corners[(k + 1) % 4]
        d, e = p0 - m, p1 - p0
        eAe = e @ A @ e
        t = 0.0 if eAe == 0 else min(1.0, max(0.0, -(d @ A @ e) / eAe))
        q = (d + t * e) @ A @ (d + t * e)
        best = min(best, q)
    return best <= rho2


def footprint_band_extent(r, rho2, tau, y0, y1, nsamp=4001):
    """The tile rule's x-extent (relative to mu_x) of a record's footprint
    within the heights [y0, y1] (relative to mu_y), evaluated by dense
    sampling of the ellipses' boundaries instead of their closed-form extreme
    points: E1's extent cut by the hull of the half-plane beta^T d >= 0 (the
    band clipped to E1's heights) and E2's.  None if the band misses."""
    a, b, c, bx, by = r[2], r[3], r[4], r[5], r[6]

    def ext(a, b, c, q, lo, hi):
        if q <= 0:
            return None
        D = a * c - b * b
        ymax = np.sqrt(a * q / D)
        lo, hi = max(lo, -ymax), min(hi, ymax)
        if lo > hi:
            return None
        ys = np.linspace(lo, hi, nsamp)
        s = np.sqrt(np.maximum(0.0, a * q - D * ys * ys))
        return ((-b * ys - s) / a).min(), ((-b * ys + s) / a).max(), lo, hi

    e1 = ext(a, b, c, rho2, y0, y1)
    if e1 is None:
        return None
    xl, xr, c0, c1 = e1
    if bx == 0 and by == 0:
        return xl, xr
    if bx != 0:
        line = -by * np.array([c0, c1]) / bx
        h = (line.min(), np.inf) if bx > 0 else (-np.inf, line.max())
    else:
        h = (-np.inf, np.inf) if ((by > 0 and c1 >= 0) or (by < 0 and c0 <= 0)) else None
    omax = r[14] * max(r[15], r[16])
    e2 = ext(a + bx * bx, b + bx * by, c + by * by, 2 * np.log(omax / tau) * (1 + 2.0 ** -10), y0, y1)
    parts = [p for p in (h, None if e2 is None else e2[:2]) if p is not None]
    if not parts:
        return None
    return max(xl, min(p[0] for p in parts)), min(xr, max(p[1] for p in parts))


def test_skew_side_bound_dense_sampling():
    """On the side beta^T d < 0 (z < 0), 1 + erf z <= exp(-z^2), so every
    pixel centre with alpha >= alpha_min lies in E2 = {d^T (A + beta beta^T) d
    <= 2 ln(o_max comp / tau)}; on the other side it lies in E1 (rho2).  Dense
    sampling around strongly skewed Gaussians with two opacities and a split
    direction."""
    sc = _footprint_scene(seed=11, n=300)
    cam = oracle.camera_from_gl(scenes.identity_camera(96, 72))
    cfg = oracle.config()
    pre = oracle.preprocess(sc, cam, cfg)
    tau = float(cfg.alpha_min)
    n_minus = 0
    for i in np.nonzero(pre["ext"][:, 0] > 0)[0]:
        r = pre["rec"][i]
        lo = np.floor(r[0:2] - 60).astype(int)
        xs, ys = np.arange(lo[0], lo[0] + 120), np.arange(lo[1], lo[1] + 120)
        pix = np.stack(np.meshgrid(xs, ys, indexing="xy"), -1).reshape(-1, 2).astype(np.int32)
        hit = np.minimum(oracle.alpha_at(r, pix), cfg.alpha_max) >= tau
        d = pix[hit] + 0.5 - r[0:2]
        a, b, c, bx, by = r[2], r[3], r[4], r[5], r[6]
        q1 = a * d[:, 0] ** 2 + 2 * b * d[:, 0] * d[:, 1] + c * d[:, 1] ** 2
        zb = bx * d[:, 0] + by * d[:, 1]
        q2 = q1 + zb * zb
        omax = r[14] * max(r[15], r[16])
        assert np.all(q1 <= pre["ext"][i, 2] * (1 + 1e-12)), i
        neg = zb < 0
        assert np.all(q2[neg] <= 2 * np.log(omax / tau) * (1 + 1e-12)), i
        n_minus += int(neg.sum())
    assert n_minus > 1000


def test_tile_sets_and_sorted_keys_match_brute_force():
    """A tile is touched iff a pixel-centre column of it lies in the
    footprint's x-extent within the tile row's band of pixel-centre heights
    (footprint_band_extent, by dense sampling), and the rule stays inside the
    E1 tiles (edge-minimisation test above) and equals them for zero skew;
    brute force over every tile against the oracle's key lists, then the
    sorted keys against numpy's lexsort."""
    sc = _footprint_scene(seed=6, n=400)
    cam = oracle.camera_from_gl(scenes.identity_camera(100, 75))
    cfg = oracle.config(tile=16)
    pre = oracle.preprocess(sc, cam, cfg)
    W, H, T = cam.width, cam.height, 16
    tx, ty = -(-W // T), -(-H // T)
    keys, vals = [], []
    skip = []
    n_box = 0
    for i in range(sc.n):
        if not pre["visible"][i]:
            continue
        r = pre["rec"][i]
        ex, ey, rho2 = pre["ext"][i]
        touched, e1_tiles = [], []
        near = False
        if ex > 0:
            A = np.array([[r[2], r[3]], [r[3], r[4]]])
            for by in range(ty):
                y0, y1 = by * T + 0.5, min(H, by * T + T) - 0.5
                span = footprint_band_extent(r, rho2, float(cfg.alpha_min), y0 - r[1], y1 - r[1])
                if span is not None:
                    xl, xr = r[0] + span[0] - 0.5, r[0] + span[1] - 0.5
                    # sampled extents are exact to ~1e-6 px: skip near-boundary rows
                    near = near or min(abs(xl - np.round(xl)), abs(xr - np.round(xr))) < 5e-3
                    lo, hi = max(np.ceil(xl), 0), min(np.floor(xr), W - 1)
                    if lo <= hi:
                        touched += [by * tx + t for t in range(int(lo) // T, int(hi) // T + 1)]
                for bx in range(tx):
                    x0, x1 = bx * T + 0.5, min(W, bx * T + T) - 0.5
                    if ellipse_meets_rect(r[0], r[1], A, rho2, x0, x1, y0, y1):
                        e1_tiles.append(by * tx + bx)
            rc = pre["rect"][i]
            n_box += (rc[2] - rc[0]) * (rc[3] - rc[1])
            assert set(touched) <= {y * tx + x for y in range(rc[1], rc[3]) for x in range(rc[0], rc[2])}, i
            assert set(touched) <= set(e1_tiles), i
            if r[5] == 0 and r[6] == 0:
                assert set(touched) == set(e1_tiles), i
        if not pre["rect_ambig"][i] and not near:
            assert len(touched) == pre["ntouch"][i], i
        if near:
            skip.append(i)
        for t in touched:
            keys.append((t << 32) | int(pre["depth_bits"][i]))
            vals.append(i)
    keys = np.array(keys, np.uint64)
    vals = np.array(vals, np.int64)
    ok, ov = oracle.bin_keys(pre, cam, cfg)
    amb = np.concatenate([np.nonzero(pre["rect_ambig"])[0], np.array(skip, np.int64)])
    keep_b = ~np.isin(vals, amb)
    keep_o = ~np.isin(ov, amb)
    order = np.lexsort((vals[keep_b], keys[keep_b]))
    np.testing.assert_array_equal(ok[keep_o], keys[keep_b][order])
    np.testing.assert_array_equal(ov[keep_o], vals[keep_b][order])
    assert len(ok) < n_box  # the ellipse test drops corner tiles of the boxes


def test_touched_tiles_cover_every_pixel_reaching_alpha_min():
    """Conservativeness of the tile test itself: every pixel centre where a
    Gaussian reaches alpha_min lies in a tile of that Gaussian's key list."""
    sc = _footprint_scene(seed=8, n=250)
    cam = oracle.camera_from_gl(scenes.identity_camera(96, 72))
    cfg = oracle.config()
    pre = oracle.preprocess(sc, cam, cfg)
    keys, vals = oracle.bin_keys(pre, cam, cfg)
    tiles_x = -(-96 // 16)
    pix = np.stack(np.meshgrid(np.arange(96), np.arange(72), indexing="xy"), -1).reshape(-1, 2).astype(np.int32)
    tile_of_pix = (pix[:, 1] // 16) * tiles_x + pix[:, 0] // 16
    for i in np.nonzero(pre["visible"])[0]:
        al = np.minimum(oracle.alpha_at(pre["rec"][i], pix), cfg.alpha_max)
        need = set(tile_of_pix[al >= cfg.alpha_min].tolist())
        have = set((keys[vals == i] >> np.uint64(32)).astype(np.int64).tolist())
        assert need <= have, i
