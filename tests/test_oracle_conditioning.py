"""Pins of the oracle's Beta-modulated conditioning (Sec. 4.3) away from its
two Gaussian ends, and of its camera convention (Sec. 3 projection, Sec. 4.4
view direction) under rotated and translated cameras.

Every expected value here is formed from the primitive's parameters by a
route other than the oracle's own matrix product: scalar closed forms for a
one-dimensional query, per-dimension sums where the query covariance is
diagonal, the regression matrix from the precision blocks of the full
covariance, limits in which the modulation must vanish, invariance of the
rendered image under one rigid motion of scene and camera together, and a
view direction computed from a camera placed at a known position.
"""
import math

import numpy as np
import pytest
import torch
from scipy.spatial.transform import Rotation

from oracle import fp32_spec
from oracle import render64 as R64
from paper_2510_03312_gb300 import scenes as S


def _cam(position, W=64, H=48, f=60.0, time=0.0, dtype=np.float64):
    """Camera at a known centre c looking at the origin: x_cam = R x + t with
    t = -R c, so that c maps to the camera origin."""
    R, _ = S.look_at(position)
    c = np.asarray(position, np.float64)
    t = -R @ c
    return S.View(R=np.asarray(R, dtype), t=np.asarray(t, dtype), fx=f, fy=f, cx=W / 2, cy=H / 2,
                  width=W, height=H, time=time), c


def _rot_scale(sc):
    """[P,3,3] R diag(s) from the quaternion plane, with SciPy's rotation."""
    q = sc.plane("rot").astype(np.float64)
    R = Rotation.from_quat(np.stack([q[1], q[2], q[3], q[0]], 1)).as_matrix()
    return R * sc.plane("scale_x").T.astype(np.float64)[:, None, :]


def _blocks(sc):
    """Sigma_x, Sigma_xq [P,3,C], Sigma_q [P,C,C] from the appendix's block
    form of L L^T (pinned there against the oracle's product)."""
    C = sc.N - 3
    Rs = _rot_scale(sc)
    lqx = sc.plane("L_qx").T.astype(np.float64).reshape(-1, C, 3)
    lq = np.zeros((sc.P, C, C))
    pk = sc.plane("L_q").astype(np.float64)
    for i in range(C):
        for j in range(i + 1):
            lq[:, i, j] = pk[i * (i + 1) // 2 + j]
    Sx = Rs @ Rs.transpose(0, 2, 1)
    Sxq = Rs @ lqx.transpose(0, 2, 1)
    Sq = lqx @ lqx.transpose(0, 2, 1) + lq @ lq.transpose(0, 2, 1)
    return Sx, Sxq, Sq


def _one_minus_tanh(x):
    """1 - tanh(x) = 2 e^{-2x} / (1 + e^{-2x}), accurate where tanh(x) has
    rounded to 1."""
    e = np.exp(-2.0 * x)
    return 2.0 * e / (1.0 + e)


def _query(sc, c, time):
    """q = [t, d] with d = (mu_x - c)/|mu_x - c| for a camera centred at c."""
    C = sc.N - 3
    mx = sc.plane("mean_x").T.astype(np.float64)
    parts = []
    if C in (1, 4):
        parts.append(np.full((sc.P, 1), float(time)))
    if C >= 3:
        v = mx - c[None, :]
        parts.append(v / np.linalg.norm(v, axis=1, keepdims=True))
    return np.concatenate(parts, 1)


# ---------------------------------------------------------------- Sec. 4.3, scalar query

@pytest.mark.parametrize("bt", [0.2, 0.5, 0.8])
def test_scalar_query_closed_form(bt):
    """N = 4 (q = [t]): with a scalar query the modulation is one number, and
    mu_{x|q} = mu_x + beta~ Sigma_xq (t - mu_t)/Sigma_q,
    Sigma_{x|q} = Sigma_x - beta~ Sigma_xq Sigma_qx / Sigma_q,
    o(q) = o (1 - tanh((t - mu_t)^2 / Sigma_q))^(4 beta_q)."""
    sc = S.make_scene(21, 4, 60)
    sc.plane("b")[1] = np.float32(math.log(bt))
    time = 0.37
    v, c = _cam([0.4, 0.5, 3.5], time=time)
    mu_c, Sc, oq, _ = R64.condition(R64.scene_leaves(sc), 4, 0, v)
    Sx, Sxq, Sq = _blocks(sc)
    sxq, sq = Sxq[:, :, 0], Sq[:, 0, 0]
    beta_q = np.exp(sc.plane("b")[1].astype(np.float64))
    assert np.all(np.abs(beta_q - bt) < 1e-6)           # 0 < beta~ = beta_q < 1
    delta = time - sc.plane("mean_q")[0].astype(np.float64)
    mx = sc.plane("mean_x").T.astype(np.float64)
    np.testing.assert_allclose(mu_c.numpy(), mx + (beta_q * delta / sq)[:, None] * sxq, rtol=1e-12, atol=1e-15)
    Sref = Sx - (beta_q / sq)[:, None, None] * sxq[:, :, None] * sxq[:, None, :]
    np.testing.assert_allclose(Sc.numpy(), Sref, rtol=1e-11, atol=1e-17)
    o = sc.plane("opacity")[0].astype(np.float64)
    np.testing.assert_allclose(oq.numpy(), o * _one_minus_tanh(delta ** 2 / sq) ** (4 * beta_q), rtol=1e-11, atol=1e-280)
    # the conditioned covariance lies strictly between the conditional (beta~ = 1)
    # and the marginal (beta~ = 0): Sigma_{x|q} - Sigma_gauss = (1 - beta~) rank-one term
    Sgauss = Sx - (1.0 / sq)[:, None, None] * sxq[:, :, None] * sxq[:, None, :]
    np.testing.assert_allclose(Sc.numpy() - Sgauss, (1 - beta_q)[:, None, None] * (Sx - Sgauss),
                               rtol=1e-9, atol=1e-16)


def test_scalar_query_opacity_takes_the_unclamped_exponent():
    """beta_q > 1: the conditioning is Gaussian (beta~ = 1), while the opacity
    exponent is 4 beta_q = 4 e^{b_q}, not 4 beta~."""
    sc = S.make_scene(22, 4, 40)
    sc.plane("b")[1] = np.float32(0.6)
    v, c = _cam([0.1, -0.3, 3.0], time=0.8)
    mu_c, Sc, oq, _ = R64.condition(R64.scene_leaves(sc), 4, 0, v)
    Sx, Sxq, Sq = _blocks(sc)
    sxq, sq = Sxq[:, :, 0], Sq[:, 0, 0]
    delta = 0.8 - sc.plane("mean_q")[0].astype(np.float64)
    mx = sc.plane("mean_x").T.astype(np.float64)
    np.testing.assert_allclose(mu_c.numpy(), mx + (delta / sq)[:, None] * sxq, rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(Sc.numpy(), Sx - (1 / sq)[:, None, None] * sxq[:, :, None] * sxq[:, None, :],
                               rtol=1e-11, atol=1e-17)
    o = sc.plane("opacity")[0].astype(np.float64)
    bq = math.exp(float(np.float32(0.6)))
    np.testing.assert_allclose(oq.numpy(), o * _one_minus_tanh(delta ** 2 / sq) ** (4 * bq), rtol=1e-11, atol=1e-280)


# ---------------------------------------------------------------- Sec. 4.3, vanishing modulation

@pytest.mark.parametrize("N", [4, 6, 7])
def test_vanishing_beta_keeps_the_marginal(N):
    """beta_q -> 0 (b_q = -60) with a nonzero cross block L_qx: the modulation
    switches conditioning off, mu_{x|q} = mu_x and Sigma_{x|q} = Sigma_x, and
    the opacity keeps o."""
    sc = S.make_scene(23, N, 50)
    assert np.abs(sc.plane("L_qx")).min() > 0
    sc.plane("b")[1:] = -60.0
    v, _ = _cam([1.0, 0.7, -3.0], time=0.9)
    mu_c, Sc, oq, _ = R64.condition(R64.scene_leaves(sc), N, 0, v)
    Sx, _, _ = _blocks(sc)
    np.testing.assert_allclose(mu_c.numpy(), sc.plane("mean_x").T.astype(np.float64), rtol=0, atol=1e-24)
    np.testing.assert_allclose(Sc.numpy(), Sx, rtol=1e-13, atol=1e-24)
    np.testing.assert_allclose(oq.numpy(), sc.plane("opacity")[0].astype(np.float64), rtol=1e-20, atol=1e-20)


# ---------------------------------------------------------------- Sec. 4.3, one dimension at a time

def _diagonal_query_scene(N, seed):
    """Scene whose Sigma_q is diagonal by construction: the rows of L_qx that
    are nonzero are mutually orthogonal, and L_q is diagonal (for N = 7 the
    time row of L_qx is zero)."""
    sc = S.make_scene(seed, N, 40)
    rng = np.random.default_rng(seed)
    C = N - 3
    # integer rows [1,2,2], [2,1,-2], [2,-2,1] are mutually orthogonal; signed
    # column permutations keep them so, and scaling each row by a float32
    # amplitude keeps every entry (and so the orthogonality) exact in float32
    base = np.array([[1.0, 2.0, 2.0], [2.0, 1.0, -2.0], [2.0, -2.0, 1.0]])
    lqx = np.zeros((sc.P, C, 3))
    for p in range(sc.P):
        Qm = base[rng.permutation(3)][:, rng.permutation(3)] * rng.choice([-1.0, 1.0], 3)[None, :]
        amp = rng.uniform(0.07, 0.27, 3).astype(np.float32).astype(np.float64)
        lqx[p, C - 3:, :] = amp[:, None] * Qm
    sc.plane("L_qx")[:] = lqx.reshape(sc.P, 3 * C).T.astype(np.float32)
    lq = sc.plane("L_q")
    for i in range(C):
        for j in range(i):
            lq[i * (i + 1) // 2 + j] = 0.0
    # distinct modulations per dimension, all strictly inside (0, 1)
    sc.plane("b")[1:] = np.log(rng.uniform(0.1, 0.9, (C, sc.P))).astype(np.float32)
    return sc


@pytest.mark.parametrize("N", [6, 7])
def test_diagonal_query_covariance_interpolates_each_dimension(N):
    """With Sigma_q diagonal, diag(beta~) commutes with Sigma_q^{-1}, so each
    query dimension i moves the kernel independently, a fraction beta~_i of
    the way from the marginal to its own Gaussian conditional:
    mu_{x|q} = mu_x + sum_i beta~_i Sigma_xq[:, i] delta_i / Sigma_q[i, i],
    Sigma_{x|q} = Sigma_x - sum_i beta~_i Sigma_xq[:, i] Sigma_xq[:, i]^T / Sigma_q[i, i]."""
    sc = _diagonal_query_scene(N, 24 + N)
    v, c = _cam([-2.0, 1.5, 2.5], time=0.55)
    mu_c, Sc, oq, _ = R64.condition(R64.scene_leaves(sc), N, 0, v)
    Sx, Sxq, Sq = _blocks(sc)
    off = Sq - np.einsum("pii->pi", Sq)[:, :, None] * np.eye(N - 3)[None]
    assert np.abs(off).max() < 1e-12 * np.abs(Sq).max()
    bt = np.exp(sc.plane("b")[1:].T.astype(np.float64))
    delta = _query(sc, c, 0.55) - sc.plane("mean_q").T.astype(np.float64)
    sii = np.einsum("pii->pi", Sq)
    mu_ref = sc.plane("mean_x").T.astype(np.float64).copy()
    S_ref = Sx.copy()
    for i in range(N - 3):
        w = bt[:, i] / sii[:, i]
        mu_ref += (w * delta[:, i])[:, None] * Sxq[:, :, i]
        S_ref -= w[:, None, None] * Sxq[:, :, i, None] * Sxq[:, None, :, i]
    np.testing.assert_allclose(mu_c.numpy(), mu_ref, rtol=1e-11, atol=1e-14)
    np.testing.assert_allclose(Sc.numpy(), S_ref, rtol=1e-10, atol=1e-16)
    # and the opacity: the Cholesky factor of a diagonal Sigma_q is its square
    # root, so d_i = tanh(delta_i^2 / Sigma_q[i, i])
    o = sc.plane("opacity")[0].astype(np.float64)
    bq = np.exp(sc.plane("b")[1:].T.astype(np.float64))
    ref = o * np.prod(_one_minus_tanh(delta ** 2 / sii) ** (4 * bq), axis=1)
    np.testing.assert_allclose(oq.numpy(), ref, rtol=1e-10, atol=1e-280)


# ---------------------------------------------------------------- Sec. 4.3, general Sigma_q

@pytest.mark.parametrize("N", [6, 7])
def test_general_modulation_through_the_precision_blocks(N):
    """General Sigma_q and distinct beta~_i in (0, 1).  The Gaussian regression
    matrix K0 = Sigma_xq Sigma_q^{-1} equals -(Lambda_xx)^{-1} Lambda_xq with
    Lambda the inverse of the whole covariance, and diag(beta~) scales its
    columns: mu_{x|q} = mu_x + sum_j beta~_j delta_j K0[:, j],
    Sigma_{x|q} = Sigma_x - sym(sum_j beta~_j K0[:, j] Sigma_qx[j, :])."""
    sc = S.make_scene(30 + N, N, 60)
    rng = np.random.default_rng(N)
    C = N - 3
    sc.plane("b")[1:] = np.log(rng.uniform(0.1, 0.9, (C, sc.P))).astype(np.float32)
    v, c = _cam([2.5, -1.0, 2.0], time=0.15)
    mu_c, Sc, _, _ = R64.condition(R64.scene_leaves(sc), N, 0, v)
    Sx, Sxq, Sq = _blocks(sc)
    full = np.zeros((sc.P, N, N))
    full[:, :3, :3], full[:, :3, 3:], full[:, 3:, :3], full[:, 3:, 3:] = Sx, Sxq, Sxq.transpose(0, 2, 1), Sq
    Lam = np.linalg.inv(full)
    K0 = -np.linalg.solve(Lam[:, :3, :3], Lam[:, :3, 3:])
    bt = np.exp(sc.plane("b")[1:].T.astype(np.float64))
    delta = _query(sc, c, 0.15) - sc.plane("mean_q").T.astype(np.float64)
    mu_ref = sc.plane("mean_x").T.astype(np.float64).copy()
    M = np.zeros((sc.P, 3, 3))
    for j in range(C):
        mu_ref += (bt[:, j] * delta[:, j])[:, None] * K0[:, :, j]
        M += bt[:, j, None, None] * K0[:, :, j, None] * Sxq.transpose(0, 2, 1)[:, None, j, :]
    S_ref = Sx - 0.5 * (M + M.transpose(0, 2, 1))
    np.testing.assert_allclose(mu_c.numpy(), mu_ref, rtol=1e-9, atol=1e-12)
    np.testing.assert_allclose(Sc.numpy(), S_ref, rtol=1e-8, atol=1e-14)


@pytest.mark.parametrize("N", [6, 7])
def test_dimension_with_vanishing_beta_is_ignored_by_the_mean(N):
    """diag(beta~) multiplies (q - mu_q): a query dimension whose beta~ is zero
    (b_q = -60) cannot move the conditioned mean, however far mu_q is moved
    along it, while the other dimensions still do."""
    C = N - 3
    sc = S.make_scene(40 + N, N, 30)
    sc.plane("b")[1:] = np.abs(sc.plane("b")[1:]) * -1 - 0.2
    j = C - 2
    sc.plane("b")[1 + j] = -60.0
    v, _ = _cam([1.5, 2.0, 2.5], time=0.4)
    mu_a, _, _, _ = R64.condition(R64.scene_leaves(sc), N, 0, v)
    moved = S.Scene(N, 0, sc.params.copy())
    moved.plane("mean_q")[j] += 0.75
    mu_b, _, _, _ = R64.condition(R64.scene_leaves(moved), N, 0, v)
    np.testing.assert_allclose(mu_b.numpy(), mu_a.numpy(), rtol=0, atol=1e-20)
    other = S.Scene(N, 0, sc.params.copy())
    other.plane("mean_q")[C - 1] += 0.75
    mu_c, _, _, _ = R64.condition(R64.scene_leaves(other), N, 0, v)
    assert np.abs(mu_c.numpy() - mu_a.numpy()).min(1).max() > 1e-6


# ---------------------------------------------------------------- Sec. 4.4, view direction

@pytest.mark.parametrize("N", [6, 7])
def test_view_direction_from_a_camera_at_a_known_centre(N):
    """The query's direction is the unit vector from the camera centre to the
    primitive's spatial mean, for a rotated and translated camera placed at a
    known point; for N = 7 the time comes first."""
    sc = S.make_scene(50 + N, N, 80)
    lv = R64.scene_leaves(sc)
    for pos, time in (([3.0, -1.0, 2.0], 0.25), ([-0.5, 4.0, -1.5], 0.9)):
        v, c = _cam(pos, time=time)
        q = R64.query(lv, N, v).numpy()
        mx = sc.plane("mean_x").T.astype(np.float64)
        d = (mx - c) / np.linalg.norm(mx - c, axis=1, keepdims=True)
        if N == 7:
            np.testing.assert_array_equal(q[:, 0], np.float64(time))
            q = q[:, 1:]
        np.testing.assert_allclose(q, d, rtol=0, atol=1e-14)


# ---------------------------------------------------------------- Sec. 3, rigid motion

def _image64(sc, v, cfg):
    """Float64 image of an N = 3 scene by the oracle's conditioning,
    projection and per-pixel compositing, every pixel blending all records
    beyond the near plane in float64 depth order (no float32 stage)."""
    lv = R64.scene_leaves(sc) if not isinstance(sc, dict) else sc
    mu_c, Sc, oq, beta = R64.condition(lv, 3, 0, v)
    tz, mu2, cov2, conic = R64.project(mu_c, Sc, v, cfg)
    keep = torch.nonzero(tz > cfg.near)[:, 0]
    lst = keep[torch.argsort(tz[keep])]
    ys, xs = np.meshgrid(np.arange(v.height), np.arange(v.width), indexing="ij")
    px = torch.tensor(xs.ravel() + 0.5, dtype=torch.float64)
    py = torch.tensor(ys.ravel() + 0.5, dtype=torch.float64)
    col, T, _, _ = R64._composite_block(px, py, mu2[lst], conic[lst], oq[lst], beta[lst],
                                        lv["rgb"].T[lst], cfg)
    return col.T.reshape(3, v.height, v.width), (tz, mu2, cov2)


def test_rigid_motion_of_scene_and_camera_leaves_the_image_unchanged():
    """One rotation Q and translation u applied to every mean (mu -> Q mu + u),
    every orientation (R_x -> Q R_x) and the camera (W -> W Q^T,
    t -> t - W Q^T u) leaves camera-space geometry, so depths, screen means,
    footprints and the float64 image, unchanged.  A transposed W or Jacobian
    product would not be invariant."""
    sc = S.make_scene(60, 3, 300)
    cfg = S.RasterConfig()
    v, _ = _cam([2.0, 1.0, 3.2])
    lv = R64.scene_leaves(sc)
    img_a, (tz_a, mu_a, cov_a) = _image64(lv, v, cfg)
    rng = np.random.default_rng(60)
    Qr = Rotation.random(random_state=7)
    Q = Qr.as_matrix()
    u = rng.uniform(-2, 2, 3)
    lv2 = {k: t.clone() for k, t in lv.items()}
    lv2["mean_x"] = torch.tensor(Q @ lv["mean_x"].numpy() + u[:, None])
    qa = lv["rot"].numpy()
    comp = (Qr * Rotation.from_quat(np.stack([qa[1], qa[2], qa[3], qa[0]], 1))).as_quat()
    lv2["rot"] = torch.tensor(np.stack([comp[:, 3], comp[:, 0], comp[:, 1], comp[:, 2]], 0))
    Rc = np.asarray(v.R, np.float64) @ Q.T
    v2 = S.View(R=Rc, t=np.asarray(v.t, np.float64) - Rc @ u, fx=v.fx, fy=v.fy, cx=v.cx, cy=v.cy,
                width=v.width, height=v.height)
    img_b, (tz_b, mu_b, cov_b) = _image64(lv2, v2, cfg)
    np.testing.assert_allclose(tz_b.numpy(), tz_a.numpy(), rtol=1e-13)
    np.testing.assert_allclose(mu_b.numpy(), mu_a.numpy(), rtol=1e-12, atol=1e-10)
    np.testing.assert_allclose(cov_b.numpy(), cov_a.numpy(), rtol=1e-11)
    assert float(img_a.max()) > 0.1
    assert float((img_b - img_a).abs().max()) <= 1e-12


def test_sign_flip_motion_keeps_every_float32_decision():
    """The half-turn Q = diag(1, -1, -1) about x changes no magnitude in
    float32: mu -> Q mu, quaternion (w, x, y, z) -> (w, x, -y, -z) (so
    R_x -> Q R_x Q, the same covariance up to the signs Q), W -> W Q.  The
    float32 decision stage must then give bit-identical culls, depth keys and
    rectangles, and the whole oracle render the same image, through a
    rotated camera that does not commute with Q."""
    wl = S.workload_static_small(seed=61, P=400, size=64)
    sc = wl.scenes[0]
    R, t = S.look_at([1.3, 2.1, -2.2])
    v = S.make_view(R, t, 64, 48)
    sc2 = S.Scene(3, 0, sc.params.copy())
    sc2.plane("mean_x")[1:] *= -1
    sc2.plane("rot")[2:] *= -1
    Q = np.diag([1.0, -1.0, -1.0]).astype(np.float32)
    v2 = S.View(R=np.asarray(v.R, np.float32) @ Q, t=v.t.copy(), fx=v.fx, fy=v.fy, cx=v.cx, cy=v.cy,
                width=v.width, height=v.height)
    cfg = wl.cfg
    a = fp32_spec.preprocess([sc], [v], cfg)[0]
    b = fp32_spec.preprocess([sc2], [v2], cfg)[0]
    for k in ("valid", "depth_bits", "rect", "tiles_touched"):
        np.testing.assert_array_equal(a[k], b[k])
    assert int(a["tiles_touched"].sum()) > 100
    ia = R64.Oracle([sc], [v], cfg).render()["image"][0]
    ib = R64.Oracle([sc2], [v2], cfg).render()["image"][0]
    assert float((ia - ib).abs().max()) <= 1e-12
    assert float(ia.max()) > 0.1
