"""Pins of the float64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: values the
paper prints (tests/golden), closed forms, identities from linear algebra,
library routines for special cases, and brute force on tiny inputs.
"""
import math
import os

import numpy as np
import pytest
import torch

from oracle import fp32_spec
from oracle import render64 as R64
from paper_2510_03312_gb300 import scenes as S

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _rows(name):
    out = []
    for line in open(os.path.join(GOLD, name)):
        line = line.strip()
        if line and not line.startswith("#"):
            out.append([float(x) for x in line.split()])
    return out


def _view_at(R, t, W=64, H=48, f=60.0, time=0.0):
    return S.View(R=np.asarray(R, np.float32), t=np.asarray(t, np.float32), fx=f, fy=f,
                  cx=W / 2, cy=H / 2, width=W, height=H, time=time)


def _one_scene(N, rot_mode, cols):
    """Scene from explicit per-plane values; cols maps plane -> [rows, P]."""
    rows = S.plane_rows(N, rot_mode)
    P = np.asarray(cols["opacity"]).reshape(1, -1).shape[1]
    planes = []
    for k in S.PLANE_ORDER:
        a = np.asarray(cols.get(k, np.zeros((rows[k], P))), np.float64).reshape(rows[k], P)
        planes.append(a)
    return S.Scene(N, rot_mode, np.concatenate(planes, 0).astype(np.float32))


# ---------------------------------------------------------------- printed values

def test_beta_map_matches_printed_values():
    """Appendix, Property 1: beta(b) = 4 exp(b) at b = -5, 0, 5."""
    for b, printed, tol in _rows("beta_map.txt"):
        sc = _one_scene(3, S.ROT_QUAT, {"rot": [[1], [0], [0], [0]], "scale_x": [[.1]] * 3,
                                        "b": [[b]], "opacity": [[.5]]})
        lv = R64.scene_leaves(sc)
        _, _, _, beta_x = R64.condition(lv, 3, 0, _view_at(np.eye(3), [0, 0, 3]))
        assert abs(float(beta_x[0]) - printed) <= tol + 1e-12


def test_parameter_counts_match_table():
    """Per-primitive parameter table: 35 (UBS-6D) and 44 (UBS-7D) in the
    paper's skew-symmetric rotation mode; covariance N(N+1)/2."""
    for N, total, cov, nb in _rows("param_counts.txt"):
        N = int(N)
        rows = S.plane_rows(N, S.ROT_SKEW1)
        assert S.params_per_primitive(N, S.ROT_SKEW1) == total
        assert rows["rot"] + rows["scale_x"] + rows["L_qx"] + rows["L_q"] == cov == N * (N + 1) // 2
        assert rows["b"] == nb == N - 2


def test_storage_column_is_float32():
    """The storage column equals primitives x parameters x 4 bytes."""
    for n, k, mb in _rows("storage_mb.txt"):
        assert round(n * k * 4 / 2 ** 20, 1) == mb


# ---------------------------------------------------------------- Sec. 4.2

def test_quaternion_rotation_matches_scipy():
    from scipy.spatial.transform import Rotation
    rng = np.random.default_rng(0)
    q = rng.standard_normal((4, 50)) * rng.uniform(0.2, 3.0, 50)
    R = R64.rotation64(torch.tensor(q), 0).numpy()
    ref = Rotation.from_quat(np.stack([q[1], q[2], q[3], q[0]], 1)).as_matrix()
    np.testing.assert_allclose(R, ref, atol=1e-13)


def test_skew_rotation_determinant():
    """R = I + A(omega): det = 1 + |omega|^2 (so Sigma stays PSD) and the
    deviation from orthogonality is second order."""
    rng = np.random.default_rng(1)
    w = rng.normal(0, 0.3, (3, 40))
    R = R64.rotation64(torch.tensor(w), 1).numpy()
    np.testing.assert_allclose(np.linalg.det(R), 1 + (w * w).sum(0), rtol=1e-12)
    small = R64.rotation64(torch.tensor(w * 1e-4), 1).numpy()
    dev = np.abs(np.einsum("pji,pjk->pik", small, small) - np.eye(3)).max()
    assert dev < 1e-7


def test_cayley_rotation_is_the_rotation_by_twice_atan():
    """The Cayley transform of A(omega) is a proper rotation about omega by
    the angle 2 atan |omega| (the Gibbs-vector form), checked against SciPy's
    rotation-vector map."""
    from scipy.spatial.transform import Rotation
    rng = np.random.default_rng(3)
    w = rng.normal(0, 0.8, (3, 40))
    R = R64.rotation64(torch.tensor(w), S.ROT_CAYLEY).numpy()
    n = np.linalg.norm(w, axis=0)
    ref = Rotation.from_rotvec((w * (2 * np.arctan(n) / n)).T).as_matrix()
    np.testing.assert_allclose(R, ref, atol=1e-13)
    np.testing.assert_allclose(np.linalg.det(R), 1.0, atol=1e-13)


def test_second_order_taylor_rotation():
    """R = I + A + A^2/2: the matrix-product form, and within O(|omega|^3) of
    the matrix exponential (SciPy's expm)."""
    from scipy.linalg import expm
    rng = np.random.default_rng(4)
    w = rng.normal(0, 0.3, (3, 20))
    R = R64.rotation64(torch.tensor(w), S.ROT_SKEW2).numpy()
    for p in range(w.shape[1]):
        o1, o2, o3 = w[:, p]
        A = np.array([[0, -o3, o2], [o3, 0, -o1], [-o2, o1, 0]])
        np.testing.assert_allclose(R[p], np.eye(3) + A + A @ A / 2, atol=1e-15)
        assert np.abs(R[p] - expm(A)).max() <= np.linalg.norm(w[:, p]) ** 3 / 6 + 1e-15
        small = 1e-2 * A
        Rs = R64.rotation64(torch.tensor(1e-2 * w[:, p:p + 1]), S.ROT_SKEW2).numpy()[0]
        assert np.abs(Rs - expm(small)).max() <= 1e-6 * np.linalg.norm(w[:, p]) ** 3


def test_plain_cholesky_factor_is_recovered_by_cholesky():
    """The table's plain Cholesky row: Sigma_x = L L^T with L lower-triangular
    (diagonal s_x, strictly-lower rot), so NumPy's Cholesky factorisation of
    the oracle's Sigma_x returns those entries."""
    sc = S.make_scene(12, 3, 50, rot_mode=S.ROT_CHOL)
    leaves = R64.scene_leaves(sc)
    L = R64.build_L(leaves, 3, S.ROT_CHOL)
    Sx = (L @ L.transpose(-1, -2)).numpy()
    ch = np.linalg.cholesky(Sx)
    s, lo = sc.plane("scale_x").astype(np.float64), sc.plane("rot").astype(np.float64)
    np.testing.assert_allclose(ch[:, [0, 1, 2], [0, 1, 2]], s.T, rtol=1e-12)
    np.testing.assert_allclose(ch[:, [1, 2, 2], [0, 0, 1]], lo.T, rtol=1e-10, atol=1e-14)
    np.testing.assert_allclose(ch[:, [0, 0, 1], [1, 2, 2]], 0.0)


def test_exponential_rotation_matches_scipy_expm():
    """R = exp(A(omega)) against SciPy's expm, and a proper rotation."""
    from scipy.linalg import expm
    rng = np.random.default_rng(5)
    w = rng.normal(0, 1.0, (3, 30))
    R = R64.rotation64(torch.tensor(w), S.ROT_EXP).numpy()
    for p in range(w.shape[1]):
        o1, o2, o3 = w[:, p]
        A = np.array([[0, -o3, o2], [o3, 0, -o1], [-o2, o1, 0]])
        np.testing.assert_allclose(R[p], expm(A), atol=1e-13)
    np.testing.assert_allclose(np.einsum("pji,pjk->pik", R, R), np.broadcast_to(np.eye(3), R.shape), atol=1e-13)


def test_float32_sine_and_cosine():
    """The decision stage's binary32 sin and cos against float64 libm."""
    x = np.concatenate([np.linspace(0, 1, 20001), np.linspace(1, 200, 200001)]).astype(np.float32)
    s, c = fp32_spec.sincos_spec(x)
    xd = x.astype(np.float64)
    assert np.abs(s.astype(np.float64) - np.sin(xd)).max() < 2.5e-7
    assert np.abs(c.astype(np.float64) - np.cos(xd)).max() < 2.5e-7
    small = x[(x > 0) & (x < 0.5)]
    ss, _ = fp32_spec.sincos_spec(small)
    rel = np.abs(ss.astype(np.float64) / np.sin(small.astype(np.float64)) - 1)
    assert rel.max() < 3e-7


@pytest.mark.parametrize("mode", [S.ROT_SKEW1, S.ROT_SKEW2, S.ROT_CAYLEY, S.ROT_EXP])
def test_float32_rotation_closed_forms_match_float64(mode):
    """The decision stage's entry-by-entry float32 rotation against the
    float64 definitions (I + A, the product form, the linear solve)."""
    sc = S.make_scene(11, 3, 300, rot_mode=mode)
    r64 = R64.rotation64(torch.tensor(sc.plane("rot").astype(np.float64)), mode).numpy()
    r32 = np.array(fp32_spec.rotation(sc), dtype=np.float64).transpose(2, 0, 1)
    np.testing.assert_allclose(r32, r64, rtol=0, atol=4e-7)


@pytest.mark.parametrize("N,mode", [(6, 0), (7, 0), (6, 1), (7, 1), (4, 0), (6, 2), (7, 3), (6, 4), (7, 5)])
def test_sigma_blocks_match_appendix_closed_form(N, mode):
    """Sigma = L L^T has the block form printed in the appendix:
    [[R diag(s)^2 R^T, R diag(s) L_qx^T], [L_qx diag(s) R^T, L_qx L_qx^T + L_q L_q^T]],
    and is positive semi-definite."""
    sc = S.make_scene(5, N, 64, rot_mode=mode)
    lv = R64.scene_leaves(sc)
    terms = {}
    R64.condition(lv, N, mode, _view_at(np.eye(3), [0, 0, 3]), terms)
    Sig = terms["Sigma"].numpy()
    C = N - 3
    s = sc.plane("scale_x").T.astype(np.float64)
    lqx = sc.plane("L_qx").T.astype(np.float64).reshape(-1, C, 3)
    lq = np.zeros((sc.P, C, C))
    pk = sc.plane("L_q").astype(np.float64)
    for i in range(C):
        for j in range(i + 1):
            lq[:, i, j] = pk[i * (i + 1) // 2 + j]
    if mode == S.ROT_CHOL:  # the plain Cholesky row: the spatial block is the factor itself
        lo = sc.plane("rot").T.astype(np.float64)
        Rs = np.zeros((sc.P, 3, 3))
        Rs[:, [0, 1, 2], [0, 1, 2]] = s
        Rs[:, [1, 2, 2], [0, 0, 1]] = lo
        np.testing.assert_allclose(Sig[:, :3, :3], Rs @ Rs.transpose(0, 2, 1), atol=1e-14)
    else:
        R = R64.rotation64(lv["rot"], mode).numpy()
        Rs = R * s[:, None, :]
        np.testing.assert_allclose(Sig[:, :3, :3], np.einsum("pij,pj,pkj->pik", R, s * s, R), atol=1e-14)
    np.testing.assert_allclose(Sig[:, :3, 3:], Rs @ lqx.transpose(0, 2, 1), atol=1e-14)
    np.testing.assert_allclose(Sig[:, 3:, :3], lqx @ Rs.transpose(0, 2, 1), atol=1e-14)
    np.testing.assert_allclose(Sig[:, 3:, 3:], lqx @ lqx.transpose(0, 2, 1) + lq @ lq.transpose(0, 2, 1),
                               atol=1e-14)
    ev = np.linalg.eigvalsh(Sig)
    assert ev.min() > -1e-12 * np.abs(ev).max()


# ---------------------------------------------------------------- Sec. 4.3

@pytest.mark.parametrize("N", [6, 7])
def test_conditioning_at_unit_beta_is_gaussian_conditioning(N):
    """With beta~ = 1 (b_q >= 0) the Beta-modulated conditioning is the
    Gaussian conditioning quoted for 6DGS/7DGS (Sec. 3).  Checked against the
    precision-block form: Sigma_{x|q} = (Lambda_xx)^{-1},
    mu_{x|q} = mu_x - Lambda_xx^{-1} Lambda_xq (q - mu_q), Lambda = Sigma^{-1}."""
    sc = S.make_scene(7, N, 40)
    sc.plane("b")[1:] = np.abs(sc.plane("b")[1:]) + 0.05
    lv = R64.scene_leaves(sc)
    v = _view_at(np.eye(3), [0.1, -0.2, 3.0], time=0.3)
    terms = {}
    mu_c, Sc, _, _ = R64.condition(lv, N, 0, v, terms)
    Sig = terms["Sigma"].numpy()
    Lam = np.linalg.inv(Sig)
    Lxx_inv = np.linalg.inv(Lam[:, :3, :3])
    np.testing.assert_allclose(Sc.numpy(), Lxx_inv, rtol=1e-9, atol=1e-14)
    delta = terms["delta"].numpy()
    mu_ref = sc.plane("mean_x").T - np.einsum("pij,pjk,pk->pi", Lxx_inv, Lam[:, :3, 3:], delta)
    np.testing.assert_allclose(mu_c.numpy(), mu_ref, rtol=1e-9, atol=1e-12)


@pytest.mark.parametrize("N", [6, 7])
def test_zero_cross_block_leaves_spatial_kernel_unchanged(N):
    sc = S.make_scene(8, N, 30)
    sc.plane("L_qx")[:] = 0
    lv = R64.scene_leaves(sc)
    mu_c, Sc, _, _ = R64.condition(lv, N, 0, _view_at(np.eye(3), [0, 0, 3], time=0.7))
    terms = {}
    R64.condition(lv, N, 0, _view_at(np.eye(3), [0, 0, 3]), terms)
    np.testing.assert_array_equal(mu_c.numpy(), sc.plane("mean_x").T.astype(np.float64))
    np.testing.assert_allclose(Sc.numpy(), terms["Sigma"].numpy()[:, :3, :3], atol=0)


@pytest.mark.parametrize("N", [6, 7])
def test_opacity_distances_sum_to_mahalanobis(N):
    """L^_q is the Cholesky factor of Sigma_q, so sum_i d_i^raw equals the
    Mahalanobis distance (q - mu_q)^T Sigma_q^{-1} (q - mu_q)."""
    sc = S.make_scene(9, N, 50)
    lv = R64.scene_leaves(sc)
    terms = {}
    R64.condition(lv, N, 0, _view_at(np.eye(3), [0.3, 0.1, 4.0], time=0.2), terms)
    Sq = terms["Sigma"].numpy()[:, 3:, 3:]
    dl = terms["delta"].numpy()
    maha = np.einsum("pi,pij,pj->p", dl, np.linalg.inv(Sq), dl)
    np.testing.assert_allclose(terms["d_raw"].numpy().sum(1), maha, rtol=1e-10)
    Lh = terms["Lh"].numpy()
    np.testing.assert_allclose(Lh @ Lh.transpose(0, 2, 1), Sq, rtol=1e-12, atol=1e-14)
    assert np.allclose(np.triu(Lh, 1), 0)


@pytest.mark.parametrize("N", [6, 7])
def test_opacity_special_cases(N):
    """q = mu_q gives o(q) = o; beta_q -> 0 gives o(q) -> o; for small
    distances o(q) = o exp(-4 sum beta_qi d_i^raw) to first order."""
    sc = S.make_scene(10, N, 20)
    v = _view_at(np.eye(3), [0, 0, 3], time=0.4)
    lv = R64.scene_leaves(sc)
    terms = {}
    R64.condition(lv, N, 0, v, terms)
    q = terms["q"].numpy()
    sc2 = S.Scene(N, 0, sc.params.copy())
    sc2.plane("mean_q")[:] = q.T.astype(np.float32)
    lv2 = R64.scene_leaves(sc2)
    t2 = {}
    _, _, oq, _ = R64.condition(lv2, N, 0, v, t2)
    # mean_q rounded to float32: distances are ~1e-8, so o(q) = o to ~1e-14
    np.testing.assert_allclose(oq.numpy(), sc.plane("opacity")[0], rtol=1e-9)
    sc3 = S.Scene(N, 0, sc.params.copy())
    sc3.plane("b")[1:] = -60.0
    _, _, oq3, _ = R64.condition(R64.scene_leaves(sc3), N, 0, v)
    np.testing.assert_allclose(oq3.numpy(), sc.plane("opacity")[0], rtol=1e-20, atol=1e-12)
    # first order: push mu_q to within a small distance of q
    sc4 = S.Scene(N, 0, sc.params.copy())
    sc4.plane("mean_q")[:] = (q.T + 1e-3 * sc.plane("L_q")[[i * (i + 1) // 2 + i for i in range(N - 3)]]
                              ).astype(np.float32)
    t4 = {}
    _, _, oq4, _ = R64.condition(R64.scene_leaves(sc4), N, 0, v, t4)
    approx = sc.plane("opacity")[0] * np.exp(-4 * (t4["beta_q"].numpy() * t4["d_raw"].numpy()).sum(1))
    np.testing.assert_allclose(oq4.numpy(), approx, rtol=1e-9)


@pytest.mark.parametrize("N", [6, 7])
def test_static_reduction_renders_like_n3(N):
    """N=6/7 with L_qx = 0 and beta_q -> 0 (b_q = -60) renders the N=3 image
    (backward compatibility, Sec. 4.4)."""
    wl = S.workload_static_small(P=300, size=48)
    s3 = wl.scenes[0]
    sN = S.make_scene(11, N, s3.P)
    for k in ("mean_x", "rot", "scale_x", "opacity", "rgb"):
        sN.plane(k)[:] = s3.plane(k)
    sN.plane("b")[0] = s3.plane("b")[0]
    sN.plane("b")[1:] = -60.0
    sN.plane("L_qx")[:] = 0
    v = wl.views[0]
    v = S.View(v.R, v.t, v.fx, v.fy, v.cx, v.cy, v.width, v.height, time=0.5)
    a = R64.Oracle([s3], [v], wl.cfg).render()["image"][0].numpy()
    b = R64.Oracle([sN], [v], wl.cfg).render()["image"][0].numpy()
    assert np.abs(a - b).max() <= 1e-12


# ---------------------------------------------------------------- Sec. 3

def _iso_scene(s, o, b, rgb=(1.0, 0.5, 0.25), pos=(0.0, 0.0, 0.0)):
    return _one_scene(3, S.ROT_QUAT, {"mean_x": [[pos[0]], [pos[1]], [pos[2]]], "rot": [[1], [0], [0], [0]],
                                      "scale_x": [[s]] * 3, "b": [[b]], "opacity": [[o]],
                                      "rgb": [[rgb[0]], [rgb[1]], [rgb[2]]]})


def test_single_primitive_closed_form_footprint():
    """Isotropic primitive on the optical axis at depth z: Sigma' = (f s/z)^2 I
    + eps I, mu' = (cx, cy); alpha(p) = min(a_max, o (1 - |p-mu'|^2/rho^2)^beta)
    inside the support, C = c alpha per pixel (single primitive)."""
    W, H, f, z, s, o, b = 64, 48, 60.0, 3.0, 0.1, 0.8, 0.2
    sc = _iso_scene(s, o, b)
    v = _view_at(np.eye(3), [0, 0, z], W, H, f)
    cfg = S.RasterConfig()
    orc = R64.Oracle([sc], [v], cfg)
    rec = orc.records(orc.leaves())[0]
    s32 = float(np.float32(s))
    rho2 = (f * s32 / z) ** 2 + float(np.float32(cfg.eps2d))
    np.testing.assert_allclose(rec["cov2d"][0].numpy(), rho2 * np.eye(2), rtol=1e-12)
    np.testing.assert_allclose(rec["mean2d"][0].numpy(), [W / 2, H / 2], atol=1e-12)
    beta = 4 * math.exp(float(np.float32(b)))
    out = orc.render()
    img = out["image"][0].numpy()
    o32 = float(np.float32(o))
    amin = float(np.float32(cfg.alpha_min))
    for (x, y) in [(32, 24), (33, 24), (35, 26), (29, 21), (38, 24), (32, 30), (40, 24)]:
        d2 = (x + 0.5 - W / 2) ** 2 + (y + 0.5 - H / 2) ** 2
        r = d2 / rho2
        a = min(cfg.alpha_max, o32 * (1 - r) ** beta) if r < 1 else 0.0
        a = a if a >= amin else 0.0
        np.testing.assert_allclose(img[:, y, x], a * np.array([1.0, 0.5, 0.25]), atol=1e-12)
    # the tile rectangle: tight radius rho^2 r_cut with r_cut = 1 - (a_min/o)^(1/beta)
    rcut = 1 - (amin / o32) ** (1 / beta)
    ext = math.sqrt(rcut * rho2)
    x0 = math.ceil(W / 2 - ext - 0.5) // 16
    x1 = math.floor(W / 2 + ext - 0.5) // 16 + 1
    y0 = math.ceil(H / 2 - ext - 0.5) // 16
    y1 = math.floor(H / 2 + ext - 0.5) // 16 + 1
    assert list(orc.pre32[0]["rect"][:, 0]) == [x0, y0, x1, y1]


def test_area_integral_of_beta_footprint():
    """sum over pixels of (1 - r)^beta o approximates the exact integral
    o pi sqrt(det Sigma') / (beta + 1) for a large footprint."""
    for b in (-0.7, 0.0, 0.9):
        sc = _iso_scene(0.5, 0.6, b)
        sc.plane("scale_x")[1] = 0.3
        sc.plane("rot")[:, 0] = [0.9, 0.1, 0.3, 0.2]
        v = _view_at(np.eye(3), [0, 0, 3], 256, 256, 120.0)
        cfg = S.RasterConfig(alpha_min=0.0, alpha_max=1.0, T_min=0.0, tight_cut=False)
        orc = R64.Oracle([sc], [v], cfg)
        img = orc.render()["image"][0].numpy()
        rec = orc.records(orc.leaves())[0]
        beta = 4 * math.exp(float(np.float32(b)))
        total = img[0].sum()
        exact = float(np.float32(0.6)) * math.pi * math.sqrt(np.linalg.det(rec["cov2d"][0].numpy())) / (beta + 1)
        assert abs(total / exact - 1) < 5e-3


def test_two_primitives_by_hand():
    """Front-to-back compositing of two overlapping primitives at one pixel:
    C = c1 a1 + c2 a2 (1 - a1), T = (1 - a1)(1 - a2)."""
    sc1 = _iso_scene(0.2, 0.7, 0.0, rgb=(1, 0, 0), pos=(0.0, 0.0, 0.0))
    sc2 = _iso_scene(0.3, 0.5, 0.3, rgb=(0, 1, 0), pos=(0.05, 0.0, 1.0))
    sc = S.Scene(3, 0, np.concatenate([sc1.params, sc2.params], 1))
    W, H, f = 32, 32, 40.0
    v = _view_at(np.eye(3), [0, 0, 3], W, H, f)
    cfg = S.RasterConfig()
    orc = R64.Oracle([sc], [v], cfg)
    out = orc.render()
    x, y = 17, 15
    col = np.zeros(3)
    T = 1.0
    for p, z in ((0, 3.0), (1, 4.0)):
        s = float(np.float32([0.2, 0.3][p]))
        o = float(np.float32([0.7, 0.5][p]))
        beta = 4 * math.exp(float(np.float32([0.0, 0.3][p])))
        u = float(np.float32([0.0, 0.05][p])) / z
        mx = W / 2 + f * u
        # J J^T s^2 + eps I with J = [[f/z, 0, -f u/z], [0, f/z, 0]] (v = 0)
        eps = float(np.float32(0.3))
        s00 = (f * s / z) ** 2 * (1 + u * u) + eps
        s11 = (f * s / z) ** 2 + eps
        r = (x + 0.5 - mx) ** 2 / s00 + (y + 0.5 - H / 2) ** 2 / s11
        a = min(0.99, o * (1 - r) ** beta)
        col += T * a * np.array([[1, 0, 0], [0, 1, 0]][p])
        T *= 1 - a
    np.testing.assert_allclose(out["image"][0].numpy()[:, y, x], col, atol=1e-12)
    np.testing.assert_allclose(out["T"][0].numpy()[y, x], T, atol=1e-12)
    assert int(out["last"][0][y, x]) == 2


def test_compositing_invariants_and_brute_force():
    """Tiled == tile-free brute force; T in (T_min (1 - a_max), 1]; weights
    plus final T sum to one; invariance to the order primitives are listed."""
    wl = S.workload_static_small(seed=3, P=500, size=64)
    cfg = wl.cfg
    orc = R64.Oracle(wl.scenes, wl.views, cfg)
    tiled = orc.render()
    free = orc.render(tile_free=True)
    assert torch.equal(tiled["last"][0] >= 0, torch.ones_like(tiled["last"][0], dtype=torch.bool))
    assert (tiled["image"][0] - free["image"][0]).abs().max() <= 1e-13
    assert (tiled["T"][0] - free["T"][0]).abs().max() <= 1e-13
    T = tiled["T"][0].numpy()
    assert (T <= 1).all() and (T > cfg.T_min * (1 - cfg.alpha_max)).all()
    # weights sum: render white primitives on a black background: C = 1 - T
    sw = S.Scene(3, 0, wl.scenes[0].params.copy())
    sw.plane("rgb")[:] = 1.0
    w = R64.Oracle([sw], wl.views, cfg).render()
    np.testing.assert_allclose(w["image"][0].numpy()[0], 1 - w["T"][0].numpy(), atol=1e-12)
    # permutation of the primitive order
    perm = np.random.default_rng(0).permutation(wl.scenes[0].P)
    sp = wl.scenes[0].subset(perm)
    pimg = R64.Oracle([sp], wl.views, cfg).render()["image"][0]
    assert (pimg - tiled["image"][0]).abs().max() <= 1e-12


def test_transmittance_is_non_increasing_along_the_list():
    wl = S.workload_static_small(seed=4, P=400, size=48)
    orc = R64.Oracle(wl.scenes, wl.views, wl.cfg)
    rec = orc.records(orc.leaves())[0]
    s, e = orc.bins["ranges"][5]
    lst = torch.from_numpy(orc.bins["record"][s:e])
    px = torch.tensor([5 * 16 % 48 + 3.5], dtype=torch.float64)
    py = torch.tensor([(5 * 16 // 48) * 16 + 7.5], dtype=torch.float64)
    # per-prefix transmittance from the compositing of growing prefixes
    Ts = []
    for k in range(len(lst) + 1):
        _, T, _, _ = R64._composite_block(px, py, rec["mean2d"][lst[:k]], rec["conic"][lst[:k]],
                                          rec["opacity"][lst[:k]], rec["beta_x"][lst[:k]],
                                          rec["rgb"][lst[:k]], wl.cfg)
        Ts.append(float(T[0]))
    assert all(a >= b for a, b in zip(Ts, Ts[1:]))


# ---------------------------------------------------------------- Gaussian limit

def test_gaussian_approximation_at_b_zero():
    """Appendix Property 3 (read as (1 - r)^4 ~ exp(-4.5 r), r the squared
    normalised distance): the printed approximation holds within 0.0433."""
    r = np.linspace(0, 1, 200001)[:-1]
    gap = np.abs((1 - r) ** 4 - np.exp(-4.5 * r)).max()
    assert gap <= 0.0433


def _gauss_render(sc, v):
    """3DGS density exp(-r/2) o, brute force per pixel (Sec. 3), no thresholds."""
    lv = R64.scene_leaves(sc)
    mu_c, Sc, oq, _ = R64.condition(lv, 3, 0, v)
    cfg = S.RasterConfig(eps2d=0.0)
    tz, mu2, cov2, conic = R64.project(mu_c, Sc, v, cfg)
    order = np.argsort(tz.numpy())
    img = np.zeros((3, v.height, v.width))
    ys, xs = np.mgrid[0:v.height, 0:v.width]
    T = np.ones((v.height, v.width))
    for p in order:
        dx = xs + 0.5 - float(mu2[p, 0])
        dy = ys + 0.5 - float(mu2[p, 1])
        cn = conic[p].numpy()
        r = cn[0, 0] * dx * dx + 2 * cn[0, 1] * dx * dy + cn[1, 1] * dy * dy
        a = float(oq[p]) * np.exp(-0.5 * r)
        img += T * a * lv["rgb"][:, p].detach().numpy()[:, None, None]
        T = T * (1 - a)
    return img


def test_beta_kernel_converges_to_gaussian():
    """(1 - r/(2 beta))^beta -> exp(-r/2): a Beta primitive with covariance
    2 beta Sigma_G renders the 3DGS image of Sigma_G, error O(1/beta)."""
    base = S.make_scene(12, 3, 6, means="uniform", extent=0.4, scale_range=(0.05, 0.12))
    v = _view_at(np.eye(3), [0, 0, 3], 40, 40, 50.0)
    ref = _gauss_render(base, v)
    errs = []
    for b in (2.0, 4.0, 6.0):
        beta = 4 * math.exp(b)
        sc = S.Scene(3, 0, base.params.copy())
        sc.plane("scale_x")[:] = (base.plane("scale_x").astype(np.float64) * math.sqrt(2 * beta)).astype(np.float32)
        sc.plane("b")[:] = b
        cfg = S.RasterConfig(alpha_min=0.0, alpha_max=1.0, T_min=0.0, eps2d=0.0, tight_cut=False)
        img = R64.Oracle([sc], [v], cfg).render()["image"][0].numpy()
        errs.append(np.abs(img - ref).max())
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 2e-3
    # O(1/beta): each step multiplies beta by e^2
    assert errs[1] / errs[0] < 0.3 and errs[2] / errs[1] < 0.3


def test_admissible_branches():
    """The branch enumeration equals the vectorised loop on an unambiguous
    pixel and yields both results when alpha sits on alpha_min."""
    cfg = S.RasterConfig()
    amin = float(np.float32(cfg.alpha_min))
    r = np.array([0.1, 0.3, 0.5])
    beta = np.array([4.0, 4.0, 4.0])
    rgb = np.array([[1.0, 0, 0], [0, 1.0, 0], [0, 0, 1.0]])
    oq = np.array([0.6, 0.5, 0.9])
    alpha = np.minimum(cfg.alpha_max, oq * (1 - r) ** beta)
    res = R64.composite_branches(r, alpha, beta, oq, rgb, cfg)
    assert len(res) == 1
    T = 1.0
    col = np.zeros(3)
    for k in range(3):
        col += rgb[k] * alpha[k] * T
        T *= 1 - alpha[k]
    np.testing.assert_allclose(res[0][0], col, atol=1e-15)
    assert res[0][2] == 3
    alpha2 = alpha.copy()
    alpha2[1] = amin
    res2 = R64.composite_branches(r, alpha2, beta, oq, rgb, cfg)
    assert len(res2) == 2
    assert sorted(x[2] for x in res2) == [3, 3]
    greens = sorted(x[0][1] for x in res2)
    assert greens[0] == 0.0 and greens[1] > 0
