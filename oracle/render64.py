"""Float64 reference rasterizer of Universal Beta Splatting (test infrastructure only).

Plain PyTorch CPU float64 operations, written to be read against the paper:

* Sec. 4.2, spatial-orthogonal Cholesky parameterisation:
  L = [[R_x diag(s_x), 0], [L_qx, L_q]], Sigma = L L^T, with R_x the 3DGS
  quaternion rotation (Sec. 3) or R_x from the skew matrix A(omega) (appendix
  on the spatial-orthogonal Cholesky parameterisation): I + A (first-order
  Taylor, the paper's choice), I + A + A^2/2 (second order) or the Cayley
  transform (I - A)^{-1}(I + A).
* Sec. 4.3, Beta-modulated conditional slicing:
  beta_x = 4 exp(b_x), beta_q = exp(b_q), beta~ = [beta_q]_{<=1};
  mu_{x|q} = mu_x + Sigma_xq Sigma_q^{-1} diag(beta~) (q - mu_q);
  Sigma_{x|q} = Sigma_x - Sigma_xq Sigma_q^{-1} diag(beta~) Sigma_qx,
  symmetrised (the product is not symmetric when diag(beta~) does not commute
  with Sigma_q; the symmetric part is used);
  d_i = tanh(((L^_q^{-1} (q - mu_q))_i)^2) with L^_q = chol(Sigma_q),
  o(q) = o prod_i (1 - d_i)^(4 beta_q_i).
* Sec. 4.4, query specialisation: q = d (N=6), q = [t, d] (N=7), q = [t]
  (N=4), with d the unit direction from the camera centre to mu_x.
* Sec. 3, EWA projection mu' = pi(W mu), Sigma' = J W Sigma W^T J^T (+ eps I),
  Mahalanobis r (Eq. r), DBS Beta kernel (1 - r)^beta on r in [0, 1), density
  sigma = B o, and front-to-back alpha compositing
  C = sum_i c_i sigma_i prod_{j<i} (1 - sigma_j).

The discrete decisions that select and order the blended primitives (culling,
tile rectangles, depth order) come from the float32 decision stage
(``fp32_spec``) and the plain-definition sort (``binning``), as the
rasterizer takes them in float32; everything else here is float64.  The
per-pixel skip (alpha < alpha_min) and stop (T < T_min) rules are evaluated
in float64; where float32 evaluation could legitimately take the other branch
(the float64 value lies inside the float32 error band of the threshold) the
pixel is flagged and every admissible branch is enumerated.

Gradients are the autograd gradients of this float64 forward.

Parity: pinned (tests/test_oracle_*.py): the quaternion, Cayley and
second-order rotations against SciPy (rotation map, rotation vector, expm),
closed-form footprints, brute-force
depth-sorted compositing, transmittance invariants, the static reduction of
N=6/7 to N=3, Gaussian conditioning at beta~ = 1 against the precision-block
identity, the Beta-modulated conditioning at 0 < beta~ < 1 (scalar-query
closed forms, per-dimension sums where Sigma_q is diagonal, the regression
matrix from the precision blocks, the vanishing-beta limits), invariance of
the image under a rigid motion of scene and camera, the view direction of a
camera placed at a known centre, the Gaussian limit of the Beta kernel, the
paper's printed beta values, and central finite differences for the
gradients.
"""
from __future__ import annotations

import math

import numpy as np
import torch

from . import binning, fp32_spec

D = torch.float64


def scene_leaves(scene, requires_grad=False):
    """Float64 leaf tensors, one per plane block, shape [rows, P]."""
    out = {}
    for name, (o, n) in scene.offsets().items():
        t = torch.tensor(scene.params[o:o + n].astype(np.float64), dtype=D)
        t.requires_grad_(requires_grad)
        out[name] = t
    return out


def skew64(rot):
    """[P, 3, 3] skew matrix A(omega) = [[0,-w3,w2],[w3,0,-w1],[-w2,w1,0]]."""
    w1, w2, w3 = rot[0], rot[1], rot[2]
    zero = torch.zeros_like(w1)
    rows = [torch.stack([zero, -w3, w2], -1), torch.stack([w3, zero, -w1], -1),
            torch.stack([-w2, w1, zero], -1)]
    return torch.stack(rows, -2)


def rotation64(rot, rot_mode):
    """[P, 3, 3] rotation R_x.  Quaternion (w, x, y, z) normalised, 3DGS
    formula (Sec. 3); the skew-symmetric forms of the appendix on the
    spatial-orthogonal Cholesky parameterisation (its table of rotation
    parameterisations): R = I + A (first-order Taylor of exp A, the paper's
    choice), R = I + A + A^2/2 (second-order Taylor), the Cayley transform
    R = (I - A)^{-1} (I + A) and R = exp(A), each written as its definition."""
    if rot_mode == 0:
        q = rot / torch.sqrt((rot * rot).sum(0, keepdim=True))
        w, x, y, z = q[0], q[1], q[2], q[3]
        rows = [
            torch.stack([1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)], -1),
            torch.stack([2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)], -1),
            torch.stack([2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)], -1),
        ]
        return torch.stack(rows, -2)
    A = skew64(rot)
    eye = torch.eye(3, dtype=A.dtype).expand_as(A)
    if rot_mode == 1:
        return eye + A
    if rot_mode == 2:
        return eye + A + 0.5 * (A @ A)
    if rot_mode == 3:
        return torch.linalg.solve(eye - A, eye + A)
    if rot_mode == 5:
        return torch.linalg.matrix_exp(A)
    raise ValueError(f"rotation mode {rot_mode}")


def spatial_factor64(leaves, rot_mode):
    """[P, 3, 3] spatial block of L: R_x diag(s_x) (Sec. 4.2), or, for the
    appendix's plain Cholesky row (rot_mode 4), the lower-triangular factor
    with diagonal s_x and strictly-lower entries (l10, l20, l21) = rot."""
    s = leaves["scale_x"].T                       # [P, 3]
    if rot_mode == 4:
        l10, l20, l21 = leaves["rot"][0], leaves["rot"][1], leaves["rot"][2]
        zero = torch.zeros_like(l10)
        rows = [torch.stack([s[:, 0], zero, zero], -1), torch.stack([l10, s[:, 1], zero], -1),
                torch.stack([l20, l21, s[:, 2]], -1)]
        return torch.stack(rows, -2)
    R = rotation64(leaves["rot"], rot_mode)
    return R * s[:, None, :]                     # R diag(s)


def build_L(leaves, N, rot_mode):
    """[P, N, N] spatial-orthogonal Cholesky factor (Sec. 4.2)."""
    top_left = spatial_factor64(leaves, rot_mode)
    s = leaves["scale_x"].T
    C = N - 3
    P = s.shape[0]
    if C == 0:
        return top_left
    lqx = leaves["L_qx"].T.reshape(P, C, 3)
    rows = []
    packed = leaves["L_q"]
    for i in range(C):
        row = []
        for j in range(C):
            row.append(packed[i * (i + 1) // 2 + j] if j <= i else torch.zeros_like(packed[0]))
        rows.append(torch.stack(row, -1))
    lq = torch.stack(rows, -2)                   # [P, C, C] lower triangular
    zeros = torch.zeros(P, 3, C, dtype=D)
    top = torch.cat([top_left, zeros], -1)
    bottom = torch.cat([lqx, lq], -1)
    return torch.cat([top, bottom], -2)


def camera_centre(view):
    R = torch.tensor(np.asarray(view.R, np.float64), dtype=D)
    t = torch.tensor(np.asarray(view.t, np.float64), dtype=D)
    return -(R.T @ t)


def query(leaves, N, view):
    """[P, C] query q of Sec. 4.4: [t, d] order, d = (mu_x - c)/|mu_x - c|."""
    C = N - 3
    P = leaves["mean_x"].shape[1]
    parts = []
    if C in (1, 4):
        parts.append(torch.full((P, 1), float(view.time), dtype=D))
    if C >= 3:
        v = leaves["mean_x"].T - camera_centre(view)[None, :]
        parts.append(v / torch.sqrt((v * v).sum(-1, keepdim=True)))
    return torch.cat(parts, -1)


def condition(leaves, N, rot_mode, view, terms=None):
    """Sec. 4.3: conditioned 3-D mean [P,3], covariance [P,3,3], opacity [P],
    and beta_x [P].  If ``terms`` is a dict, intermediate quantities (Sigma,
    q, delta, y, d_raw, d) are stored in it."""
    L = build_L(leaves, N, rot_mode)
    Sigma = L @ L.transpose(-1, -2)
    mu_x = leaves["mean_x"].T
    o = leaves["opacity"][0]
    beta_x = 4.0 * torch.exp(leaves["b"][0])
    C = N - 3
    if terms is not None:
        terms["Sigma"] = Sigma
    if C == 0:
        return mu_x, Sigma, o, beta_x
    Sx, Sxq = Sigma[:, :3, :3], Sigma[:, :3, 3:]
    Sqx, Sq = Sigma[:, 3:, :3], Sigma[:, 3:, 3:]
    beta_q = torch.exp(leaves["b"][1:]).T        # [P, C]
    beta_t = torch.clamp(beta_q, max=1.0)
    K = Sxq @ torch.linalg.inv(Sq) @ torch.diag_embed(beta_t)
    q = query(leaves, N, view)
    delta = q - leaves["mean_q"].T
    mu_c = mu_x + (K @ delta[..., None])[..., 0]
    Sc = Sx - K @ Sqx
    Sc = 0.5 * (Sc + Sc.transpose(-1, -2))
    Lh = torch.linalg.cholesky(Sq)
    y = torch.linalg.solve_triangular(Lh, delta[..., None], upper=False)[..., 0]
    d_raw = y * y
    d = torch.tanh(d_raw)
    # (1 - d_i)^(4 beta_q_i) = exp(4 beta_q_i log(1 - tanh d_raw_i)), with the
    # exact identity log(1 - tanh x) = ln 2 - 2x - log1p(exp(-2x)) (x >= 0),
    # which stays accurate where tanh has rounded to 1 in float64
    log_1md = math.log(2.0) - 2.0 * d_raw - torch.log1p(torch.exp(-2.0 * d_raw))
    oq = o * torch.exp((4.0 * beta_q * log_1md).sum(-1))
    if terms is not None:
        terms.update(Sigma=Sigma, q=q, delta=delta, y=y, d_raw=d_raw, d=d, beta_q=beta_q,
                     beta_t=beta_t, Lh=Lh)
    return mu_c, Sc, oq, beta_x


def project(mu_c, Sc, view, cfg):
    """Sec. 3: camera-space mean, screen mean mu', Sigma' = J W Sigma W^T J^T
    + eps I (the Jacobian evaluated at the clamped screen ray), and conic."""
    Rv = torch.tensor(np.asarray(view.R, np.float64), dtype=D)
    tv = torch.tensor(np.asarray(view.t, np.float64), dtype=D)
    t = mu_c @ Rv.T + tv
    tx, ty, tz = t[:, 0], t[:, 1], t[:, 2]
    fx, fy, cx, cy = float(view.fx), float(view.fy), float(view.cx), float(view.cy)
    u, v = tx / tz, ty / tz
    mu2 = torch.stack([fx * u + cx, fy * v + cy], -1)
    clip = float(np.float32(cfg.jac_clip))
    limx = clip * (0.5 * view.width / fx)
    limy = clip * (0.5 * view.height / fy)
    uc = torch.clamp(u, -limx, limx)
    vc = torch.clamp(v, -limy, limy)
    zero = torch.zeros_like(tz)
    J = torch.stack([torch.stack([fx / tz, zero, -fx * uc / tz], -1),
                     torch.stack([zero, fy / tz, -fy * vc / tz], -1)], -2)
    T = J @ Rv
    eps = float(np.float32(cfg.eps2d))
    cov2 = T @ Sc @ T.transpose(-1, -2) + eps * torch.eye(2, dtype=D)
    conic = torch.linalg.inv(cov2)
    return tz, mu2, cov2, conic


# ----------------------------------------------------------------------------
# compositing
# ----------------------------------------------------------------------------

def alpha_band(r, beta):
    """Relative width of the float32 error band around alpha = alpha_min for
    a pair at Mahalanobis r with exponent beta (conic, opacity and MUFU
    errors of the GPU evaluation, with a safety factor of 4)."""
    return 8e-5 + beta * (1.2e-5 * r + 1.2e-6) / np.maximum(1.0 - r, 1e-12)


T_BAND = 1e-4
R_BAND = 4e-6   # |r - 1| within which float32 may decide r < 1 either way


def _composite_block(px, py, mu2, conic, oq, beta, rgb, cfg, extra=None):
    """Vectorised compositing of M pixels over one front-to-back list of K
    records (tensors gathered in list order).  Returns colour [M,3], final T
    [M], last-contributor count [M] and a per-pixel ambiguity flag.  With a
    dict ``extra``, also the pair count of each pixel, the number of list
    entries with r < 1 visited before the pixel terminates (the stopping
    entry included), as the interval [pairs_lo, pairs_hi] that float32
    evaluation of r admits: r < 1 is decided on the float32 conic
    (``extra["count_conic"]``, [K, 3] a, b, c, when given) and is ambiguous
    within R_BAND plus 1e-6 of the magnitude of r's three terms (the float32
    rounding of terms that cancel)."""
    M, K = px.shape[0], mu2.shape[0]
    bg = torch.tensor(cfg.bg, dtype=D)
    if K == 0:
        if extra is not None:
            extra["pairs_lo"] = torch.zeros(M, dtype=torch.long)
            extra["pairs_hi"] = torch.zeros(M, dtype=torch.long)
        return (bg.expand(M, 3).clone(), torch.ones(M, dtype=D),
                torch.zeros(M, dtype=torch.long), torch.zeros(M, dtype=torch.bool))
    dx = px[:, None] - mu2[None, :, 0]
    dy = py[:, None] - mu2[None, :, 1]
    a, b, c = conic[None, :, 0, 0], conic[None, :, 0, 1], conic[None, :, 1, 1]
    r = a * dx * dx + 2.0 * b * dx * dy + c * dy * dy
    inside = r < 1.0
    base = torch.where(inside, 1.0 - r, torch.ones_like(r))
    kern = torch.where(inside, base ** beta[None, :], torch.zeros_like(r))
    alpha = torch.clamp(oq[None, :] * kern, max=cfg.alpha_max)
    amin = float(np.float32(cfg.alpha_min))
    tmin = float(np.float32(cfg.T_min))
    with torch.no_grad():
        used = inside & (alpha >= amin)
    om = torch.where(used, 1.0 - alpha, torch.ones_like(alpha))
    Tc = torch.cumprod(om, dim=1)
    Tb = torch.cat([torch.ones(M, 1, dtype=D), Tc[:, :-1]], 1)
    with torch.no_grad():
        stop = used & (Tb * (1.0 - alpha) < tmin)
        has = stop.any(1)
        first = torch.where(has, stop.float().argmax(1), torch.full((M,), K, dtype=torch.long))
        ar = torch.arange(K)[None, :]
        incl = used & (ar < first[:, None])
        last = torch.where(incl.any(1), (incl * (ar + 1)).max(1).values, torch.zeros(M, dtype=torch.long))
        # ambiguity flags
        rn, an, bn = r.detach().numpy(), alpha.detach().numpy(), beta.detach().numpy()[None, :]
        band = alpha_band(np.clip(rn, 0, 1), bn)
        fa = inside.numpy() & (np.abs(an - amin) <= band * amin)
        fr = (np.abs(rn - 1.0) <= 4e-6) & (oq.detach().numpy()[None, :] * (4e-6 ** bn) >= amin * 0.5)
        Tp = (Tb * (1.0 - alpha)).detach().numpy()
        reach = (ar <= first[:, None]).numpy()
        ft = used.numpy() & reach & (np.abs(Tp - tmin) <= T_BAND * tmin)
        flag = torch.from_numpy((fa | fr | ft).any(1))
        if extra is not None:
            dxd, dyd = dx.detach(), dy.detach()
            cc = extra.get("count_conic")
            if cc is None:
                ca, cb, ccc = a.detach(), b.detach(), c.detach()
            else:
                ca, cb, ccc = cc[None, :, 0], cc[None, :, 1], cc[None, :, 2]
            rc = ca * dxd * dxd + 2.0 * cb * dxd * dyd + ccc * dyd * dyd
            mag = (ca * dxd * dxd).abs() + (2.0 * cb * dxd * dyd).abs() + (ccc * dyd * dyd).abs()
            band = R_BAND + 1e-6 * mag
            vis = ar <= first[:, None]
            extra["pairs_lo"] = ((rc < 1.0 - band) & vis).sum(1)
            extra["pairs_hi"] = ((rc < 1.0 + band) & vis).sum(1)
    w = torch.where(incl, alpha * Tb, torch.zeros_like(alpha))
    Text = torch.cat([Tb, Tc[:, -1:]], 1)
    Tfin = torch.gather(Text, 1, first[:, None])[:, 0]
    color = w @ rgb + Tfin[:, None] * bg[None, :]
    return color, Tfin, last, flag


def composite_branches(r, alpha, beta, oq, rgb, cfg, max_results=64):
    """All admissible results (colour, T, last) of one pixel: the scalar
    front-to-back loop of Sec. 3 with the skip/stop rules, branching at every
    decision whose float64 margin lies inside the float32 error band."""
    amin = float(np.float32(cfg.alpha_min))
    tmin = float(np.float32(cfg.T_min))
    bg = np.asarray(cfg.bg, np.float64)
    K = len(r)
    out = []
    stack = [(0, 1.0, np.zeros(3), 0)]
    while stack:
        k, T, C, last = stack.pop()
        while k < K:
            rk, ak = r[k], alpha[k]
            inside = rk < 1.0
            amb_r = abs(rk - 1.0) <= 4e-6 and oq[k] * (4e-6 ** beta[k]) >= amin * 0.5
            if not inside and not amb_r:
                k += 1
                continue
            amb_a = abs(ak - amin) <= alpha_band(min(max(rk, 0.0), 1.0), beta[k]) * amin
            use = inside and ak >= amin
            if amb_a or amb_r:
                if len(stack) + len(out) < max_results:
                    # the other branch
                    if use:
                        stack.append((k + 1, T, C.copy(), last))
                    else:
                        ak_alt = max(ak, 0.0)
                        Tn = T * (1.0 - ak_alt)
                        if Tn >= tmin:
                            stack.append((k + 1, Tn, C + rgb[k] * ak_alt * T, k + 1))
                        else:
                            stack.append((K, T, C.copy(), last))
            if not use:
                k += 1
                continue
            Tn = T * (1.0 - ak)
            if abs(Tn - tmin) <= T_BAND * tmin and len(stack) + len(out) < max_results:
                if Tn < tmin:
                    stack.append((k + 1, Tn, C + rgb[k] * ak * T, k + 1))
                else:
                    stack.append((K, T, C.copy(), last))
            if Tn < tmin:
                break
            C = C + rgb[k] * ak * T
            T = Tn
            last = k + 1
            k += 1
        out.append((C + T * bg, T, last))
    return out


class Oracle:
    """Decisions from the float32 stage, values in float64.

    ``render`` composites the requested global tiles (default: all) of every
    view.  With ``tile_free=True`` each pixel blends every non-culled record
    of its view in (depth bits, record) order instead of its tile's list.
    """

    def __init__(self, scenes, views, cfg):
        self.scenes, self.views, self.cfg = scenes, views, cfg
        self.pre32 = fp32_spec.preprocess(scenes, views, cfg)
        self.bins = binning.bin_and_sort(scenes, views, cfg, self.pre32)
        self.rec_off = self.bins["record_offset"]
        self.tile_off = self.bins["tile_offset"]

    def leaves(self, requires_grad=False):
        return [scene_leaves(s, requires_grad) for s in self.scenes]

    def records(self, leaves, views=None):
        """Per view: float64 mean2d [P,2], conic [P,2,2], opacity [P],
        beta_x [P], rgb [P,3], depth [P], cov2d [P,2,2], mean3 [P,3].  With
        ``views`` (indices), only those views' records are computed and the
        others are None (a render restricted to their tiles needs no more)."""
        out = []
        for vi, v in enumerate(self.views):
            if views is not None and vi not in views:
                out.append(None)
                continue
            sc = self.scenes[v.scene_id]
            lv = leaves[v.scene_id]
            mu_c, Sc, oq, beta_x = condition(lv, sc.N, sc.rot_mode, v)
            tz, mu2, cov2, conic = project(mu_c, Sc, v, self.cfg)
            out.append({"mean2d": mu2, "conic": conic, "opacity": oq, "beta_x": beta_x,
                        "rgb": lv["rgb"].T, "depth": tz, "cov2d": cov2, "mean3": mu_c})
        return out

    def view_of_tile(self, g):
        return int(np.searchsorted(self.tile_off, g, side="right") - 1)

    def render(self, leaves=None, tiles=None, tile_free=False, recs=None):
        cfg = self.cfg
        if leaves is None:
            leaves = self.leaves(False)
        if recs is None:
            recs = self.records(leaves)
        images, Ts, lasts, flags, plo, phi = [], [], [], [], [], []
        for vi, v in enumerate(self.views):
            H, W = v.height, v.width
            images.append(torch.full((3, H, W), float("nan"), dtype=D))
            Ts.append(torch.full((H, W), float("nan"), dtype=D))
            lasts.append(torch.full((H, W), -1, dtype=torch.long))
            flags.append(torch.zeros((H, W), dtype=torch.bool))
            plo.append(torch.full((H, W), -1, dtype=torch.long))
            phi.append(torch.full((H, W), -1, dtype=torch.long))
        if tiles is None:
            tiles = range(int(self.tile_off[-1]))
        ranges = self.bins["ranges"]
        rec_sorted = self.bins["record"]
        # tile-free order per view: all valid records by (depth bits, index)
        order_cache = {}
        for g in tiles:
            vi = self.view_of_tile(g)
            v = self.views[vi]
            ntx, _ = binning.tile_grid(v, cfg)
            loc = g - self.tile_off[vi]
            tx, ty = loc % ntx, loc // ntx
            x0, y0 = tx * cfg.tile_w, ty * cfg.tile_h
            x1, y1 = min(x0 + cfg.tile_w, v.width), min(y0 + cfg.tile_h, v.height)
            ys, xs = np.meshgrid(np.arange(y0, y1), np.arange(x0, x1), indexing="ij")
            px = torch.tensor(xs.ravel() + 0.5, dtype=D)
            py = torch.tensor(ys.ravel() + 0.5, dtype=D)
            if tile_free:
                if vi not in order_cache:
                    pre = self.pre32[vi]
                    idx = np.nonzero(pre["valid"] & (pre["tiles_touched"] > 0))[0]
                    o = np.lexsort((idx, pre["depth_bits"][idx]))
                    order_cache[vi] = idx[o]
                lst = torch.from_numpy(order_cache[vi])
            else:
                s, e = ranges[g]
                lst = torch.from_numpy(rec_sorted[s:e] - self.rec_off[vi])
            R = recs[vi]
            c32 = self.pre32[vi]["conic"]
            ext = {"count_conic": torch.from_numpy(c32.T[lst.numpy()].astype(np.float64))}
            col, T, last, flag = _composite_block(px, py, R["mean2d"][lst], R["conic"][lst],
                                                  R["opacity"][lst], R["beta_x"][lst],
                                                  R["rgb"][lst], cfg, ext)
            hh, ww = y1 - y0, x1 - x0
            plo[vi][y0:y1, x0:x1] = ext["pairs_lo"].reshape(hh, ww)
            phi[vi][y0:y1, x0:x1] = ext["pairs_hi"].reshape(hh, ww)
            images[vi][:, y0:y1, x0:x1] = col.T.reshape(3, hh, ww)
            Ts[vi][y0:y1, x0:x1] = T.reshape(hh, ww)
            lasts[vi][y0:y1, x0:x1] = last.reshape(hh, ww)
            flags[vi][y0:y1, x0:x1] = flag.reshape(hh, ww)
        return {"image": images, "T": Ts, "last": lasts, "flag": flags, "pairs_lo": plo, "pairs_hi": phi}

    def admissible(self, vi, x, y, recs=None, tile_free=False):
        """All admissible (colour, T, last) results of pixel (x, y) of view vi."""
        cfg = self.cfg
        if recs is None:
            recs = self.records(self.leaves(False))
        v = self.views[vi]
        ntx, _ = binning.tile_grid(v, cfg)
        g = self.tile_off[vi] + (y // cfg.tile_h) * ntx + (x // cfg.tile_w)
        s, e = self.bins["ranges"][g]
        lst = self.bins["record"][s:e] - self.rec_off[vi]
        R = recs[vi]
        with torch.no_grad():
            mu2 = R["mean2d"][lst].numpy()
            con = R["conic"][lst].numpy()
            oq = R["opacity"][lst].numpy()
            beta = R["beta_x"][lst].numpy()
            rgb = R["rgb"][lst].numpy()
        dx = (x + 0.5) - mu2[:, 0]
        dy = (y + 0.5) - mu2[:, 1]
        r = con[:, 0, 0] * dx * dx + 2 * con[:, 0, 1] * dx * dy + con[:, 1, 1] * dy * dy
        base = np.where(r < 1, 1 - r, 1.0)
        alpha = np.minimum(cfg.alpha_max, oq * np.where(r < 1, base ** beta, 0.0))
        return composite_branches(r, alpha, beta, oq, rgb, cfg)


def loss_grads(oracle, dL_dimage, tiles=None, views=None):
    """Gradient of sum(image * dL_dimage) with respect to every parameter
    plane block of every scene (autograd of the float64 forward), plus the
    per-record gradients of the projected quantities.  ``views``: restrict the
    records to these views (dL_dimage must vanish on the others)."""
    leaves = oracle.leaves(True)
    recs = oracle.records(leaves, views=views)
    for R in recs:
        if R is None:
            continue
        for k in ("mean2d", "conic", "opacity", "beta_x", "rgb"):
            R[k].retain_grad()
    out = oracle.render(leaves=leaves, tiles=tiles, recs=recs)
    loss = torch.zeros((), dtype=D)
    for img, g in zip(out["image"], dL_dimage):
        gg = torch.as_tensor(np.asarray(g, np.float64))
        mask = ~torch.isnan(img)
        loss = loss + (torch.where(mask, img, torch.zeros_like(img)) * gg).sum()
    loss.backward()
    grads = [{k: (t.grad.numpy().copy() if t.grad is not None else np.zeros(tuple(t.shape)))
              for k, t in lv.items()} for lv in leaves]
    rec_grads = []
    for R in recs:
        if R is None:
            rec_grads.append(None)
            continue
        rec_grads.append({k: (R[k].grad.numpy().copy() if R[k].grad is not None
                              else np.zeros(tuple(R[k].shape))) for k in
                          ("mean2d", "conic", "opacity", "beta_x", "rgb")})
    return {"params": grads, "records": rec_grads, "image": out}
