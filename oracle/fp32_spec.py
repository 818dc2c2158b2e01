"""FP32 decision stage of the oracle (test infrastructure only).

The rasterizer turns floating-point values into integers in three places:
primitive culling, the depth sort key, and the tile rectangle of each
projected primitive.  For the sorted instance lists to be comparable bit for
bit, both the oracle and the CUDA path take these decisions in float32 by the
same written rules.  This module is the oracle's statement of those rules:

* every arithmetic operation is a single IEEE-754 binary32 operation rounded
  to nearest-even (numpy float32 arrays: no fused multiply-add, no
  reassociation); sums are evaluated left to right exactly as written;
* division and square root are correctly rounded;
* exp and log are project-written (no libm):
    exp: Cody & Waite (1980) argument reduction x = k ln2 + r with a two-part
         ln2 (hi part with 16 significant bits), then the degree-7 Taylor
         polynomial of e^r in Horner form with float32-rounded 1/k!
         coefficients, scaled by 2^k built from the exponent bits; inputs are
         clamped to [-87, 88] and return 0 below -87;
    log: x = m 2^e with m in [sqrt(1/2), sqrt(2)), s = (m-1)/(m+1), then
         log m = 2 atanh(s) = s (2 + z (2/3 + z (2/5 + z (2/7 + z (2/9 +
         z 2/11))))) with z = s^2, and log x = e ln2_hi + (poly + e ln2_lo).
    sin, cos (x >= 0): Cody & Waite reduction x = j pi/2 + r with j =
         rint(x 2/pi) and pi/2 split into three parts (12, 12 and 24
         significant bits), r = ((x - j P1) - j P2) - j P3; the Taylor
         polynomials sin r = r + r (z (-1/3! + z (1/5! + z (-1/7! + z 1/9!))))
         and cos r = 1 + z (-1/2! + z (1/4! + z (-1/6! + z (1/8! - z 1/10!))))
         with z = r^2 and binary32-rounded coefficients; the quadrant j mod 4
         picks (s, c), (c, -s), (-s, -c) or (-c, s).
  Both are within a few ulp of the true functions (tests pin this).

The quantities follow the paper: Sec. 4.2 (L, Sigma blocks), Sec. 4.3
(beta_x = 4 exp(b_x), beta_q = exp(b_q), clamped beta, conditional mean and
covariance, modulated opacity with d_i = tanh(d_i^raw)), Sec. 3 (EWA
projection Sigma' = J W Sigma W^T J^T, Mahalanobis r, compact support r < 1).
Rasterizer constants (alpha_min = 1/255, alpha_max = 0.99, transmittance stop
1e-4, the 0.3 low-pass dilation) and the tight cut radius follow standard
3DGS practice, which the paper's rasterizer inherits without restating.

Parity: pinned.  Each float output is compared against the float64
definition in ``render64`` (tests/test_oracle_fp32_spec.py), exp/log against
float64 libm within an ulp bound, and rectangle conservativeness against a
per-pixel float64 evaluation.
"""
from __future__ import annotations

import numpy as np

F = np.float32
I32 = np.int32

# exact binary32 constants (hex), derived from the mathematics
LOG2E = F(float.fromhex("0x1.715476p+0"))      # 1/ln 2 rounded to binary32
LN2 = F(float.fromhex("0x1.62e430p-1"))        # ln 2 rounded to binary32
LN2_HI = F(float.fromhex("0x1.62e4p-1"))       # 16 significant bits
LN2_LO = F(float.fromhex("0x1.7f7d1cp-20"))    # ln 2 - LN2_HI rounded
SQRT2 = F(float.fromhex("0x1.6a09e6p+0"))
EXP_C = [F(1) / F(f) for f in (5040, 720, 120, 24, 6, 2, 1, 1)]   # 1/7! ... 1/0!
LOG_C = [F(2) / F(k) for k in (11, 9, 7, 5, 3, 1)]                 # 2/11 ... 2/1
# pi/2 = PIO2_A + PIO2_B + PIO2_C (12, 12, 24 significant bits), 2/pi, and the
# alternating 1/k! of the sine (odd k) and cosine (even k) series
TWO_OVER_PI = F(float.fromhex("0x1.45f306p-1"))
PIO2_A = F(float.fromhex("0x1.92p+0"))
PIO2_B = F(float.fromhex("0x1.fb4p-12"))
PIO2_C = F(float.fromhex("0x1.4442d2p-24"))
SIN_C = [F(float.fromhex(h)) for h in ("-0x1.555556p-3", "0x1.111112p-7", "-0x1.a01a02p-13", "0x1.71de3ap-19")]
COS_C = [F(float.fromhex(h)) for h in ("-0x1p-1", "0x1.555556p-5", "-0x1.6c16c2p-10", "0x1.a01a02p-16",
                                         "-0x1.27e4fcp-22")]
MARG_R = F(float.fromhex("0x1.004p+0"))        # 1 + 2^-10
MARG_A = F(float.fromhex("0x1p-6"))            # 2^-6 pixel


def exp_spec(x):
    """e^x in binary32 (Cody-Waite reduction + degree-7 Taylor, Horner)."""
    x = np.asarray(x, dtype=F)
    under = x < F(-87.0)
    xc = np.minimum(np.maximum(x, F(-87.0)), F(88.0))
    k = np.rint(xc * LOG2E).astype(F)
    r = (xc - k * LN2_HI) - k * LN2_LO
    p = EXP_C[0]
    for c in EXP_C[1:]:
        p = p * r + c
    scale = ((k.astype(I32) + I32(127)) << I32(23)).astype(I32).view(F)
    out = (p * scale).astype(F)
    return np.where(under, F(0), out).astype(F)


def log_spec(x):
    """log x in binary32 for normal x > 0 (atanh series); -inf for x <= 0."""
    x = np.asarray(x, dtype=F)
    bad = ~(x > F(0))
    xs = np.where(bad, F(1), x).astype(F)
    bits = xs.view(I32)
    e = ((bits >> I32(23)) & I32(0xFF)) - I32(127)
    m = ((bits & I32(0x7FFFFF)) | I32(0x3F800000)).astype(I32).view(F)
    big = m > SQRT2
    m = np.where(big, m * F(0.5), m).astype(F)
    e = np.where(big, e + I32(1), e)
    s = (m - F(1)) / (m + F(1))
    z = s * s
    p = LOG_C[0]
    for c in LOG_C[1:]:
        p = p * z + c
    poly = s * p
    ef = e.astype(F)
    out = ef * LN2_HI + (poly + ef * LN2_LO)
    return np.where(bad, F(-np.inf), out).astype(F)


def sincos_spec(x):
    """(sin x, cos x) in binary32 for x >= 0 (Cody-Waite by pi/2, Taylor)."""
    x = np.asarray(x, dtype=F)
    j = np.rint(x * TWO_OVER_PI).astype(F)
    r = ((x - j * PIO2_A) - j * PIO2_B) - j * PIO2_C
    z = r * r
    ps = SIN_C[3]
    for c in (SIN_C[2], SIN_C[1], SIN_C[0]):
        ps = c + z * ps
    s = r + r * (z * ps)
    pc = COS_C[4]
    for c in (COS_C[3], COS_C[2], COS_C[1], COS_C[0]):
        pc = c + z * pc
    c = F(1) + z * pc
    q = j.astype(np.int64) & 3
    sin = np.select([q == 0, q == 1, q == 2], [s, c, -s], -c).astype(F)
    cos = np.select([q == 0, q == 1, q == 2], [c, -s, -c], s).astype(F)
    return sin, cos


# ----------------------------------------------------------------------------
# per-primitive, view-independent stage (Sec. 4.2 and the view-independent
# part of Sec. 4.3)
# ----------------------------------------------------------------------------

def _planes(scene):
    off = scene.offsets()
    p = {k: scene.params[o:o + n].astype(F) for k, (o, n) in off.items()}
    return p


def rotation(scene):
    """R_x rows as a 3x3 nested list of [P] arrays.  Quaternion mode: the
    3DGS rotation of the normalised quaternion (Sec. 3).  Skew modes, from
    omega (appendix on the spatial-orthogonal Cholesky parameterisation):
    R = I + A (first-order Taylor), and with the squares and products
    a_ij = o_i o_j
        R = I + l A + k A^2,  (A^2)_ij = a_ij - delta_ij (a11 + a22 + a33),
    k = 1/2, l = 1 (second-order Taylor) or k = l = 2 / (1 + ((a11 + a22) + a33))
    (Cayley: (I - A)^{-1}(I + A) in closed form), or, for exp(A), Rodrigues'
    l = sin t / t and k = (1 - cos t) / t^2 (t = |omega|; Taylor series in t^2
    below t^2 = 1/4, else sincos_spec), evaluated entry by entry as
        R00 = 1 - k (a22 + a33)   R01 = k a12 - l o3   R02 = k a13 + l o2
        R10 = k a12 + l o3        R11 = 1 - k (a11 + a33)   R12 = k a23 - l o1
        R20 = k a13 - l o2        R21 = k a23 + l o1   R22 = 1 - k (a11 + a22)."""
    pl = _planes(scene)
    rot = pl["rot"]
    if scene.rot_mode == 0:
        w, x, y, z = rot[0], rot[1], rot[2], rot[3]
        nn = ((w * w + x * x) + y * y) + z * z
        n = np.sqrt(nn)
        w, x, y, z = w / n, x / n, y / n, z / n
        one, two = F(1), F(2)
        R = [[one - two * (y * y + z * z), two * (x * y - w * z), two * (x * z + w * y)],
             [two * (x * y + w * z), one - two * (x * x + z * z), two * (y * z - w * x)],
             [two * (x * z - w * y), two * (y * z + w * x), one - two * (x * x + y * y)]]
    elif scene.rot_mode == 1:
        o1, o2, o3 = rot[0], rot[1], rot[2]
        one = np.ones_like(o1)
        R = [[one, -o3, o2], [o3, one, -o1], [-o2, o1, one]]
    elif scene.rot_mode in (2, 3, 5):
        o1, o2, o3 = rot[0], rot[1], rot[2]
        a11, a22, a33 = o1 * o1, o2 * o2, o3 * o3
        a12, a13, a23 = o1 * o2, o1 * o3, o2 * o3
        one = F(1)
        if scene.rot_mode == 2:
            k = np.full_like(o1, F(0.5))
            l = np.ones_like(o1)
        elif scene.rot_mode == 3:
            k = F(2) / (one + ((a11 + a22) + a33))
            l = k
        else:
            # exp(A) (Rodrigues): l = sin t / t, k = (1 - cos t) / t^2 with t^2 = n;
            # below n = 1/4 their Taylor series in n (Horner), else sincos_spec
            n = (a11 + a22) + a33
            s1, s2, s3, s4 = SIN_C
            c2, c3, c4, c5 = COS_C[1:]
            l_ser = one + n * (s1 + n * (s2 + n * (s3 + n * s4)))
            k_ser = F(0.5) + n * (-c2 + n * (-c3 + n * (-c4 + n * -c5)))
            t = np.sqrt(n)
            sn, cs = sincos_spec(t)
            small = n < F(0.25)
            with np.errstate(divide="ignore", invalid="ignore"):
                l_big = sn / t
                k_big = (one - cs) / n
            l = np.where(small, l_ser, l_big).astype(F)
            k = np.where(small, k_ser, k_big).astype(F)
        R = [[one - k * (a22 + a33), k * a12 - l * o3, k * a13 + l * o2],
             [k * a12 + l * o3, one - k * (a11 + a33), k * a23 - l * o1],
             [k * a13 - l * o2, k * a23 + l * o1, one - k * (a11 + a22)]]
    else:
        raise ValueError(f"rotation mode {scene.rot_mode}")
    return R


def prim_stage(scene):
    """View-independent per-primitive quantities in binary32."""
    pl = _planes(scene)
    C = scene.C
    P = scene.P
    s = pl["scale_x"]
    if scene.rot_mode == 4:
        # the plain Cholesky row: M is the factor itself, no arithmetic
        lo = pl["rot"]
        zero = np.zeros_like(s[0])
        M = [[s[0], zero, zero], [lo[0], s[1], zero], [lo[1], lo[2], s[2]]]
        R = None
    else:
        R = rotation(scene)
        M = [[R[i][j] * s[j] for j in range(3)] for i in range(3)]
    Sx = {}
    for i in range(3):
        for j in range(i, 3):
            Sx[(i, j)] = (M[i][0] * M[j][0] + M[i][1] * M[j][1]) + M[i][2] * M[j][2]
    bx = pl["b"][0]
    beta_x = F(4) * exp_spec(bx)
    out = {"R": R, "M": M, "Sx": Sx, "beta_x": beta_x, "valid": np.ones(P, bool),
           "opacity": pl["opacity"][0], "rgb": pl["rgb"], "mean_x": pl["mean_x"], "C": C}
    if C == 0:
        out["Sc"] = Sx
        return out
    Lqx = [[pl["L_qx"][3 * k + j] for j in range(3)] for k in range(C)]
    Lq = {}
    for i in range(C):
        for j in range(i + 1):
            Lq[(i, j)] = pl["L_q"][i * (i + 1) // 2 + j]
    # Sigma_qx[k][i] = sum_j M[i][j] L_qx[k][j]   (Sigma_xq = R diag(s) L_qx^T)
    Sqx = [[(M[i][0] * Lqx[k][0] + M[i][1] * Lqx[k][1]) + M[i][2] * Lqx[k][2]
            for i in range(3)] for k in range(C)]
    # Sigma_q = L_qx L_qx^T + L_q L_q^T, running sum
    Sq = {}
    for k in range(C):
        for l in range(k + 1):
            acc = Lqx[k][0] * Lqx[l][0]
            acc = acc + Lqx[k][1] * Lqx[l][1]
            acc = acc + Lqx[k][2] * Lqx[l][2]
            for m in range(l + 1):
                acc = acc + Lq[(k, m)] * Lq[(l, m)]
            Sq[(k, l)] = acc
    # Cholesky factor of Sigma_q (L-hat of Sec. 4.3)
    Lh = {}
    valid = np.ones(P, bool)
    for i in range(C):
        for j in range(i + 1):
            acc = Sq[(i, j)]
            for m in range(j):
                acc = acc - Lh[(i, m)] * Lh[(j, m)]
            if i == j:
                valid &= acc > F(0)
                Lh[(i, i)] = np.sqrt(np.where(acc > F(0), acc, F(1)).astype(F))
            else:
                Lh[(i, j)] = acc / Lh[(j, j)]
    # Z = Sigma_q^{-1} Sigma_qx  (forward then backward substitution, per column)
    Z = [[None] * 3 for _ in range(C)]
    for i in range(3):
        Y = [None] * C
        for k in range(C):
            acc = Sqx[k][i]
            for m in range(k):
                acc = acc - Lh[(k, m)] * Y[m]
            Y[k] = acc / Lh[(k, k)]
        for k in range(C - 1, -1, -1):
            acc = Y[k]
            for m in range(k + 1, C):
                acc = acc - Lh[(m, k)] * Z[m][i]
            Z[k][i] = acc / Lh[(k, k)]
    beta_q = [exp_spec(pl["b"][1 + k]) for k in range(C)]
    beta_t = [np.minimum(bq, F(1)) for bq in beta_q]
    # W3[i][k] = (Sigma_xq Sigma_q^{-1} diag(beta~))[i][k]
    W3 = [[Z[k][i] * beta_t[k] for k in range(C)] for i in range(3)]
    Sc = {}
    M2 = [[None] * 3 for _ in range(3)]
    for i in range(3):
        for j in range(3):
            acc = W3[i][0] * Sqx[0][j]
            for k in range(1, C):
                acc = acc + W3[i][k] * Sqx[k][j]
            M2[i][j] = acc
    for i in range(3):
        for j in range(i, 3):
            Sc[(i, j)] = Sx[(i, j)] - F(0.5) * (M2[i][j] + M2[j][i])
    out.update({"Sqx": Sqx, "Sq": Sq, "Lh": Lh, "Z": Z, "beta_q": beta_q, "beta_t": beta_t,
                "W3": W3, "Sc": Sc, "mean_q": pl["mean_q"]})
    out["valid"] = valid
    return out


# ----------------------------------------------------------------------------
# per (view, primitive) stage
# ----------------------------------------------------------------------------

def view_stage(scene, pre, view, cfg):
    """Conditioning on the query of ``view`` (Sec. 4.3, Sec. 4.4 query
    specialisation) and projection (Sec. 3) in binary32; returns the decision
    outputs and the binary32 values used by the rasterizer."""
    C = scene.C
    Rv = np.asarray(view.R, F)
    tv = np.asarray(view.t, F)
    mx = pre["mean_x"]
    oq = pre["opacity"]
    if C > 0:
        # camera centre c = -R^T t
        cam = [-((Rv[0, i] * tv[0] + Rv[1, i] * tv[1]) + Rv[2, i] * tv[2]) for i in range(3)]
        q = []
        if C in (1, 4):
            q.append(np.full(scene.P, F(view.time), F))
        if C >= 3:
            v = [mx[i] - F(cam[i]) for i in range(3)]
            nn = (v[0] * v[0] + v[1] * v[1]) + v[2] * v[2]
            n = np.sqrt(nn)
            q += [v[i] / n for i in range(3)]
        delta = [q[k] - pre["mean_q"][k] for k in range(C)]
        Lh = pre["Lh"]
        y = [None] * C
        for k in range(C):
            acc = delta[k]
            for m in range(k):
                acc = acc - Lh[(k, m)] * y[m]
            y[k] = acc / Lh[(k, k)]
        E = None
        for k in range(C):
            dr = y[k] * y[k]
            u = exp_spec(F(-2) * dr)
            lg = (LN2 - F(2) * dr) - log_spec(F(1) + u)
            term = (F(4) * pre["beta_q"][k]) * lg
            E = term if E is None else E + term
        oq = oq * exp_spec(E)
        W3 = pre["W3"]
        mc = []
        for i in range(3):
            acc = W3[i][0] * delta[0]
            for k in range(1, C):
                acc = acc + W3[i][k] * delta[k]
            mc.append(mx[i] + acc)
    else:
        mc = [mx[0], mx[1], mx[2]]
    S = pre["Sc"]
    Sf = lambda i, j: S[(i, j)] if i <= j else S[(j, i)]
    tc = [((Rv[j, 0] * mc[0] + Rv[j, 1] * mc[1]) + Rv[j, 2] * mc[2]) + tv[j] for j in range(3)]
    tz = tc[2]
    fx, fy, cx, cy = F(view.fx), F(view.fy), F(view.cx), F(view.cy)
    W, H = view.width, view.height
    valid = pre["valid"] & (tz > F(cfg.near))
    tzs = np.where(valid, tz, F(1)).astype(F)
    u = tc[0] / tzs
    vv = tc[1] / tzs
    mux = fx * u + cx
    muy = fy * vv + cy
    limx = F(cfg.jac_clip) * ((F(0.5) * F(W)) / fx)
    limy = F(cfg.jac_clip) * ((F(0.5) * F(H)) / fy)
    uc = np.minimum(np.maximum(u, -limx), limx)
    vc = np.minimum(np.maximum(vv, -limy), limy)
    J00 = fx / tzs
    J02 = -((fx * uc) / tzs)
    J11 = fy / tzs
    J12 = -((fy * vc) / tzs)
    T = [[J00 * Rv[0, j] + J02 * Rv[2, j] for j in range(3)],
         [J11 * Rv[1, j] + J12 * Rv[2, j] for j in range(3)]]
    U = [[(T[a][0] * Sf(0, j) + T[a][1] * Sf(1, j)) + T[a][2] * Sf(2, j) for j in range(3)]
         for a in range(2)]
    eps = F(cfg.eps2d)
    s00 = ((U[0][0] * T[0][0] + U[0][1] * T[0][1]) + U[0][2] * T[0][2]) + eps
    s01 = (U[0][0] * T[1][0] + U[0][1] * T[1][1]) + U[0][2] * T[1][2]
    s11 = ((U[1][0] * T[1][0] + U[1][1] * T[1][1]) + U[1][2] * T[1][2]) + eps
    det = s00 * s11 - s01 * s01
    valid &= det > F(0)
    dets = np.where(valid, det, F(1)).astype(F)
    ca = s11 / dets
    cb = -(s01 / dets)
    cc = s00 / dets
    amin = F(cfg.alpha_min)
    valid &= oq >= amin
    if cfg.tight_cut:
        oqs = np.where(valid, oq, F(1)).astype(F)
        with np.errstate(invalid="ignore", divide="ignore"):
            lr = log_spec(amin / oqs)
            rcut = F(1) - exp_spec(lr / pre["beta_x"])
    else:
        rcut = np.ones_like(oq)
    ex = np.sqrt(np.maximum(rcut * s00, F(0)))
    ey = np.sqrt(np.maximum(rcut * s11, F(0)))
    exm = ex * MARG_R + MARG_A
    eym = ey * MARG_R + MARG_A
    with np.errstate(invalid="ignore", over="ignore"):
        px0 = np.ceil((mux - exm) - F(0.5))
        px1 = np.floor((mux + exm) - F(0.5))
        py0 = np.ceil((muy - eym) - F(0.5))
        py1 = np.floor((muy + eym) - F(0.5))
    px0 = np.maximum(px0, F(0))
    py0 = np.maximum(py0, F(0))
    px1 = np.minimum(px1, F(W - 1))
    py1 = np.minimum(py1, F(H - 1))
    valid &= (px0 <= px1) & (py0 <= py1)
    tw, th = cfg.tile_w, cfg.tile_h
    z = np.zeros_like(px0)
    ix0 = np.where(valid, px0, z).astype(np.int64)
    ix1 = np.where(valid, px1, z).astype(np.int64)
    iy0 = np.where(valid, py0, z).astype(np.int64)
    iy1 = np.where(valid, py1, z).astype(np.int64)
    tx0, tx1 = ix0 // tw, ix1 // tw + 1
    ty0, ty1 = iy0 // th, iy1 // th + 1
    tiles = np.where(valid, (tx1 - tx0) * (ty1 - ty0), 0).astype(np.int64)
    rect = np.stack([tx0, ty0, tx1, ty1], axis=0)
    rect[:, ~valid] = 0
    return {
        "valid": valid, "depth": tz.astype(F), "depth_bits": tz.astype(F).view(np.uint32),
        "rect": rect, "tiles_touched": tiles,
        "mean2d": np.stack([mux, muy]).astype(F), "conic": np.stack([ca, cb, cc]).astype(F),
        "opacity": oq.astype(F), "beta_x": pre["beta_x"].astype(F), "rcut": rcut.astype(F),
        "cov2d": np.stack([s00, s01, s11]).astype(F), "mean3": np.stack(mc).astype(F),
    }


def preprocess(scenes, views, cfg):
    """All (view, primitive) records; record index = record_offset[v] + p."""
    pres = {}
    out = []
    for v in views:
        sid = v.scene_id
        if sid not in pres:
            pres[sid] = prim_stage(scenes[sid])
        out.append(view_stage(scenes[sid], pres[sid], v, cfg))
    return out
