// prim_forward.cuh -- per-primitive forward math of the preprocess step.
//
// Follows Sec. 4.2 (spatial-orthogonal Cholesky L and the blocks of
// Sigma = L L^T), Sec. 4.3 (beta_x = 4 e^{b_x}, beta_q = e^{b_q},
// beta~ = min(beta_q, 1), mu_{x|q}, Sigma_{x|q}, d_i = tanh(d_i^raw),
// o(q) = o prod (1 - d_i)^{4 beta_qi}), Sec. 4.4 (q = [t, d]) and Sec. 3
// (EWA projection, Mahalanobis conic, compact Beta support).
//
// Every value that decides an integer is computed under the float32 rule
// set of spec32.cuh.  The screen mean used for blending is additionally
// carried as an unevaluated double-float (hi + lo) sum from an error-free
// evaluation of mu' = f (W mu_{x|q} + t)_xy / (W mu_{x|q} + t)_z + c, so
// that pixel offsets keep their precision at large image coordinates.
//
// Restatement of the rules used by the opacity factor: with x = d_raw >= 0,
// log(1 - tanh x) = (ln 2 - 2x) - log(1 + e^{-2x}) (exact identity), and
// o(q) = o exp(sum_k (4 beta_qk) log(1 - tanh x_k)).
#pragma once

#include "common.cuh"
#include "spec32.cuh"

namespace ubs {

template <int C>
struct CDim {
  static constexpr int M = C > 0 ? C : 1;
  static constexpr int T = C > 0 ? C * (C + 1) / 2 : 1;
};

UBS_HD int tri(int i, int j) { return i * (i + 1) / 2 + j; }

template <int C>
struct PrimIn {
  float mx[3];
  float rot[4];
  float s[3];
  float lqx[3 * CDim<C>::M];
  float lq[CDim<C>::T];
  float b[1 + C];
  float o;
  float mq[CDim<C>::M];
};

// view-independent quantities
template <int C>
struct PrimVI {
  float R[9];
  float M[9];
  float Sc[6];  // symmetric 3x3, packed 00 01 02 11 12 22
  float beta_x;
  bool valid;
  float Sqx[CDim<C>::M][3];
  float Lh[CDim<C>::T];
  float Z[CDim<C>::M][3];
  float beta_q[CDim<C>::M];
  float beta_t[CDim<C>::M];
  float W3[3][CDim<C>::M];
};

UBS_HD int sym(int i, int j) {
  // index of (i, j) in the packed 00 01 02 11 12 22 order
  int a = i < j ? i : j, b = i < j ? j : i;
  return a == 0 ? b : (a == 1 ? 2 + b : 5);
}

UBS_HD void rotation_spec(const float* rot, int rot_mode, float* R) {
  if (rot_mode == 0) {
    float w = rot[0], x = rot[1], y = rot[2], z = rot[3];
    float nn = ((w * w + x * x) + y * y) + z * z;
    float n = sqrtf(nn);
    w = w / n;
    x = x / n;
    y = y / n;
    z = z / n;
    R[0] = 1.0f - 2.0f * (y * y + z * z);
    R[1] = 2.0f * (x * y - w * z);
    R[2] = 2.0f * (x * z + w * y);
    R[3] = 2.0f * (x * y + w * z);
    R[4] = 1.0f - 2.0f * (x * x + z * z);
    R[5] = 2.0f * (y * z - w * x);
    R[6] = 2.0f * (x * z - w * y);
    R[7] = 2.0f * (y * z + w * x);
    R[8] = 1.0f - 2.0f * (x * x + y * y);
  } else if (rot_mode == 1) {
    float o1 = rot[0], o2 = rot[1], o3 = rot[2];
    R[0] = 1.0f; R[1] = -o3;  R[2] = o2;
    R[3] = o3;   R[4] = 1.0f; R[5] = -o1;
    R[6] = -o2;  R[7] = o1;   R[8] = 1.0f;
  } else {
    // R = I + l A + k A^2 with (A^2)_ij = o_i o_j - delta_ij |o|^2: k = 1/2,
    // l = 1 (second-order Taylor of exp A), k = l = 2 / (1 + |o|^2) (the
    // Cayley transform (I - A)^-1 (I + A) in closed form), or exp A itself
    const float o1 = rot[0], o2 = rot[1], o3 = rot[2];
    const float a11 = o1 * o1, a22 = o2 * o2, a33 = o3 * o3;
    const float a12 = o1 * o2, a13 = o1 * o3, a23 = o2 * o3;
    float k, l;
    if (rot_mode == 2) {
      k = 0.5f;
      l = 1.0f;
    } else if (rot_mode == 3) {
      k = 2.0f / (1.0f + ((a11 + a22) + a33));
      l = k;
    } else {
      // exp(A) by Rodrigues: l = sin t / t, k = (1 - cos t) / t^2, t = |o|;
      // below t^2 = 1/4 their Taylor series in t^2, else the rule set's sin, cos
      const float n = (a11 + a22) + a33;
      if (n < 0.25f) {
        l = 1.0f + n * (spec::kInv3 + n * (spec::kInv5 + n * (spec::kInv7 + n * spec::kInv9)));
        k = 0.5f + n * (-spec::kInv4 + n * (-spec::kInv6 + n * (-spec::kInv8 + n * -spec::kInv10)));
      } else {
        const float t = sqrtf(n);
        float s, c;
        spec::sincos32(t, &s, &c);
        l = s / t;
        k = (1.0f - c) / n;
      }
    }
    R[0] = 1.0f - k * (a22 + a33);
    R[1] = k * a12 - l * o3;
    R[2] = k * a13 + l * o2;
    R[3] = k * a12 + l * o3;
    R[4] = 1.0f - k * (a11 + a33);
    R[5] = k * a23 - l * o1;
    R[6] = k * a13 - l * o2;
    R[7] = k * a23 + l * o1;
    R[8] = 1.0f - k * (a11 + a22);
  }
}

template <int C>
UBS_HD void prim_stage(const PrimIn<C>& in, int rot_mode, PrimVI<C>& vi) {
  if (rot_mode == 4) {
    // the plain Cholesky row: M is the lower-triangular factor itself
    vi.M[0] = in.s[0];  vi.M[1] = 0.0f;      vi.M[2] = 0.0f;
    vi.M[3] = in.rot[0]; vi.M[4] = in.s[1];  vi.M[5] = 0.0f;
    vi.M[6] = in.rot[1]; vi.M[7] = in.rot[2]; vi.M[8] = in.s[2];
  } else {
    rotation_spec(in.rot, rot_mode, vi.R);
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) vi.M[3 * i + j] = vi.R[3 * i + j] * in.s[j];
  }
  const float* M = vi.M;
  float Sx[6];
  for (int i = 0; i < 3; ++i)
    for (int j = i; j < 3; ++j)
      Sx[sym(i, j)] = (M[3 * i] * M[3 * j] + M[3 * i + 1] * M[3 * j + 1]) + M[3 * i + 2] * M[3 * j + 2];
  vi.beta_x = 4.0f * spec::exp32(in.b[0]);
  vi.valid = true;
  if constexpr (C == 0) {
    for (int k = 0; k < 6; ++k) vi.Sc[k] = Sx[k];
  } else {
    const float* Lqx = in.lqx;
    for (int k = 0; k < C; ++k)
      for (int i = 0; i < 3; ++i)
        vi.Sqx[k][i] = (M[3 * i] * Lqx[3 * k] + M[3 * i + 1] * Lqx[3 * k + 1]) + M[3 * i + 2] * Lqx[3 * k + 2];
    float Sq[CDim<C>::T];
    for (int k = 0; k < C; ++k)
      for (int l = 0; l <= k; ++l) {
        float acc = Lqx[3 * k] * Lqx[3 * l];
        acc = acc + Lqx[3 * k + 1] * Lqx[3 * l + 1];
        acc = acc + Lqx[3 * k + 2] * Lqx[3 * l + 2];
        for (int m = 0; m <= l; ++m) acc = acc + in.lq[tri(k, m)] * in.lq[tri(l, m)];
        Sq[tri(k, l)] = acc;
      }
    for (int i = 0; i < C; ++i)
      for (int j = 0; j <= i; ++j) {
        float acc = Sq[tri(i, j)];
        for (int m = 0; m < j; ++m) acc = acc - vi.Lh[tri(i, m)] * vi.Lh[tri(j, m)];
        if (i == j) {
          vi.valid = vi.valid && (acc > 0.0f);
          vi.Lh[tri(i, i)] = sqrtf(acc > 0.0f ? acc : 1.0f);
        } else {
          vi.Lh[tri(i, j)] = acc / vi.Lh[tri(j, j)];
        }
      }
    for (int i = 0; i < 3; ++i) {
      float Y[CDim<C>::M];
      for (int k = 0; k < C; ++k) {
        float acc = vi.Sqx[k][i];
        for (int m = 0; m < k; ++m) acc = acc - vi.Lh[tri(k, m)] * Y[m];
        Y[k] = acc / vi.Lh[tri(k, k)];
      }
      for (int k = C - 1; k >= 0; --k) {
        float acc = Y[k];
        for (int m = k + 1; m < C; ++m) acc = acc - vi.Lh[tri(m, k)] * vi.Z[m][i];
        vi.Z[k][i] = acc / vi.Lh[tri(k, k)];
      }
    }
    for (int k = 0; k < C; ++k) {
      vi.beta_q[k] = spec::exp32(in.b[1 + k]);
      vi.beta_t[k] = fminf(vi.beta_q[k], 1.0f);
    }
    for (int i = 0; i < 3; ++i)
      for (int k = 0; k < C; ++k) vi.W3[i][k] = vi.Z[k][i] * vi.beta_t[k];
    float M2[3][3];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) {
        float acc = vi.W3[i][0] * vi.Sqx[0][j];
        for (int k = 1; k < C; ++k) acc = acc + vi.W3[i][k] * vi.Sqx[k][j];
        M2[i][j] = acc;
      }
    for (int i = 0; i < 3; ++i)
      for (int j = i; j < 3; ++j) vi.Sc[sym(i, j)] = Sx[sym(i, j)] - 0.5f * (M2[i][j] + M2[j][i]);
  }
}

// ---------------------------------------------------------------- double-float

struct DF {
  float hi, lo;
};

UBS_HD DF two_sum(float a, float b) {
  float s = a + b;
  float bb = s - a;
  float e = (a - (s - bb)) + (b - bb);
  return {s, e};
}

UBS_HD DF quick_two_sum(float a, float b) {
  float s = a + b;
  float e = b - (s - a);
  return {s, e};
}

UBS_HD DF two_prod(float a, float b) {
  float p = a * b;
  float e = fmaf(a, b, -p);
  return {p, e};
}

UBS_HD DF df_add(DF a, DF b) {
  DF s = two_sum(a.hi, b.hi);
  float e = (s.lo + a.lo) + b.lo;
  return quick_two_sum(s.hi, e);
}

UBS_HD DF df_mul_f(DF a, float b) {
  DF p = two_prod(a.hi, b);
  float e = fmaf(a.lo, b, p.lo);
  return quick_two_sum(p.hi, e);
}

UBS_HD DF df_div(DF a, DF b) {
  float q1 = a.hi / b.hi;
  DF p = df_mul_f(b, q1);
  DF r = df_add(a, DF{-p.hi, -p.lo});
  float q2 = r.hi / b.hi;
  return quick_two_sum(q1, q2);
}

// ---------------------------------------------------------------- per view

struct ViewOut {
  bool valid;
  float depth;
  int32_t tx0, ty0, tx1, ty1;
  uint32_t tiles;
  float mu_hi[2], mu_lo[2];
  float conic[3];
  float oq;
};

// The conditioning of one record on its view's query (Sec. 4.3, 4.4): the
// modulated opacity o(q), the mean shift and the conditioned mean.
struct ViewCond {
  float oq;
  float shift[3];
  float mc[3];
};

//
// cull_below (a natural log): a record whose opacity is certain to fall
// below alpha_min skips the opacity's exp/log and the mean shift, with
// cond.oq = 0 (culled).  Since log(1 - tanh x) <= ln 2 - 2x and log32 of
// 1 + u is never negative, each term of the exponent E is, in float32 (the
// roundings are monotone), at most the matching term of
// E_ub = sum 4 beta_q (ln 2 - 2 y^2); where E_ub < cull_below =
// ln(alpha_min / o) - 0.01, o(q) = o exp(E) lies 1% below alpha_min, far
// beyond the rounding of exp32 and of the product, and the full evaluation
// would cull the record too.  No decision changes.
template <int C>
UBS_HD void view_condition(const PrimIn<C>& in, const PrimVI<C>& vi, const ViewDev& v, ViewCond& cond,
                           float cull_below = -INFINITY) {
  const float* Rv = v.R;
  float mc[3], shift[3] = {0.0f, 0.0f, 0.0f};
  float oq = in.o;
  if constexpr (C > 0) {
    float q[CDim<C>::M];
    int qi = 0;
    if constexpr (C == 1 || C == 4) q[qi++] = v.time;
    if constexpr (C >= 3) {
      float cam[3], vv[3];
      for (int i = 0; i < 3; ++i) cam[i] = -((Rv[i] * v.t[0] + Rv[3 + i] * v.t[1]) + Rv[6 + i] * v.t[2]);
      for (int i = 0; i < 3; ++i) vv[i] = in.mx[i] - cam[i];
      float nn = (vv[0] * vv[0] + vv[1] * vv[1]) + vv[2] * vv[2];
      float n = sqrtf(nn);
      for (int i = 0; i < 3; ++i) q[qi++] = vv[i] / n;
    }
    float delta[CDim<C>::M], y[CDim<C>::M];
    for (int k = 0; k < C; ++k) delta[k] = q[k] - in.mq[k];
    for (int k = 0; k < C; ++k) {
      float acc = delta[k];
      for (int m = 0; m < k; ++m) acc = acc - vi.Lh[tri(k, m)] * y[m];
      y[k] = acc / vi.Lh[tri(k, k)];
    }
    float Eub = 0.0f;
    for (int k = 0; k < C; ++k) {
      const float bound = (4.0f * vi.beta_q[k]) * (spec::kLn2 - 2.0f * (y[k] * y[k]));
      Eub = (k == 0) ? bound : Eub + bound;
    }
    if (Eub < cull_below) {  // culled whatever the exact exponent
      cond.oq = 0.0f;
      for (int i = 0; i < 3; ++i) {
        cond.shift[i] = 0.0f;
        cond.mc[i] = in.mx[i];
      }
      return;
    }
    float E = 0.0f;
    for (int k = 0; k < C; ++k) {
      float dr = y[k] * y[k];
      float u = spec::exp32(-2.0f * dr);
      float lg = (spec::kLn2 - 2.0f * dr) - spec::log32(1.0f + u);
      float term = (4.0f * vi.beta_q[k]) * lg;
      E = (k == 0) ? term : E + term;
    }
    oq = in.o * spec::exp32(E);
    for (int i = 0; i < 3; ++i) {
      float acc = vi.W3[i][0] * delta[0];
      for (int k = 1; k < C; ++k) acc = acc + vi.W3[i][k] * delta[k];
      shift[i] = acc;
      mc[i] = in.mx[i] + acc;
    }
  } else {
    for (int i = 0; i < 3; ++i) mc[i] = in.mx[i];
  }
  cond.oq = oq;
  for (int i = 0; i < 3; ++i) {
    cond.shift[i] = shift[i];
    cond.mc[i] = mc[i];
  }
}

// Whether a conditioned record can be drawn at all: the tests of
// view_project that come before its projection (kernel valid, o(q) at least
// alpha_min, depth beyond the near plane), with the same arithmetic.
UBS_HD bool view_candidate(bool kernel_valid, const ViewCond& c, const ViewDev& v, const CfgDev& cfg) {
  const float* Rv = v.R;
  const float tz = ((Rv[6] * c.mc[0] + Rv[7] * c.mc[1]) + Rv[8] * c.mc[2]) + v.t[2];
  return kernel_valid && (tz > cfg.near_plane) && (c.oq >= cfg.amin);
}

// The projection of a conditioned record (Sec. 3, EWA splatting of the Beta
// kernel): depth, screen mean, conic, tight support radius and tile
// rectangle, and the error-free screen mean.  mx: the primitive's spatial
// mean; Sc, beta_x, kernel_valid: its view-independent covariance, spatial
// exponent and validity.
UBS_HD void view_project(const float* mx, const float* Sc, float beta_x, bool kernel_valid, const ViewCond& c,
                         const ViewDev& v, const CfgDev& cfg, ViewOut& out) {
  const float* Rv = v.R;
  const float* mc = c.mc;
  const float* shift = c.shift;
  const float oq = c.oq;
  float tc[3];
  for (int j = 0; j < 3; ++j) tc[j] = ((Rv[3 * j] * mc[0] + Rv[3 * j + 1] * mc[1]) + Rv[3 * j + 2] * mc[2]) + v.t[j];
  const float tz = tc[2];
  bool valid = kernel_valid && (tz > cfg.near_plane);
  const float tzs = valid ? tz : 1.0f;
  const float u = tc[0] / tzs;
  const float vq = tc[1] / tzs;
  const float mux = v.fx * u + v.cx;
  const float muy = v.fy * vq + v.cy;
  const float limx = cfg.clip * ((0.5f * (float)v.W) / v.fx);
  const float limy = cfg.clip * ((0.5f * (float)v.H) / v.fy);
  const float uc = fminf(fmaxf(u, -limx), limx);
  const float vc = fminf(fmaxf(vq, -limy), limy);
  const float J00 = v.fx / tzs;
  const float J02 = -((v.fx * uc) / tzs);
  const float J11 = v.fy / tzs;
  const float J12 = -((v.fy * vc) / tzs);
  float T[2][3];
  for (int j = 0; j < 3; ++j) {
    T[0][j] = J00 * Rv[j] + J02 * Rv[6 + j];
    T[1][j] = J11 * Rv[3 + j] + J12 * Rv[6 + j];
  }
  const float* S = Sc;
  float U[2][3];
  for (int a = 0; a < 2; ++a)
    for (int j = 0; j < 3; ++j)
      U[a][j] = (T[a][0] * S[sym(0, j)] + T[a][1] * S[sym(1, j)]) + T[a][2] * S[sym(2, j)];
  const float s00 = ((U[0][0] * T[0][0] + U[0][1] * T[0][1]) + U[0][2] * T[0][2]) + cfg.eps;
  const float s01 = (U[0][0] * T[1][0] + U[0][1] * T[1][1]) + U[0][2] * T[1][2];
  const float s11 = ((U[1][0] * T[1][0] + U[1][1] * T[1][1]) + U[1][2] * T[1][2]) + cfg.eps;
  const float det = s00 * s11 - s01 * s01;
  valid = valid && (det > 0.0f);
  const float dets = valid ? det : 1.0f;
  out.conic[0] = s11 / dets;
  out.conic[1] = -(s01 / dets);
  out.conic[2] = s00 / dets;
  valid = valid && (oq >= cfg.amin);
  float rcut = 1.0f;
  if (cfg.flags & 1) {
    const float oqs = valid ? oq : 1.0f;
    const float lr = spec::log32(cfg.amin / oqs);
    rcut = 1.0f - spec::exp32(lr / beta_x);
  }
  const float ex = sqrtf(fmaxf(rcut * s00, 0.0f));
  const float ey = sqrtf(fmaxf(rcut * s11, 0.0f));
  const float exm = ex * spec::kMargR + spec::kMargA;
  const float eym = ey * spec::kMargR + spec::kMargA;
  float px0 = ceilf((mux - exm) - 0.5f);
  float px1 = floorf((mux + exm) - 0.5f);
  float py0 = ceilf((muy - eym) - 0.5f);
  float py1 = floorf((muy + eym) - 0.5f);
  px0 = fmaxf(px0, 0.0f);
  py0 = fmaxf(py0, 0.0f);
  px1 = fminf(px1, (float)(v.W - 1));
  py1 = fminf(py1, (float)(v.H - 1));
  valid = valid && (px0 <= px1) && (py0 <= py1);
  out.valid = valid;
  out.depth = tz;
  out.oq = oq;
  if (valid) {
    const int ix0 = (int)px0, ix1 = (int)px1, iy0 = (int)py0, iy1 = (int)py1;
    out.tx0 = ix0 / cfg.tw;
    out.tx1 = ix1 / cfg.tw + 1;
    out.ty0 = iy0 / cfg.th;
    out.ty1 = iy1 / cfg.th + 1;
    out.tiles = (uint32_t)((out.tx1 - out.tx0) * (out.ty1 - out.ty0));
  } else {
    out.tx0 = out.tx1 = out.ty0 = out.ty1 = 0;
    out.tiles = 0;
  }
  // error-free screen mean: m = mx + shift exactly, t = Rv m + t, mu' = f t/t_z + c
  DF m[3];
  for (int i = 0; i < 3; ++i) m[i] = two_sum(mx[i], shift[i]);
  DF t3[3];
  for (int j = 0; j < 3; ++j) {
    DF acc = {v.t[j], 0.0f};
    for (int i = 0; i < 3; ++i) {
      DF p = two_prod(Rv[3 * j + i], m[i].hi);
      p.lo = fmaf(Rv[3 * j + i], m[i].lo, p.lo);
      acc = df_add(acc, p);
    }
    t3[j] = acc;
  }
  if (!(t3[2].hi > 0.0f)) t3[2] = DF{1.0f, 0.0f};
  DF uu = df_div(t3[0], t3[2]);
  DF vv2 = df_div(t3[1], t3[2]);
  DF mx2 = df_add(df_mul_f(uu, v.fx), DF{v.cx, 0.0f});
  DF my2 = df_add(df_mul_f(vv2, v.fy), DF{v.cy, 0.0f});
  out.mu_hi[0] = mx2.hi;
  out.mu_lo[0] = mx2.lo;
  out.mu_hi[1] = my2.hi;
  out.mu_lo[1] = my2.lo;
}

template <int C>
UBS_HD void view_stage(const PrimIn<C>& in, const PrimVI<C>& vi, const ViewDev& v, const CfgDev& cfg,
                       ViewOut& out) {
  ViewCond c;
  view_condition<C>(in, vi, v, c);
  view_project(in.mx, vi.Sc, vi.beta_x, vi.valid, c, v, cfg, out);
}

}  // namespace ubs
