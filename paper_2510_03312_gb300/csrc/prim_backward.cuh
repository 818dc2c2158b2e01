// prim_backward.cuh -- G2: reverse-mode derivative of the preprocess step.
//
// Input per (view, primitive) record: the gradient of the loss with respect
// to the record's screen quantities, as accumulated by the backward blend:
//   g[0..1] d mu'            g[2..4] d (a, b, c) of the conic, with
//                             r = a dx^2 + 2 b dx dy + c dy^2
//   g[5]    d log2 o(q)      g[6]    d beta_x      g[7..9] d rgb
// Output: gradients with respect to the parameters of Sec. 4.2-4.3 (mu_x,
// mu_q, rotation, s_x, L_qx, L_q, b, o, rgb), summed over the views.
//
// The forward quantities are recomputed in float32 (contractions allowed);
// the chain follows the forward of prim_forward.cuh step by step:
//   conic = Sigma'^{-1}          dSigma' = -K dK K (K with off-diagonal b)
//   Sigma' = T S T^T + eps I     dT = 2 dSigma' T S,  dS += T^T dSigma' T
//   T = J W                      dJ = dT W^T
//   J = [[fx/z, 0, -fx u~/z], [0, fy/z, -fy v~/z]], u~ = clamp(x/z)
//   mu' = f (x, y)/z + c
//   t = W mu_{x|q} + t_v
//   mu_{x|q} = mu_x + W3 delta, W3 = Sigma_xq Sigma_q^{-1} diag(beta~)
//   o(q) = o exp(sum_k 4 beta_qk log(1 - tanh(y_k^2))), L^ y = delta
//   S = Sigma_x - sym(W3 Sigma_qx)
//   Z = Sigma_q^{-1} Sigma_qx      dSigma_qx += Sigma_q^{-1} dZ,
//                                  dSigma_q -= (Sigma_q^{-1} dZ) Z^T
//   L^ = chol(Sigma_q)             dSigma_q += L^{-T} Phi(L^T dL^) L^{-1}
//                                  (Phi: lower triangle, halved diagonal)
//   Sigma_q = L_qx L_qx^T + L_q L_q^T,  Sigma_qx = L_qx M^T,  Sigma_x = M M^T,
//   M = R diag(s_x), R from the normalised quaternion or from A(omega):
//   I + A, I + A + A^2/2, the Cayley transform (I - A)^-1 (I + A) or exp(A).
#pragma once

#include "prim_forward.cuh"

namespace ubs {

template <int C>
struct PrimAcc {
  float gmx[3];
  float gmq[CDim<C>::M];
  float gS[3][3];
  float gW3[3][CDim<C>::M];
  float gLh[CDim<C>::M][CDim<C>::M];
  float go;
  float gbq[CDim<C>::M];
  float gbx;
  float grgb[3];
};

template <int C>
UBS_HD void acc_zero(PrimAcc<C>& a) {
  float* p = (float*)&a;
  for (unsigned i = 0; i < sizeof(PrimAcc<C>) / sizeof(float); ++i) p[i] = 0.0f;
}

// Accumulate the contribution of one view's screen-space gradient g[10].
template <int C>
UBS_HD void prim_backward_view(const PrimIn<C>& in, const PrimVI<C>& vi, const ViewDev& v, const CfgDev& cfg,
                               const float* g, PrimAcc<C>& acc) {
  const float* Rv = v.R;
  float mc[3];
  float oq = in.o;
  float delta[CDim<C>::M], y[CDim<C>::M], uk[CDim<C>::M], lg[CDim<C>::M], d3[3] = {0.f, 0.f, 0.f};
  float nrm = 1.0f, eE = 1.0f;
  if constexpr (C > 0) {
    float q[CDim<C>::M];
    int qi = 0;
    if constexpr (C == 1 || C == 4) q[qi++] = v.time;
    if constexpr (C >= 3) {
      float cam[3], vv[3];
      for (int i = 0; i < 3; ++i) cam[i] = -(Rv[i] * v.t[0] + Rv[3 + i] * v.t[1] + Rv[6 + i] * v.t[2]);
      for (int i = 0; i < 3; ++i) vv[i] = in.mx[i] - cam[i];
      nrm = sqrtf(vv[0] * vv[0] + vv[1] * vv[1] + vv[2] * vv[2]);
      for (int i = 0; i < 3; ++i) {
        d3[i] = vv[i] / nrm;
        q[qi++] = d3[i];
      }
    }
    for (int k = 0; k < C; ++k) delta[k] = q[k] - in.mq[k];
    for (int k = 0; k < C; ++k) {
      float a = delta[k];
      for (int m = 0; m < k; ++m) a -= vi.Lh[tri(k, m)] * y[m];
      y[k] = a / vi.Lh[tri(k, k)];
    }
    float E = 0.0f;
    for (int k = 0; k < C; ++k) {
      const float dr = y[k] * y[k];
      uk[k] = expf(-2.0f * dr);
      lg[k] = (kLn2f - 2.0f * dr) - log1pf(uk[k]);
      E += 4.0f * vi.beta_q[k] * lg[k];
    }
    eE = expf(E);
    oq = in.o * eE;
    for (int i = 0; i < 3; ++i) {
      float a = 0.0f;
      for (int k = 0; k < C; ++k) a += vi.W3[i][k] * delta[k];
      mc[i] = in.mx[i] + a;
    }
  } else {
    for (int i = 0; i < 3; ++i) mc[i] = in.mx[i];
  }
  float tc[3];
  for (int j = 0; j < 3; ++j) tc[j] = Rv[3 * j] * mc[0] + Rv[3 * j + 1] * mc[1] + Rv[3 * j + 2] * mc[2] + v.t[j];
  const float tz = tc[2], iz = 1.0f / tz;
  const float u = tc[0] * iz, vq = tc[1] * iz;
  const float limx = cfg.clip * ((0.5f * (float)v.W) / v.fx);
  const float limy = cfg.clip * ((0.5f * (float)v.H) / v.fy);
  const bool inx = u >= -limx && u <= limx, iny = vq >= -limy && vq <= limy;
  const float uc = fminf(fmaxf(u, -limx), limx), vc = fminf(fmaxf(vq, -limy), limy);
  const float J00 = v.fx * iz, J02 = -v.fx * uc * iz, J11 = v.fy * iz, J12 = -v.fy * vc * iz;
  float T[2][3];
  for (int j = 0; j < 3; ++j) {
    T[0][j] = J00 * Rv[j] + J02 * Rv[6 + j];
    T[1][j] = J11 * Rv[3 + j] + J12 * Rv[6 + j];
  }
  float S[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) S[i][j] = vi.Sc[sym(i, j)];
  float A[2][3];  // T S
  for (int a = 0; a < 2; ++a)
    for (int j = 0; j < 3; ++j) A[a][j] = T[a][0] * S[0][j] + T[a][1] * S[1][j] + T[a][2] * S[2][j];
  const float s00 = A[0][0] * T[0][0] + A[0][1] * T[0][1] + A[0][2] * T[0][2] + cfg.eps;
  const float s01 = A[0][0] * T[1][0] + A[0][1] * T[1][1] + A[0][2] * T[1][2];
  const float s11 = A[1][0] * T[1][0] + A[1][1] * T[1][1] + A[1][2] * T[1][2] + cfg.eps;
  const float idet = 1.0f / (s00 * s11 - s01 * s01);
  const float K[2][2] = {{s11 * idet, -s01 * idet}, {-s01 * idet, s00 * idet}};
  // conic -> Sigma'
  const float gK[2][2] = {{g[2], 0.5f * g[3]}, {0.5f * g[3], g[4]}};
  float M1[2][2], gSp[2][2];
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 2; ++b) M1[a][b] = K[a][0] * gK[0][b] + K[a][1] * gK[1][b];
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 2; ++b) gSp[a][b] = -(M1[a][0] * K[0][b] + M1[a][1] * K[1][b]);
  // Sigma' = T S T^T + eps I
  float gT[2][3];
  for (int a = 0; a < 2; ++a)
    for (int j = 0; j < 3; ++j) gT[a][j] = 2.0f * (gSp[a][0] * A[0][j] + gSp[a][1] * A[1][j]);
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      float s = 0.0f;
      for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) s += T[a][i] * gSp[a][b] * T[b][j];
      acc.gS[i][j] += s;
    }
  // T = J W
  float gJ00 = 0.f, gJ02 = 0.f, gJ11 = 0.f, gJ12 = 0.f;
  for (int j = 0; j < 3; ++j) {
    gJ00 += gT[0][j] * Rv[j];
    gJ02 += gT[0][j] * Rv[6 + j];
    gJ11 += gT[1][j] * Rv[3 + j];
    gJ12 += gT[1][j] * Rv[6 + j];
  }
  float gtz = (-(gJ00 * v.fx + gJ11 * v.fy) + gJ02 * v.fx * uc + gJ12 * v.fy * vc) * iz * iz;
  const float gu = g[0] * v.fx + (inx ? -gJ02 * v.fx * iz : 0.0f);
  const float gv = g[1] * v.fy + (iny ? -gJ12 * v.fy * iz : 0.0f);
  const float gt[3] = {gu * iz, gv * iz, gtz - (gu * tc[0] + gv * tc[1]) * iz * iz};
  float gmc[3];
  for (int i = 0; i < 3; ++i) gmc[i] = Rv[i] * gt[0] + Rv[3 + i] * gt[1] + Rv[6 + i] * gt[2];
  for (int i = 0; i < 3; ++i) {
    acc.grgb[i] += g[7 + i];
    acc.gmx[i] += gmc[i];
  }
  acc.gbx += g[6];
  const float goq = oq > 0.0f ? g[5] / (oq * kLn2f) : 0.0f;
  if constexpr (C == 0) {
    acc.go += goq;
  } else {
    float gdelta[CDim<C>::M];
    for (int k = 0; k < C; ++k) {
      float s = 0.0f;
      for (int i = 0; i < 3; ++i) {
        acc.gW3[i][k] += gmc[i] * delta[k];
        s += vi.W3[i][k] * gmc[i];
      }
      gdelta[k] = s;
    }
    acc.go += goq * eE;
    const float gE = goq * oq;
    float gy[CDim<C>::M];
    for (int k = 0; k < C; ++k) {
      acc.gbq[k] += gE * 4.0f * lg[k];
      const float glg = gE * 4.0f * vi.beta_q[k];
      const float gdr = -glg * 2.0f / (1.0f + uk[k]);
      gy[k] = 2.0f * y[k] * gdr;
    }
    // L^ y = delta  ->  w = L^{-T} gy;  d delta += w;  dL^_ij -= w_i y_j
    float w[CDim<C>::M];
    for (int k = C - 1; k >= 0; --k) {
      float a = gy[k];
      for (int m = k + 1; m < C; ++m) a -= vi.Lh[tri(m, k)] * w[m];
      w[k] = a / vi.Lh[tri(k, k)];
    }
    for (int i = 0; i < C; ++i) {
      gdelta[i] += w[i];
      for (int j = 0; j <= i; ++j) acc.gLh[i][j] -= w[i] * y[j];
    }
    for (int k = 0; k < C; ++k) acc.gmq[k] -= gdelta[k];
    if constexpr (C >= 3) {
      const int off = (C == 4) ? 1 : 0;
      const float gd[3] = {gdelta[off], gdelta[off + 1], gdelta[off + 2]};
      const float dd = d3[0] * gd[0] + d3[1] * gd[1] + d3[2] * gd[2];
      for (int i = 0; i < 3; ++i) acc.gmx[i] += (gd[i] - d3[i] * dd) / nrm;
    }
  }
}

// Output gradient of one primitive, same plane order as the parameters.
template <int C>
struct PrimGrad {
  float mx[3];
  float mq[CDim<C>::M];
  float rot[4];
  float s[3];
  float lqx[3 * CDim<C>::M];
  float lq[CDim<C>::T];
  float b[1 + C];
  float o;
  float rgb[3];
};

template <int C>
UBS_HD void prim_backward_final(const PrimIn<C>& in, const PrimVI<C>& vi, int rot_mode, PrimAcc<C>& acc,
                                PrimGrad<C>& out) {
  float gM[3][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
  const float* M = vi.M;
  // gS is symmetric; Sigma_x receives it whole
  float gSx[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) gSx[i][j] = acc.gS[i][j];
  if constexpr (C > 0) {
    // S = Sigma_x - 1/2 (M2 + M2^T), M2 = W3 Sigma_qx  ->  dM2 = -dS
    float gSqx[CDim<C>::M][3];
    for (int k = 0; k < C; ++k)
      for (int j = 0; j < 3; ++j) {
        float s = 0.0f;
        for (int i = 0; i < 3; ++i) s -= vi.W3[i][k] * acc.gS[i][j];
        gSqx[k][j] = s;
      }
    for (int i = 0; i < 3; ++i)
      for (int k = 0; k < C; ++k) {
        float s = 0.0f;
        for (int j = 0; j < 3; ++j) s -= acc.gS[i][j] * vi.Sqx[k][j];
        acc.gW3[i][k] += s;
      }
    // W3 = Z^T diag(beta~)
    float gZ[CDim<C>::M][3];
    for (int k = 0; k < C; ++k) {
      float gbt = 0.0f;
      for (int i = 0; i < 3; ++i) {
        gZ[k][i] = acc.gW3[i][k] * vi.beta_t[k];
        gbt += acc.gW3[i][k] * vi.Z[k][i];
      }
      if (vi.beta_q[k] <= 1.0f) acc.gbq[k] += gbt;
      out.b[1 + k] = acc.gbq[k] * vi.beta_q[k];
    }
    // inverse of L^ (lower triangular)
    float Li[CDim<C>::M][CDim<C>::M];
    for (int i = 0; i < C; ++i)
      for (int j = 0; j < C; ++j) Li[i][j] = 0.0f;
    for (int j = 0; j < C; ++j) {
      Li[j][j] = 1.0f / vi.Lh[tri(j, j)];
      for (int i = j + 1; i < C; ++i) {
        float s = 0.0f;
        for (int m = j; m < i; ++m) s += vi.Lh[tri(i, m)] * Li[m][j];
        Li[i][j] = -s / vi.Lh[tri(i, i)];
      }
    }
    // Z = Sigma_q^{-1} Sigma_qx: Wz = Sigma_q^{-1} gZ = Li^T Li gZ
    float gSq[CDim<C>::M][CDim<C>::M];
    {
      float t1[CDim<C>::M][3], Wz[CDim<C>::M][3];
      for (int i = 0; i < C; ++i)
        for (int j = 0; j < 3; ++j) {
          float s = 0.0f;
          for (int m = 0; m <= i; ++m) s += Li[i][m] * gZ[m][j];
          t1[i][j] = s;
        }
      for (int i = 0; i < C; ++i)
        for (int j = 0; j < 3; ++j) {
          float s = 0.0f;
          for (int m = i; m < C; ++m) s += Li[m][i] * t1[m][j];
          Wz[i][j] = s;
        }
      for (int k = 0; k < C; ++k)
        for (int j = 0; j < 3; ++j) gSqx[k][j] += Wz[k][j];
      for (int a = 0; a < C; ++a)
        for (int b = 0; b < C; ++b) {
          float s = 0.0f;
          for (int j = 0; j < 3; ++j) s -= Wz[a][j] * vi.Z[b][j];
          gSq[a][b] = s;
        }
    }
    // Cholesky: dSigma_q += Li^T Phi(L^T gL) Li
    {
      float X[CDim<C>::M][CDim<C>::M];
      for (int i = 0; i < C; ++i)
        for (int j = 0; j < C; ++j) {
          float s = 0.0f;
          for (int m = 0; m < C; ++m) {
            const float Lmi = m >= i ? vi.Lh[tri(m, i)] : 0.0f;
            const float gmj = j <= m ? acc.gLh[m][j] : 0.0f;
            s += Lmi * gmj;
          }
          X[i][j] = (j < i) ? s : (j == i ? 0.5f * s : 0.0f);
        }
      float Y[CDim<C>::M][CDim<C>::M];  // Phi Li
      for (int i = 0; i < C; ++i)
        for (int j = 0; j < C; ++j) {
          float s = 0.0f;
          for (int m = 0; m < C; ++m) s += X[i][m] * Li[m][j];
          Y[i][j] = s;
        }
      for (int i = 0; i < C; ++i)
        for (int j = 0; j < C; ++j) {
          float s = 0.0f;
          for (int m = 0; m < C; ++m) s += Li[m][i] * Y[m][j];
          gSq[i][j] += s;
        }
    }
    // Sigma_q = L_qx L_qx^T + L_q L_q^T  (G = gSq + gSq^T)
    const float* Lqx = in.lqx;
    for (int k = 0; k < C; ++k)
      for (int j = 0; j < 3; ++j) {
        float s = 0.0f;
        for (int m = 0; m < C; ++m) s += (gSq[k][m] + gSq[m][k]) * Lqx[3 * m + j];
        out.lqx[3 * k + j] = s;
      }
    for (int i = 0; i < C; ++i)
      for (int j = 0; j <= i; ++j) {
        float s = 0.0f;
        for (int m = j; m < C; ++m) s += (gSq[i][m] + gSq[m][i]) * in.lq[tri(m, j)];
        out.lq[tri(i, j)] = s;
      }
    // Sigma_qx[k][i] = sum_j M[i][j] L_qx[k][j]
    for (int k = 0; k < C; ++k)
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
          gM[i][j] += gSqx[k][i] * Lqx[3 * k + j];
          out.lqx[3 * k + j] += gSqx[k][i] * M[3 * i + j];
        }
    for (int k = 0; k < C; ++k) out.mq[k] = acc.gmq[k];
  }
  // Sigma_x = M M^T  ->  dM += 2 gSx M
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      float s = 0.0f;
      for (int m = 0; m < 3; ++m) s += (gSx[i][m] + gSx[m][i]) * M[3 * m + j];
      gM[i][j] += s;
    }
  float gR[9];
  if (rot_mode == 4) {
    // the plain Cholesky row: M is the factor (diagonal s_x, strictly-lower rot)
    for (int j = 0; j < 3; ++j) out.s[j] = gM[j][j];
    out.rot[0] = gM[1][0];
    out.rot[1] = gM[2][0];
    out.rot[2] = gM[2][1];
    out.rot[3] = 0.0f;
  } else {
    for (int j = 0; j < 3; ++j) {
      float s = 0.0f;
      for (int i = 0; i < 3; ++i) {
        gR[3 * i + j] = gM[i][j] * in.s[j];
        s += gM[i][j] * vi.R[3 * i + j];
      }
      out.s[j] = s;
    }
  }
  if (rot_mode == 0) {
    const float qw = in.rot[0], qx = in.rot[1], qy = in.rot[2], qz = in.rot[3];
    const float n = sqrtf(qw * qw + qx * qx + qy * qy + qz * qz);
    const float w = qw / n, x = qx / n, y = qy / n, z = qz / n;
    const float gw = 2.0f * (-z * gR[1] + y * gR[2] + z * gR[3] - x * gR[5] - y * gR[6] + x * gR[7]);
    const float gx = 2.0f * (y * gR[1] + z * gR[2] + y * gR[3] - w * gR[5] + z * gR[6] + w * gR[7]) -
                     4.0f * x * (gR[4] + gR[8]);
    const float gy = 2.0f * (x * gR[1] + w * gR[2] + x * gR[3] + z * gR[5] - w * gR[6] + z * gR[7]) -
                     4.0f * y * (gR[0] + gR[8]);
    const float gz = 2.0f * (-w * gR[1] + x * gR[2] + w * gR[3] + y * gR[5] + x * gR[6] + y * gR[7]) -
                     4.0f * z * (gR[0] + gR[4]);
    const float dot = w * gw + x * gx + y * gy + z * gz;
    out.rot[0] = (gw - w * dot) / n;
    out.rot[1] = (gx - x * dot) / n;
    out.rot[2] = (gy - y * dot) / n;
    out.rot[3] = (gz - z * dot) / n;
  } else if (rot_mode != 4) {
    // through A(omega): L_k = sum_ij gR_ij dA_ij/domega_k
    const float L[3] = {gR[7] - gR[5], gR[2] - gR[6], gR[3] - gR[1]};
    if (rot_mode == 1) {
      for (int k = 0; k < 3; ++k) out.rot[k] = L[k];
    } else {
      // R = I + l A + k A^2: through A^2, Q_k = sum_ij gR_ij d(A^2)_ij/domega_k
      //   = (gR o)_k + (gR^T o)_k - 2 o_k tr(gR)
      const float o[3] = {in.rot[0], in.rot[1], in.rot[2]};
      const float tr = gR[0] + gR[4] + gR[8];
      float Q[3];
      for (int k = 0; k < 3; ++k)
        Q[k] = (gR[3 * k] * o[0] + gR[3 * k + 1] * o[1] + gR[3 * k + 2] * o[2]) +
               (gR[k] * o[0] + gR[3 + k] * o[1] + gR[6 + k] * o[2]) - 2.0f * o[k] * tr;
      // l, k and their derivatives in n = |o|^2: grad_k = l L_k + k Q_k +
      // 2 o_k (l' <gR, A> + k' <gR, A^2>), <gR, A> = sum_k o_k L_k and
      // <gR, A^2> = o^T gR o - n tr(gR)
      const float n = o[0] * o[0] + o[1] * o[1] + o[2] * o[2];
      float l, kk, dl, dk;
      if (rot_mode == 2) {  // second-order Taylor
        l = 1.0f;
        kk = 0.5f;
        dl = dk = 0.0f;
      } else if (rot_mode == 3) {  // Cayley: l = k = 2 / (1 + n), derivative -l^2 / 2
        l = kk = 2.0f / (1.0f + n);
        dl = dk = -0.5f * l * l;
      } else if (n < 0.25f) {  // exp A, Taylor series in n
        l = 1.0f + n * (spec::kInv3 + n * (spec::kInv5 + n * (spec::kInv7 + n * spec::kInv9)));
        kk = 0.5f + n * (-spec::kInv4 + n * (-spec::kInv6 + n * (-spec::kInv8 + n * -spec::kInv10)));
        dl = spec::kInv3 + n * (2.0f * spec::kInv5 + n * (3.0f * spec::kInv7 + n * 4.0f * spec::kInv9));
        dk = -spec::kInv4 + n * (-2.0f * spec::kInv6 + n * (-3.0f * spec::kInv8 + n * -4.0f * spec::kInv10));
      } else {  // exp A: l = sin t / t, k = (1 - cos t) / n, l' = (cos t - l) / (2n), k' = (l/2 - k) / n
        const float t = sqrtf(n);
        float s, c;
        spec::sincos32(t, &s, &c);
        l = s / t;
        kk = (1.0f - c) / n;
        dl = (c - l) / (2.0f * n);
        dk = (0.5f * l - kk) / n;
      }
      float oGo = 0.0f;
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) oGo += o[i] * gR[3 * i + j] * o[j];
      const float inA = o[0] * L[0] + o[1] * L[1] + o[2] * L[2];
      const float inA2 = oGo - n * tr;
      for (int k = 0; k < 3; ++k) out.rot[k] = l * L[k] + kk * Q[k] + 2.0f * o[k] * (dl * inA + dk * inA2);
    }
    out.rot[3] = 0.0f;
  }
  for (int i = 0; i < 3; ++i) {
    out.mx[i] = acc.gmx[i];
    out.rgb[i] = acc.grgb[i];
  }
  out.o = acc.go;
  out.b[0] = acc.gbx * vi.beta_x;
}

}  // namespace ubs
