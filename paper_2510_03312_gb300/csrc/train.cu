// train.cu -- the training step around the rasterizer: the image loss of
// Sec. 4.5 with its gradient (ubs_image_loss) and the optimiser step of
// Sec. 5.1 fused with the activations, penalties and noise of Sec. 4.5
// (ubs_adam_step).
//
// Image loss, per view, L = (1 - lambda) L1 + lambda (1 - SSIM): L1 the mean
// |x - y| over pixels and channels, SSIM the mean map of Wang et al. (2004)
// per channel under an 11 x 11 Gaussian window (sigma 1.5), zero-padded.
// With the window statistics mu_x = G * x, E_xx = G * x^2, E_xy = G * (x y)
// (and the same for y), the map is
//   S = A B / (Cc D),  A = 2 mu_x mu_y + C1,  B = 2 (E_xy - mu_x mu_y) + C2,
//   Cc = mu_x^2 + mu_y^2 + C1,  D = (E_xx - mu_x^2) + (E_yy - mu_y^2) + C2,
// and its gradient with respect to x at pixel q gathers, over the output
// pixels p whose window covers q,
//   dS/dx(q) = sum_p G(p - q) [S_mu(p) + 2 x(q) S_xx(p) + y(q) S_xy(p)]
// with S_mu = dS/dmu_x (through A, B, Cc, D), S_xx = dS/dE_xx = dS/dD and
// S_xy = dS/dE_xy = 2 dS/dB.  G is symmetric and separable, so both passes
// are two 1-D convolutions (rows, then columns) over a shared-memory tile
// of 32 x 32 outputs with a 5-pixel halo, each thread computing four
// neighbouring outputs of a pass from registers (the row pass reads five
// aligned 16-byte words per plane for four outputs, the column pass 14
// values per statistic for four), so that the passes are not bound by
// shared-memory loads:
//   ssim_fwd_kernel   the five window statistics, S, the three partials
//                     (to the workspace) and per-block sums of S and |x - y|
//   ssim_bwd_kernel   the three partials convolved back, combined with the
//                     L1 term into dL/dimage
//   loss_reduce_kernel  per-view and total losses from the block sums, in a
//                     fixed order (deterministic).
//
// Adam (Kingma and Ba 2015) runs one thread per four parameters of a plane
// (float4 loads and stores where the plane stride allows), reading raw, grad,
// m, v and writing raw, m, v and the activated value the rasterizer reads:
// 32 bytes of traffic per parameter.
#include <math.h>
#include <string.h>

#include "ubs.h"
#include "kernels.cuh"

namespace ubs {
namespace {

constexpr int kLossMaxViews = 256;
constexpr int kWin = 11, kRad = 5;
constexpr int kTX = 32, kTY = 32;   // output tile
constexpr int kHY = kTY + 2 * kRad; // halo rows
constexpr int kCOff = 8;            // shared-memory column of tile column 0
constexpr int kSW = kCOff + kTX + 8;  // shared-memory row: tile columns -8 .. 39
constexpr int kLossThreads = 256;
constexpr float kC1 = 0.0001f, kC2 = 0.0009f;  // (0.01)^2, (0.03)^2

struct LossView {
  int32_t W, H, tiles_x, tiles;  // tiles: per channel
  uint32_t pix_off, blk_off;     // first pixel, first block of the view
};
struct LossParams {
  LossView v[kLossMaxViews];
  float2 g2[kWin];     // 1-D window (g_k, g_k), sums to 1
  int32_t n;           // views
  uint32_t n_blocks;   // blocks of the two convolution kernels
  float lam;           // lambda_SSIM
  float inv_views;     // 1 / n
  uint64_t plane;      // floats in one partial plane (3 * all pixels)
};

inline size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }

// the view owning block b: the last view whose first block is <= b
__device__ __forceinline__ int loss_view_of(const LossParams& P, uint32_t b) {
  int lo = 0, hi = P.n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (P.v[mid].blk_off <= b) lo = mid; else hi = mid - 1;
  }
  return lo;
}

struct TileAt {
  int v, ch, gx0, gy0;  // view, channel, first output pixel
  size_t base;          // float offset of the channel plane in the packed images
};
__device__ __forceinline__ TileAt tile_at(const LossParams& P, int v) {
  const LossView& w = P.v[v];
  const uint32_t lb = blockIdx.x - w.blk_off;
  TileAt t;
  t.v = v;
  t.ch = lb / w.tiles;
  const uint32_t ti = lb % w.tiles;
  t.gx0 = (ti % w.tiles_x) * kTX;
  t.gy0 = (ti / w.tiles_x) * kTY;
  t.base = (size_t)w.pix_off * 3 + (size_t)t.ch * w.W * w.H;
  return t;
}

// 4-byte asynchronous copy global -> shared (sm_80 and later); with
// valid == false it writes zero and reads nothing (src-size 0), src then only
// has to be some mapped address.
__device__ __forceinline__ void cp_async4(void* dst, const float* src, bool valid) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(d), "l"(src), "r"(valid ? 4 : 0) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Fills the tile with its halo (rows -5 .. 36, columns -8 .. 39 of the tile)
// in shared memory, zero outside the image, with asynchronous copies: one
// warp per row, each lane two columns, every copy of the thread in flight
// before it waits.  copy(r, c, offset, in) issues the copies of one element
// (offset: of the pixel within its plane set; clamped to the tile's first
// pixel when !in).
template <typename Copy>
__device__ __forceinline__ void load_halo(const TileAt& t, int W, int H, Copy copy) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int gxa = t.gx0 - kCOff + lane, gxb = gxa + 32;
  const bool ca = gxa >= 0 && gxa < W, cb = lane < kSW - 32 && gxb >= 0 && gxb < W;
  constexpr int kRows = (kHY + kLossThreads / 32 - 1) / (kLossThreads / 32);
#pragma unroll
  for (int i = 0; i < kRows; ++i) {
    const int r = warp + i * (kLossThreads / 32);
    if (r < kHY) {
      const int gy = t.gy0 - kRad + r;
      const bool ry = gy >= 0 && gy < H;
      const size_t row = t.base + (size_t)(ry ? gy : t.gy0) * W;
      copy(r, lane, row + (ry && ca ? gxa : t.gx0), ry && ca);
      if (lane < kSW - 32) copy(r, lane + 32, row + (ry && cb ? gxb : t.gx0), ry && cb);
    }
  }
  cp_async_wait_all();
}

// Row pass over one halo row r: the 11-tap window sums at output columns c0
// and c0 + 1 (tile coordinates), from the 16-byte words of shared columns
// c0 + 2 .. c0 + 15 (tile columns c0 - 6 .. c0 + 7).  F receives each loaded
// column with, per output o, its tap k (or -1).
template <typename F>
__device__ __forceinline__ void row_taps(int c0, F f) {
#pragma unroll
  for (int ch = 0; ch < 7; ++ch)
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      const int j = 2 * ch + e;  // tile column c0 - 6 + j
      const int k0 = j - 1, k1 = j - 2;
      f(c0 + 2 + 2 * ch, e, (k0 >= 0 && k0 < kWin) ? k0 : -1, (k1 >= 0 && k1 < kWin) ? k1 : -1);
    }
}

__global__ void __launch_bounds__(kLossThreads, 5)
    ssim_fwd_kernel(const __grid_constant__ LossParams P, const float* __restrict__ img,
                    const float* __restrict__ tgt, float* __restrict__ part, float2* __restrict__ bsum) {
  wait_prior_grid();
  __shared__ __align__(16) float2 sxy[kHY][kSW];  // (x, y)
  __shared__ __align__(16) float2 hm[kHY][kTX];   // row sums of (x, y)
  __shared__ __align__(16) float2 hq[kHY][kTX];   // row sums of (x^2, y^2)
  __shared__ __align__(16) float hc[kHY][kTX];    // row sums of x y
  __shared__ float red[2][kLossThreads / 32];
  __shared__ int s_v;
  if (threadIdx.x == 0) s_v = loss_view_of(P, blockIdx.x);
  __syncthreads();
  const TileAt t = tile_at(P, s_v);
  const int W = P.v[t.v].W, H = P.v[t.v].H;
  load_halo(t, W, H, [&](int r, int c, size_t o, bool in) {
    cp_async4(&sxy[r][c].x, img + o, in);
    cp_async4(&sxy[r][c].y, tgt + o, in);
  });
  __syncthreads();
  // rows: two output columns per work item, (x, y) and (x^2, y^2) in packed pairs
  for (int it = threadIdx.x; it < kHY * (kTX / 2); it += kLossThreads) {
    const int r = it / (kTX / 2), c0 = 2 * (it % (kTX / 2));
    float2 m0 = make_float2(0.0f, 0.0f), m1 = m0, q0 = m0, q1 = m0;
    float x0 = 0.0f, x1 = 0.0f;
    float4 w = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    row_taps(c0, [&](int col, int e, int k0, int k1) {
      if (e == 0) w = *reinterpret_cast<const float4*>(&sxy[r][col]);
      const float2 v = e == 0 ? make_float2(w.x, w.y) : make_float2(w.z, w.w);
      const float2 sq = mul2(v, v);
      const float cr = v.x * v.y;
      if (k0 >= 0) {
        m0 = fma2(P.g2[k0], v, m0);
        q0 = fma2(P.g2[k0], sq, q0);
        x0 = fmaf(P.g2[k0].x, cr, x0);
      }
      if (k1 >= 0) {
        m1 = fma2(P.g2[k1], v, m1);
        q1 = fma2(P.g2[k1], sq, q1);
        x1 = fmaf(P.g2[k1].x, cr, x1);
      }
    });
    *reinterpret_cast<float4*>(&hm[r][c0]) = make_float4(m0.x, m0.y, m1.x, m1.y);
    *reinterpret_cast<float4*>(&hq[r][c0]) = make_float4(q0.x, q0.y, q1.x, q1.y);
    *reinterpret_cast<float2*>(&hc[r][c0]) = make_float2(x0, x1);
  }
  __syncthreads();
  // columns: four output rows per thread
  const int c = threadIdx.x % kTX, r0 = 4 * (threadIdx.x / kTX);
  float2 am[4], aq[4];
  float ac[4];
#pragma unroll
  for (int o = 0; o < 4; ++o) {
    am[o] = aq[o] = make_float2(0.0f, 0.0f);
    ac[o] = 0.0f;
  }
#pragma unroll
  for (int j = 0; j < kWin + 3; ++j) {
    const float2 m = hm[r0 + j][c], q = hq[r0 + j][c];
    const float x = hc[r0 + j][c];
#pragma unroll
    for (int o = 0; o < 4; ++o) {
      const int k = j - o;
      if (k < 0 || k >= kWin) continue;
      am[o] = fma2(P.g2[k], m, am[o]);
      aq[o] = fma2(P.g2[k], q, aq[o]);
      ac[o] = fmaf(P.g2[k].x, x, ac[o]);
    }
  }
  float ssum = 0.0f, lsum = 0.0f;
  const size_t plane = P.plane;
#pragma unroll
  for (int o = 0; o < 4; ++o) {
    const int r = r0 + o;
    const int gx = t.gx0 + c, gy = t.gy0 + r;
    if (gx >= W || gy >= H) continue;
    const float mx = am[o].x, my = am[o].y, exx = aq[o].x, eyy = aq[o].y, exy = ac[o];
    const float A = 2.0f * mx * my + kC1;
    const float B = 2.0f * (exy - mx * my) + kC2;
    const float Cc = mx * mx + my * my + kC1;
    const float D = (exx - mx * mx) + (eyy - my * my) + kC2;
    const float icd = __fdividef(1.0f, Cc * D);
    const float S = A * B * icd;
    const float dA = B * icd, dB = A * icd, dC = -__fdividef(S, Cc), dD = -__fdividef(S, D);
    // through A (2 mu_y), B (-2 mu_y), Cc (2 mu_x) and D (-2 mu_x)
    const float s_mu = 2.0f * (my * (dA - dB) + mx * (dC - dD));
    const size_t idx = t.base + (size_t)gy * W + gx;
    part[idx] = s_mu;
    part[plane + idx] = dD;
    part[2 * plane + idx] = 2.0f * dB;
    ssum += S;
    const float2 xy = sxy[r + kRad][c + kCOff];
    lsum += fabsf(xy.x - xy.y);
  }
  // block sums (fixed shuffle tree, then the warps in order)
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) {
    ssum += __shfl_xor_sync(0xffffffffu, ssum, d);
    lsum += __shfl_xor_sync(0xffffffffu, lsum, d);
  }
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = ssum;
    red[1][threadIdx.x >> 5] = lsum;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    float a = 0.0f, b = 0.0f;
    for (int w = 0; w < kLossThreads / 32; ++w) {
      a += red[0][w];
      b += red[1][w];
    }
    bsum[blockIdx.x] = make_float2(a, b);
  }
}

__global__ void __launch_bounds__(kLossThreads, 5)
    ssim_bwd_kernel(const __grid_constant__ LossParams P, const float* __restrict__ img,
                    const float* __restrict__ tgt, const float* __restrict__ part, float* __restrict__ dL) {
  wait_prior_grid();
  __shared__ __align__(16) float2 sp[kHY][kSW];  // (S_mu, S_xx)
  __shared__ __align__(16) float sc[kHY][kSW];   // S_xy
  __shared__ __align__(16) float2 hp[kHY][kTX];
  __shared__ __align__(16) float hs[kHY][kTX];
  __shared__ int s_v;
  if (threadIdx.x == 0) s_v = loss_view_of(P, blockIdx.x);
  __syncthreads();
  const TileAt t = tile_at(P, s_v);
  const int W = P.v[t.v].W, H = P.v[t.v].H;
  const size_t plane = P.plane;
  // this thread's four outputs (column c, rows r0 .. r0 + 3): their image and
  // target values are loaded first, to arrive during the passes
  const int c = threadIdx.x % kTX, r0 = 4 * (threadIdx.x / kTX);
  float xo[4], yo[4];
  size_t io[4];
  bool ok[4];
#pragma unroll
  for (int o = 0; o < 4; ++o) {
    const int gx = t.gx0 + c, gy = t.gy0 + r0 + o;
    ok[o] = gx < W && gy < H;
    io[o] = t.base + (size_t)(ok[o] ? gy : 0) * W + (ok[o] ? gx : 0);
    xo[o] = ok[o] ? img[io[o]] : 0.0f;
    yo[o] = ok[o] ? tgt[io[o]] : 0.0f;
  }
  load_halo(t, W, H, [&](int r, int cc, size_t o, bool in) {
    cp_async4(&sp[r][cc].x, part + o, in);
    cp_async4(&sp[r][cc].y, part + plane + o, in);
    cp_async4(&sc[r][cc], part + 2 * plane + o, in);
  });
  __syncthreads();
  for (int it = threadIdx.x; it < kHY * (kTX / 2); it += kLossThreads) {
    const int r = it / (kTX / 2), c0 = 2 * (it % (kTX / 2));
    float2 a0 = make_float2(0.0f, 0.0f), a1 = a0;
    float b0 = 0.0f, b1 = 0.0f;
    float4 w = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    float2 z = make_float2(0.0f, 0.0f);
    row_taps(c0, [&](int col, int e, int k0, int k1) {
      if (e == 0) {
        w = *reinterpret_cast<const float4*>(&sp[r][col]);
        z = *reinterpret_cast<const float2*>(&sc[r][col]);
      }
      const float2 v = e == 0 ? make_float2(w.x, w.y) : make_float2(w.z, w.w);
      const float u = e == 0 ? z.x : z.y;
      if (k0 >= 0) {
        a0 = fma2(P.g2[k0], v, a0);
        b0 = fmaf(P.g2[k0].x, u, b0);
      }
      if (k1 >= 0) {
        a1 = fma2(P.g2[k1], v, a1);
        b1 = fmaf(P.g2[k1].x, u, b1);
      }
    });
    *reinterpret_cast<float4*>(&hp[r][c0]) = make_float4(a0.x, a0.y, a1.x, a1.y);
    *reinterpret_cast<float2*>(&hs[r][c0]) = make_float2(b0, b1);
  }
  __syncthreads();
  float2 am[4];
  float ab[4];
#pragma unroll
  for (int o = 0; o < 4; ++o) {
    am[o] = make_float2(0.0f, 0.0f);
    ab[o] = 0.0f;
  }
#pragma unroll
  for (int j = 0; j < kWin + 3; ++j) {
    const float2 m = hp[r0 + j][c];
    const float u = hs[r0 + j][c];
#pragma unroll
    for (int o = 0; o < 4; ++o) {
      const int k = j - o;
      if (k < 0 || k >= kWin) continue;
      am[o] = fma2(P.g2[k], m, am[o]);
      ab[o] = fmaf(P.g2[k].x, u, ab[o]);
    }
  }
  const float n_inv = 1.0f / (3.0f * (float)W * (float)H);
  const float w1 = P.inv_views * n_inv * (1.0f - P.lam), ws = P.inv_views * n_inv * P.lam;
#pragma unroll
  for (int o = 0; o < 4; ++o) {
    if (!ok[o]) continue;
    const float x = xo[o], y = yo[o];
    const float sg = (float)(x > y) - (float)(x < y);
    // d(1 - SSIM)/dx = -dSSIM/dx
    dL[io[o]] = w1 * sg - ws * (am[o].x + 2.0f * x * am[o].y + y * ab[o]);
  }
}

// Per-view losses from the block sums: one block per view, float sums in a
// fixed order (deterministic).
__global__ void __launch_bounds__(256)
    loss_reduce_kernel(const __grid_constant__ LossParams P, const float2* __restrict__ bsum,
                       float* __restrict__ loss) {
  wait_prior_grid();
  __shared__ float red[2][256];
  const LossView& w = P.v[blockIdx.x];
  const uint32_t b0 = w.blk_off, nb = 3u * (uint32_t)w.tiles;
  float s = 0.0f, l = 0.0f;
  for (uint32_t i = threadIdx.x; i < nb; i += 256) {
    const float2 q = bsum[b0 + i];
    s += q.x;
    l += q.y;
  }
  red[0][threadIdx.x] = s;
  red[1][threadIdx.x] = l;
  __syncthreads();
  for (int d = 128; d > 0; d >>= 1) {
    if (threadIdx.x < d) {
      red[0][threadIdx.x] += red[0][threadIdx.x + d];
      red[1][threadIdx.x] += red[1][threadIdx.x + d];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const float n = 3.0f * (float)w.W * (float)w.H;
    loss[1 + blockIdx.x] = (1.0f - P.lam) * (red[1][0] / n) + P.lam * (1.0f - red[0][0] / n);
  }
}

// the mean of the view losses, summed in view order
__global__ void loss_total_kernel(int n, float* __restrict__ loss) {
  wait_prior_grid();
  float s = 0.0f;
  for (int v = 0; v < n; ++v) s += loss[1 + v];
  loss[0] = s / (float)n;
}

// ---------------------------------------------------------------------------
// Adam
// ---------------------------------------------------------------------------

constexpr int kAdamMaxPlanes = 64;
struct AdamParams {
  float lr[kAdamMaxPlanes];
  float l1[kAdamMaxPlanes];
  int32_t act[kAdamMaxPlanes];
  int32_t noise_row[kAdamMaxPlanes];
  int64_t P;
  int32_t K;
  float b1, b2, eps, bc1, bc2, leps;  // bc = 1 / (1 - beta^t)
};

__device__ __forceinline__ float activate(float r, int act) {
  if (act == UBS_ACT_SIGMOID) return 1.0f / (1.0f + expf(-r));
  if (act == UBS_ACT_EXP) return expf(r);
  return r;
}

__device__ __forceinline__ void adam_one(const AdamParams& A, int k, float& r, float& a, float g, float& m,
                                         float& v, float noise) {
  const int act = A.act[k];
  const float a0 = activate(r, act);
  g += A.l1[k] * ((float)(a0 > 0.0f) - (float)(a0 < 0.0f));
  if (act == UBS_ACT_SIGMOID) g *= a0 * (1.0f - a0);
  else if (act == UBS_ACT_EXP) g *= a0;
  m = fmaf(A.b1, m, (1.0f - A.b1) * g);
  v = fmaf(A.b2, v, (1.0f - A.b2) * g * g);
  r -= A.lr[k] * (m * A.bc1) / (sqrtf(v * A.bc2) + A.eps);
  r = fmaf(A.leps, noise, r);
  a = activate(r, act);
}

template <bool VEC>
__global__ void __launch_bounds__(256)
    adam_kernel(const __grid_constant__ AdamParams A, float* __restrict__ raw, float* __restrict__ act,
                const float* __restrict__ grad, float* __restrict__ m, float* __restrict__ v,
                const float* __restrict__ noise) {
  wait_prior_grid();
  const int64_t n = (int64_t)A.K * A.P;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  if constexpr (VEC) {
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n / 4; q += stride) {
      const int64_t e = 4 * q;
      const int k = (int)(e / A.P);  // P % 4 == 0: the four share a plane
      float4 r = reinterpret_cast<float4*>(raw)[q];
      const float4 g = reinterpret_cast<const float4*>(grad)[q];
      float4 mm = reinterpret_cast<float4*>(m)[q];
      float4 vv = reinterpret_cast<float4*>(v)[q];
      float4 z = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
      const int row = A.noise_row[k];
      if (row >= 0) z = reinterpret_cast<const float4*>(noise + (size_t)row * A.P)[(e - (int64_t)k * A.P) / 4];
      float4 a;
      adam_one(A, k, r.x, a.x, g.x, mm.x, vv.x, z.x);
      adam_one(A, k, r.y, a.y, g.y, mm.y, vv.y, z.y);
      adam_one(A, k, r.z, a.z, g.z, mm.z, vv.z, z.z);
      adam_one(A, k, r.w, a.w, g.w, mm.w, vv.w, z.w);
      reinterpret_cast<float4*>(raw)[q] = r;
      reinterpret_cast<float4*>(act)[q] = a;
      reinterpret_cast<float4*>(m)[q] = mm;
      reinterpret_cast<float4*>(v)[q] = vv;
    }
  } else {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += stride) {
      const int k = (int)(e / A.P);
      const int row = A.noise_row[k];
      const float z = row >= 0 ? noise[(size_t)row * A.P + (e - (int64_t)k * A.P)] : 0.0f;
      float r = raw[e], mm = m[e], vv = v[e], a;
      adam_one(A, k, r, a, grad[e], mm, vv, z);
      raw[e] = r;
      act[e] = a;
      m[e] = mm;
      v[e] = vv;
    }
  }
}

bool loss_views(int32_t n, const int32_t* w, const int32_t* h, LossParams* P, size_t* ws) {
  if (n < 1 || n > kLossMaxViews || !w || !h) return false;
  uint64_t pix = 0, blk = 0;
  for (int i = 0; i < n; ++i) {
    if (w[i] < 1 || h[i] < 1 || w[i] > 65535 || h[i] > 65535) return false;
    const int tx = (w[i] + kTX - 1) / kTX, ty = (h[i] + kTY - 1) / kTY;
    if (P) {
      P->v[i].W = w[i];
      P->v[i].H = h[i];
      P->v[i].tiles_x = tx;
      P->v[i].tiles = tx * ty;
      P->v[i].pix_off = (uint32_t)pix;
      P->v[i].blk_off = (uint32_t)blk;
    }
    pix += (uint64_t)w[i] * h[i];
    blk += 3ull * tx * ty;
    if (pix > 0x7fffffffull / 3 || blk > 0x7fffffffull) return false;
  }
  if (P) {
    P->n = n;
    P->n_blocks = (uint32_t)blk;
    P->plane = 3 * pix;
  }
  *ws = align256(3 * 3 * pix * sizeof(float)) + align256(blk * sizeof(float2));
  return true;
}

}  // namespace
}  // namespace ubs

using namespace ubs;

extern "C" size_t ubs_loss_workspace_size(int32_t n_views, const int32_t* widths, const int32_t* heights) {
  size_t ws = 0;
  return loss_views(n_views, widths, heights, nullptr, &ws) ? ws : 0;
}

extern "C" ubs_status ubs_image_loss(int32_t n_views, const int32_t* widths, const int32_t* heights,
                                     const float* image, const float* target, float lambda_ssim, float* dL_dimage,
                                     float* loss, void* workspace, size_t workspace_bytes, cudaStream_t stream) {
  ubs::TraceRange trace_("ubs_image_loss");
  LossParams p;
  memset(&p, 0, sizeof(p));
  size_t need = 0;
  if (!loss_views(n_views, widths, heights, &p, &need)) return UBS_ERR_INVALID_ARG;
  if (!image || !target || !dL_dimage || !loss || !workspace) return UBS_ERR_INVALID_ARG;
  if (!(lambda_ssim >= 0.0f && lambda_ssim <= 1.0f)) return UBS_ERR_INVALID_ARG;
  if (((uintptr_t)workspace & 255u) != 0) return UBS_ERR_ALIGNMENT;
  if (((uintptr_t)image | (uintptr_t)target | (uintptr_t)dL_dimage | (uintptr_t)loss) & 3u) return UBS_ERR_ALIGNMENT;
  if (workspace_bytes < need) return UBS_ERR_WORKSPACE;
  // the 1-D window: exp(-(i - 5)^2 / (2 * 1.5^2)), normalised to sum 1
  double g[kWin], s = 0.0;
  for (int i = 0; i < kWin; ++i) {
    g[i] = exp(-(double)((i - kRad) * (i - kRad)) / (2.0 * 1.5 * 1.5));
    s += g[i];
  }
  for (int i = 0; i < kWin; ++i) p.g2[i] = make_float2((float)(g[i] / s), (float)(g[i] / s));
  p.lam = lambda_ssim;
  p.inv_views = 1.0f / (float)n_views;
  char* ws = (char*)workspace;
  float* part = (float*)ws;
  float2* bsum = (float2*)(ws + align256(3 * p.plane * sizeof(float)));
  cudaError_t e = launch_dependent(ssim_fwd_kernel, dim3(p.n_blocks), dim3(kLossThreads), 0, stream, p, image,
                                   target, part, bsum);
  if (e == cudaSuccess)
    e = launch_dependent(ssim_bwd_kernel, dim3(p.n_blocks), dim3(kLossThreads), 0, stream, p, image, target,
                         (const float*)part, dL_dimage);
  if (e == cudaSuccess)
    e = launch_dependent(loss_reduce_kernel, dim3(p.n), dim3(256), 0, stream, p, (const float2*)bsum, loss);
  if (e == cudaSuccess) e = launch_dependent(loss_total_kernel, dim3(1), dim3(1), 0, stream, p.n, loss);
  return e == cudaSuccess ? UBS_OK : UBS_ERR_CUDA;
}

extern "C" ubs_status ubs_adam_step(int32_t K, int64_t P, const ubs_adam_plane* planes, const ubs_adam_config* cfg,
                                    float* raw, float* act_out, const float* grad, float* m, float* v,
                                    const float* noise, cudaStream_t stream) {
  ubs::TraceRange trace_("ubs_adam_step");
  if (K < 1 || K > kAdamMaxPlanes || P < 0 || !planes || !cfg) return UBS_ERR_INVALID_ARG;
  if (P == 0) return UBS_OK;
  if (!raw || !act_out || !grad || !m || !v || raw == act_out) return UBS_ERR_INVALID_ARG;
  if (cfg->step < 1 || !(cfg->beta1 >= 0.0f && cfg->beta1 < 1.0f) || !(cfg->beta2 >= 0.0f && cfg->beta2 < 1.0f) ||
      !(cfg->eps >= 0.0f))
    return UBS_ERR_INVALID_ARG;
  AdamParams A;
  memset(&A, 0, sizeof(A));
  bool any_noise = false;
  for (int k = 0; k < K; ++k) {
    const ubs_adam_plane& q = planes[k];
    if (q.activation < UBS_ACT_IDENTITY || q.activation > UBS_ACT_EXP || !(q.lr >= 0.0f)) return UBS_ERR_INVALID_ARG;
    A.lr[k] = q.lr;
    A.l1[k] = q.l1_weight;
    A.act[k] = q.activation;
    A.noise_row[k] = q.noise_row < 0 ? -1 : q.noise_row;
    any_noise = any_noise || q.noise_row >= 0;
  }
  if (any_noise && !noise) return UBS_ERR_INVALID_ARG;
  const uintptr_t all = (uintptr_t)raw | (uintptr_t)act_out | (uintptr_t)grad | (uintptr_t)m | (uintptr_t)v |
                        (uintptr_t)(noise ? noise : raw);
  if (all & 3u) return UBS_ERR_ALIGNMENT;
  A.P = P;
  A.K = K;
  A.b1 = cfg->beta1;
  A.b2 = cfg->beta2;
  A.eps = cfg->eps;
  A.bc1 = (float)(1.0 / (1.0 - pow((double)cfg->beta1, (double)cfg->step)));
  A.bc2 = (float)(1.0 / (1.0 - pow((double)cfg->beta2, (double)cfg->step)));
  A.leps = cfg->lambda_eps;
  const bool vec = (P % 4 == 0) && (all & 15u) == 0;
  const int64_t units = vec ? (int64_t)K * P / 4 : (int64_t)K * P;
  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t want = (units + 255) / 256;
  const unsigned grid = (unsigned)(want < (int64_t)sms * 8 ? want : (int64_t)sms * 8);
  cudaError_t e = vec ? launch_dependent(adam_kernel<true>, dim3(grid), dim3(256), 0, stream, A, raw, act_out, grad, m,
                                         v, noise)
                      : launch_dependent(adam_kernel<false>, dim3(grid), dim3(256), 0, stream, A, raw, act_out, grad,
                                         m, v, noise);
  return e == cudaSuccess ? UBS_OK : UBS_ERR_CUDA;
}
