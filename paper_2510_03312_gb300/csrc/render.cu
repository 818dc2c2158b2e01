// render.cu -- R1 (forward blend) and G1 (backward blend).
//
// One CTA per screen tile, one thread per pixel.  The tile's front-to-back
// list (sorted record ids) is consumed in batches of one record per thread:
// each batch's 48-byte render records are staged in shared memory, then every
// thread walks the batch.  Per pair (Sec. 3, Eq. r; Sec. 4.3 final density):
//   dx = (px - hi_x) - lo_x,  r = a dx^2 + 2 b dx dy + c dy^2,
//   skip if r >= 1;  alpha = min(alpha_max, 2^(beta_x log2(1 - r) + log2 o(q)))
//   skip if alpha < alpha_min;  stop before T (1 - alpha) < T_min;
//   C += c alpha T;  T *= 1 - alpha.
// log2/exp2 are the MUFU approximations (lg2.approx, ex2.approx).  The pair
// evaluation is one inline function with explicit rounding so that the
// backward kernel re-derives exactly the forward's alpha and decisions.
// A CTA stops loading batches once every pixel of the tile has terminated
// (__syncthreads_count).
//
// The backward walks each tile's list back to front from the last
// contributor, recovers T by division, and forms per-pair gradients of
// (mu', conic, log2 o(q), beta_x, rgb).  They are summed over the warp's 32
// pixels with shuffles (only for records some lane of the warp touches),
// accumulated per record in shared memory across the CTA's warps, and
// flushed with one vector atomic add per (record, tile) -- never one global
// atomic per pixel.
#include "kernels.cuh"

namespace ubs {

namespace {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ float lg2_approx(float x) {
  float y;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

struct PairEval {
  float dx, dy, r, lg, alpha;
};

// the one definition of a pair's alpha, shared by forward and backward
__device__ __forceinline__ void eval_pair(float px, float py, const float4& a, const float4& c, float beta,
                                          float amax, PairEval& e) {
  e.dx = __fsub_rn(__fsub_rn(px, a.x), a.z);
  e.dy = __fsub_rn(__fsub_rn(py, a.y), a.w);
  const float t0 = __fmul_rn(c.x, e.dx);
  const float t1 = __fmul_rn(c.z, e.dy);
  const float bxy = __fmul_rn(__fmul_rn(2.0f, c.y), e.dy);
  e.r = __fmaf_rn(t0, e.dx, __fmaf_rn(t1, e.dy, __fmul_rn(bxy, e.dx)));
  e.lg = lg2_approx(__fsub_rn(1.0f, e.r));
  e.alpha = fminf(amax, ex2_approx(__fmaf_rn(beta, e.lg, c.w)));
}

__device__ __forceinline__ int find_view(const ViewDev* __restrict__ views, int V, uint32_t g) {
  int lo = 0, hi = V - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (views[mid].tile_off <= g) lo = mid; else hi = mid - 1;
  }
  return lo;
}

template <int TW, int TH, bool COUNT>
__global__ void __launch_bounds__(TW * TH) render_fwd_kernel(const ViewDev* __restrict__ views, int V, CfgDev cfg,
                                                             const uint32_t* __restrict__ tstart,
                                                             const uint32_t* __restrict__ ivals,
                                                             const float4* __restrict__ rec4,
                                                             float* __restrict__ image, float* __restrict__ Tfin,
                                                             uint32_t* __restrict__ lastc, const Header* hdr,
                                                             uint32_t R, uint32_t* __restrict__ pairs) {
  constexpr int B = TW * TH;
  constexpr int BS = B < 256 ? B : 256;  // records staged per batch
  __shared__ float4 s_a[BS], s_c[BS], s_d[BS];
  __shared__ int s_v;
  if (hdr->status != 0) return;
  const uint32_t g = blockIdx.x;
  if (threadIdx.x == 0) s_v = find_view(views, V, g);
  __syncthreads();
  const ViewDev& v = views[s_v];
  const uint32_t lt = g - v.tile_off;
  const int tx = lt % v.tiles_x, ty = lt / v.tiles_x;
  const int x = tx * TW + (threadIdx.x % TW), y = ty * TH + (threadIdx.x / TW);
  const bool inside = x < v.W && y < v.H;
  const float px = (float)x + 0.5f, py = (float)y + 0.5f;
  const uint32_t start = tstart[g], end = tstart[g + 1];
  float T = 1.0f, C0 = 0.0f, C1 = 0.0f, C2 = 0.0f;
  uint32_t last = 0, np = 0;
  bool done = !inside;
  for (uint32_t base = start; base < end; base += BS) {
    if (__syncthreads_count(done) == B) break;
    const uint32_t idx = base + threadIdx.x;
    if (threadIdx.x < BS && idx < end) {
      const uint32_t r = min(ivals[idx], R - 1);  // ids are < R by construction
      s_a[threadIdx.x] = rec4[3 * (size_t)r];
      s_c[threadIdx.x] = rec4[3 * (size_t)r + 1];
      s_d[threadIdx.x] = rec4[3 * (size_t)r + 2];
    }
    __syncthreads();
    const int n = (int)min((uint32_t)BS, end - base);
    for (int j = 0; j < n && !done; ++j) {
      const float4 a = s_a[j], c = s_c[j], d = s_d[j];
      PairEval e;
      eval_pair(px, py, a, c, d.x, cfg.amax, e);
      if (!(e.r < 1.0f)) continue;
      if constexpr (COUNT) ++np;
      if (e.alpha < cfg.amin) continue;
      const float Tn = T * (1.0f - e.alpha);
      if (Tn < cfg.tmin) {
        done = true;
        break;
      }
      const float w = e.alpha * T;
      C0 = fmaf(d.y, w, C0);
      C1 = fmaf(d.z, w, C1);
      C2 = fmaf(d.w, w, C2);
      T = Tn;
      last = base - start + j + 1;
    }
  }
  if (inside) {
    const size_t plane = (size_t)v.W * v.H;
    const size_t pix = (size_t)y * v.W + x;
    float* img = image + (size_t)v.pix_off * 3;
    img[pix] = fmaf(T, cfg.bg[0], C0);
    img[plane + pix] = fmaf(T, cfg.bg[1], C1);
    img[2 * plane + pix] = fmaf(T, cfg.bg[2], C2);
    Tfin[v.pix_off + pix] = T;
    lastc[v.pix_off + pix] = last;
    if constexpr (COUNT) pairs[v.pix_off + pix] = np;
  }
}

template <int TW, int TH>
__global__ void __launch_bounds__(TW * TH) render_bwd_kernel(const ViewDev* __restrict__ views, int V, CfgDev cfg,
                                                             const uint32_t* __restrict__ tstart,
                                                             const uint32_t* __restrict__ ivals,
                                                             const float4* __restrict__ rec4,
                                                             const float* __restrict__ dLdimg,
                                                             const float* __restrict__ Tfin,
                                                             const uint32_t* __restrict__ lastc,
                                                             float4* __restrict__ g2d, const Header* hdr, uint32_t R) {
  constexpr int B = TW * TH;
  constexpr int BS = B < 256 ? B : 256;  // records staged per batch
  __shared__ float4 s_a[BS], s_c[BS], s_d[BS];
  __shared__ uint32_t s_rec[BS];
  __shared__ float s_acc[10][BS];
  __shared__ int s_hit[BS];
  __shared__ int s_v;
  __shared__ uint32_t s_max;
  if (hdr->status != 0) return;
  const uint32_t g = blockIdx.x;
  if (threadIdx.x == 0) {
    s_v = find_view(views, V, g);
    s_max = 0;
  }
  for (int i = threadIdx.x; i < 10 * BS; i += B) (&s_acc[0][0])[i] = 0.0f;
  if (threadIdx.x < BS) s_hit[threadIdx.x] = 0;
  __syncthreads();
  const ViewDev& v = views[s_v];
  const uint32_t lt = g - v.tile_off;
  const int tx = lt % v.tiles_x, ty = lt / v.tiles_x;
  const int x = tx * TW + (threadIdx.x % TW), y = ty * TH + (threadIdx.x / TW);
  const bool inside = x < v.W && y < v.H;
  const float px = (float)x + 0.5f, py = (float)y + 0.5f;
  const uint32_t start = tstart[g];
  float T = 1.0f, G0 = 0.0f, G1 = 0.0f, G2 = 0.0f;
  uint32_t last = 0;
  if (inside) {
    const size_t plane = (size_t)v.W * v.H;
    const size_t pix = (size_t)y * v.W + x;
    const float* gi = dLdimg + (size_t)v.pix_off * 3;
    G0 = gi[pix];
    G1 = gi[plane + pix];
    G2 = gi[2 * plane + pix];
    T = Tfin[v.pix_off + pix];
    last = lastc[v.pix_off + pix];
  }
  // colour behind the current record, normalised by the transmittance after it
  float B0 = cfg.bg[0], B1 = cfg.bg[1], B2 = cfg.bg[2];
  if (last) atomicMax(&s_max, last);
  __syncthreads();
  const uint32_t nmax = s_max;
  const uint32_t lane = threadIdx.x & 31;
  // batches from the back: entries [lo, hi) with hi = nmax, nmax - BS, ...
  for (int hi = (int)nmax; hi > 0; hi -= BS) {
    const int lo = hi - BS > 0 ? hi - BS : 0;
    const int n = hi - lo;
    __syncthreads();
    if ((int)threadIdx.x < n) {
      const uint32_t r = min(ivals[start + lo + threadIdx.x], R - 1);  // ids are < R by construction
      s_rec[threadIdx.x] = r;
      s_a[threadIdx.x] = rec4[3 * (size_t)r];
      s_c[threadIdx.x] = rec4[3 * (size_t)r + 1];
      s_d[threadIdx.x] = rec4[3 * (size_t)r + 2];
    }
    __syncthreads();
    for (int j = n - 1; j >= 0; --j) {
      const uint32_t entry = (uint32_t)(lo + j);
      float g[10];
      bool hit = false;
      if (entry < last) {
        const float4 a = s_a[j], c = s_c[j], d = s_d[j];
        PairEval e;
        eval_pair(px, py, a, c, d.x, cfg.amax, e);
        if (e.r < 1.0f && e.alpha >= cfg.amin) {
          hit = true;
          const float om = 1.0f - e.alpha;
          T = __fdividef(T, om);
          const float w = e.alpha * T;
          g[7] = w * G0;
          g[8] = w * G1;
          g[9] = w * G2;
          const float dalpha = T * ((d.y - B0) * G0 + (d.z - B1) * G1 + (d.w - B2) * G2);
          B0 = fmaf(e.alpha, d.y - B0, B0);
          B1 = fmaf(e.alpha, d.z - B1, B1);
          B2 = fmaf(e.alpha, d.w - B2, B2);
          if (e.alpha < cfg.amax) {
            const float ga = dalpha * e.alpha;
            g[5] = ga * kLn2f;                       // d log2 o(q)
            g[6] = ga * e.lg * kLn2f;                // d beta_x = alpha ln(1 - r)
            const float dr = -ga * d.x / (1.0f - e.r);
            g[0] = -2.0f * dr * (c.x * e.dx + c.y * e.dy);  // d mu'_x
            g[1] = -2.0f * dr * (c.y * e.dx + c.z * e.dy);  // d mu'_y
            g[2] = dr * e.dx * e.dx;
            g[3] = 2.0f * dr * e.dx * e.dy;
            g[4] = dr * e.dy * e.dy;
          } else {
#pragma unroll
            for (int k = 0; k < 7; ++k) g[k] = 0.0f;
          }
        }
      }
      if (!hit) {
#pragma unroll
        for (int k = 0; k < 10; ++k) g[k] = 0.0f;
      }
      const unsigned any = __ballot_sync(kFull, hit);
      if (any) {
#pragma unroll
        for (int k = 0; k < 10; ++k) {
          float s = g[k];
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(kFull, s, o);
          g[k] = s;
        }
        if (lane == 0) {
#pragma unroll
          for (int k = 0; k < 10; ++k) atomicAdd(&s_acc[k][j], g[k]);
          s_hit[j] = 1;
        }
      }
    }
    __syncthreads();
    if ((int)threadIdx.x < n && s_hit[threadIdx.x]) {
      const int j = threadIdx.x;
      float4* dst = g2d + 3 * (size_t)s_rec[j];
      atomicAdd(dst, make_float4(s_acc[0][j], s_acc[1][j], s_acc[2][j], s_acc[3][j]));
      atomicAdd(dst + 1, make_float4(s_acc[4][j], s_acc[5][j], s_acc[6][j], s_acc[7][j]));
      atomicAdd((float2*)(dst + 2), make_float2(s_acc[8][j], s_acc[9][j]));
#pragma unroll
      for (int k = 0; k < 10; ++k) s_acc[k][j] = 0.0f;
      s_hit[j] = 0;
    }
  }
}

template <int TW, int TH>
cudaError_t fwd_t(const Layout& L, const CfgDev& cfg, char* ws, float* image, cudaStream_t st) {
  const ViewDev* views = (const ViewDev*)(ws + L.views);
  const uint32_t* tstart = (const uint32_t*)(ws + L.tstart);
  const float4* rec4 = (const float4*)(ws + L.rec4);
  float* Tfin = (float*)(ws + L.Tfin);
  uint32_t* last = (uint32_t*)(ws + L.last);
  const Header* hdr = (const Header*)(ws + L.header);
  const uint32_t R = L.R > 0 ? L.R : 1;
  if (cfg.flags & 2)  // diagnostic variant: also count visited pairs with r < 1 per pixel
    render_fwd_kernel<TW, TH, true><<<L.NT, TW * TH, 0, st>>>(views, L.V, cfg, tstart, sorted_instances(L, ws),
                                                            rec4, image, Tfin, last, hdr, R,
                                                            (uint32_t*)(ws + L.pairs));
  else
    render_fwd_kernel<TW, TH, false><<<L.NT, TW * TH, 0, st>>>(views, L.V, cfg, tstart, sorted_instances(L, ws),
                                                             rec4, image, Tfin, last, hdr, R, nullptr);
  return cudaGetLastError();
}

template <int TW, int TH>
cudaError_t bwd_t(const Layout& L, const CfgDev& cfg, char* ws, const float* dL, cudaStream_t st) {
  render_bwd_kernel<TW, TH><<<L.NT, TW * TH, 0, st>>>(
      (const ViewDev*)(ws + L.views), L.V, cfg, (const uint32_t*)(ws + L.tstart), sorted_instances(L, ws),
      (const float4*)(ws + L.rec4), dL, (const float*)(ws + L.Tfin), (const uint32_t*)(ws + L.last),
      (float4*)(ws + L.g2d), (const Header*)(ws + L.header), L.R > 0 ? L.R : 1);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_render_fwd(const Layout& L, const CfgDev& cfg, char* ws, float* image, cudaStream_t st) {
  if (L.NT == 0) return cudaSuccess;
  if (cfg.tw == 16 && cfg.th == 16) return fwd_t<16, 16>(L, cfg, ws, image, st);
  if (cfg.tw == 8 && cfg.th == 8) return fwd_t<8, 8>(L, cfg, ws, image, st);
  if (cfg.tw == 16 && cfg.th == 32) return fwd_t<16, 32>(L, cfg, ws, image, st);
  if (cfg.tw == 32 && cfg.th == 32) return fwd_t<32, 32>(L, cfg, ws, image, st);
  return cudaErrorInvalidValue;
}

cudaError_t launch_render_bwd(const Layout& L, const CfgDev& cfg, char* ws, const float* dL, cudaStream_t st) {
  if (L.NT == 0 || L.R == 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(ws + L.g2d, 0, (size_t)L.R * kGradFloats * sizeof(float), st);
  if (e != cudaSuccess) return e;
  if (cfg.tw == 16 && cfg.th == 16) return bwd_t<16, 16>(L, cfg, ws, dL, st);
  if (cfg.tw == 8 && cfg.th == 8) return bwd_t<8, 8>(L, cfg, ws, dL, st);
  if (cfg.tw == 16 && cfg.th == 32) return bwd_t<16, 32>(L, cfg, ws, dL, st);
  if (cfg.tw == 32 && cfg.th == 32) return bwd_t<32, 32>(L, cfg, ws, dL, st);
  return cudaErrorInvalidValue;
}

}  // namespace ubs
