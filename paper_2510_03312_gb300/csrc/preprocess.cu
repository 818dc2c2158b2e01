// preprocess.cu -- P1-P3: kernel construction, Beta-modulated conditioning
// and projection of every (view, primitive) record.
//
// Compiled with --fmad=false -prec-div=true -prec-sqrt=true -ftz=false so
// that the float32 rule set of spec32.cuh holds (see prim_forward.cuh).
//
// One thread per primitive of one scene; the thread builds the view-
// independent part once (Sigma blocks, Cholesky of Sigma_q, Sigma_q^{-1}
// Sigma_qx, beta) and then loops over the scene's views, so each primitive's
// parameters are read from HBM once per batch of views.  Parameter planes
// are structure-of-arrays: a warp reads 32 consecutive floats per plane.
#include <atomic>

#include "kernels.cuh"
#include "prim_forward.cuh"

namespace ubs {

template <int C>
__device__ __forceinline__ void load_prim(const SceneDev& sc, int64_t p, PrimIn<C>& in) {
  const int64_t P = sc.P;
  for (int i = 0; i < 3; ++i) in.mx[i] = __ldg(sc.mean_x + i * P + p);
  const int nr = sc.rot_mode == 0 ? 4 : 3;
  for (int i = 0; i < 4; ++i) in.rot[i] = i < nr ? __ldg(sc.rot + i * P + p) : 0.0f;
  for (int i = 0; i < 3; ++i) in.s[i] = __ldg(sc.scale_x + i * P + p);
  for (int i = 0; i < 1 + C; ++i) in.b[i] = __ldg(sc.b + i * P + p);
  in.o = __ldg(sc.opacity + p);
  if constexpr (C > 0) {
    for (int i = 0; i < C; ++i) in.mq[i] = __ldg(sc.mean_q + i * P + p);
    for (int i = 0; i < 3 * C; ++i) in.lqx[i] = __ldg(sc.L_qx + i * P + p);
    for (int i = 0; i < C * (C + 1) / 2; ++i) in.lq[i] = __ldg(sc.L_q + i * P + p);
  }
}

// Zeroes zero[0, n) over the grid (the binning's counters, with the first
// scene's launch).
__device__ __forceinline__ void zero_words(uint32_t* __restrict__ zero, uint32_t n) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) zero[i] = 0;
}

template <int C>
__global__ void __launch_bounds__(256) preprocess_kernel(SceneDev sc, ViewList vl, const ViewDev* __restrict__ views,
                                                         CfgDev cfg, float4* __restrict__ rec4,
                                                         uint32_t* __restrict__ key, uint32_t* __restrict__ tiles,
                                                         uint2* __restrict__ rect, uint32_t* __restrict__ vis_mask,
                                                         uint32_t* __restrict__ act_list, uint32_t* act_count,
                                                         uint32_t* __restrict__ zero, uint32_t nzero) {
  wait_prior_grid();
  zero_words(zero, nzero);
  extern __shared__ ViewDev s_views[];
  for (int i = threadIdx.x; i < vl.n; i += blockDim.x) s_views[i] = views[vl.idx[i]];
  __syncthreads();
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= sc.P) return;
  PrimIn<C> in;
  load_prim<C>(sc, p, in);
  PrimVI<C> vi;
  prim_stage<C>(in, sc.rot_mode, vi);
  const float cr = __ldg(sc.rgb + p), cg = __ldg(sc.rgb + sc.P + p), cb = __ldg(sc.rgb + 2 * sc.P + p);
  bool any = false;  // visible in some view
  for (int k = 0; k < vl.n; ++k) {
    const ViewDev& v = s_views[k];
    ViewOut o;
    view_stage<C>(in, vi, v, cfg, o);
    any = any || o.valid;
    const uint32_t r = v.rec_off + (uint32_t)p;
    tiles[r] = o.tiles;
    {
      // the warp's 32 primitives (p aligned to 32) are one word of the
      // view's visibility mask: lane l's bit for primitive 32 (p / 32) + l
      const unsigned act = __activemask();
      const unsigned vis = __ballot_sync(act, o.valid);
      if ((threadIdx.x & 31) == (unsigned)(__ffs(act) - 1)) vis_mask[v.mask_off + (uint32_t)(p >> 5)] = vis;
    }
    if (o.valid) {
      key[r] = __float_as_uint(o.depth);
      rect[r] = make_uint2((uint32_t)o.tx0 | ((uint32_t)o.ty0 << 16), (uint32_t)o.tx1 | ((uint32_t)o.ty1 << 16));
      rec4[3 * (size_t)r + 0] = make_float4(o.mu_hi[0], o.mu_hi[1], o.mu_lo[0], o.mu_lo[1]);
      rec4[3 * (size_t)r + 1] = make_float4(o.conic[0], o.conic[1], o.conic[2], log2f(o.oq));
      rec4[3 * (size_t)r + 2] = make_float4(vi.beta_x, cr, cg, cb);
    }
  }
  // scenes with several views: the primitives some view sees, listed for the
  // parameter backward (one add per warp)
  if (vl.n > 1) {
    const unsigned act = __activemask();
    const unsigned m = __ballot_sync(act, any);
    if (m) {
      const int lane = threadIdx.x & 31, leader = __ffs(act) - 1;
      uint32_t base = 0;
      if (lane == leader) base = atomicAdd(act_count, (uint32_t)__popc(m));
      base = __shfl_sync(act, base, leader);
      if (any) act_list[base + __popc(m & ((1u << lane) - 1u))] = (uint32_t)p;
    }
  }
}

// Scenes with query dimensions (N > 3): the conditioning runs per (view,
// primitive) as in preprocess_kernel, but only the records that pass the
// early tests (view_candidate) are projected, from a per-warp queue in
// shared memory, 32 at a time.  Where the query culls most records (o(q)
// below alpha_min), the projection -- over half of a record's arithmetic --
// then runs on full warps instead of on the few lanes whose record survives.
// The projection of a queued record is the same arithmetic on the same
// values as in view_stage.
constexpr int kQCap = 64;   // queue entries per warp: 31 carried over + 32 new
constexpr int kQWarps = 8;  // warps per CTA (256 threads)
// Held to 80 registers (three CTAs per SM, from two at 108-116): the
// kernel's dependent float32 chains need the warps (the 16-view N=6 batch
// 253 -> 232 us, the 8-view N=7 one 99 -> 91 us).

template <int C>
__global__ void __launch_bounds__(256, 3) preprocess_queued_kernel(SceneDev sc, ViewList vl,
                                                                const ViewDev* __restrict__ views, CfgDev cfg,
                                                                float4* __restrict__ rec4, uint32_t* __restrict__ key,
                                                                uint32_t* __restrict__ tiles, uint2* __restrict__ rect,
                                                                uint32_t* __restrict__ vis_mask,
                                                                uint32_t* __restrict__ act_list, uint32_t* act_count,
                                                                uint32_t* __restrict__ zero, uint32_t nzero) {
  wait_prior_grid();
  zero_words(zero, nzero);
  extern __shared__ ViewDev s_views[];
  // per warp: the lanes' view-independent values (mean, Sigma, beta_x, rgb),
  // and the queue (record, view | owner lane << 16, shift, o(q))
  __shared__ float s_prim[kQWarps][13][32];
  __shared__ float s_qf[kQWarps][4][kQCap];
  __shared__ uint32_t s_qr[kQWarps][kQCap], s_qk[kQWarps][kQCap];
  __shared__ uint32_t s_any[kQWarps];
  __shared__ uint32_t s_vis[kQWarps][kMaxViews];  // per warp and view: the visibility mask word
  for (int i = threadIdx.x; i < vl.n; i += blockDim.x) s_views[i] = views[vl.idx[i]];
  if (threadIdx.x < kQWarps) s_any[threadIdx.x] = 0;
  for (int i = threadIdx.x; i < kQWarps * vl.n; i += blockDim.x) s_vis[i / vl.n][i % vl.n] = 0;
  __syncthreads();
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool live = p < sc.P;  // every lane stays: the queue is warp-synchronous
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const unsigned lt = (1u << lane) - 1u;
  float(*prim)[32] = s_prim[w];
  float(*qf)[kQCap] = s_qf[w];
  uint32_t* qr = s_qr[w];
  uint32_t* qk = s_qk[w];
  PrimIn<C> in;
  PrimVI<C> vi;
  // the log-opacity bound below which a record is certainly culled (see
  // view_condition): approximate log and quotient, inside the bound's margin
  float cull_below = -INFINITY;
  if (live) {
    load_prim<C>(sc, p, in);
    prim_stage<C>(in, sc.rot_mode, vi);
    if (cfg.amin > 0.0f) cull_below = __logf(__fdividef(cfg.amin, in.o)) - 0.01f;
    for (int i = 0; i < 3; ++i) prim[i][lane] = in.mx[i];
    for (int i = 0; i < 6; ++i) prim[3 + i][lane] = vi.Sc[i];
    prim[9][lane] = vi.beta_x;
    for (int i = 0; i < 3; ++i) prim[10 + i][lane] = __ldg(sc.rgb + i * sc.P + p);
  }
  __syncwarp();
  // projects queue entry j (any lane may take any entry)
  auto project = [&](int j) {
    const uint32_t r = qr[j], kk = qk[j];
    const int k = (int)(kk & 0xffffu), owner = (int)(kk >> 16);
    float mx[3], Sc[6];
    ViewCond c;
    for (int i = 0; i < 3; ++i) {
      mx[i] = prim[i][owner];
      c.shift[i] = qf[i][j];
      c.mc[i] = mx[i] + c.shift[i];
    }
    c.oq = qf[3][j];
    for (int i = 0; i < 6; ++i) Sc[i] = prim[3 + i][owner];
    const float beta_x = prim[9][owner];
    ViewOut o;
    view_project(mx, Sc, beta_x, true, c, s_views[k], cfg, o);
    tiles[r] = o.tiles;
    if (o.valid) {
      atomicOr(&s_vis[w][k], 1u << owner);
      key[r] = __float_as_uint(o.depth);
      rect[r] = make_uint2((uint32_t)o.tx0 | ((uint32_t)o.ty0 << 16), (uint32_t)o.tx1 | ((uint32_t)o.ty1 << 16));
      rec4[3 * (size_t)r + 0] = make_float4(o.mu_hi[0], o.mu_hi[1], o.mu_lo[0], o.mu_lo[1]);
      rec4[3 * (size_t)r + 1] = make_float4(o.conic[0], o.conic[1], o.conic[2], log2f(o.oq));
      rec4[3 * (size_t)r + 2] = make_float4(beta_x, prim[10][owner], prim[11][owner], prim[12][owner]);
      atomicOr(&s_any[w], 1u << owner);
    }
  };
  int qn = 0;  // warp-uniform
  for (int k = 0; k < vl.n; ++k) {
    const ViewDev& v = s_views[k];
    bool cand = false;
    ViewCond c;
    uint32_t r = 0;
    if (live) {
      view_condition<C>(in, vi, v, c, cull_below);
      r = v.rec_off + (uint32_t)p;
      cand = view_candidate(vi.valid, c, v, cfg);
      if (!cand) tiles[r] = 0;
    }
    const unsigned m = __ballot_sync(0xffffffffu, cand);
    if (cand) {
      const int j = qn + __popc(m & lt);
      qr[j] = r;
      qk[j] = (uint32_t)k | ((uint32_t)lane << 16);
      for (int i = 0; i < 3; ++i) qf[i][j] = c.shift[i];
      qf[3][j] = c.oq;
    }
    qn += __popc(m);
    __syncwarp();
    if (qn >= 32) {  // the 32 newest entries, one per lane
      project(qn - 32 + lane);
      qn -= 32;
      __syncwarp();
    }
  }
  if (lane < qn) project(lane);
  __syncwarp();
  // the warp's visibility mask word of each view (its primitives start at a
  // multiple of 32)
  const int64_t p0 = p - lane;
  if (p0 < sc.P)
    for (int k = lane; k < vl.n; k += 32) vis_mask[s_views[k].mask_off + (uint32_t)(p0 >> 5)] = s_vis[w][k];
  // scenes with several views: the primitives some view sees, listed for the
  // parameter backward (one add per warp)
  const bool any = live && ((s_any[w] >> lane) & 1u);
  if (vl.n > 1) {
    const unsigned m = __ballot_sync(0xffffffffu, any);
    if (m) {
      uint32_t base = 0;
      if (lane == 0) base = atomicAdd(act_count, (uint32_t)__popc(m));
      base = __shfl_sync(0xffffffffu, base, 0);
      if (any) act_list[base + __popc(m & lt)] = (uint32_t)p;
    }
  }
}

constexpr int kMaxDevices = 64;
std::atomic<bool> g_queued_smem_set[kMaxDevices];

// the queued kernels' view table plus their static queues can pass 48 KB of
// shared memory (256 views): opt in once per device
cudaError_t prepare_queued() {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev >= 0 && dev < kMaxDevices && g_queued_smem_set[dev].load(std::memory_order_acquire)) return cudaSuccess;
  const int bytes = (int)(kMaxViews * sizeof(ViewDev));
  e = cudaFuncSetAttribute(preprocess_queued_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(preprocess_queued_kernel<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(preprocess_queued_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess && dev >= 0 && dev < kMaxDevices) g_queued_smem_set[dev].store(true, std::memory_order_release);
  return e;
}

cudaError_t launch_preprocess(const SceneDev& sc, const ViewList& vl, const ViewDev* views, const CfgDev& cfg,
                              const Layout& L, char* ws, uint32_t* act_list, uint32_t* act_count, uint32_t* zero,
                              uint32_t nzero, cudaStream_t st) {
  if (sc.P == 0 || vl.n == 0) return cudaSuccess;
  if (sc.N > 3) {
    const cudaError_t e = prepare_queued();
    if (e != cudaSuccess) return e;
  }
  const int threads = 256;
  const unsigned blocks = (unsigned)((sc.P + threads - 1) / threads);
  const size_t smem = sizeof(ViewDev) * vl.n;
  float4* rec4 = (float4*)(ws + L.rec4);
  uint32_t* key = (uint32_t*)(ws + L.key);
  uint32_t* tiles = (uint32_t*)(ws + L.tiles);
  uint2* rect = (uint2*)(ws + L.rect);
  uint32_t* vis = (uint32_t*)(ws + L.vis_mask);
  switch (sc.N) {
    case 3: launch_dependent(preprocess_kernel<0>, dim3(blocks), dim3(threads), smem, st, sc, vl, views, cfg, rec4, key, tiles, rect, vis, act_list, act_count, zero, nzero); break;
    case 4: launch_dependent(preprocess_queued_kernel<1>, dim3(blocks), dim3(threads), smem, st, sc, vl, views, cfg, rec4, key, tiles, rect, vis, act_list, act_count, zero, nzero); break;
    case 6: launch_dependent(preprocess_queued_kernel<3>, dim3(blocks), dim3(threads), smem, st, sc, vl, views, cfg, rec4, key, tiles, rect, vis, act_list, act_count, zero, nzero); break;
    case 7: launch_dependent(preprocess_queued_kernel<4>, dim3(blocks), dim3(threads), smem, st, sc, vl, views, cfg, rec4, key, tiles, rect, vis, act_list, act_count, zero, nzero); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace ubs
