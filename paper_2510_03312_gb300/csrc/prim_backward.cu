// prim_backward.cu -- G2: chain the per-record screen gradients back to the
// primitive parameters (math in prim_backward.cuh).
//
// One thread per primitive (scenes with one view: every primitive; with
// several: the list of primitives some view sees, built by preprocess); it
// rebuilds the view-independent quantities once, walks its visible views
// accumulating in registers, and writes every parameter gradient once: no
// atomics and a deterministic sum over views.
#include "kernels.cuh"
#include "prim_backward.cuh"

namespace ubs {

namespace {

template <int C>
__device__ __forceinline__ void load_prim_b(const SceneDev& sc, int64_t p, PrimIn<C>& in) {
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

// N = 3 (C = 0) is held to 72 registers (7 CTAs per SM): G2 is bound by
// memory latency and gains more from occupancy than it loses to a few spills
// to L1 (63.5 us unbounded, 53.7 at 6 CTAs, 51.9 at 7 on the 1M-primitive
// view; 8 gained nothing more); the larger query dimensions would spill too
// much
template <int C>
__global__ void __launch_bounds__(128, C == 0 ? 7 : 1) prim_backward_kernel(SceneDev sc, SceneGradDev gr, ViewList vl,
                                                            const ViewDev* __restrict__ views, CfgDev cfg,
                                                            const uint32_t* __restrict__ tiles,
                                                            const float4* __restrict__ g2d) {
  wait_prior_grid();
  extern __shared__ ViewDev s_views[];
  for (int i = threadIdx.x; i < vl.n; i += blockDim.x) s_views[i] = views[vl.idx[i]];
  __syncthreads();
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= sc.P) return;
  PrimIn<C> in;
  load_prim_b<C>(sc, p, in);
  PrimVI<C> vi;
  prim_stage<C>(in, sc.rot_mode, vi);
  PrimAcc<C> acc;
  acc_zero<C>(acc);
  for (int k = 0; k < vl.n; ++k) {
    const ViewDev& v = s_views[k];
    const uint32_t r = v.rec_off + (uint32_t)p;
    if (tiles[r] == 0) continue;
    const float4 a = g2d[3 * (size_t)r], b = g2d[3 * (size_t)r + 1], c = g2d[3 * (size_t)r + 2];
    const float g[10] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w, c.x, c.y};
    prim_backward_view<C>(in, vi, v, cfg, g, acc);
  }
  PrimGrad<C> out;
  prim_backward_final<C>(in, vi, sc.rot_mode, acc, out);
  const int64_t P = sc.P;
  // written, or added to the caller's running sum (UBS_FLAG_ACCUMULATE_GRADS)
  const bool add = (cfg.flags & 4) != 0;
  auto put = [&](float* dst, float v) { *dst = add ? *dst + v : v; };
  for (int i = 0; i < 3; ++i) put(gr.mean_x + i * P + p, out.mx[i]);
  const int nr = sc.rot_mode == 0 ? 4 : 3;
  for (int i = 0; i < nr; ++i) put(gr.rot + i * P + p, out.rot[i]);
  for (int i = 0; i < 3; ++i) put(gr.scale_x + i * P + p, out.s[i]);
  for (int i = 0; i < 1 + C; ++i) put(gr.b + i * P + p, out.b[i]);
  put(gr.opacity + p, out.o);
  for (int i = 0; i < 3; ++i) put(gr.rgb + i * P + p, out.rgb[i]);
  if constexpr (C > 0) {
    for (int i = 0; i < C; ++i) put(gr.mean_q + i * P + p, out.mq[i]);
    for (int i = 0; i < 3 * C; ++i) put(gr.L_qx + i * P + p, out.lqx[i]);
    for (int i = 0; i < C * (C + 1) / 2; ++i) put(gr.L_q + i * P + p, out.lq[i]);
  }
}


// Zeroes one scene's gradient planes (the primitives that no view sees keep
// these zeros; the others are overwritten by prim_backward_kernel).
__global__ void __launch_bounds__(256) zero_scene_grads_kernel(SceneGradDev gr, int64_t P, int C, int nr) {
  wait_prior_grid();
  const int64_t p = (int64_t)blockIdx.x * 256 + threadIdx.x;
  if (p >= P) return;
  for (int i = 0; i < 3; ++i) gr.mean_x[i * P + p] = 0.0f;
  for (int i = 0; i < nr; ++i) gr.rot[i * P + p] = 0.0f;
  for (int i = 0; i < 3; ++i) gr.scale_x[i * P + p] = 0.0f;
  for (int i = 0; i < 1 + C; ++i) gr.b[i * P + p] = 0.0f;
  gr.opacity[p] = 0.0f;
  for (int i = 0; i < 3; ++i) gr.rgb[i * P + p] = 0.0f;
  for (int i = 0; i < C; ++i) gr.mean_q[i * P + p] = 0.0f;
  for (int i = 0; i < 3 * C; ++i) gr.L_qx[i * P + p] = 0.0f;
  for (int i = 0; i < C * (C + 1) / 2; ++i) gr.L_q[i * P + p] = 0.0f;
}

// Scenes with several views: one thread per primitive some view sees (the
// scene's list from preprocess, walked grid-stride), so that warps stay full
// however sparse the visibility; the other primitives keep the zeros of
// zero_scene_grads_kernel (or their sum, when accumulating).  Each lane walks
// only its own visible views (a bit mask per 32 views), so a warp runs as
// many per-view steps as its busiest lane needs.  The C = 3 instantiation
// (216 registers unbounded) is held to 128 so that four CTAs share an SM: it
// is bound by memory latency, and the occupancy outweighs its spills (the
// 16-view N=6 batch 135 -> 122 us); the C = 4 one lost time that way.
template <int C>
__global__ void __launch_bounds__(128, C == 3 ? 4 : 1) prim_backward_listed_kernel(SceneDev sc, SceneGradDev gr, ViewList vl,
                                                            const ViewDev* __restrict__ views, CfgDev cfg,
                                                            const uint32_t* __restrict__ tiles,
                                                            const float4* __restrict__ g2d,
                                                            const uint32_t* __restrict__ act_list,
                                                            const uint32_t* act_count) {
  wait_prior_grid();
  extern __shared__ ViewDev s_views[];
  for (int i = threadIdx.x; i < vl.n; i += blockDim.x) s_views[i] = views[vl.idx[i]];
  __syncthreads();
  const int64_t P = sc.P;
  const int64_t n_items = (int64_t)*act_count;
  const bool add = (cfg.flags & 4) != 0;  // add to the caller's running sum (UBS_FLAG_ACCUMULATE_GRADS)
  auto put = [&](float* dst, float v) { *dst = add ? *dst + v : v; };
  const int nr = sc.rot_mode == 0 ? 4 : 3;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_items; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p = act_list[i];
    PrimIn<C> in;
    load_prim_b<C>(sc, p, in);
    PrimVI<C> vi;
    prim_stage<C>(in, sc.rot_mode, vi);
    PrimAcc<C> acc;
    acc_zero<C>(acc);
    // each lane walks only its own visible views (a bit mask per 32 views),
    // so a warp runs as many per-view steps as its busiest lane needs rather
    // than one per view that any lane sees
    for (int k0 = 0; k0 < vl.n; k0 += 32) {
      const int k1 = min(vl.n, k0 + 32);
      unsigned vis = 0;
      for (int k = k0; k < k1; ++k) vis |= (tiles[s_views[k].rec_off + (uint32_t)p] != 0 ? 1u : 0u) << (k - k0);
      while (vis) {
        const int k = k0 + __ffs(vis) - 1;
        vis &= vis - 1;
        const ViewDev& v = s_views[k];
        const uint32_t r = v.rec_off + (uint32_t)p;
        const float4 a = g2d[3 * (size_t)r], b = g2d[3 * (size_t)r + 1], c = g2d[3 * (size_t)r + 2];
        const float g[10] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w, c.x, c.y};
        prim_backward_view<C>(in, vi, v, cfg, g, acc);
      }
    }
    PrimGrad<C> out;
    prim_backward_final<C>(in, vi, sc.rot_mode, acc, out);
    for (int j = 0; j < 3; ++j) put(gr.mean_x + j * P + p, out.mx[j]);
    for (int j = 0; j < nr; ++j) put(gr.rot + j * P + p, out.rot[j]);
    for (int j = 0; j < 3; ++j) put(gr.scale_x + j * P + p, out.s[j]);
    for (int j = 0; j < 1 + C; ++j) put(gr.b + j * P + p, out.b[j]);
    put(gr.opacity + p, out.o);
    for (int j = 0; j < 3; ++j) put(gr.rgb + j * P + p, out.rgb[j]);
    if constexpr (C > 0) {
      for (int j = 0; j < C; ++j) put(gr.mean_q + j * P + p, out.mq[j]);
      for (int j = 0; j < 3 * C; ++j) put(gr.L_qx + j * P + p, out.lqx[j]);
      for (int j = 0; j < C * (C + 1) / 2; ++j) put(gr.L_q + j * P + p, out.lq[j]);
    }
  }
}

}  // namespace

cudaError_t launch_prim_backward(const SceneDev& sc, const SceneGradDev& g, const ViewList& vl, const ViewDev* views,
                                 const CfgDev& cfg, const Layout& L, char* ws, const uint32_t* act_list,
                                 const uint32_t* act_count, cudaStream_t st) {
  if (sc.P == 0) return cudaSuccess;
  const int threads = 128;
  const int64_t nblk = (sc.P + threads - 1) / threads;
  const size_t smem = sizeof(ViewDev) * vl.n;
  const uint32_t* tiles = (const uint32_t*)(ws + L.tiles);
  const float4* g2d = (const float4*)(ws + L.g2d);
  cudaError_t e = cudaSuccess;
  if (vl.n <= 1) {  // one view: every primitive, directly
    const unsigned blocks = (unsigned)nblk;
    switch (sc.N) {
      case 3: e = launch_dependent(prim_backward_kernel<0>, dim3(blocks), dim3(threads), smem, st, sc, g, vl, views, cfg, tiles, g2d); break;
      case 4: e = launch_dependent(prim_backward_kernel<1>, dim3(blocks), dim3(threads), smem, st, sc, g, vl, views, cfg, tiles, g2d); break;
      case 6: e = launch_dependent(prim_backward_kernel<3>, dim3(blocks), dim3(threads), smem, st, sc, g, vl, views, cfg, tiles, g2d); break;
      case 7: e = launch_dependent(prim_backward_kernel<4>, dim3(blocks), dim3(threads), smem, st, sc, g, vl, views, cfg, tiles, g2d); break;
      default: return cudaErrorInvalidValue;
    }
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
  }
  // several views: the listed primitives, the others zeroed first unless accumulating
  if (!(cfg.flags & 4)) {
    e = launch_dependent(zero_scene_grads_kernel, dim3((unsigned)((sc.P + 255) / 256)), dim3(256), 0, st, g, sc.P,
                         sc.N - 3, sc.rot_mode == 0 ? 4 : 3);
    if (e != cudaSuccess) return e;
  }
  const unsigned blocks = (unsigned)(nblk < 152 * 8 ? nblk : 152 * 8);
  switch (sc.N) {
    case 3: e = launch_dependent(prim_backward_listed_kernel<0>, dim3(blocks), dim3(threads), smem, st, sc, g, vl, views, cfg, tiles, g2d, act_list, act_count); break;
    case 4: e = launch_dependent(prim_backward_listed_kernel<1>, dim3(blocks), dim3(threads), smem, st, sc, g, vl, views, cfg, tiles, g2d, act_list, act_count); break;
    case 6: e = launch_dependent(prim_backward_listed_kernel<3>, dim3(blocks), dim3(threads), smem, st, sc, g, vl, views, cfg, tiles, g2d, act_list, act_count); break;
    case 7: e = launch_dependent(prim_backward_listed_kernel<4>, dim3(blocks), dim3(threads), smem, st, sc, g, vl, views, cfg, tiles, g2d, act_list, act_count); break;
    default: return cudaErrorInvalidValue;
  }
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

}  // namespace ubs
