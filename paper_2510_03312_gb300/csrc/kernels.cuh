// kernels.cuh -- launchers of the device kernels (one translation unit each).
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include "common.cuh"

namespace ubs {

// An NVTX range named after a C-ABI entry point, open for the call (host
// side; header-only NVTX3, a few nanoseconds when no profiler is attached),
// so that profiler timelines group each call's launches.
struct TraceRange {
  explicit TraceRange(const char* name) { nvtxRangePushA(name); }
  ~TraceRange() { nvtxRangePop(); }
  TraceRange(const TraceRange&) = delete;
  TraceRange& operator=(const TraceRange&) = delete;
};

// Programmatic dependent launch (sm_90 and later): a kernel started with
// launch_dependent may be scheduled while the previous kernel on the stream
// drains.  It must call wait_prior_grid() before its first access to memory
// written by earlier work: griddepcontrol.wait returns once the previous
// grid has completed and its writes are visible (and at once for a kernel
// launched without the attribute).  Every kernel waiting first keeps the
// ordering transitive.
__device__ __forceinline__ void wait_prior_grid() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
// Whether the blend kernels take the tiles in the order of bin_sort's tile
// order (longest lists first) or in their own order: reordering pays where
// lists are long on average (a few long tiles would otherwise trail the
// grid) and costs locality where they are short.
constexpr uint32_t kOrdDense = 64;  // instances per tile from which the tiles are reordered
__device__ __forceinline__ bool order_dense(const Header* hdr, uint32_t NT, uint32_t cap) {
  const uint64_t n = hdr->n_inst < cap ? hdr->n_inst : cap;
  return n >= (uint64_t)kOrdDense * NT;
}
// whether an order can pay at all: more tiles than a few waves of blend
// CTAs (with fewer, every tile starts at once) and an instance capacity that
// allows dense lists; where not, no order is made and the blend kernels get
// none
constexpr uint32_t kOrdMinTiles = 1024;
inline bool order_possible(const Layout& L) {
  return L.NT > kOrdMinTiles && (uint64_t)L.cap >= (uint64_t)kOrdDense * L.NT;
}

// The binning walks a record's rectangle of up to kSoloTiles tiles in its
// own lane and a larger one with the whole warp.
constexpr uint32_t kSoloTiles = 8;

// Calls f(g, rec) for every tile g of each active lane's rectangle that has
// more than kSoloTiles tiles (n tiles: columns x0 <= tx < x1 of
// rc.x/rc.y's low halves, rows y0 <= ty < y1 of their high halves, at tile
// toff + ty tsx + tx of the view), the active lanes, which must be converged
// at the call, taking the rectangles in turn.
template <class F>
__device__ __forceinline__ void walk_large_rects(uint32_t n, uint2 rc, uint32_t toff, uint32_t tsx, uint32_t rec,
                                                 F&& f) {
  const unsigned act = __activemask();
  unsigned big = __ballot_sync(act, n > kSoloTiles);
  if (!big) return;
  const unsigned lane = threadIdx.x & 31;
  const uint32_t nact = (uint32_t)__popc(act), me = (uint32_t)__popc(act & ((1u << lane) - 1u));
  while (big) {
    const int src = __ffs(big) - 1;
    big &= big - 1;
    const uint32_t sn = __shfl_sync(act, n, src), sx = __shfl_sync(act, rc.x, src), sy = __shfl_sync(act, rc.y, src);
    const uint32_t so = __shfl_sync(act, toff, src), ss = __shfl_sync(act, tsx, src), sr = __shfl_sync(act, rec, src);
    const uint32_t sx0 = sx & 0xFFFFu, w = (sy & 0xFFFFu) - sx0, sy0 = sx >> 16;
    for (uint32_t k = me; k < sn; k += nact) f(so + (sy0 + k / w) * ss + sx0 + k % w, sr);
  }
}

// The tiles of a rectangle of at most kSoloTiles tiles, row-major; entries
// k >= n are left as they are.
__device__ __forceinline__ void solo_tiles(uint32_t n, uint2 rc, uint32_t toff, uint32_t tsx,
                                           uint32_t (&g)[kSoloTiles]) {
  const uint32_t x0 = rc.x & 0xFFFFu, x1 = rc.y & 0xFFFFu;
  uint32_t tx = x0, ty = rc.x >> 16;
#pragma unroll
  for (uint32_t k = 0; k < kSoloTiles; ++k) {
    if (k < n) g[k] = toff + ty * tsx + tx;
    if (++tx == x1) tx = x0, ++ty;
  }
}

template <typename... Params, typename... Args>
cudaError_t launch_dependent(void (*kernel)(Params...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                             Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, args...);
}

// the views that render one scene, by index into the view table
struct ViewList {
  int32_t n;
  int16_t idx[kMaxViews];
};

// act_list/act_count: the scene's list of primitives visible in some view
// (appended by preprocess, read by the parameter backward)
// zero/nzero: words the launch zeroes besides its own work (the binning's
// counters), or none
cudaError_t launch_preprocess(const SceneDev& sc, const ViewList& vl, const ViewDev* views, const CfgDev& cfg,
                              const Layout& L, char* ws, uint32_t* act_list, uint32_t* act_count, uint32_t* zero,
                              uint32_t nzero, cudaStream_t st);

// count, scan (ranges), scatter, per-tile sort and merge; leaves the sorted
// instance records in the buffer reported by sorted_instances()
cudaError_t launch_bin_sort(const Layout& L, const CfgDev& cfg, char* ws, cudaStream_t st);
const uint32_t* sorted_instances(const Layout& L, const char* ws);
// blocks of the binning's walks over the visible records (each count block
// writes its visible records to vis_part[block])
uint32_t walk_blocks(const Layout& L);

cudaError_t launch_render_fwd(const Layout& L, const CfgDev& cfg, char* ws, float* image, cudaStream_t st);
cudaError_t launch_render_bwd(const Layout& L, const CfgDev& cfg, char* ws, const float* dL_dimage, cudaStream_t st);
cudaError_t launch_prim_backward(const SceneDev& sc, const SceneGradDev& g, const ViewList& vl, const ViewDev* views,
                                 const CfgDev& cfg, const Layout& L, char* ws, const uint32_t* act_list,
                                 const uint32_t* act_count, cudaStream_t st);

}  // namespace ubs
