// abi.cu -- the extern "C" entry points of include/ubs.h: argument checks,
// workspace layout and kernel launches.  No entry point allocates device or
// host memory; ubs_read_status is the only one that synchronises.
#include <string.h>

#include "ubs.h"
#include "kernels.cuh"

namespace ubs {
namespace {

constexpr int kUploadChunk = 16;
struct ViewChunk {
  ViewDev v[kUploadChunk];
};

// Copies a chunk of the view table; the first chunk's launch also zeroes
// the status header and the per-scene counts of drawn primitives (hdr and
// act_count non-null).
__global__ void upload_views_kernel(ViewChunk chunk, int n, ViewDev* dst, uint32_t* hdr, uint32_t hdr_words,
                                    uint32_t* act_count, int S) {
  const int i = threadIdx.x;
  if (i < n) dst[i] = chunk.v[i];
  if (hdr) {
    for (uint32_t k = i; k < hdr_words; k += blockDim.x) hdr[k] = 0;
    for (int k = i; k < S; k += blockDim.x) act_count[k] = 0;
  }
}

inline size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

bool aligned4(const void* p) { return ((uintptr_t)p & 3u) == 0; }

ubs_status check_scene(const ubs_scene& s) {
  if (!(s.N == 3 || s.N == 4 || s.N == 6 || s.N == 7)) return UBS_ERR_INVALID_ARG;
  if (s.rot_mode < UBS_ROT_QUAT || s.rot_mode > UBS_ROT_EXP) return UBS_ERR_INVALID_ARG;
  if (s.P < 0 || s.P > (int64_t)0x7fffffff) return UBS_ERR_INVALID_ARG;
  if (s.P == 0) return UBS_OK;
  const void* req[] = {s.mean_x, s.rot, s.scale_x, s.b, s.opacity, s.rgb};
  for (const void* p : req) {
    if (!p) return UBS_ERR_INVALID_ARG;
    if (!aligned4(p)) return UBS_ERR_ALIGNMENT;
  }
  if (s.N > 3) {
    const void* q[] = {s.mean_q, s.L_qx, s.L_q};
    for (const void* p : q) {
      if (!p) return UBS_ERR_INVALID_ARG;
      if (!aligned4(p)) return UBS_ERR_ALIGNMENT;
    }
  }
  return UBS_OK;
}

bool tile_ok(int tw, int th) {
  return (tw == 16 && th == 16) || (tw == 8 && th == 8) || (tw == 16 && th == 32) || (tw == 32 && th == 32);
}

ubs_status make_layout(const ubs_problem* pr, Layout& L) {
  if (!pr || !pr->scenes || !pr->views) return UBS_ERR_INVALID_ARG;
  if (pr->n_scenes < 1 || pr->n_scenes > kMaxScenes) return UBS_ERR_INVALID_ARG;
  if (pr->n_views < 1 || pr->n_views > kMaxViews) return UBS_ERR_INVALID_ARG;
  const ubs_config& c = pr->cfg;
  if (!tile_ok(c.tile_w, c.tile_h)) return UBS_ERR_INVALID_ARG;
  if (!(c.alpha_max > 0.0f && c.alpha_max <= 1.0f) || !(c.alpha_min >= 0.0f) || !(c.T_min >= 0.0f) ||
      !(c.eps2d >= 0.0f) || !(c.jac_clip > 0.0f))
    return UBS_ERR_INVALID_ARG;
  if (pr->instance_capacity < 0 || pr->instance_capacity > (int64_t)0x7fffffff) return UBS_ERR_INVALID_ARG;
  for (int s = 0; s < pr->n_scenes; ++s) {
    const ubs_status st = check_scene(pr->scenes[s]);
    if (st != UBS_OK) return st;
  }
  uint64_t R = 0, NT = 0, NPIX = 0;
  for (int v = 0; v < pr->n_views; ++v) {
    const ubs_view& w = pr->views[v];
    if (w.scene_id < 0 || w.scene_id >= pr->n_scenes) return UBS_ERR_INVALID_ARG;
    if (w.width < 1 || w.height < 1 || w.width > 16384 || w.height > 16384) return UBS_ERR_INVALID_ARG;
    if (!(w.fx > 0.0f) || !(w.fy > 0.0f)) return UBS_ERR_INVALID_ARG;
    const uint64_t tx = (w.width + c.tile_w - 1) / c.tile_w, ty = (w.height + c.tile_h - 1) / c.tile_h;
    R += (uint64_t)pr->scenes[w.scene_id].P;
    NT += tx * ty;
    NPIX += (uint64_t)w.width * w.height;
  }
  if (R > 0x7fffffffull || NT * kTileSub > 0x7fffffffull || NPIX > 0x7fffffffull) return UBS_ERR_INVALID_ARG;
  memset(&L, 0, sizeof(L));
  L.V = pr->n_views;
  L.S = pr->n_scenes;
  L.R = (uint32_t)R;
  L.NT = (uint32_t)NT;
  L.NPIX = (uint32_t)NPIX;
  L.cap = (uint32_t)(pr->instance_capacity > 0 ? pr->instance_capacity : 1);
  L.n_scan_blocks = (L.NT + kScanTiles - 1) / kScanTiles;
  uint64_t words = 0;
  for (int v = 0; v < pr->n_views; ++v) words += (uint64_t)(pr->scenes[pr->views[v].scene_id].P + 31) / 32;
  L.mask_words = (uint32_t)words;
  L.max_items = L.NT + L.cap / kSortChunk + 1;
  size_t o = 0;
  auto take = [&](size_t bytes) {
    const size_t at = o;
    o = align256(o + bytes);
    return at;
  };
  L.header = take(sizeof(Header));
  L.views = take(sizeof(ViewDev) * L.V);
  L.rec4 = take((size_t)L.R * kRecFloats * 4);
  L.key = take((size_t)L.R * 4);
  L.tiles = take((size_t)L.R * 4);
  L.rect = take((size_t)L.R * 8);
  L.g2d = take((size_t)L.R * kGradFloats * 4);
  L.tcount = take((size_t)L.NT * kTileSub * 4 + 4 * 132 * 4 + kVisBlocks * 4);
  L.order_count = L.tcount + (size_t)L.NT * kTileSub * 4;
  L.vis_part = L.order_count + 4 * 132 * 4;
  L.cursor = take((size_t)L.NT * kTileSub * 4);
  L.vis_mask = take((size_t)L.mask_words * 4);
  L.bucket = take((size_t)L.cap * 4);
  L.ivals = take((size_t)L.cap * 4);
  L.chunk64 = take((size_t)L.cap * 8);
  L.tmp64 = take((size_t)L.cap * 8);
  L.items = take((size_t)L.max_items * 8);
  L.scan_part = take(((size_t)2 * L.n_scan_blocks + 1) * 16);
  L.tstart = take((size_t)(L.NT + 1) * 4);
  L.tile_order = take((size_t)L.NT * 4);
  // the primitives some view sees, per scene
  uint64_t Ptot = 0;
  for (int sc = 0; sc < pr->n_scenes; ++sc) Ptot += (uint64_t)pr->scenes[sc].P;
  L.act_list = take((size_t)Ptot * 4);
  L.act_count = take((size_t)kMaxScenes * 4);
  L.Tfin = take((size_t)L.NPIX * 4);
  L.last = take((size_t)L.NPIX * 4);
  L.pairs = take((size_t)L.NPIX * 8);  // pairs with r < 1, then visited entries
  if (c.flags & kFlagSplit) {
    // a split tile holds more than kSegLen instances, and its segments number
    // at most its instances / kSegLen + 1: bounds from the capacity
    L.seg_max_split = L.cap / kSegLen + 1;
    L.seg_max_extra = L.cap / kSegLen + 1;
    L.seg_slots = 2 * (L.cap / kSegLen) + 2;
    L.split_list = take((size_t)L.seg_max_split * 16);
    L.tile_slot = take((size_t)L.NT * 4);
    L.seg_buf = take((size_t)L.seg_slots * (size_t)c.tile_w * (size_t)c.tile_h * 32);
    L.slot_owner = take((size_t)L.seg_slots * 4);
    L.ext_owner = take((size_t)L.seg_max_extra * 4);
    L.split_term = take((size_t)L.seg_max_split * 4);
  }
  L.total = o;
  return UBS_OK;
}

ubs_status prepare(const ubs_problem* pr, void* ws, size_t ws_bytes, Layout& L) {
  const ubs_status st = make_layout(pr, L);
  if (st != UBS_OK) return st;
  if (!ws) return UBS_ERR_INVALID_ARG;
  if (((uintptr_t)ws & 255u) != 0) return UBS_ERR_ALIGNMENT;
  if (ws_bytes < L.total) return UBS_ERR_WORKSPACE;
  return UBS_OK;
}

CfgDev cfg_dev(const ubs_config& c) {
  CfgDev d;
  d.tw = c.tile_w;
  d.th = c.tile_h;
  d.amin = c.alpha_min;
  d.amax = c.alpha_max;
  d.tmin = c.T_min;
  d.eps = c.eps2d;
  d.near_plane = c.near_plane;
  d.clip = c.jac_clip;
  d.bg[0] = c.bg[0];
  d.bg[1] = c.bg[1];
  d.bg[2] = c.bg[2];
  d.flags = c.flags;
  if (c.flags & kFlagNoThresholds) {  // the gradient-check mode: every pair with r < 1 is composited
    d.amin = 0.0f;
    d.amax = 1.0f;
    d.tmin = 0.0f;
  }
  return d;
}

SceneDev scene_dev(const ubs_scene& s) {
  SceneDev d;
  d.mean_x = s.mean_x;
  d.mean_q = s.mean_q;
  d.rot = s.rot;
  d.scale_x = s.scale_x;
  d.L_qx = s.L_qx;
  d.L_q = s.L_q;
  d.b = s.b;
  d.opacity = s.opacity;
  d.rgb = s.rgb;
  d.N = s.N;
  d.rot_mode = s.rot_mode;
  d.P = s.P;
  return d;
}

void view_list(const ubs_problem* pr, int scene, ViewList& vl) {
  vl.n = 0;
  for (int v = 0; v < pr->n_views; ++v)
    if (pr->views[v].scene_id == scene) vl.idx[vl.n++] = (int16_t)v;
}

ubs_status cuda_status(cudaError_t e) { return e == cudaSuccess ? UBS_OK : UBS_ERR_CUDA; }

ubs_status check_grads(const ubs_problem* pr, const Layout& L, const ubs_scene_grad* grads) {
  for (int s = 0; s < L.S; ++s) {
    const ubs_scene& sc = pr->scenes[s];
    if (sc.P == 0) continue;
    const ubs_scene_grad& g = grads[s];
    const void* req[] = {g.mean_x, g.rot, g.scale_x, g.b, g.opacity, g.rgb};
    for (const void* p : req) {
      if (!p) return UBS_ERR_INVALID_ARG;
      if (!aligned4(p)) return UBS_ERR_ALIGNMENT;
    }
    if (sc.N > 3) {
      const void* q[] = {g.mean_q, g.L_qx, g.L_q};
      for (const void* p : q) {
        if (!p) return UBS_ERR_INVALID_ARG;
        if (!aligned4(p)) return UBS_ERR_ALIGNMENT;
      }
    }
  }
  return UBS_OK;
}

}  // namespace
}  // namespace ubs

using namespace ubs;

extern "C" {

size_t ubs_workspace_size(const ubs_problem* problem) {
  Layout L;
  if (make_layout(problem, L) != UBS_OK) return 0;
  return L.total;
}

ubs_status ubs_preprocess(const ubs_problem* pr, void* ws, size_t ws_bytes, cudaStream_t stream) {
  ubs::TraceRange trace_("ubs_preprocess");
  Layout L;
  ubs_status st = prepare(pr, ws, ws_bytes, L);
  if (st != UBS_OK) return st;
  char* w = (char*)ws;
  cudaError_t e = cudaSuccess;
  // view table: per-view constants, tile/record/pixel/mask offsets
  ViewDev* views = (ViewDev*)(w + L.views);
  uint32_t tile_off = 0, rec_off = 0, pix_off = 0, mask_off = 0;
  for (int c0 = 0; c0 < L.V; c0 += kUploadChunk) {
    ViewChunk chunk;
    memset(&chunk, 0, sizeof(chunk));
    const int n = (L.V - c0) < kUploadChunk ? (L.V - c0) : kUploadChunk;
    for (int i = 0; i < n; ++i) {
      const ubs_view& v = pr->views[c0 + i];
      ViewDev& d = chunk.v[i];
      memcpy(d.R, v.R, sizeof(d.R));
      memcpy(d.t, v.t, sizeof(d.t));
      d.fx = v.fx;
      d.fy = v.fy;
      d.cx = v.cx;
      d.cy = v.cy;
      d.W = v.width;
      d.H = v.height;
      d.time = v.time;
      d.scene = v.scene_id;
      d.tiles_x = (v.width + pr->cfg.tile_w - 1) / pr->cfg.tile_w;
      d.tiles_y = (v.height + pr->cfg.tile_h - 1) / pr->cfg.tile_h;
      d.tile_off = tile_off;
      d.rec_off = rec_off;
      d.pix_off = pix_off;
      d.mask_off = mask_off;
      tile_off += (uint32_t)(d.tiles_x * d.tiles_y);
      rec_off += (uint32_t)pr->scenes[v.scene_id].P;
      pix_off += (uint32_t)(v.width * v.height);
      mask_off += (uint32_t)((pr->scenes[v.scene_id].P + 31) / 32);
    }
    static_assert(sizeof(Header) % 4 == 0, "the header is zeroed by words");
    upload_views_kernel<<<1, kUploadChunk, 0, stream>>>(chunk, n, views + c0,
                                                         c0 == 0 ? (uint32_t*)(w + L.header) : nullptr,
                                                         (uint32_t)(sizeof(Header) / 4), (uint32_t*)(w + L.act_count),
                                                         L.S);
    e = cudaGetLastError();
    if (e != cudaSuccess) return UBS_ERR_CUDA;
  }
  const CfgDev cfg = cfg_dev(pr->cfg);
  uint64_t act_off = 0;
  // the first scene that launches also zeroes the binning's counters (tile
  // counters, length buckets, visible records per count block); where no
  // scene launches there are no records and the binning reads none of them
  bool zeroed = false;
  const uint32_t nzero = L.NT * kTileSub + 4 * 132 + kVisBlocks;
  for (int s = 0; s < L.S; ++s) {
    ViewList vl;
    view_list(pr, s, vl);
    const bool launches = pr->scenes[s].P > 0 && vl.n > 0;
    uint32_t* zero = launches && !zeroed ? (uint32_t*)(w + L.tcount) : nullptr;
    zeroed = zeroed || launches;
    e = launch_preprocess(scene_dev(pr->scenes[s]), vl, views, cfg, L, w, (uint32_t*)(w + L.act_list) + act_off,
                          (uint32_t*)(w + L.act_count) + s, zero, zero ? nzero : 0u, stream);
    act_off += (uint64_t)pr->scenes[s].P;
    if (e != cudaSuccess) return UBS_ERR_CUDA;
  }
  return UBS_OK;
}

ubs_status ubs_bin_sort(const ubs_problem* pr, void* ws, size_t ws_bytes, cudaStream_t stream) {
  ubs::TraceRange trace_("ubs_bin_sort");
  Layout L;
  ubs_status st = prepare(pr, ws, ws_bytes, L);
  if (st != UBS_OK) return st;
  return cuda_status(launch_bin_sort(L, cfg_dev(pr->cfg), (char*)ws, stream));
}

ubs_status ubs_render_fwd(const ubs_problem* pr, void* ws, size_t ws_bytes, float* image, cudaStream_t stream) {
  ubs::TraceRange trace_("ubs_render_fwd");
  Layout L;
  ubs_status st = prepare(pr, ws, ws_bytes, L);
  if (st != UBS_OK) return st;
  if (!image) return UBS_ERR_INVALID_ARG;
  if (!aligned4(image)) return UBS_ERR_ALIGNMENT;
  return cuda_status(launch_render_fwd(L, cfg_dev(pr->cfg), (char*)ws, image, stream));
}

ubs_status ubs_render_bwd_blend(const ubs_problem* pr, void* ws, size_t ws_bytes, const float* dL_dimage,
                                cudaStream_t stream) {
  ubs::TraceRange trace_("ubs_render_bwd_blend");
  Layout L;
  ubs_status st = prepare(pr, ws, ws_bytes, L);
  if (st != UBS_OK) return st;
  if (!dL_dimage) return UBS_ERR_INVALID_ARG;
  if (!aligned4(dL_dimage)) return UBS_ERR_ALIGNMENT;
  return cuda_status(launch_render_bwd(L, cfg_dev(pr->cfg), (char*)ws, dL_dimage, stream));
}

ubs_status ubs_render_bwd_params(const ubs_problem* pr, void* ws, size_t ws_bytes, const ubs_scene_grad* grads,
                                 cudaStream_t stream) {
  ubs::TraceRange trace_("ubs_render_bwd_params");
  Layout L;
  ubs_status st = prepare(pr, ws, ws_bytes, L);
  if (st != UBS_OK) return st;
  if (!grads) return UBS_ERR_INVALID_ARG;
  st = check_grads(pr, L, grads);
  if (st != UBS_OK) return st;
  char* w = (char*)ws;
  const CfgDev cfg = cfg_dev(pr->cfg);
  const ViewDev* views = (const ViewDev*)(w + L.views);
  uint64_t act_off = 0;
  for (int s = 0; s < L.S; ++s) {
    ViewList vl;
    view_list(pr, s, vl);
    const ubs_scene_grad& g = grads[s];
    SceneGradDev gd = {g.mean_x, g.mean_q, g.rot, g.scale_x, g.L_qx, g.L_q, g.b, g.opacity, g.rgb};
    if (launch_prim_backward(scene_dev(pr->scenes[s]), gd, vl, views, cfg, L, w,
                             (const uint32_t*)(w + L.act_list) + act_off, (const uint32_t*)(w + L.act_count) + s,
                             stream) != cudaSuccess)
      return UBS_ERR_CUDA;
    act_off += (uint64_t)pr->scenes[s].P;
  }
  return UBS_OK;
}

ubs_status ubs_render_bwd(const ubs_problem* pr, void* ws, size_t ws_bytes, const float* dL_dimage,
                          const ubs_scene_grad* grads, cudaStream_t stream) {
  ubs::TraceRange trace_("ubs_render_bwd");
  Layout L;
  ubs_status st = prepare(pr, ws, ws_bytes, L);
  if (st != UBS_OK) return st;
  if (!dL_dimage || !grads) return UBS_ERR_INVALID_ARG;
  if (!aligned4(dL_dimage)) return UBS_ERR_ALIGNMENT;
  st = check_grads(pr, L, grads);
  if (st != UBS_OK) return st;
  st = ubs_render_bwd_blend(pr, ws, ws_bytes, dL_dimage, stream);
  if (st != UBS_OK) return st;
  return ubs_render_bwd_params(pr, ws, ws_bytes, grads, stream);
}


ubs_status ubs_read_status(const ubs_problem* pr, void* ws, size_t ws_bytes, ubs_device_status* out,
                           cudaStream_t stream) {
  ubs::TraceRange trace_("ubs_read_status");
  Layout L;
  ubs_status st = prepare(pr, ws, ws_bytes, L);
  if (st != UBS_OK) return st;
  if (!out) return UBS_ERR_INVALID_ARG;
  if (cudaStreamSynchronize(stream) != cudaSuccess) return UBS_ERR_CUDA;
  Header h;
  if (cudaMemcpy(&h, (char*)ws + L.header, sizeof(Header), cudaMemcpyDeviceToHost) != cudaSuccess)
    return UBS_ERR_CUDA;
  out->status = (int32_t)h.status;
  out->reserved = 0;
  uint32_t part[kVisBlocks];
  if (cudaMemcpy(part, (char*)ws + L.vis_part, sizeof(part), cudaMemcpyDeviceToHost) != cudaSuccess)
    return UBS_ERR_CUDA;
  int64_t vis = 0;
  const uint32_t nb = L.R ? walk_blocks(L) : 0u;
  for (uint32_t i = 0; i < nb; ++i) vis += part[i];
  out->visible_records = vis;
  out->instances = (int64_t)h.n_inst;
  return UBS_OK;
}

ubs_status ubs_export(const ubs_problem* pr, void* ws, size_t ws_bytes, int32_t what, void* dst, size_t dst_bytes,
                      size_t* bytes_needed, cudaStream_t stream) {
  ubs::TraceRange trace_("ubs_export");
  Layout L;
  ubs_status st = prepare(pr, ws, ws_bytes, L);
  if (st != UBS_OK) return st;
  size_t off = 0, n = 0;
  switch (what) {
    case 0: off = L.key; n = (size_t)L.R * 4; break;
    case 1: off = L.tiles; n = (size_t)L.R * 4; break;
    case 2: off = L.rect; n = (size_t)L.R * 8; break;
    case 3: off = L.rec4; n = (size_t)L.R * kRecFloats * 4; break;
    case 4: off = (size_t)((const char*)sorted_instances(L, (const char*)ws) - (const char*)ws); n = (size_t)L.cap * 4; break;
    case 5: off = L.tstart; n = (size_t)(L.NT + 1) * 4; break;
    case 6: off = L.Tfin; n = (size_t)L.NPIX * 4; break;
    case 7: off = L.last; n = (size_t)L.NPIX * 4; break;
    case 8: off = L.g2d; n = (size_t)L.R * kGradFloats * 4; break;
    case 9: off = L.pairs; n = (size_t)L.NPIX * 4; break;
    case 10: off = L.pairs + (size_t)L.NPIX * 4; n = (size_t)L.NPIX * 4; break;
    default: return UBS_ERR_INVALID_ARG;
  }
  if (bytes_needed) *bytes_needed = n;
  if (!dst) return UBS_OK;
  if (dst_bytes < n) return UBS_ERR_INVALID_ARG;
  return cuda_status(cudaMemcpyAsync(dst, (char*)ws + off, n, cudaMemcpyDeviceToDevice, stream));
}

const char* ubs_status_string(ubs_status s) {
  switch (s) {
    case UBS_OK: return "ok";
    case UBS_ERR_INVALID_ARG: return "invalid argument";
    case UBS_ERR_ALIGNMENT: return "misaligned pointer";
    case UBS_ERR_CAPACITY: return "instance capacity exceeded";
    case UBS_ERR_CUDA: return "CUDA error";
    case UBS_ERR_TIMEOUT: return "device-side wait timed out";
    case UBS_ERR_INTERNAL: return "internal error";
    case UBS_ERR_WORKSPACE: return "workspace too small";
  }
  return "unknown status";
}

}  // extern "C"
