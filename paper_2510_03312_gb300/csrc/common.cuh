// common.cuh -- types shared by the kernels and the C-ABI layer.
#pragma once

#include <stddef.h>
#include <stdint.h>

#ifndef UBS_HD
#define UBS_HD __host__ __device__ __forceinline__
#endif

namespace ubs {

constexpr int kMaxViews = 256;
constexpr int kMaxScenes = 64;
constexpr float kLn2f = 0x1.62e430p-1f;

// View constants as the kernels see them (one per view, in the workspace).
struct ViewDev {
  float R[9];
  float t[3];
  float fx, fy, cx, cy;
  int32_t W, H;
  float time;
  int32_t scene;
  int32_t tiles_x, tiles_y;
  uint32_t tile_off;  // first global tile id of the view
  uint32_t rec_off;   // first record of the view
  uint32_t pix_off;   // first pixel of the view (images are packed)
  uint32_t mask_off;  // first word of the view's visibility mask (a bit per primitive)
  uint32_t pad[2];
};
static_assert(sizeof(ViewDev) == 112, "ViewDev layout");

struct CfgDev {
  int32_t tw, th;
  float amin, amax, tmin, eps, near_plane, clip;
  float bg[3];
  int32_t flags;
};

struct SceneDev {
  const float* mean_x;
  const float* mean_q;
  const float* rot;
  const float* scale_x;
  const float* L_qx;
  const float* L_q;
  const float* b;
  const float* opacity;
  const float* rgb;
  int32_t N, rot_mode;
  int64_t P;
};

struct SceneGradDev {
  float* mean_x;
  float* mean_q;
  float* rot;
  float* scale_x;
  float* L_qx;
  float* L_q;
  float* b;
  float* opacity;
  float* rgb;
};

// Device status block at the start of the workspace.
struct Header {
  uint32_t status;       // ubs_status of device-side work (0 = ok)
  uint32_t n_items;      // work items of the per-tile sort (0 after a capacity overflow)
  uint64_t n_inst;       // instances required
  uint32_t n_long;       // of those, the chunks of lists longer than kSortChunk (listed first)
  uint32_t pad0;
  uint32_t ctr[32];      // dynamic tile counters, one per single-pass kernel
};

// Workspace layout, computed on the host from the problem.
struct Layout {
  int32_t V, S;
  uint32_t R;       // records
  uint32_t NT;      // tiles
  uint32_t NPIX;    // pixels
  uint32_t cap;     // instance capacity
  uint32_t n_scan_blocks;  // blocks of the tile-count scan (kScanTiles tiles each)
  uint32_t mask_words;     // words of the visibility masks: the sum over views of ceil(P / 32)
  uint32_t max_items;      // bound on the per-tile sort's work items: NT + cap / kSortChunk + 1
  size_t header, views, rec4, key, tiles, rect, g2d;
  size_t tcount;     // instances per (tile, sub-bucket) [kTileSub][NT], then per length bucket
                     // the totals and cursors of the tile order and of the short lists' sort
                     // items [4 x 132], then the visible records per count block [kVisBlocks]
                     // (zeroed together by ubs_preprocess)
  size_t cursor;     // next free slot of each (tile, sub-bucket) [kTileSub][NT]
  size_t vis_mask;   // per view, a bit per primitive: visible (written whole by preprocess) [mask_words]
  size_t bucket;     // the instances grouped by tile, unordered within a tile [cap]
  size_t ivals;      // the sorted instance lists [cap]
  size_t chunk64;    // sorted chunks (depth << 32 | record) of lists longer than kSortChunk [cap]
  size_t tmp64;      // the other buffer of their merge rounds [cap]
  size_t items;      // (tile, chunk) work items of the per-tile sort [max_items]
  size_t scan_part;  // per scan block: instances (u64) and items, then their exclusive prefixes
  size_t tstart;
  size_t tile_order;   // the order the blend kernels take the tiles in [NT]
  size_t order_count;  // the length buckets' totals and cursors [4 x 132] (after tcount)
  size_t vis_part;     // visible records per block of the binning's count walk [kVisBlocks] (after order_count)
  size_t act_list;   // per scene (at the sum of the earlier scenes' P): primitives visible in some view
  size_t act_count;  // their number per scene [kMaxScenes]
  size_t Tfin, last, pairs;
  // long tile lists split across CTAs (UBS_FLAG_SPLIT_LISTS): the split
  // tiles [seg_max_split] x (tile, first slot, segments, first extra
  // segment), each tile's first slot or ~0 [NT], and per (slot, pixel of
  // the tile) 8 floats of segment state [seg_slots][tile pixels][8]
  size_t split_list, tile_slot, seg_buf;
  size_t slot_owner;  // split tile of each slot [seg_slots]
  size_t ext_owner;   // split tile of each extra segment [seg_max_extra]
  size_t split_term;  // per split tile: the first segment after which every pixel had ended [seg_max_split]
  uint32_t seg_max_split, seg_max_extra, seg_slots;
  size_t total;
};

// Tiles whose lists are longer than kSegLen entries are split into segments
// of kSegLen entries (a multiple of every blend batch size) when
// UBS_FLAG_SPLIT_LISTS is set.
constexpr uint32_t kSegLen = 2048;
constexpr uint32_t kFlagSplit = 16;
constexpr uint32_t kFlagNoThresholds = 32;
constexpr uint32_t kFlagChecked = 64;

// float record of one (view, primitive) for the blend kernels: 3 x float4
//   [mu'_x hi, mu'_y hi, mu'_x lo, mu'_y lo]
//   [conic a, conic b, conic c, log2 o(q)]
//   [beta_x, r, g, b]
// r = a dx^2 + 2 b dx dy + c dy^2 with dx = (px - hi_x) - lo_x.
constexpr int kRecFloats = 12;
// per-record screen-space gradient: 3 x float4
//   [d mu'_x, d mu'_y, d a, d b] [d c, d log2 o(q), d beta_x, d r] [d g, d b, -, -]
constexpr int kGradFloats = 12;


// the binning: tiles per block of the tile-count scan; sub-buckets per tile
// (a record's is its index mod kTileSub: the atomic adds on one tile's
// counters spread over that many addresses); the longest list one warp
// sorts whole (longer lists are sorted in chunks of this many entries and
// then merged)
constexpr uint32_t kScanTiles = 1024;
constexpr uint32_t kTileSub = 8;
constexpr uint32_t kSortChunk = 512;
constexpr int kCtrSortItems = 8;   // header counter of the per-tile sort's next item
constexpr int kCtrMergeItems = 9;  // and of the merge's
constexpr uint32_t kVisBlocks = 1024;  // bound on the blocks of the binning's count walk

enum DevStatus : uint32_t { kDevOk = 0, kDevCapacity = 3, kDevTimeout = 5, kDevInternal = 6 };

}  // namespace ubs
