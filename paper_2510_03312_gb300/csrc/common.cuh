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
  uint32_t pad[3];
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
  uint32_t pad0;
  uint64_t n_visible;    // records with tiles_touched > 0
  uint64_t n_inst;       // instances required
  uint32_t ctr[32];      // dynamic tile counters, one per single-pass kernel
};

// Workspace layout, computed on the host from the problem.
struct Layout {
  int32_t V, S;
  uint32_t R;       // records
  uint32_t NT;      // tiles
  uint32_t NPIX;    // pixels
  uint32_t cap;     // instance capacity
  int32_t tile_bits, tile_passes;
  uint32_t n_cmp_tiles;   // compaction blocks
  uint32_t n_emit_tiles;  // emission offset blocks (records)
  uint32_t n_dsort_tiles; // depth radix pass blocks (records)
  uint32_t n_isort_tiles; // tile-key radix pass blocks = emission fill blocks (instances)
  size_t header, views, rec4, key, tiles, rect, g2d;
  size_t ckA, cvA, ckB, cvB;
  size_t ikA, ivA, ikB, ivB;
  size_t tstart;
  size_t tile_order;   // the order the blend kernels take the tiles in [NT]
  size_t order_count;  // tiles per list-length bucket and bucket cursors [2 x 132]
  size_t vis_count;  // visible records per compaction block [n_cmp_tiles] (made by preprocess)
  size_t vis_prefix; // its exclusive prefix [n_cmp_tiles]
  size_t ioff;       // first instance of each depth-sorted record [R]
  // rewritten whole by every bin_sort (no zeroing needed)
  size_t hist_d;     // per (pass block, digit) counts of the 4 depth passes [4][n_dsort_tiles][256]
  size_t hist_i;     // the same for the tile-key passes [tile_passes][n_isort_tiles][256]
  size_t icount;     // instances per emission block [n_emit_tiles]
  size_t ghist;      // digit totals per pass [4 + 3][256]
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


// block sizes of the binning kernels (items per block)
constexpr int kCmpTile = 2048;  // compaction
constexpr int kDsTile = 2048;   // one depth radix pass (records)
constexpr int kIsTile = 2048;   // one tile-key radix pass and one emission fill block (instances)
constexpr int kEmTile = 1024;   // instance offsets of the depth-sorted records

enum DevStatus : uint32_t { kDevOk = 0, kDevCapacity = 3, kDevTimeout = 5, kDevInternal = 6 };

}  // namespace ubs
