// render.cu -- R1 (forward blend) and G1 (backward blend).
//
// Both kernels give each warp an 8x8 pixel block of a tile and each lane two
// pixels of one column (rows y and y + 4).  The two pixels' state and
// arithmetic are carried in packed float32 pairs (add/mul/fma .f32x2 of
// sm_100 and later), so one instruction serves both pixels; each record
// scalar the pair arithmetic needs is staged twice in shared memory to sit
// in such a pair.  Forward: one CTA per screen tile.  The tile's
// front-to-back list (sorted record ids) is consumed in batches of up to 256
// records: each batch's 48-byte render records are staged in shared memory
// together with a conservative screen box of each record's support (the
// ellipse r <= r_cut, r_cut the radius beyond which alpha < alpha_min,
// widened by a margin).  Each warp first lists the batch entries whose
// support meets its block (32 boxes per ballot) and then walks only that
// list -- a cull that can only drop pairs whose alpha is below alpha_min, so
// no decision changes.  Backward: one single-warp CTA per 8x8 block.
//
// Per pair (Sec. 3, Eq. r; Sec. 4.3 final density), with the screen mean
// staged relative to the tile origin o as m = (hi - o) + lo:
//   dx = (px - o) - m,  r = a dx^2 + 2 b dx dy + c dy^2,
//   skip if r >= 1;  alpha = min(alpha_max, 2^(beta_x log2(1 - r) + log2 o(q)))
//   skip if alpha < alpha_min;  stop before T (1 - alpha) < T_min;
//   C += c alpha T;  T *= 1 - alpha.
// log2/exp2 are the MUFU approximations (lg2.approx, ex2.approx).  The pair
// evaluation is one inline function with explicit rounding so that the
// backward kernel re-derives exactly the forward's alpha and decisions.
// A CTA stops loading batches once every pixel of the tile has terminated.
//
// The backward walks each tile's list back to front from the last
// contributor, recovers T by division and forms per-pair gradients of
// (mu', conic, log2 o(q), beta_x, rgb).  A lane first adds its two pixels'
// contributions; the warp then sums its lanes with a transposed butterfly
// (reduce-scatter: 12 shuffles for the 10 values, leaving each total in one
// lane), and one vector atomic add per (record, block) flushes the sum --
// never one global atomic per pixel.
#include <atomic>

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

__device__ __forceinline__ float rcp_approx(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float sqrt_approx(float x) {
  float y;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
// Packed float32 pairs (sm_100 and later): one instruction rounds each half
// exactly as the scalar operation would (round to nearest even).
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 lo2(const float4& v) { return make_float2(v.x, v.y); }
__device__ __forceinline__ float2 hi2(const float4& v) { return make_float2(v.z, v.w); }

// A record id of a tile list, which is below R by construction: clamped, and
// with UBS_FLAG_CHECKED an id out of range is also recorded in the device
// status (UBS_ERR_INTERNAL), which ubs_read_status reports.
__device__ __forceinline__ void set_status_dev(const Header* h, uint32_t s) {
  atomicCAS(const_cast<uint32_t*>(&h->status), 0u, s);
}
__device__ __forceinline__ uint32_t record_id(uint32_t id, uint32_t R, const CfgDev& cfg, const Header* hdr) {
  if (id >= R) {
    if (cfg.flags & kFlagChecked) set_status_dev(hdr, kDevInternal);
    return R - 1;
  }
  return id;
}

// A staged record, tile-relative: the screen mean is re-expressed relative to
// the tile origin (hi - origin) + lo, exact for the subtraction and rounded
// once, so that per pair dx = (pixel centre - origin) - mean costs one add.
struct Staged {
  float4 p;  // mean_x, mean_y (tile-relative), a, 2b
  float4 q;  // c, log2 o(q), beta_x, red
  float2 s;  // green, blue
};

__device__ __forceinline__ void stage_record(const float4* __restrict__ rec4, uint32_t r, float ox, float oy,
                                             float lg2_amin, Staged& st, float4& box, float& rcut) {
  const float4 a = rec4[3 * (size_t)r], c = rec4[3 * (size_t)r + 1], d = rec4[3 * (size_t)r + 2];
  st.p = make_float4(__fadd_rn(__fsub_rn(a.x, ox), a.z), __fadd_rn(__fsub_rn(a.y, oy), a.w), c.x,
                     __fmul_rn(2.0f, c.y));
  st.q = make_float4(c.z, c.w, d.x, d.y);
  st.s = make_float2(d.z, d.w);
  // conservative box of the pixels with alpha >= alpha_min: the ellipse
  // r <= r_cut, r_cut = 1 - (alpha_min/o(q))^(1/beta_x), widened by 2% + 0.02
  // in r_cut and 0.1 px; empty when o(q) < alpha_min.  Approximate
  // reciprocals and square roots (relative errors near 1e-7) are far inside
  // those margins.
  const float det = c.x * c.z - c.y * c.y;
  const float idet = rcp_approx(det);
  const float s00 = c.z * idet, s11 = c.x * idet;
  float rc = 1.0f - ex2_approx((lg2_amin - c.w) * rcp_approx(d.x));
  if (!(rc > -0.02f)) {
    box = make_float4(1.0f, -1.0f, 1.0f, -1.0f);
    rcut = -1.0f;
  } else {
    rc = fminf(1.0f, fmaf(rc, 1.02f, 0.02f));
    rcut = rc;
    const float ex = sqrt_approx(fmaxf(rc * s00, 0.0f)) + 0.1f, ey = sqrt_approx(fmaxf(rc * s11, 0.0f)) + 0.1f;
    box = make_float4(st.p.x - ex, st.p.x + ex, st.p.y - ey, st.p.y + ey);
  }
}

// A staged record, each scalar the pair arithmetic needs held twice so that
// one packed instruction serves a lane's two pixels (rows y and y + 4 of
// its column): A = (-mx, -mx, -my, -my), Bc = (a, a, 2b, 2b),
// Cc = (c, c, beta_x, beta_x), D = (log2 o(q), log2 o(q), red, red),
// E = (green, green, blue, blue).  Kept as one 80-byte structure per entry
// in shared memory, so that an entry's five loads share one address.
struct __align__(16) Staged2 {
  float4 A, Bc, Cc, D, E;
};
__device__ __forceinline__ Staged2 pack_staged(const Staged& st) {
  Staged2 s;
  s.A = make_float4(-st.p.x, -st.p.x, -st.p.y, -st.p.y);
  s.Bc = make_float4(st.p.z, st.p.z, st.p.w, st.p.w);
  s.Cc = make_float4(st.q.x, st.q.x, st.q.z, st.q.z);
  s.D = make_float4(st.q.y, st.q.y, st.q.w, st.q.w);
  s.E = make_float4(st.s.x, st.s.x, st.s.y, st.s.y);
  return s;
}

struct PairEval2 {
  float2 dx, dy, r, om, lg, alpha;
};

// The one definition of a pair's r and alpha, shared by the forward and
// backward kernels, for a lane's two pixels at once: (lx, ly.x) and
// (lx, ly.y), pixel centres relative to the tile origin (dx is the same for
// both).  Each half of a packed operation rounds as the scalar one would
// (x + (-m) is x - m; fma(r, -1, 1) is 1 - r).  A pair is used when r < 1 and
// alpha >= alpha_min.  HOLD keeps 1 - r above zero for the backward, which
// divides by it; the forward skips that (a pair with r >= 1 is never used,
// whatever its alpha), and for r < 1 both give the same values.
template <bool HOLD>
__device__ __forceinline__ void eval_pair2(float2 lx, float2 ly, const float4& A, const float4& Bc,
                                           const float4& Cc, const float4& D, float amax, PairEval2& e) {
  e.dx = add2(lx, lo2(A));
  e.dy = add2(ly, hi2(A));
  const float2 t = fma2(lo2(Bc), e.dx, mul2(hi2(Bc), e.dy));
  e.r = fma2(e.dx, t, mul2(mul2(lo2(Cc), e.dy), e.dy));
  // 1 - r, held above 0 with HOLD: a pair with r < 1 has 1 - r >= 2^-24
  // and is unchanged; for the others (never composited) log2 and
  // 1/(1 - r) stay finite
  const float2 om = fma2(e.r, make_float2(-1.0f, -1.0f), make_float2(1.0f, 1.0f));
  e.om = HOLD ? make_float2(fmaxf(om.x, 1.0e-30f), fmaxf(om.y, 1.0e-30f)) : om;
  e.lg = make_float2(lg2_approx(e.om.x), lg2_approx(e.om.y));
  const float2 ex = fma2(hi2(Cc), e.lg, lo2(D));
  e.alpha = make_float2(fminf(amax, ex2_approx(ex.x)), fminf(amax, ex2_approx(ex.y)));
}

// The view holding global tile g: the last view whose first tile is at or
// before g (views are numbered in tile order and view 0 starts at tile 0).
// Called by a whole warp: a ballot over 32 views, after one over the first
// views of 32-view chunks when there are more than 32 -- at most two
// dependent loads, where a binary search takes log2(V).
__device__ __forceinline__ int find_view_warp(const ViewDev* __restrict__ views, int V, uint32_t g) {
  if (V == 1) return 0;
  const int lane = threadIdx.x & 31;
  int c = 0;
  if (V > 32) {
    const int i = lane * 32;
    c = 31 - __clz(__ballot_sync(kFull, i < V && views[i].tile_off <= g));
  }
  const int i = c * 32 + lane;
  return c * 32 + (31 - __clz(__ballot_sync(kFull, i < V && views[i].tile_off <= g)));
}

// the warp's 8 x RB block (bx, by) within a TW-wide tile and this lane's
// first pixel (lx, ly); with RB = 8 the lane's second pixel is (lx, ly + 4)
template <int TW, int RB>
__device__ __forceinline__ void pixel_of(int& lx, int& ly, int& bx, int& by) {
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  constexpr int WPR = TW / 8;  // warps per row of blocks
  bx = (w % WPR) * 8;
  by = (w / WPR) * RB;
  lx = bx + (lane & 7);
  ly = by + (lane >> 3);
}

__device__ __forceinline__ bool box_hits(const float4& bb, float x0, float x1, float y0, float y1) {
  return bb.x <= x1 && bb.y >= x0 && bb.z <= y1 && bb.w >= y0;
}

// Whether the ellipse r <= rcut meets the rectangle [x0, x1] x [y0, y1]:
// the smallest r = a dx^2 + 2b dx dy + c dy^2 over the rectangle is 0 when it
// holds the mean, else it lies on an edge, where r is a 1-D convex quadratic
// minimised by clamping its stationary point to the edge.  Rounding here is
// far inside the margin by which rcut was widened.
__device__ __forceinline__ bool ellipse_hits(const float4& p, float c, float rcut, float x0, float x1, float y0,
                                             float y1) {
  const float dx0 = x0 - p.x, dx1 = x1 - p.x, dy0 = y0 - p.y, dy1 = y1 - p.y;
  const float a = p.z, b2 = p.w, hb = 0.5f * p.w;  // b2 = 2b
  const float ia = __frcp_rn(a), ic = __frcp_rn(c);
  auto rq = [&](float dx, float dy) { return fmaf(dx, fmaf(a, dx, b2 * dy), c * dy * dy); };
  float m = rq(dx0, fminf(fmaxf(-hb * dx0 * ic, dy0), dy1));
  m = fminf(m, rq(dx1, fminf(fmaxf(-hb * dx1 * ic, dy0), dy1)));
  m = fminf(m, rq(fminf(fmaxf(-hb * dy0 * ia, dx0), dx1), dy0));
  m = fminf(m, rq(fminf(fmaxf(-hb * dy1 * ia, dx0), dx1), dy1));
  const bool inside = dx0 <= 0.0f && dx1 >= 0.0f && dy0 <= 0.0f && dy1 >= 0.0f;
  return inside || m <= rcut;
}

// Whether staged entry j's support (the ellipse r <= r_cut, widened) meets the
// block [x0, x1] x [y0, y1]: its box first, then the ellipse itself.
__device__ __forceinline__ bool entry_hits(const float4* s_bb, const Staged2* s_st, const float* s_rc, int j,
                                           float x0, float x1, float y0, float y1) {
  if (!box_hits(s_bb[j], x0, x1, y0, y1)) return false;
  const float4 A = s_st[j].A, Bc = s_st[j].Bc;
  return ellipse_hits(make_float4(-A.x, -A.z, Bc.x, Bc.z), s_st[j].Cc.x, s_rc[j], x0, x1, y0, y1);
}

// Forward blend: a CTA per tile, a warp per 8x8 block, two pixels per lane
// (rows y and y + 4) carried in packed pairs, so that the pair evaluation
// and the compositing update run once per entry for both pixels.  Each half
// takes the operations of the scalar rule above in the same order.  The
// warp walks the entries its cull keeps two per step between checks that
// its 64 pixels are all done; the CTA stops loading batches once its
// tile's are.
template <int TW, int TH>
struct FwdSmem {
  static constexpr int NT = TW * TH / 2;           // threads: two pixels each
  static constexpr int BS = NT < 256 ? NT : 256;  // records staged per batch
  Staged2 st[BS];
  float4 bb[BS];
  float rc[BS];
  int v;
  uint32_t next;
};

struct FwdArgs {
  const ViewDev* __restrict__ views;
  int V;
  CfgDev cfg;
  const uint32_t* __restrict__ tstart;
  const uint32_t* __restrict__ ivals;
  const float4* __restrict__ rec4;
  float* __restrict__ image;
  float* __restrict__ Tfin;
  uint32_t* __restrict__ lastc;
  const Header* hdr;
  uint32_t R;
  uint32_t* __restrict__ pairs;
  uint32_t* __restrict__ visited;
  const uint32_t* __restrict__ tile_order;
  uint32_t n_tiles, cap;
  uint32_t* queue;  // persistent form: [next tile, finished CTAs], zero between launches
  // split lists (UBS_FLAG_SPLIT_LISTS): the plan made by split_plan_kernel
  const uint4* split_list;
  const uint32_t* tile_split;  // split index of each tile, or ~0
  const uint32_t* slot_owner;  // split index of each slot
  const uint32_t* ext_owner;   // split index of each extra segment
  uint32_t* split_term;        // per split tile: first segment after which every pixel had ended
  float4* seg_buf;
  uint32_t max_extra;
};

// One tile g, by the whole CTA (every thread calls it).  With SPLIT it
// walks only the list positions [wbeg, wend) of the tile and, when `slot`
// is given, writes each pixel's state there (colour, T, last contributor
// and whether the pixel terminated) instead of the image: the part of one
// segment of a split list.
// A segment k > 0 that learns (through `term`) that an earlier segment ended
// every pixel of the tile stops: no pixel's result can use it.  A segment
// whose walk ends every pixel records its index there.
template <int TW, int TH, bool COUNT, bool SPLIT = false>
__device__ __forceinline__ void fwd_tile(const FwdArgs& A, uint32_t g, FwdSmem<TW, TH>& sm, uint32_t wbeg = 0,
                                         uint32_t wend = 0xffffffffu, float4* slot = nullptr,
                                         bool resume = false, uint32_t* term = nullptr, uint32_t seg = 0) {
  constexpr int NT = FwdSmem<TW, TH>::NT, BS = FwdSmem<TW, TH>::BS;
  const CfgDev& cfg = A.cfg;
  uint32_t start = A.tstart[g], end = A.tstart[g + 1];  // loaded while warp 0 finds the view
  const uint32_t list0 = start;  // positions are numbered from the tile list's first entry
  if constexpr (SPLIT) {
    start = min(end, list0 + wbeg);
    end = min(end, list0 + min(wend, 0xffffffffu - list0));
  }
  if (threadIdx.x < 32) {
    const int vi = find_view_warp(A.views, A.V, g);
    if (threadIdx.x == 0) sm.v = vi;
  }
  __syncthreads();
  const ViewDev& v = A.views[sm.v];
  const uint32_t lt = g - v.tile_off;
  const int tx = lt % v.tiles_x, ty = lt / v.tiles_x;
  int lx, ly, bx, by;
  pixel_of<TW, 8>(lx, ly, bx, by);
  const int x = tx * TW + lx, y0 = ty * TH + ly, y1 = y0 + 4;
  const bool in0 = x < v.W && y0 < v.H, in1 = x < v.W && y1 < v.H;
  const float ox = (float)(tx * TW), oy = (float)(ty * TH);
  const float2 fx = make_float2((float)lx + 0.5f, (float)lx + 0.5f);  // pixel centres, tile-relative
  const float2 fy = make_float2((float)ly + 0.5f, (float)(ly + 4) + 0.5f);
  const float wx0 = (float)bx + 0.5f, wx1 = wx0 + 7.0f, wy0 = (float)by + 0.5f, wy1 = wy0 + 7.0f;
  const float lg2_amin = lg2_approx(cfg.amin);
  const float2 one = make_float2(1.0f, 1.0f), neg1 = make_float2(-1.0f, -1.0f);
  float2 T = one, C0 = make_float2(0.0f, 0.0f), C1 = C0, C2 = C0;
  uint32_t last0 = 0, last1 = 0, np0 = 0, np1 = 0, nv = 0;
  bool done0 = !in0, done1 = !in1;
  bool need0 = true, need1 = true;
  if constexpr (SPLIT) {
    if (resume) {  // a pixel whose walk ends in this segment resumes from its T and last contributor
      const float4 a0 = slot[2 * (ly * TW + lx)], a1 = slot[2 * (ly * TW + lx) + 1];
      const float4 b0 = slot[2 * ((ly + 4) * TW + lx)], b1 = slot[2 * ((ly + 4) * TW + lx) + 1];
      need0 = __float_as_uint(a1.y) != 0u;
      need1 = __float_as_uint(b1.y) != 0u;
      T = make_float2(a0.w, b0.w);
      last0 = __float_as_uint(a1.x);
      last1 = __float_as_uint(b1.x);
      done0 = done0 || !need0;
      done1 = done1 || !need1;
    }
  }
  for (uint32_t base = start; base < end; base += BS) {
    if constexpr (SPLIT) {
      // read by one thread before the barrier, by all after it; rewritten only
      // after this batch's staging barrier, which every reader has passed
      if (term && seg > 0 && threadIdx.x == 0) sm.next = *(volatile const uint32_t*)term < seg ? 1u : 0u;
    }
    if (__syncthreads_count(done0 && done1) == NT) break;
    if constexpr (SPLIT) {
      if (term && seg > 0 && sm.next) return;  // an earlier segment ended every pixel of the tile
    }
    const uint32_t idx = base + threadIdx.x;
    if (threadIdx.x < BS && idx < end) {
      Staged st;
      float4 box;
      stage_record(A.rec4, record_id(A.ivals[idx], A.R, cfg, A.hdr), ox, oy, lg2_amin, st, box, sm.rc[threadIdx.x]);
      sm.st[threadIdx.x] = pack_staged(st);
      sm.bb[threadIdx.x] = box;
    }
    __syncthreads();
    const int n = (int)min((uint32_t)BS, end - base);
    const uint32_t rel = base - list0;
    // one entry for both pixels; branch-free: a pair that is skipped (or
    // stops its pixel) adds c * 0 and keeps T, which leaves C and T exactly
    auto blend = [&](int j) {
      const Staged2& sj = sm.st[j];
      const float4 D = sj.D;
      PairEval2 e;
      eval_pair2<false>(fx, fy, sj.A, sj.Bc, sj.Cc, D, cfg.amax, e);
      const float2 r = e.r;
      const float al0 = e.alpha.x, al1 = e.alpha.y;
      if constexpr (COUNT) {
        np0 += (!done0 && r.x < 1.0f);
        np1 += (!done1 && r.y < 1.0f);
        nv += entry_hits(sm.bb, sm.st, sm.rc, j, wx0, wx1, wy0, wy1);
      }
      const bool u0 = !done0 && r.x < 1.0f && al0 >= cfg.amin;
      const bool u1 = !done1 && r.y < 1.0f && al1 >= cfg.amin;
      const float2 a = make_float2(u0 ? al0 : 0.0f, u1 ? al1 : 0.0f);
      const float2 Tn = mul2(T, fma2(a, neg1, one));
      const bool term0 = u0 && Tn.x < cfg.tmin, term1 = u1 && Tn.y < cfg.tmin;
      done0 = done0 || term0;
      done1 = done1 || term1;
      const bool ok0 = u0 && !term0, ok1 = u1 && !term1;
      float2 w = mul2(a, T);
      w.x = ok0 ? w.x : 0.0f;
      w.y = ok1 ? w.y : 0.0f;
      const float4 E = sj.E;
      C0 = fma2(hi2(D), w, C0);
      C1 = fma2(lo2(E), w, C1);
      C2 = fma2(hi2(E), w, C2);
      T.x = ok0 ? Tn.x : T.x;
      T.y = ok1 ? Tn.y : T.y;
      last0 = ok0 ? rel + j + 1 : last0;
      last1 = ok1 ? rel + j + 1 : last1;
    };
    // 32 entries at a time: the warp's ballot of those whose support meets
    // its block (every entry in the counting variant, which counts every pair
    // with r < 1 and, apart, the entries the cull keeps), then those entries
    // in order, two between checks that the block's pixels are all done;
    // the entry index stays warp-uniform, from the ballot
    bool all_done = false;
    for (int k = 0; k < n && !all_done; k += 32) {
      const int jl = k + (int)(threadIdx.x & 31);
      const bool hit = jl < n && (COUNT || entry_hits(sm.bb, sm.st, sm.rc, jl, wx0, wx1, wy0, wy1));
      unsigned mm = __ballot_sync(kFull, hit);
      while (mm) {
        if (__all_sync(kFull, done0 && done1)) {
          all_done = true;
          break;
        }
        blend(k + __ffs(mm) - 1);
        mm &= mm - 1;
        if (mm) {
          blend(k + __ffs(mm) - 1);
          mm &= mm - 1;
        }
      }
    }
  }
  if constexpr (SPLIT) {
    if (term && __syncthreads_count(done0 && done1) == NT && threadIdx.x == 0) atomicMin(term, seg);
    if (slot) {  // one segment's state of the lane's two pixels (only the resumed ones when resuming)
      float4* s0 = slot + 2 * (ly * TW + lx);
      float4* s1 = slot + 2 * ((ly + 4) * TW + lx);
      if (need0) {
        s0[0] = make_float4(C0.x, C1.x, C2.x, T.x);
        s0[1] = make_float4(__uint_as_float(last0), __uint_as_float(done0 ? 1u : 0u), 0.0f, 0.0f);
      }
      if (need1) {
        s1[0] = make_float4(C0.y, C1.y, C2.y, T.y);
        s1[1] = make_float4(__uint_as_float(last1), __uint_as_float(done1 ? 1u : 0u), 0.0f, 0.0f);
      }
      return;
    }
  }
  const size_t plane = (size_t)v.W * v.H;
  float* img = A.image + (size_t)v.pix_off * 3;
  if (in0) {
    const size_t pix = (size_t)y0 * v.W + x;
    img[pix] = fmaf(T.x, cfg.bg[0], C0.x);
    img[plane + pix] = fmaf(T.x, cfg.bg[1], C1.x);
    img[2 * plane + pix] = fmaf(T.x, cfg.bg[2], C2.x);
    A.Tfin[v.pix_off + pix] = T.x;
    A.lastc[v.pix_off + pix] = last0;
    if constexpr (COUNT) {
      A.pairs[v.pix_off + pix] = np0;
      A.visited[v.pix_off + pix] = nv;
    }
  }
  if (in1) {
    const size_t pix = (size_t)y1 * v.W + x;
    img[pix] = fmaf(T.y, cfg.bg[0], C0.y);
    img[plane + pix] = fmaf(T.y, cfg.bg[1], C1.y);
    img[2 * plane + pix] = fmaf(T.y, cfg.bg[2], C2.y);
    A.Tfin[v.pix_off + pix] = T.y;
    A.lastc[v.pix_off + pix] = last1;
    if constexpr (COUNT) {
      A.pairs[v.pix_off + pix] = np1;
      A.visited[v.pix_off + pix] = nv;
    }
  }
}

// The grid form: one CTA per tile, in bin_sort's tile order where the lists
// are dense.  With SPLIT a split tile's own CTA walks its first segment, and
// A.max_extra more CTAs after the tiles' walk the later segments (those that
// split_plan_kernel did not assign exit): started after the tiles, they can
// find their tile already ended by its first segment, as dense tiles are.
template <int TW, int TH, bool COUNT, bool SPLIT>
__global__ void __launch_bounds__(TW * TH / 2, (TW * TH / 2 >= 128 ? 1024 / (TW * TH / 2) : 16))
    render_fwd_kernel(FwdArgs A) {
  wait_prior_grid();
  __shared__ FwdSmem<TW, TH> sm;
  if (A.hdr->status != 0) return;
  uint32_t t = blockIdx.x;
  if constexpr (SPLIT) {
    constexpr int TP = TW * TH;  // pixels per tile: the float4 pairs of a slot
    if (t >= A.n_tiles) {
      // extra segment e: the split tile whose extra segments [w, w + m - 1) hold it
      const uint32_t e = t - A.n_tiles;
      if (e >= A.hdr->ctr[6]) return;
      const uint32_t i = A.ext_owner[e];
      const uint4 sp = A.split_list[i];
      const uint32_t k = e - sp.w + 1;
      fwd_tile<TW, TH, COUNT, true>(A, sp.x, sm, k * kSegLen, (k + 1) * kSegLen,
                                    A.seg_buf + (size_t)(sp.y + k) * TP * 2, false, A.split_term + i, k);
      return;
    }
    const uint32_t g = A.tile_order && order_dense(A.hdr, A.n_tiles, A.cap) ? A.tile_order[t] : t;
    const uint32_t i = A.tile_split[g];
    if (i != 0xffffffffu)
      fwd_tile<TW, TH, COUNT, true>(A, g, sm, 0, kSegLen, A.seg_buf + (size_t)A.split_list[i].y * TP * 2, false,
                                    A.split_term + i, 0);
    else
      fwd_tile<TW, TH, COUNT, true>(A, g, sm);
  } else {
    const uint32_t g = A.tile_order && order_dense(A.hdr, A.n_tiles, A.cap) ? A.tile_order[t] : t;
    fwd_tile<TW, TH, COUNT>(A, g, sm);
  }
}


// The plan of split lists: every tile whose list holds more than kSegLen
// entries gets a split index i, m = ceil(n / kSegLen) consecutive slots of
// segment state and m - 1 extra segments (CTAs of the split grids), in the
// order the atomics hand them out; tile_split, slot_owner and ext_owner map
// tiles, slots and extra segments to i.  The counters (header ctr[4..6]) are
// zeroed before the launch.
__global__ void __launch_bounds__(256) split_plan_kernel(const uint32_t* __restrict__ tstart, uint32_t NT,
                                                         uint4* __restrict__ split_list,
                                                         uint32_t* __restrict__ tile_split,
                                                         uint32_t* __restrict__ slot_owner,
                                                         uint32_t* __restrict__ ext_owner,
                                                         uint32_t* __restrict__ split_term, uint32_t max_split,
                                                         uint32_t max_slots, uint32_t max_extra, Header* hdr) {
  wait_prior_grid();
  if (hdr->status != 0) return;
  for (uint32_t g = blockIdx.x * 256 + threadIdx.x; g < NT; g += gridDim.x * 256) {
    const uint32_t n = tstart[g + 1] - tstart[g];
    uint32_t split = 0xffffffffu;
    if (n > kSegLen) {
      const uint32_t m = (n + kSegLen - 1) / kSegLen;
      const uint32_t i = atomicAdd(&hdr->ctr[4], 1u);
      const uint32_t b = atomicAdd(&hdr->ctr[5], m);
      const uint32_t e = atomicAdd(&hdr->ctr[6], m - 1);
      // within the bounds by construction (at most the capacity's instances)
      if (i < max_split && b + m <= max_slots && e + m - 1 <= max_extra) {
        split_list[i] = make_uint4(g, b, m, e);
        split_term[i] = 0xffffffffu;
        for (uint32_t k = 0; k < m; ++k) slot_owner[b + k] = i;
        for (uint32_t k = 0; k + 1 < m; ++k) ext_owner[e + k] = i;
        split = i;
      } else {
        set_status_dev(hdr, kDevInternal);
      }
    }
    tile_split[g] = split;
  }
}

// The persistent form: as many CTAs as fit on the GPU at once, each taking
// the next tile (same order) from a counter until none is left.  No CTA
// waits on another; the last CTA to finish resets the counters for the
// next launch.
template <int TW, int TH, bool COUNT>
__global__ void __launch_bounds__(TW * TH / 2, (TW * TH / 2 >= 128 ? 1024 / (TW * TH / 2) : 16))
    render_fwd_persistent_kernel(FwdArgs A) {
  wait_prior_grid();
  __shared__ FwdSmem<TW, TH> sm;
  if (A.hdr->status != 0) return;
  const bool dense = A.tile_order && order_dense(A.hdr, A.n_tiles, A.cap);
  for (;;) {
    if (threadIdx.x == 0) sm.next = atomicAdd(A.queue, 1u);
    __syncthreads();  // also: every thread is done with the previous tile's shared memory
    const uint32_t t = sm.next;
    if (t >= A.n_tiles) break;
    fwd_tile<TW, TH, COUNT>(A, dense ? A.tile_order[t] : t, sm);
  }
  if (threadIdx.x == 0 && atomicAdd(A.queue + 1, 1u) == gridDim.x - 1) {
    A.queue[0] = 0;  // every CTA has taken its last tile
    A.queue[1] = 0;
  }
}

// The merge of a split tile's segments takes three kernels.  Every
// segment but the first was walked from T = 1 (and stopped only where its
// own T fell below T_min, which the true T, no larger, would have done
// sooner).  Front to back, the over operator joins them exactly
// (C += T C_k, T *= T_k) as long as the pixel's true transmittance stays at
// or above T_min through segment k; the first segment k* where it would not
// (the local walk stopped, or T T_k < T_min) is where the pixel's walk ends,
// and that segment is walked again from the pixel's true T.
//
// Pass 1 (one CTA per split tile, a thread per pixel): the over operator up
// to k*.  Slot k < k* gets the colour segment k adds (absolute) and T at its
// end; slot k* gets the pixel's T and last contributor at its start and a
// "walk again" mark; slot 0 records k* (m when the walk never ends early)
// and the last contributor.
template <int TW, int TH>
__global__ void __launch_bounds__(TW * TH) split_join_kernel(FwdArgs A) {
  wait_prior_grid();
  constexpr int TP = TW * TH;
  if (A.hdr->status != 0) return;
  if (blockIdx.x >= A.hdr->ctr[4]) return;
  const uint4 sp = A.split_list[blockIdx.x];
  const uint32_t m = sp.z;
  float4* my = A.seg_buf + (size_t)sp.y * TP * 2 + 2 * threadIdx.x;  // slot k: my[2 k TP], my[2 k TP + 1]
  const CfgDev& cfg = A.cfg;
  const float4 s0 = my[0], s1 = my[1];
  float T = s0.w;
  uint32_t last = __float_as_uint(s1.x);
  bool done = __float_as_uint(s1.y) != 0u;  // ended in the first segment (exact), or outside the image
  uint32_t kstar = m;
  my[1] = make_float4(s1.x, 0.0f, 0.0f, 0.0f);
  for (uint32_t k = 1; k < m; ++k) {
    float4* mk = my + (size_t)2 * k * TP;
    const float4 a0 = mk[0], a1 = mk[1];
    if (kstar < m || done) {  // after the walk ended: the segment adds nothing
      mk[0] = make_float4(0.0f, 0.0f, 0.0f, T);
      mk[1] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
      continue;
    }
    const float Tk = __fmul_rn(T, a0.w);
    if (__float_as_uint(a1.y) != 0u || Tk < cfg.tmin) {
      kstar = k;
      mk[0] = make_float4(0.0f, 0.0f, 0.0f, T);
      mk[1] = make_float4(__uint_as_float(last), __uint_as_float(1u), 0.0f, 0.0f);
      continue;
    }
    mk[0] = make_float4(__fmul_rn(T, a0.x), __fmul_rn(T, a0.y), __fmul_rn(T, a0.z), Tk);
    mk[1] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    T = Tk;
    const uint32_t lk = __float_as_uint(a1.x);
    last = lk ? lk : last;
  }
  my[1] = make_float4(__uint_as_float(last), 0.0f, __uint_as_float(kstar), 0.0f);
}

// Pass 2 (one CTA per slot): the segments that pass 1 marked are walked
// again, with the forward blend's own tile walk, only for the marked pixels,
// from their true T (colour from zero); all the segments run at once.
template <int TW, int TH>
__global__ void __launch_bounds__(TW * TH / 2, (TW * TH / 2 >= 128 ? 1024 / (TW * TH / 2) : 16))
    split_resume_kernel(FwdArgs A) {
  wait_prior_grid();
  constexpr int TP = TW * TH;
  __shared__ FwdSmem<TW, TH> sm;
  if (A.hdr->status != 0) return;
  const uint32_t s = blockIdx.x;
  if (s >= A.hdr->ctr[5]) return;  // unused
  const uint4 sp = A.split_list[A.slot_owner[s]];
  const uint32_t k = s - sp.y;
  if (k == 0) return;  // the first segment is exact
  fwd_tile<TW, TH, false, true>(A, sp.x, sm, k * kSegLen, (k + 1) * kSegLen, A.seg_buf + (size_t)s * TP * 2, true);
}

// Pass 3 (one CTA per split tile, a thread per pixel): the pixel's colour,
// final T and last contributor, written to the image; and, for the
// backward, each segment's T at its end and the colour behind it
// (everything after it and the background), normalised by that T.
template <int TW, int TH>
__global__ void __launch_bounds__(TW * TH) split_finish_kernel(FwdArgs A) {
  wait_prior_grid();
  constexpr int TP = TW * TH;
  __shared__ int s_v;
  if (A.hdr->status != 0) return;
  if (blockIdx.x >= A.hdr->ctr[4]) return;
  const uint4 sp = A.split_list[blockIdx.x];
  const uint32_t g = sp.x, m = sp.z;
  if (threadIdx.x < 32) {
    const int vi = find_view_warp(A.views, A.V, g);
    if (threadIdx.x == 0) s_v = vi;
  }
  __syncthreads();
  const ViewDev& v = A.views[s_v];
  const CfgDev& cfg = A.cfg;
  float4* my = A.seg_buf + (size_t)sp.y * TP * 2 + 2 * threadIdx.x;
  const float4 h1 = my[1];
  uint32_t last = __float_as_uint(h1.x);
  const uint32_t kstar = __float_as_uint(h1.z);
  float C0 = 0.0f, C1 = 0.0f, C2 = 0.0f, T = 1.0f;
  const uint32_t kend = kstar < m ? kstar : m - 1;  // the segment the walk ends in
  for (uint32_t k = 0; k <= kend; ++k) {
    const float4 a0 = my[(size_t)2 * k * TP];
    C0 += a0.x;
    C1 += a0.y;
    C2 += a0.z;
    T = a0.w;
  }
  if (kstar < m) last = __float_as_uint(my[(size_t)2 * kstar * TP + 1].x);
  const uint32_t lt = g - v.tile_off;
  const int tx = lt % v.tiles_x, ty = lt / v.tiles_x;
  const int x = tx * TW + (int)(threadIdx.x % TW), y = ty * TH + (int)(threadIdx.x / TW);
  if (x < v.W && y < v.H) {
    const size_t plane = (size_t)v.W * v.H, pix = (size_t)y * v.W + x;
    float* img = A.image + (size_t)v.pix_off * 3;
    img[pix] = fmaf(T, cfg.bg[0], C0);
    img[plane + pix] = fmaf(T, cfg.bg[1], C1);
    img[2 * plane + pix] = fmaf(T, cfg.bg[2], C2);
    A.Tfin[v.pix_off + pix] = T;
    A.lastc[v.pix_off + pix] = last;
  }
  float b0 = T * cfg.bg[0], b1 = T * cfg.bg[1], b2 = T * cfg.bg[2];
  for (int k = (int)m - 1; k >= 0; --k) {
    float4* mk = my + (size_t)2 * k * TP;
    float4 a0 = make_float4(0.0f, 0.0f, 0.0f, T);  // after the walk ended: nothing added, T final
    if ((uint32_t)k <= kend) a0 = mk[0];
    const float inv = a0.w > 0.0f ? 1.0f / a0.w : 0.0f;
    mk[1] = make_float4(b0 * inv, b1 * inv, b2 * inv, a0.w);
    b0 += a0.x;
    b1 += a0.y;
    b2 += a0.z;
  }
}

// Transposed-butterfly reduction of g[0..9] over the warp: each exchange
// step halves the values a lane keeps, so 12 shuffles sum all 10; the adds
// of neighbouring slots run as packed float32 pairs.  On return lane l holds
// the warp total of value writer_of(l) (when that is >= 0).
__device__ __forceinline__ float warp_reduce10(const float (&g)[10], int lane) {
  const bool b4 = lane & 16, b3 = lane & 8, b2 = lane & 4, b1 = lane & 2;
  float2 k01 = b4 ? make_float2(g[5], g[6]) : make_float2(g[0], g[1]);
  float2 k23 = b4 ? make_float2(g[7], g[8]) : make_float2(g[2], g[3]);
  const float k4 = b4 ? g[9] : g[4];
  const float e0 = b4 ? g[0] : g[5], e1 = b4 ? g[1] : g[6], e2 = b4 ? g[2] : g[7], e3 = b4 ? g[3] : g[8],
              e4 = b4 ? g[4] : g[9];
  const float2 p01 = add2(k01, make_float2(__shfl_xor_sync(kFull, e0, 16), __shfl_xor_sync(kFull, e1, 16)));
  const float2 p23 = add2(k23, make_float2(__shfl_xor_sync(kFull, e2, 16), __shfl_xor_sync(kFull, e3, 16)));
  const float p4 = k4 + __shfl_xor_sync(kFull, e4, 16);
  // bit 3: slots (p0|p3, p1|p4, p2)
  const float2 kk = b3 ? make_float2(p23.y, p4) : make_float2(p01.x, p01.y);
  const float f0 = b3 ? p01.x : p23.y, f1 = b3 ? p01.y : p4;
  const float2 s01 = add2(kk, make_float2(__shfl_xor_sync(kFull, f0, 8), __shfl_xor_sync(kFull, f1, 8)));
  const float s2 = p23.x + __shfl_xor_sync(kFull, p23.x, 8);
  // bit 2: slots (s0|s1, s2)
  const float m0 = b2 ? s01.y : s01.x, h0 = b2 ? s01.x : s01.y;
  const float2 t01 = add2(make_float2(m0, s2),
                          make_float2(__shfl_xor_sync(kFull, h0, 4), __shfl_xor_sync(kFull, s2, 4)));
  // bit 1: slot t0|t1
  const float k = b1 ? t01.y : t01.x, e = b1 ? t01.x : t01.y;
  float u = k + __shfl_xor_sync(kFull, e, 2);
  // bit 0
  u += __shfl_xor_sync(kFull, u, 1);
  return u;
}

// value index whose total `lane` holds after warp_reduce10, or -1 if the
// lane is not that value's designated writer
__device__ __forceinline__ int writer_of(int lane) {
  if (lane & 1) return -1;
  const int base = (lane & 16) ? 5 : 0;
  if (lane & 2) return (lane & 12) ? -1 : base + 2;
  return base + ((lane & 4) ? ((lane & 8) ? 4 : 1) : ((lane & 8) ? 3 : 0));
}

// Per-record sums accumulated by the backward blend (record constants a, b,
// c, beta_x and ln 2 are applied once per record when flushing):
//   v0 = sum q dx, v1 = sum q dy, v2 = sum q dx^2, v3 = sum q dx dy,
//   v4 = sum q dy^2 with q = alpha dL/dalpha / (1 - r),
//   v5 = sum alpha dL/dalpha, v6 = sum alpha dL/dalpha log2(1 - r),
//   v7..9 = sum alpha T dL/dC.
// With dr = -beta q:  d mu' = 2 beta [[a, b], [b, c]] (v0, v1),
// d(a, b, c) = -beta (v2, 2 v3, v4), d log2 o = ln2 v5, d beta = ln2 v6.
//
// One CTA of one warp per 8x8 block of a tile (two pixels a lane, rows y and
// y + 4), with no block-wide barrier: warps of a tile finish independently
// and free their slot at once.  The warp walks the tile's list back to front
// from its block's last contributor in batches of 32 entries: each lane
// stages one record, the batch is culled to the entries whose support meets
// the block, those are processed, and each record the block used is flushed
// by its lane with one vector atomic add per (record, block).  The pair
// evaluation and the per-pixel recurrences (T, the colour behind) run in
// packed pairs over the lane's two pixels; the two share dx, so a lane's
// sums of q dx, q dx^2 and q dx dy take dx out of the sum.
struct BwdSmem {
  static constexpr int WB = 32;  // entries per batch: one per lane
  Staged2 st[WB];
  uint32_t rec[WB];
  float acc[10][WB + 1];  // +1: the 10 writer lanes hit 10 different banks
};

struct BwdArgs {
  const ViewDev* __restrict__ views;
  int V;
  CfgDev cfg;
  const uint32_t* __restrict__ tstart;
  const uint32_t* __restrict__ ivals;
  const float4* __restrict__ rec4;
  const float* __restrict__ dLdimg;
  const float* __restrict__ Tfin;
  const uint32_t* __restrict__ lastc;
  float4* __restrict__ g2d;
  const Header* hdr;
  uint32_t R;
  const uint32_t* __restrict__ tile_order;
  uint32_t n_tiles, cap;
  uint32_t* queue;  // persistent form: [next block, finished CTAs], zero between launches
  // split lists: the forward's plan and segment state
  const uint4* split_list;
  const uint32_t* tile_split;
  const uint32_t* ext_owner;
  const float4* seg_buf;
  uint32_t max_extra;
};

// One 8x8 block wb of tile g, by one warp.  With SPLIT and a slot, only the
// list positions [wbeg, wend) of one segment are walked, from the
// transmittance and colour behind at the segment's end that the forward's
// merge left in the slot.
template <int TW, int TH, bool SPLIT = false>
__device__ __forceinline__ void bwd_block(const BwdArgs& A, uint32_t g, int wb, BwdSmem& sm, uint32_t wbeg = 0,
                                          uint32_t wend = 0xffffffffu, const float4* slot = nullptr) {
  constexpr int WB = BwdSmem::WB;
  constexpr int WPR = TW / 8;  // blocks per row of the tile
  const CfgDev& cfg = A.cfg;
  const int lane = threadIdx.x & 31;
  const uint32_t start = A.tstart[g], end = A.tstart[g + 1];  // loaded while the view is found
  const int vi = find_view_warp(A.views, A.V, g);
  if (start == end) return;  // an empty list: no pixel of the tile has a contributor
  const ViewDev& v = A.views[vi];
  const uint32_t lt = g - v.tile_off;
  const int tx = lt % v.tiles_x, ty = lt / v.tiles_x;
  const int bx = (wb % WPR) * 8, by = (wb / WPR) * 8;
  const int lx = bx + (lane & 7), ly = by + (lane >> 3);
  const int x = tx * TW + lx;
  // per-pixel state of the lane's two pixels, packed: .x row ly, .y row ly + 4
  const float2 fx = make_float2((float)lx + 0.5f, (float)lx + 0.5f);
  const float2 fy = make_float2((float)ly + 0.5f, (float)(ly + 4) + 0.5f);
  float2 T = make_float2(1.0f, 1.0f), G0 = make_float2(0.0f, 0.0f), G1 = G0, G2 = G0;
  // colour behind the current record, normalised by the transmittance after it
  float2 B0 = make_float2(cfg.bg[0], cfg.bg[0]), B1 = make_float2(cfg.bg[1], cfg.bg[1]),
         B2 = make_float2(cfg.bg[2], cfg.bg[2]);
  uint32_t last0 = 0, last1 = 0;
  {
    const size_t plane = (size_t)v.W * v.H;
    const float* gi = A.dLdimg + (size_t)v.pix_off * 3;
    const int y0 = ty * TH + ly, y1 = y0 + 4;
    if (x < v.W && y0 < v.H) {
      const size_t pix = (size_t)y0 * v.W + x;
      G0.x = gi[pix];
      G1.x = gi[plane + pix];
      G2.x = gi[2 * plane + pix];
      T.x = A.Tfin[v.pix_off + pix];
      last0 = A.lastc[v.pix_off + pix];
    }
    if (x < v.W && y1 < v.H) {
      const size_t pix = (size_t)y1 * v.W + x;
      G0.y = gi[pix];
      G1.y = gi[plane + pix];
      G2.y = gi[2 * plane + pix];
      T.y = A.Tfin[v.pix_off + pix];
      last1 = A.lastc[v.pix_off + pix];
    }
  }
  if constexpr (SPLIT) {
    if (slot) {  // the segment's end: T and the normalised colour behind it
      const float4 s0 = slot[2 * (ly * TW + lx) + 1], s1 = slot[2 * ((ly + 4) * TW + lx) + 1];
      T = make_float2(s0.w, s1.w);
      B0 = make_float2(s0.x, s1.x);
      B1 = make_float2(s0.y, s1.y);
      B2 = make_float2(s0.z, s1.z);
    }
  }
  uint32_t wlast = __reduce_max_sync(kFull, max(last0, last1));
  if constexpr (SPLIT) {
    wlast = min(wlast, wend);
    if (wlast <= wbeg) return;
  }
  if (wlast == 0) return;
  const float ox = (float)(tx * TW), oy = (float)(ty * TH);
  const float wx0 = (float)bx + 0.5f, wx1 = wx0 + 7.0f, wy0 = (float)by + 0.5f, wy1 = wy0 + 7.0f;
  const float lg2_amin = lg2_approx(cfg.amin);
  const float2 one = make_float2(1.0f, 1.0f), neg1 = make_float2(-1.0f, -1.0f);
  const int wslot = writer_of(lane);
  const int wfirst = SPLIT ? (int)wbeg : 0;
  for (int hi = (int)wlast; hi > wfirst; hi -= WB) {
    const int lo = hi - WB > wfirst ? hi - WB : wfirst;
    const int n = hi - lo;
    bool listed = false;
    if (lane < n) {
      const uint32_t r = record_id(A.ivals[start + lo + lane], A.R, cfg, A.hdr);
      Staged st;
      float4 box;
      float rc;
      stage_record(A.rec4, r, ox, oy, lg2_amin, st, box, rc);
      sm.rec[lane] = r;
      sm.st[lane] = pack_staged(st);
      listed = box_hits(box, wx0, wx1, wy0, wy1) && ellipse_hits(st.p, st.q.x, rc, wx0, wx1, wy0, wy1);
    }
    const unsigned lm = __ballot_sync(kFull, listed);
    __syncwarp();
    unsigned touched = 0;  // entries the block used (warp-uniform)
    // entry j of the batch is list position lo + j: the forward composited it
    // at a pixel only if lo + j < that pixel's last contributor
    const int lim0 = (int)last0 - lo, lim1 = (int)last1 - lo;
    // the listed entries back to front, the index warp-uniform from the ballot
    for (unsigned rem = lm; rem != 0;) {
      const int j = 31 - __clz(rem);
      rem ^= 1u << j;
      const Staged2& sj = sm.st[j];
      const float4 D = sj.D, E = sj.E;
      PairEval2 e;
      eval_pair2<true>(fx, fy, sj.A, sj.Bc, sj.Cc, D, cfg.amax, e);
      // pairs the forward composited
      const bool use0 = e.r.x < 1.0f && e.alpha.x >= cfg.amin && j < lim0;
      const bool use1 = e.r.y < 1.0f && e.alpha.y >= cfg.amin && j < lim1;
      const unsigned hits = __ballot_sync(kFull, use0 || use1);
      if (hits == 0) continue;  // no pixel of the block: T and B stay
      touched |= 1u << j;
      // branch-free: a pair the forward skipped contributes zero and leaves T, B
      const float2 a = make_float2(use0 ? e.alpha.x : 0.0f, use1 ? e.alpha.y : 0.0f);
      const float2 oma = fma2(a, neg1, one);
      T = mul2(T, make_float2(rcp_approx(oma.x), rcp_approx(oma.y)));  // transmittance before this record
      const float2 w = mul2(a, T);
      float gv[10];
      {
        const float2 c0 = hi2(D), c1 = lo2(E), c2 = hi2(E);
        const float2 e0 = fma2(B0, neg1, c0), e1 = fma2(B1, neg1, c1), e2 = fma2(B2, neg1, c2);
        const float2 dal = mul2(T, fma2(e0, G0, fma2(e1, G1, mul2(e2, G2))));
        B0 = fma2(a, e0, B0);
        B1 = fma2(a, e1, B1);
        B2 = fma2(a, e2, B2);
        const float2 wg0 = mul2(w, G0), wg1 = mul2(w, G1), wg2 = mul2(w, G2);
        gv[7] = wg0.x + wg0.y;
        gv[8] = wg1.x + wg1.y;
        gv[9] = wg2.x + wg2.y;
        float2 ga = mul2(dal, a);
        ga.x = a.x < cfg.amax ? ga.x : 0.0f;
        ga.y = a.y < cfg.amax ? ga.y : 0.0f;
        // q = ga / (1 - r): ga = 0 unless composited, and 1 - r > 0
        const float2 qq = mul2(ga, make_float2(rcp_approx(e.om.x), rcp_approx(e.om.y)));
        const float2 u1 = mul2(qq, e.dy);
        const float2 u1y = mul2(u1, e.dy);
        const float2 glg = mul2(ga, e.lg);
        // dx is the same for both pixels: sums of q dx and q dx dy factor it
        gv[0] = (qq.x + qq.y) * e.dx.x;
        gv[1] = u1.x + u1.y;
        gv[2] = gv[0] * e.dx.x;
        gv[3] = gv[1] * e.dx.x;
        gv[4] = u1y.x + u1y.y;
        gv[5] = ga.x + ga.y;
        gv[6] = glg.x + glg.y;
      }
      if (__popc(hits) == 1) {  // one lane: its values are the totals
        if (use0 || use1) {
#pragma unroll
          for (int m = 0; m < 10; ++m) sm.acc[m][j] = gv[m];
        }
      } else {
        const float tot = warp_reduce10(gv, lane);
        if (wslot >= 0) sm.acc[wslot][j] = tot;
      }
    }
    __syncwarp();
    if ((touched >> lane) & 1u) {
      const float a = sm.st[lane].Bc.x, b = 0.5f * sm.st[lane].Bc.z, c = sm.st[lane].Cc.x, beta = sm.st[lane].Cc.z;
      const float v0 = sm.acc[0][lane], v1 = sm.acc[1][lane];
      float4* dst = A.g2d + 3 * (size_t)sm.rec[lane];
      atomicAdd(dst, make_float4(2.0f * beta * (a * v0 + b * v1), 2.0f * beta * (b * v0 + c * v1),
                                 -beta * sm.acc[2][lane], -2.0f * beta * sm.acc[3][lane]));
      atomicAdd(dst + 1, make_float4(-beta * sm.acc[4][lane], kLn2f * sm.acc[5][lane], kLn2f * sm.acc[6][lane],
                                     sm.acc[7][lane]));
      atomicAdd((float2*)(dst + 2), make_float2(sm.acc[8][lane], sm.acc[9][lane]));
    }
    __syncwarp();
  }
}

// The grid form: one single-warp CTA per 8x8 block.  With SPLIT the grid
// first holds the blocks of A.max_extra extra segments (those the plan did
// not assign exit), and a split tile's own blocks walk its first segment.
template <int TW, int TH, bool SPLIT>
__global__ void __launch_bounds__(32, 32)  // 64 registers: 32 one-warp CTAs per SM
    render_bwd_kernel(BwdArgs A) {
  wait_prior_grid();
  constexpr int BPT = TW * TH / 64;  // 8x8 blocks per tile
  __shared__ BwdSmem sm;
  if (A.hdr->status != 0) return;
  uint32_t t = blockIdx.x / BPT;
  const int wb = blockIdx.x % BPT;
  if constexpr (SPLIT) {
    constexpr int TP = TW * TH;
    if (t < A.max_extra) {
      if (t >= A.hdr->ctr[6]) return;
      const uint4 sp = A.split_list[A.ext_owner[t]];
      const uint32_t k = t - sp.w + 1;
      bwd_block<TW, TH, true>(A, sp.x, wb, sm, k * kSegLen, (k + 1) * kSegLen,
                              A.seg_buf + (size_t)(sp.y + k) * TP * 2);
      return;
    }
    t -= A.max_extra;
    const uint32_t g = A.tile_order && order_dense(A.hdr, A.n_tiles, A.cap) ? A.tile_order[t] : t;
    const uint32_t i = A.tile_split[g];
    if (i != 0xffffffffu)
      bwd_block<TW, TH, true>(A, g, wb, sm, 0, kSegLen, A.seg_buf + (size_t)A.split_list[i].y * TP * 2);
    else
      bwd_block<TW, TH, true>(A, g, wb, sm);
  } else {
    const uint32_t g = A.tile_order && order_dense(A.hdr, A.n_tiles, A.cap) ? A.tile_order[t] : t;
    bwd_block<TW, TH>(A, g, wb, sm);
  }
}

// The persistent form: as many one-warp CTAs as fit on the GPU at once, each
// taking the next tile (same order) from a counter and walking its 8x8
// blocks in turn, until none is left (one counter update per tile, not per
// block: a single counter updated once per block by thousands of warps
// serialises); the last CTA to finish resets the counters for the next
// launch.
template <int TW, int TH>
__global__ void __launch_bounds__(32, 32)
    render_bwd_persistent_kernel(BwdArgs A) {
  wait_prior_grid();
  constexpr int BPT = TW * TH / 64;
  __shared__ BwdSmem sm;
  if (A.hdr->status != 0) return;
  const bool dense = A.tile_order && order_dense(A.hdr, A.n_tiles, A.cap);
  for (;;) {
    uint32_t t = 0;
    if (threadIdx.x == 0) t = atomicAdd(A.queue, 1u);
    t = __shfl_sync(kFull, t, 0);
    if (t >= A.n_tiles) break;
    const uint32_t g = dense ? A.tile_order[t] : t;
    for (int wb = 0; wb < BPT; ++wb) {
      bwd_block<TW, TH>(A, g, wb, sm);
      __syncwarp();
    }
  }
  if (threadIdx.x == 0 && atomicAdd(A.queue + 1, 1u) == gridDim.x - 1) {
    A.queue[0] = 0;  // every CTA has taken its last block
    A.queue[1] = 0;
  }
}

// Zeroes the per-record gradient accumulators of the visible records (those
// with tiles): the only ones the backward blend adds to and the parameter
// backward reads.
__global__ void __launch_bounds__(256) zero_visible_grads_kernel(const uint32_t* __restrict__ tiles, uint32_t R,
                                                                 float4* __restrict__ g2d) {
  wait_prior_grid();
  const uint32_t r = blockIdx.x * 256 + threadIdx.x;
  if (r >= R || tiles[r] == 0) return;
  const float4 z = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
  g2d[3 * (size_t)r] = z;
  g2d[3 * (size_t)r + 1] = z;
  g2d[3 * (size_t)r + 2] = z;
}

// CTAs of `kernel` (with `threads` threads each) that fit on the current
// device at once, for the persistent forms; 0 if the query fails.  Cached per
// kernel and device.
template <typename Kernel>
uint32_t resident_ctas(Kernel kernel, int threads) {
  static std::atomic<uint32_t> cache[64];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 0;
  uint32_t n = cache[dev].load(std::memory_order_relaxed);
  if (n) return n;
  int per_sm = 0, sms = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, 0) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  n = (uint32_t)(per_sm > 0 ? per_sm : 0) * (uint32_t)(sms > 0 ? sms : 0);
  cache[dev].store(n, std::memory_order_relaxed);
  return n;
}

template <int TW, int TH, bool COUNT>
cudaError_t fwd_launch(const FwdArgs& args, const Layout& L, bool persistent, cudaStream_t st) {
  constexpr int NT = TW * TH / 2;
  if (persistent) {
    const uint32_t n = resident_ctas(render_fwd_persistent_kernel<TW, TH, COUNT>, NT);
    if (n > 0)
      return launch_dependent(render_fwd_persistent_kernel<TW, TH, COUNT>, dim3(n < L.NT ? n : L.NT), dim3(NT), 0,
                              st, args);
  }
  return launch_dependent(render_fwd_kernel<TW, TH, COUNT, false>, dim3(L.NT), dim3(NT), 0, st, args);
}

// Split lists: the plan (after zeroing its counters), the grid of extra
// segments and tiles, and the merge of the split tiles.
template <int TW, int TH>
cudaError_t fwd_split(const FwdArgs& args, const Layout& L, char* ws, cudaStream_t st) {
  constexpr int NT = TW * TH / 2;
  Header* hdr = (Header*)(ws + L.header);
  cudaError_t e = cudaMemsetAsync(&hdr->ctr[4], 0, 3 * sizeof(uint32_t), st);
  if (e != cudaSuccess) return e;
  const uint32_t pb = (L.NT + 255) / 256;
  e = launch_dependent(split_plan_kernel, dim3(pb < 1024 ? pb : 1024), dim3(256), 0, st,
                       (const uint32_t*)(ws + L.tstart), L.NT, (uint4*)(ws + L.split_list),
                       (uint32_t*)(ws + L.tile_slot), (uint32_t*)(ws + L.slot_owner), (uint32_t*)(ws + L.ext_owner),
                       (uint32_t*)(ws + L.split_term), L.seg_max_split, L.seg_slots, L.seg_max_extra, hdr);
  if (e != cudaSuccess) return e;
  e = launch_dependent(render_fwd_kernel<TW, TH, false, true>, dim3(L.seg_max_extra + L.NT), dim3(NT), 0, st, args);
  if (e != cudaSuccess) return e;
  e = launch_dependent(split_join_kernel<TW, TH>, dim3(L.seg_max_split), dim3(TW * TH), 0, st, args);
  if (e != cudaSuccess) return e;
  e = launch_dependent(split_resume_kernel<TW, TH>, dim3(L.seg_slots), dim3(NT), 0, st, args);
  if (e != cudaSuccess) return e;
  return launch_dependent(split_finish_kernel<TW, TH>, dim3(L.seg_max_split), dim3(TW * TH), 0, st, args);
}

template <int TW, int TH>
cudaError_t fwd_t(const Layout& L, const CfgDev& cfg, char* ws, float* image, cudaStream_t st) {
  FwdArgs a;
  a.views = (const ViewDev*)(ws + L.views);
  a.V = L.V;
  a.cfg = cfg;
  a.tstart = (const uint32_t*)(ws + L.tstart);
  a.ivals = sorted_instances(L, ws);
  a.rec4 = (const float4*)(ws + L.rec4);
  a.image = image;
  a.Tfin = (float*)(ws + L.Tfin);
  a.lastc = (uint32_t*)(ws + L.last);
  a.hdr = (const Header*)(ws + L.header);
  a.R = L.R > 0 ? L.R : 1;
  const bool count = (cfg.flags & 2) != 0;  // diagnostic variant: also count pairs and visited entries
  a.pairs = count ? (uint32_t*)(ws + L.pairs) : nullptr;
  a.visited = count ? (uint32_t*)(ws + L.pairs) + L.NPIX : nullptr;
  a.tile_order = order_possible(L) ? (const uint32_t*)(ws + L.tile_order) : nullptr;
  a.n_tiles = L.NT;
  a.cap = L.cap;
  a.queue = ((Header*)(ws + L.header))->ctr;
  const bool split = (cfg.flags & kFlagSplit) && !count && L.seg_slots > 0;
  a.split_list = split ? (const uint4*)(ws + L.split_list) : nullptr;
  a.tile_split = split ? (const uint32_t*)(ws + L.tile_slot) : nullptr;
  a.slot_owner = split ? (const uint32_t*)(ws + L.slot_owner) : nullptr;
  a.ext_owner = split ? (const uint32_t*)(ws + L.ext_owner) : nullptr;
  a.split_term = split ? (uint32_t*)(ws + L.split_term) : nullptr;
  a.seg_buf = split ? (float4*)(ws + L.seg_buf) : nullptr;
  a.max_extra = split ? L.seg_max_extra : 0;
  if (split) return fwd_split<TW, TH>(a, L, ws, st);
  const bool persistent = (cfg.flags & 8) != 0;
  return count ? fwd_launch<TW, TH, true>(a, L, persistent, st) : fwd_launch<TW, TH, false>(a, L, persistent, st);
}

template <int TW, int TH>
cudaError_t bwd_t(const Layout& L, const CfgDev& cfg, char* ws, const float* dL, cudaStream_t st) {
  BwdArgs a;
  a.views = (const ViewDev*)(ws + L.views);
  a.V = L.V;
  a.cfg = cfg;
  a.tstart = (const uint32_t*)(ws + L.tstart);
  a.ivals = sorted_instances(L, ws);
  a.rec4 = (const float4*)(ws + L.rec4);
  a.dLdimg = dL;
  a.Tfin = (const float*)(ws + L.Tfin);
  a.lastc = (const uint32_t*)(ws + L.last);
  a.g2d = (float4*)(ws + L.g2d);
  a.hdr = (const Header*)(ws + L.header);
  a.R = L.R > 0 ? L.R : 1;
  a.tile_order = order_possible(L) ? (const uint32_t*)(ws + L.tile_order) : nullptr;
  a.n_tiles = L.NT;
  a.cap = L.cap;
  a.queue = ((Header*)(ws + L.header))->ctr + 2;
  const uint32_t n_blocks = L.NT * (TW * TH / 64);
  // the same choice as the forward's: split lists unless counting pairs
  const bool split = (cfg.flags & kFlagSplit) && !(cfg.flags & 2) && L.seg_slots > 0;
  a.split_list = split ? (const uint4*)(ws + L.split_list) : nullptr;
  a.tile_split = split ? (const uint32_t*)(ws + L.tile_slot) : nullptr;
  a.ext_owner = split ? (const uint32_t*)(ws + L.ext_owner) : nullptr;
  a.seg_buf = split ? (const float4*)(ws + L.seg_buf) : nullptr;
  a.max_extra = split ? L.seg_max_extra : 0;
  if (split) {
    launch_dependent(render_bwd_kernel<TW, TH, true>, dim3((L.seg_max_extra + L.NT) * (TW * TH / 64)), dim3(32), 0,
                     st, a);
    return cudaGetLastError();
  }
  if (cfg.flags & 8) {
    const uint32_t n = resident_ctas(render_bwd_persistent_kernel<TW, TH>, 32);
    if (n > 0)
      return launch_dependent(render_bwd_persistent_kernel<TW, TH>, dim3(n < L.NT ? n : L.NT), dim3(32), 0, st,
                              a);
  }
  launch_dependent(render_bwd_kernel<TW, TH, false>, dim3(n_blocks), dim3(32), 0, st, a);
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
  cudaError_t e = launch_dependent(zero_visible_grads_kernel, dim3((L.R + 255) / 256), dim3(256), 0, st,
                                   (const uint32_t*)(ws + L.tiles), L.R, (float4*)(ws + L.g2d));
  if (e != cudaSuccess) return e;
  if (cfg.tw == 16 && cfg.th == 16) return bwd_t<16, 16>(L, cfg, ws, dL, st);
  if (cfg.tw == 8 && cfg.th == 8) return bwd_t<8, 8>(L, cfg, ws, dL, st);
  if (cfg.tw == 16 && cfg.th == 32) return bwd_t<16, 32>(L, cfg, ws, dL, st);
  if (cfg.tw == 32 && cfg.th == 32) return bwd_t<32, 32>(L, cfg, ws, dL, st);
  return cudaErrorInvalidValue;
}

}  // namespace ubs
