// sort.cu -- B1-B3: tile binning, front-to-back order and tile ranges.
//
// The instance order is (global tile, float32 depth, record index).  It is
// made as a most-significant-digit radix sort whose first digit is the whole
// tile id, the rest of the key being sorted inside each tile:
//   1. count: every visible record (a set bit of the visibility masks the
//      preprocess writes, one bit per primitive and view) adds one to a
//      counter of each tile of its rectangle, one of kTileSub sub-buckets
//      by record index, so that the adds on a busy tile spread over several
//      addresses;
//   2. scan: the exclusive prefix of the counts gives each tile's range
//      (B3) and the start of its bucket; the scan also lists the work items
//      of step 4 (one per tile, or one per kSortChunk entries of a longer
//      list) and, where lists are long, the order in which the blend kernels
//      take the tiles;
//   3. scatter: every visible record writes its index into the bucket of
//      each of its tiles, at a slot taken from its sub-bucket's cursor (an
//      atomic add); the order inside a bucket is the order the adds ran in;
//   4. per-tile sort: one warp sorts a bucket by the 64-bit key
//      (depth bits << 32 | record) in registers, with a bitonic network;
//      a list longer than kSortChunk entries is sorted in chunks of that
//      many entries, and
//   5. merge: one CTA per such list merges its sorted chunks pairwise in
//      rounds (merge path: each thread an equal share of the outputs), in
//      shared memory up to kMergeSeg entries, then in global memory.
// A record meets a tile once, so the keys of a tile are distinct and the
// result does not depend on the bucket order: it is the order a stable
// sort by (tile, depth) of the records in index order gives.
//
// No kernel waits on another block: every step's inputs are made by the
// kernels before it.  A work item of the per-tile sort holds at most
// kSortChunk entries; the warps take the items from a counter, the long
// lists' chunks first and then the short lists longest first.  The scatter
// zeroes the counters the scan has used, so that the binning can run again
// on the same preprocess.
#include "kernels.cuh"

namespace ubs {

namespace {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ void set_status(Header* h, uint32_t s) { atomicCAS(&h->status, 0u, s); }

__device__ __forceinline__ uint32_t lane_id() { return threadIdx.x & 31; }

// Exclusive scan of one value per thread over a block of NT threads
// (NT / 32 <= 32); total receives the block's sum.  s_w must hold NT/32 + 1
// values.  Must be called by every thread.
template <typename T, int NT>
__device__ __forceinline__ T block_excl_scan(T v, T& total, T* s_w) {
  constexpr int NW = NT / 32;
  static_assert(NW <= 32, "one warp scans the warp sums");
  const uint32_t lane = lane_id(), warp = threadIdx.x >> 5;
  T incl = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const T t = __shfl_up_sync(kFull, incl, o);
    if (lane >= (uint32_t)o) incl += t;
  }
  if (lane == 31) s_w[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    const T w = lane < (uint32_t)NW ? s_w[lane] : T(0);
    T wi = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const T t = __shfl_up_sync(kFull, wi, o);
      if (lane >= (uint32_t)o) wi += t;
    }
    if (lane < (uint32_t)NW) s_w[lane] = wi - w;
    if (lane == (uint32_t)NW - 1) s_w[NW] = wi;
  }
  __syncthreads();
  total = s_w[NW];
  const T out = s_w[warp] + incl - v;
  __syncthreads();
  return out;
}

// block_excl_scan of two values at once (the same barriers): a 64-bit and
// a 32-bit count.  s_a / s_b must hold NT/32 + 1 values each.
template <int NT>
__device__ __forceinline__ void block_excl_scan2(unsigned long long a, uint32_t b, unsigned long long& ea, uint32_t& eb,
                                                 unsigned long long& ta, uint32_t& tb, unsigned long long* s_a,
                                                 uint32_t* s_b) {
  constexpr int NW = NT / 32;
  static_assert(NW <= 32, "one warp scans the warp sums");
  const uint32_t lane = lane_id(), warp = threadIdx.x >> 5;
  unsigned long long ia = a;
  uint32_t ib = b;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned long long x = __shfl_up_sync(kFull, ia, o);
    const uint32_t y = __shfl_up_sync(kFull, ib, o);
    if (lane >= (uint32_t)o) ia += x, ib += y;
  }
  if (lane == 31) s_a[warp] = ia, s_b[warp] = ib;
  __syncthreads();
  if (warp == 0) {
    const unsigned long long wa = lane < (uint32_t)NW ? s_a[lane] : 0ull;
    const uint32_t wb = lane < (uint32_t)NW ? s_b[lane] : 0u;
    unsigned long long xa = wa;
    uint32_t xb = wb;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned long long x = __shfl_up_sync(kFull, xa, o);
      const uint32_t y = __shfl_up_sync(kFull, xb, o);
      if (lane >= (uint32_t)o) xa += x, xb += y;
    }
    if (lane < (uint32_t)NW) s_a[lane] = xa - wa, s_b[lane] = xb - wb;
    if (lane == (uint32_t)NW - 1) s_a[NW] = xa, s_b[NW] = xb;
  }
  __syncthreads();
  ta = s_a[NW];
  tb = s_b[NW];
  ea = s_a[warp] + ia - a;
  eb = s_b[warp] + ib - b;
  __syncthreads();
}

// ---------------------------------------------------------------- tile order

constexpr int kOrdBuckets = 4 * 33;

// bucket of a list length: four per octave, longest first (bucket 0)
__device__ __forceinline__ int length_bucket(uint32_t n) {
  if (n == 0) return kOrdBuckets - 1;
  const int e = 31 - __clz(n);                                                       // 2^e <= n
  const int f = e >= 2 ? (int)((n >> (e - 2)) & 3u) : (int)((n << (2 - e)) & 3u);  // the next two bits
  return kOrdBuckets - 2 - (4 * e + f);
}

// Warp-aggregated add of 1 to s[b] (b < 0: no add): the lanes sharing a
// bucket make one shared-memory atomic, and each gets its rank among the
// lanes that came before it in the warp; returns the old value plus the rank.
// The lanes sharing the bucket are found with one ballot per bit of it.
static_assert(kOrdBuckets < 255, "bucket ids and the no-bucket id fit 8 bits");
__device__ __forceinline__ uint32_t bucket_add(uint32_t* s, int b) {
  const uint32_t key = b >= 0 ? (uint32_t)b : 255u;
  uint32_t peers = 0xffffffffu;
#pragma unroll
  for (int bit = 0; bit < 8; ++bit) {
    const bool one = (key >> bit) & 1u;
    const uint32_t m = __ballot_sync(0xffffffffu, one);
    peers &= one ? m : ~m;
  }
  const int lane = threadIdx.x & 31;
  const int leader = __ffs(peers) - 1;
  uint32_t base = 0;
  if (b >= 0 && lane == leader) base = atomicAdd(s + b, (uint32_t)__popc(peers));
  base = __shfl_sync(0xffffffffu, base, leader);
  return base + __popc(peers & ((1u << lane) - 1u));
}

// ---------------------------------------------------------------- scan

// Places each thread's item (bucket b, or none if b < 0) of this block in
// the bucket order: bucket i's range starts after the totals of the buckets
// before it (totals, complete over every block), and each block takes its
// part of that range from the bucket's cursor.  Returns the position, ~0
// where b < 0.  Block-uniform call (every thread).
template <int NT>
__device__ __forceinline__ uint32_t bucket_place(const uint32_t* __restrict__ totals, uint32_t* __restrict__ cursors,
                                                 int b, uint32_t* s_n, uint32_t* s_base) {
  for (int i = threadIdx.x; i < kOrdBuckets; i += NT) s_n[i] = 0;
  __syncthreads();
  const uint32_t rank = bucket_add(s_n, b);
  __syncthreads();
  if (threadIdx.x < 32) {  // five buckets a lane
    constexpr int PER = (kOrdBuckets + 31) / 32;
    const uint32_t lane = threadIdx.x;
    uint32_t tot[PER], sum = 0;
#pragma unroll
    for (int j = 0; j < PER; ++j) {
      const uint32_t i = lane * PER + j;
      tot[j] = i < (uint32_t)kOrdBuckets ? totals[i] : 0u;
      sum += tot[j];
    }
    uint32_t incl = sum;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const uint32_t o = __shfl_up_sync(kFull, incl, d);
      if (lane >= (uint32_t)d) incl += o;
    }
    uint32_t start = incl - sum;
#pragma unroll
    for (int j = 0; j < PER; ++j) {
      const uint32_t i = lane * PER + j;
      if (i < (uint32_t)kOrdBuckets && s_n[i]) s_base[i] = start + atomicAdd(cursors + i, s_n[i]);
      start += tot[j];
    }
  }
  __syncthreads();
  return b >= 0 ? s_base[b] + rank : ~0u;
}


// The tiles in the order the blend kernels take them.  Where lists are long
// on average, by list length, longest first (to a quarter octave; the order
// within a bucket is arbitrary), so that long tiles start early and do not
// trail the grid; where they are short, the blend kernels keep the tiles'
// own order (neighbouring tiles share records) and no order is made.
// Every tile appears once, so the order changes no result.  The scan makes
// it: its first pass counts the tiles per length bucket, its last places
// each block's tiles after the longer buckets' totals.
//
// One thread per tile; kScanTiles tiles per block.
constexpr int kScT = kScanTiles;
static_assert(kScT == 1024, "one thread per tile");

__device__ __forceinline__ uint32_t sort_items(uint32_t n) { return (n + kSortChunk - 1) / kSortChunk; }

// The counts of tile t (zero past the last tile) and their sum: sub-bucket
// u of tile t is tcount[u NT + t].
__device__ __forceinline__ uint32_t load_tile_counts(const uint32_t* __restrict__ tcount, uint32_t t, uint32_t NT,
                                                     uint32_t (&c)[kTileSub]) {
#pragma unroll
  for (int i = 0; i < (int)kTileSub; ++i) c[i] = t < NT ? tcount[(size_t)i * NT + t] : 0u;
  uint32_t n = 0;
#pragma unroll
  for (int i = 0; i < (int)kTileSub; ++i) n += c[i];
  return n;
}

// per scan block: instances (u64), chunk items of long lists, short lists
struct ScanPart {
  unsigned long long inst;
  uint32_t n_long, n_short;
};

// Pass 1: each block's sums; the short lists per length bucket (the sort
// items of short lists are placed longest first); and, with `order`, the
// tiles per length bucket of the tile order.  The bucket counts go to
// order_count: [0, 132) tiles, [264, 396) short lists.
__global__ void __launch_bounds__(kScT) scan_part_kernel(const uint32_t* __restrict__ tcount, uint32_t NT,
                                                         ScanPart* __restrict__ part,
                                                         uint32_t* __restrict__ order_count, bool order) {
  wait_prior_grid();
  __shared__ unsigned long long s_w64[kScT / 32 + 1];
  __shared__ uint32_t s_w[kScT / 32 + 1];
  __shared__ uint32_t s_n[2][kOrdBuckets];
  const uint32_t t = blockIdx.x * kScT + threadIdx.x;
  uint32_t c[kTileSub];
  const uint32_t n = load_tile_counts(tcount, t, NT, c);
  for (int i = threadIdx.x; i < 2 * kOrdBuckets; i += kScT) (&s_n[0][0])[i] = 0;
  __syncthreads();
  bucket_add(s_n[1], t < NT && n > 0 && n <= kSortChunk ? length_bucket(n) : -1);
  if (order) bucket_add(s_n[0], t < NT ? length_bucket(n) : -1);
  __syncthreads();
  for (int i = threadIdx.x; i < 2 * kOrdBuckets; i += kScT) {
    const uint32_t v = (&s_n[0][0])[i];
    if (v) atomicAdd(order_count + (i < kOrdBuckets ? i : 2 * kOrdBuckets + (i - kOrdBuckets)), v);
  }
  unsigned long long ea, ti;
  uint32_t es, ts, tl;
  block_excl_scan2<kScT>((unsigned long long)n, n > 0 && n <= kSortChunk ? 1u : 0u, ea, es, ti, ts, s_w64, s_w);
  block_excl_scan<uint32_t, kScT>(n > kSortChunk ? sort_items(n) : 0u, tl, s_w);
  if (threadIdx.x == 0) part[blockIdx.x] = ScanPart{ti, tl, ts};
}

// Pass 2 (one block; only where there are more than kFusePrefixMax scan
// blocks): every block's exclusive prefix and the totals.
constexpr uint32_t kFusePrefixMax = 2048;  // blocks up to which the last pass sums the earlier blocks' parts itself
__global__ void __launch_bounds__(kScT) scan_mid_kernel(const ScanPart* __restrict__ part, uint32_t nb,
                                                        ScanPart* __restrict__ pre, ScanPart* __restrict__ tot) {
  wait_prior_grid();
  __shared__ unsigned long long s_w64[kScT / 32 + 1];
  __shared__ uint32_t s_w[kScT / 32 + 1];
  ScanPart carry{0ull, 0u, 0u};
  for (uint32_t b0 = 0; b0 < nb; b0 += kScT) {
    const uint32_t b = b0 + threadIdx.x;
    const ScanPart v = b < nb ? part[b] : ScanPart{0ull, 0u, 0u};
    unsigned long long ti;
    uint32_t tl, ts;
    const unsigned long long ei = block_excl_scan<unsigned long long, kScT>(v.inst, ti, s_w64);
    const uint32_t el = block_excl_scan<uint32_t, kScT>(v.n_long, tl, s_w);
    const uint32_t es = block_excl_scan<uint32_t, kScT>(v.n_short, ts, s_w);
    if (b < nb) pre[b] = ScanPart{carry.inst + ei, carry.n_long + el, carry.n_short + es};
    carry.inst += ti;
    carry.n_long += tl;
    carry.n_short += ts;
  }
  if (threadIdx.x == 0) *tot = carry;
}

// The last pass: each tile's range and sub-bucket cursors, the sort items
// (every chunk of a long list first, then one per short list) and the tile
// order.  With few blocks (pre null) a block sums the earlier blocks' parts
// itself; else it reads the prefixes and totals of scan_mid_kernel.  Block
// 0 records the totals (and a capacity overflow, after which every list is
// empty and there is no item).
__global__ void __launch_bounds__(kScT) scan_place_kernel(const uint32_t* __restrict__ tcount, uint32_t NT,
                                                          uint32_t cap, const ScanPart* __restrict__ part, uint32_t nb,
                                                          const ScanPart* __restrict__ pre,
                                                          const ScanPart* __restrict__ tot, Header* hdr,
                                                          uint32_t* __restrict__ tstart,
                                                          uint32_t* __restrict__ cursor, uint2* __restrict__ items,
                                                          uint32_t* __restrict__ order_count,
                                                          uint32_t* __restrict__ order) {
  wait_prior_grid();
  __shared__ unsigned long long s_w64[kScT / 32 + 1];
  __shared__ uint32_t s_w[kScT / 32 + 1];
  __shared__ uint32_t s_n[kOrdBuckets], s_base[kOrdBuckets];
  __shared__ ScanPart s_pt[2];
  if (threadIdx.x < 32) {
    // the parts before this block (P) and of all blocks (T): one warp
    ScanPart P{0ull, 0u, 0u}, T{0ull, 0u, 0u};
    if (pre) {
      P = pre[blockIdx.x];
      T = *tot;
    } else {
      for (uint32_t b = threadIdx.x; b < nb; b += 32) {
        const ScanPart v = part[b];
        if (b < blockIdx.x) P.inst += v.inst, P.n_long += v.n_long, P.n_short += v.n_short;
        T.inst += v.inst, T.n_long += v.n_long, T.n_short += v.n_short;
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        P.inst += __shfl_xor_sync(kFull, P.inst, o);
        P.n_long += __shfl_xor_sync(kFull, P.n_long, o);
        P.n_short += __shfl_xor_sync(kFull, P.n_short, o);
        T.inst += __shfl_xor_sync(kFull, T.inst, o);
        T.n_long += __shfl_xor_sync(kFull, T.n_long, o);
        T.n_short += __shfl_xor_sync(kFull, T.n_short, o);
      }
    }
    if (threadIdx.x == 0) s_pt[0] = P, s_pt[1] = T;
  }
  __syncthreads();
  const ScanPart P = s_pt[0], T = s_pt[1];
  const bool over = T.inst > cap;
  const uint32_t t = blockIdx.x * kScT + threadIdx.x;
  uint32_t c[kTileSub];
  const uint32_t n = load_tile_counts(tcount, t, NT, c);
  const uint32_t nl = n > kSortChunk ? sort_items(n) : 0u;
  unsigned long long ei, bi;
  uint32_t el, bl;
  block_excl_scan2<kScT>((unsigned long long)n, nl, ei, el, bi, bl, s_w64, s_w);
  // the short lists' items, after every long list's chunks, longest first
  const bool is_short = t < NT && n > 0 && n <= kSortChunk;
  const uint32_t ps = bucket_place<kScT>(order_count + 2 * kOrdBuckets, order_count + 3 * kOrdBuckets,
                                         is_short ? length_bucket(n) : -1, s_n, s_base);
  if (t < NT) {
    uint32_t run = over ? 0u : (uint32_t)(P.inst + ei);
    tstart[t] = run;
#pragma unroll
    for (int i = 0; i < (int)kTileSub; ++i) {
      cursor[(size_t)i * NT + t] = run;
      if (!over) run += c[i];
    }
    if (!over) {
      const uint32_t l0 = P.n_long + el;
      for (uint32_t ch = 0; ch < nl; ++ch) items[l0 + ch] = make_uint2(t, ch);
      if (is_short && ps < T.n_short) items[T.n_long + ps] = make_uint2(t, 0u);  // ps < n_short holds
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    hdr->ctr[kCtrSortItems] = 0;  // the per-tile sort's and the merge's item counters
    hdr->ctr[kCtrMergeItems] = 0;
    tstart[NT] = over ? 0u : (uint32_t)T.inst;
    hdr->n_inst = T.inst;
    hdr->n_long = over ? 0u : T.n_long;
    hdr->n_items = over ? 0u : T.n_long + T.n_short;
    if (over) set_status(hdr, kDevCapacity);
  }
  if (order && !over && T.inst >= (unsigned long long)kOrdDense * NT) {  // uniform over the block
    const uint32_t pos = bucket_place<kScT>(order_count, order_count + kOrdBuckets, t < NT ? length_bucket(n) : -1,
                                            s_n, s_base);
    if (t < NT && pos < NT) order[pos] = t;  // pos < NT holds: the totals count every tile
  }
}

// ---------------------------------------------------------------- count and scatter

constexpr int kScatT = 256, kScatW = kScatT / 32;

// The view constants the walk over the visibility masks needs, per block.
struct ViewTable {
  uint32_t recoff[kMaxViews], maskoff[kMaxViews], toff[kMaxViews], tsx[kMaxViews];
};

__device__ __forceinline__ void stage_views(ViewTable& t, const ViewDev* __restrict__ views, int V) {
  for (int i = threadIdx.x; i < V; i += blockDim.x) {
    t.recoff[i] = views[i].rec_off;
    t.maskoff[i] = views[i].mask_off;
    t.toff[i] = views[i].tile_off;
    t.tsx[i] = (uint32_t)views[i].tiles_x;
  }
}

// Walks the visible records (the set bits of the visibility masks): each
// warp takes chunks of `chunk` (<= 32) consecutive mask words, a grid-
// stride loop over the chunks, loads the chunk's words together (one a
// lane), lists the records of their set bits in shared memory and then
// calls f(r, n, rc, toff, tsx) for 32 of them at a time, one a lane: record
// r, its tile count n (0 on the lanes past the list's end, which load
// nothing), its rectangle rc and its view's first tile and tiles per row.
// Every lane of the warp calls f together.  s_list holds 32 x 32 entries
// per warp.
template <class F>
__device__ __forceinline__ void walk_visible(const uint32_t* __restrict__ vis_mask, uint32_t mask_words,
                                             uint32_t chunk, const ViewTable& vt, int V,
                                             const uint32_t* __restrict__ tiles, const uint2* __restrict__ rect,
                                             uint32_t* s_list, F&& f) {
  const uint32_t lane = lane_id();
  const uint32_t n_chunks = (mask_words + chunk - 1) / chunk;
  const uint32_t nw = gridDim.x * kScatW;
  for (uint32_t c = blockIdx.x * kScatW + (threadIdx.x >> 5); c < n_chunks; c += nw) {
    const uint32_t word = c * chunk + lane;
    const uint32_t m = (lane < chunk && word < mask_words) ? vis_mask[word] : 0u;
    const uint32_t cnt = __popc(m);
    uint32_t off = cnt;  // inclusive scan of the counts over the lanes
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t t = __shfl_up_sync(kFull, off, o);
      if (lane >= (uint32_t)o) off += t;
    }
    const uint32_t total = __shfl_sync(kFull, off, 31);
    if (total == 0) continue;
    if (m) {
      int lo = 0, hi = V - 1;  // the word's view: the last with mask_off <= word
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (vt.maskoff[mid] <= word) lo = mid; else hi = mid - 1;
      }
      const uint32_t r0 = vt.recoff[lo] + (word - vt.maskoff[lo]) * 32;
      uint32_t at = off - cnt;
      for (uint32_t b = m; b; b &= b - 1) s_list[at++] = r0 + (uint32_t)(__ffs(b) - 1);
    }
    __syncwarp();
    for (uint32_t g = 0; g < total; g += 32) {  // warp-uniform
      const bool on = g + lane < total;
      const uint32_t r = on ? s_list[g + lane] : 0u;
      const uint32_t n = on ? tiles[r] : 0u;
      const uint2 rc = on ? rect[r] : make_uint2(0u, 0u);
      uint32_t toff = 0, tsx = 0;
      if (on) {
        int lo = 0, hi = V - 1;  // the record's view: the last with rec_off <= r
        while (lo < hi) {
          const int mid = (lo + hi + 1) >> 1;
          if (vt.recoff[mid] <= r) lo = mid; else hi = mid - 1;
        }
        toff = vt.toff[lo];
        tsx = vt.tsx[lo];
      }
      f(r, n, rc, toff, tsx);
    }
    __syncwarp();  // the list is read before the next chunk's is written
  }
}

// B1: every visible record adds one to its sub-bucket (record index mod
// kTileSub) of each tile of its rectangle; each block writes the number of
// visible records it walked to vis_block[block] (overwritten by every
// binning).
__global__ void __launch_bounds__(kScatT) count_kernel(const uint32_t* __restrict__ tiles,
                                                       const uint2* __restrict__ rect,
                                                       const uint32_t* __restrict__ vis_mask, uint32_t mask_words,
                                                       uint32_t chunk, const ViewDev* __restrict__ views, int V,
                                                       uint32_t NT, uint32_t* __restrict__ tcount,
                                                       uint32_t* __restrict__ vis_block) {
  wait_prior_grid();
  __shared__ ViewTable s_vt;
  __shared__ uint32_t s_list[kScatW][32 * 32];
  __shared__ uint32_t s_vis[kScatW];
  stage_views(s_vt, views, V);
  __syncthreads();
  uint32_t nvis = 0;
  walk_visible(vis_mask, mask_words, chunk, s_vt, V, tiles, rect, s_list[threadIdx.x >> 5],
               [&](uint32_t r, uint32_t n, uint2 rc, uint32_t toff, uint32_t tsx) {
                 nvis += n != 0;
                 uint32_t* sub = tcount + (r & (kTileSub - 1)) * NT + toff;
                 if (n != 0 && n <= kSoloTiles) {
                   const uint32_t x0 = rc.x & 0xFFFFu, x1 = rc.y & 0xFFFFu, y1 = rc.y >> 16;
                   for (uint32_t ty = rc.x >> 16; ty < y1; ++ty)
                     for (uint32_t tx = x0; tx < x1; ++tx)
                       if (toff + ty * tsx + tx < NT) atomicAdd(sub + ty * tsx + tx, 1u);  // holds: in the view
                 }
                 walk_large_rects(n, rc, toff, tsx, r, [&](uint32_t g, uint32_t rec) {
                   if (g < NT) atomicAdd(tcount + (rec & (kTileSub - 1)) * NT + g, 1u);
                 });
               });
  const uint32_t w = __reduce_add_sync(kFull, nvis);
  if (lane_id() == 0) s_vis[threadIdx.x >> 5] = w;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t b = 0;
    for (int i = 0; i < kScatW; ++i) b += s_vis[i];
    vis_block[blockIdx.x] = b;
  }
}

// Every visible record writes its index into the bucket of each tile of its
// rectangle, at a slot taken from its sub-bucket's cursor: a lane's own
// rectangle of up to kSoloTiles tiles with all its adds in flight together,
// a larger one with all lanes of the warp working on it in turn.  Nothing is
// written after a capacity overflow.  The kernel also zeroes the tile
// counters and the length buckets' totals and cursors, which the scan has
// used, for the next binning on this workspace.
__global__ void __launch_bounds__(kScatT) scatter_kernel(const uint32_t* __restrict__ tiles,
                                                         const uint2* __restrict__ rect,
                                                         const uint32_t* __restrict__ vis_mask, uint32_t mask_words,
                                                         uint32_t chunk, const ViewDev* __restrict__ views, int V,
                                                         uint32_t NT, uint32_t cap, const Header* hdr,
                                                         uint32_t* cursor, uint32_t* __restrict__ bucket,
                                                         uint32_t* __restrict__ tcount,
                                                         uint32_t* __restrict__ order_count) {
  wait_prior_grid();
  for (uint32_t i = blockIdx.x * kScatT + threadIdx.x; i < kTileSub * NT; i += gridDim.x * kScatT) tcount[i] = 0;
  if (blockIdx.x == 0)
    for (int i = threadIdx.x; i < 4 * kOrdBuckets; i += kScatT) order_count[i] = 0;
  __shared__ ViewTable s_vt;
  __shared__ uint32_t s_list[kScatW][32 * 32];
  stage_views(s_vt, views, V);
  __syncthreads();
  if (hdr->n_inst > cap) return;
  walk_visible(vis_mask, mask_words, chunk, s_vt, V, tiles, rect, s_list[threadIdx.x >> 5],
               [&](uint32_t r, uint32_t n, uint2 rc, uint32_t toff, uint32_t tsx) {
                 uint32_t* cur = cursor + (r & (kTileSub - 1)) * NT;
                 if (n != 0 && n <= kSoloTiles) {
                   uint32_t g[kSoloTiles], pos[kSoloTiles];
                   solo_tiles(n, rc, toff, tsx, g);
#pragma unroll
                   for (uint32_t k = 0; k < kSoloTiles; ++k)  // g < NT holds: rectangles lie in their view
                     pos[k] = (k < n && g[k] < NT) ? atomicAdd(cur + g[k], 1u) : cap;
#pragma unroll
                   for (uint32_t k = 0; k < kSoloTiles; ++k)
                     if (pos[k] < cap) bucket[pos[k]] = r;  // holds: the counts fit the capacity
                 }
                 walk_large_rects(n, rc, toff, tsx, r, [&](uint32_t g, uint32_t rec) {
                   if (g >= NT) return;
                   const uint32_t pos = atomicAdd(cursor + (rec & (kTileSub - 1)) * NT + g, 1u);
                   if (pos < cap) bucket[pos] = rec;
                 });
               });
}

// ---------------------------------------------------------------- per-tile sort

// A compare-exchange of two keys: afterwards a <= b if asc, else a >= b.
__device__ __forceinline__ void cmp_swap(unsigned long long& a, unsigned long long& b, bool asc) {
  const bool sw = (a > b) == asc;
  const unsigned long long lo = sw ? b : a;
  b = sw ? a : b;
  a = lo;
}

// Sorts a lane's K registers: ascending if asc, else descending (a static
// bitonic network; only the last level's direction is chosen at run time).
template <int K>
__device__ __forceinline__ void lane_sort(unsigned long long (&v)[K], bool asc) {
#pragma unroll
  for (int sz = 2; sz <= K; sz <<= 1)
#pragma unroll
    for (int j = sz >> 1; j > 0; j >>= 1)
#pragma unroll
      for (int k = 0; k < K; ++k)
        if ((k & j) == 0) cmp_swap(v[k], v[k | j], sz == K ? asc : (k & sz) == 0);
}

// The in-lane steps of a bitonic merge (distances K/2 .. 1), direction asc.
template <int K>
__device__ __forceinline__ void lane_merge(unsigned long long (&v)[K], bool asc) {
#pragma unroll
  for (int j = K >> 1; j > 0; j >>= 1)
#pragma unroll
    for (int k = 0; k < K; ++k)
      if ((k & j) == 0) cmp_swap(v[k], v[k | j], asc);
}

// One warp sorts the 32 K keys it holds, lane l holding positions
// l K .. l K + K - 1, ascending by position: a bitonic sort whose blocks of
// up to K positions are sorted inside each lane; each later round (blocks
// of 2K .. 32K positions, direction by the block's position bit) pairs lane
// l with lane l ^ (distance / K) by shuffles for the distances of K and
// more, then finishes in the lane's registers.  The rounds are a loop, so
// the code holds one copy of each step.
template <int K>
__device__ __forceinline__ void warp_sort_keys(unsigned long long (&v)[K]) {
  const uint32_t lane = lane_id();
  lane_sort<K>(v, (lane & 1u) == 0);
#pragma unroll 1
  for (uint32_t size = 2 * K; size <= 32 * K; size <<= 1) {
    const bool asc = ((lane * K) & size) == 0;
#pragma unroll 1
    for (uint32_t lm = size / (2 * K); lm > 0; lm >>= 1) {
      const bool keep_min = asc != ((lane & lm) != 0);
#pragma unroll
      for (int k = 0; k < K; ++k) {
        const unsigned long long p = __shfl_xor_sync(kFull, v[k], lm);
        v[k] = ((p < v[k]) == keep_min) ? p : v[k];
      }
    }
    lane_merge<K>(v, asc);
  }
}

// Sorts n <= 32 K entries of a bucket by (depth bits << 32 | record) and
// writes the records (out32) or the keys (out64) in order; padding is ~0.
template <int K>
__device__ __forceinline__ void warp_sort_list(const uint32_t* __restrict__ src, uint32_t n,
                                               const uint32_t* __restrict__ key, uint32_t R,
                                               uint32_t* __restrict__ out32, unsigned long long* __restrict__ out64) {
  const uint32_t lane = lane_id();
  unsigned long long v[K];
#pragma unroll
  for (int k = 0; k < K; ++k) {  // the records first, all loads in flight, then their depth keys
    const uint32_t i = lane * K + k;
    v[k] = i < n ? src[i] : ~0ull;
  }
#pragma unroll
  for (int k = 0; k < K; ++k)  // r < R holds: written by the scatter
    if (v[k] != ~0ull) v[k] |= (unsigned long long)__ldg(key + min((uint32_t)v[k], R - 1)) << 32;
  warp_sort_keys<K>(v);
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const uint32_t i = lane * K + k;
    if (i < n) {
      if (out32) out32[i] = (uint32_t)v[k];
      else out64[i] = v[k];
    }
  }
}

constexpr int kTsW = 4;  // warps per CTA of the per-tile sort
static_assert(kSortChunk == 32 * 16, "the widest warp sort holds 16 keys a lane");

// One warp per work item, taken in order from a counter: a list of at most
// kSortChunk entries is sorted
// from its bucket into the instance lists; a chunk of a longer list into
// chunk64 as keys, for the merge.  The warp takes the narrowest network
// that holds the entries (2, 8 or 16 a lane).
__global__ void __launch_bounds__(kTsW * 32, 8) tile_sort_kernel(const uint2* __restrict__ items,
                                                              const uint32_t* __restrict__ tstart,
                                                              const uint32_t* __restrict__ key, uint32_t R,
                                                              const uint32_t* __restrict__ bucket,
                                                              uint32_t* __restrict__ out,
                                                              unsigned long long* __restrict__ chunk64,
                                                              Header* hdr) {
  wait_prior_grid();
  const uint32_t n_items = hdr->n_items;
  for (;;) {
    // the next item, taken from the counter (the long lists' chunks first,
    // then the short lists longest first)
    uint32_t it = 0;
    if (lane_id() == 0) it = atomicAdd(&hdr->ctr[kCtrSortItems], 1u);
    it = __shfl_sync(kFull, it, 0);
    if (it >= n_items) break;
    const uint2 item = items[it];
    const uint32_t s = tstart[item.x], e = tstart[item.x + 1];
    const bool whole = e - s <= kSortChunk;
    const uint32_t base = whole ? s : s + item.y * kSortChunk;
    const uint32_t n = whole ? e - s : min(kSortChunk, e - base);
    uint32_t* o32 = whole ? out + base : nullptr;
    unsigned long long* o64 = whole ? nullptr : chunk64 + base;
    if (n <= 64) warp_sort_list<2>(bucket + base, n, key, R, o32, o64);
    else if (n <= 256) warp_sort_list<8>(bucket + base, n, key, R, o32, o64);
    else warp_sort_list<16>(bucket + base, n, key, R, o32, o64);
  }
}

// ---------------------------------------------------------------- merge

constexpr int kMgT = 512;  // threads of a merge CTA

// Merges the sorted runs A = src[a0, a0 + na) and B = src[b0, b0 + nb)
// (distinct keys) into dst[o0, o0 + na + nb), writing only the outputs
// [d0, d1) of the merged order: the split of output d0 between A and B is
// found by bisection (the count i of A's keys among the first d0 outputs
// is the one with A[i - 1] < B[d0 - i] and B[d0 - i - 1] < A[i]), then the
// outputs are taken in order.
__device__ __forceinline__ void merge_path(const unsigned long long* __restrict__ src, uint32_t a0, uint32_t na,
                                           uint32_t b0, uint32_t nb, unsigned long long* __restrict__ dst,
                                           uint32_t o0, uint32_t d0, uint32_t d1) {
  uint32_t lo = d0 > nb ? d0 - nb : 0u, hi = d0 < na ? d0 : na;
  while (lo < hi) {  // the smallest i with A[i] > B[d0 - i - 1]
    const uint32_t i = (lo + hi) >> 1;
    if (src[a0 + i] < src[b0 + (d0 - i - 1)]) lo = i + 1; else hi = i;
  }
  uint32_t i = lo, j = d0 - lo;
  unsigned long long x = i < na ? src[a0 + i] : ~0ull, y = j < nb ? src[b0 + j] : ~0ull;
  for (uint32_t d = d0; d < d1; ++d) {
    if (x < y) {
      dst[o0 + d] = x;
      ++i;
      x = i < na ? src[a0 + i] : ~0ull;
    } else {
      dst[o0 + d] = y;
      ++j;
      y = j < nb ? src[b0 + j] : ~0ull;
    }
  }
}

// Sorts one segment of up to kMergeSeg entries of a long list: its sorted
// kSortChunk-runs (src[0, n)) are staged in shared memory and merged
// pairwise in rounds; in each round every thread computes its share of the
// outputs (kMergePer consecutive positions, found by merge path) into
// registers, and writes them back after a barrier.  Leaves the sorted
// segment in s_seg.  Block-uniform call.
constexpr uint32_t kMergeSeg = 4096;
constexpr int kMergePer = kMergeSeg / kMgT;
__device__ __forceinline__ void merge_segment(const unsigned long long* __restrict__ src, uint32_t n,
                                              unsigned long long* s_seg) {
  for (uint32_t i = threadIdx.x; i < n; i += kMgT) s_seg[i] = src[i];
  __syncthreads();
  for (uint32_t w = kSortChunk; w < n; w <<= 1) {
    unsigned long long v[kMergePer];
    const uint32_t q0 = threadIdx.x * kMergePer;
    if (q0 < n) {
      const uint32_t p0 = q0 - q0 % (2 * w);  // kMergePer divides 2w: one pair of runs
      const uint32_t na = min(w, n - p0), nb = min(w, n - min(n, p0 + w));
      const uint32_t d0 = q0 - p0;
      uint32_t lo = d0 > nb ? d0 - nb : 0u, hi = d0 < na ? d0 : na;
      const unsigned long long* A = s_seg + p0;
      const unsigned long long* B = s_seg + p0 + na;
      while (lo < hi) {
        const uint32_t i = (lo + hi) >> 1;
        if (A[i] < B[d0 - i - 1]) lo = i + 1; else hi = i;
      }
      uint32_t i = lo, j = d0 - lo;
      unsigned long long x = i < na ? A[i] : ~0ull, y = j < nb ? B[j] : ~0ull;
#pragma unroll
      for (int k = 0; k < kMergePer; ++k) {
        const bool ta = x < y;
        v[k] = ta ? x : y;
        if (ta) {
          ++i;
          x = i < na ? A[i] : ~0ull;
        } else {
          ++j;
          y = j < nb ? B[j] : ~0ull;
        }
      }
    }
    __syncthreads();  // every share is read before any is written
    if (q0 < n)
#pragma unroll
      for (int k = 0; k < kMergePer; ++k)
        if (q0 + k < n) s_seg[q0 + k] = v[k];
    __syncthreads();
  }
}

// One CTA per list longer than kSortChunk (the items with chunk 0 among
// the first n_long, taken from a counter): its chunks, sorted by the per-tile sort in chunk64,
// are merged into segments of kMergeSeg entries in shared memory; a longer
// list's segments are then merged pairwise in rounds between chunk64 and
// tmp64 in global memory, each thread taking an equal share of every
// round's outputs (split where it crosses from one pair of runs to the
// next), with a barrier between rounds.  The records of the merged order
// are written into the instance list.
__global__ void __launch_bounds__(kMgT, 2) tile_merge_kernel(const uint2* __restrict__ items,
                                                          const uint32_t* __restrict__ tstart,
                                                          unsigned long long* __restrict__ chunk64,
                                                          unsigned long long* __restrict__ tmp64,
                                                          uint32_t* __restrict__ out, Header* hdr) {
  wait_prior_grid();
  __shared__ unsigned long long s_seg[kMergeSeg];
  __shared__ uint32_t s_it;
  const uint32_t n_long = hdr->n_long;
  for (;;) {
    // the next chunk item, from a counter: the CTAs stay busy however the
    // long lists fall among them; a list's first chunk stands for the list
    __syncthreads();  // every thread has read the previous s_it
    if (threadIdx.x == 0) s_it = atomicAdd(&hdr->ctr[kCtrMergeItems], 1u);
    __syncthreads();
    const uint32_t it = s_it;
    if (it >= n_long) break;
    const uint2 item = items[it];
    if (item.y != 0) continue;  // uniform over the block
    const uint32_t s = tstart[item.x], L = tstart[item.x + 1] - s;
    if (L <= kMergeSeg) {
      merge_segment(chunk64 + s, L, s_seg);
      for (uint32_t i = threadIdx.x; i < L; i += kMgT) out[s + i] = (uint32_t)s_seg[i];
      __syncthreads();  // the segment buffer is free for the block's next list
      continue;
    }
    for (uint32_t s0 = 0; s0 < L; s0 += kMergeSeg) {
      const uint32_t n = min(kMergeSeg, L - s0);
      merge_segment(chunk64 + s + s0, n, s_seg);
      for (uint32_t i = threadIdx.x; i < n; i += kMgT) chunk64[s + s0 + i] = s_seg[i];
      __syncthreads();
    }
    unsigned long long* src = chunk64 + s;
    unsigned long long* dst = tmp64 + s;
    const uint32_t share = (L + kMgT - 1) / kMgT;
    for (uint32_t w = kMergeSeg; w < L; w <<= 1) {
      const uint32_t q0 = min(L, threadIdx.x * share), q1 = min(L, q0 + share);
      for (uint32_t q = q0; q < q1;) {
        const uint32_t p0 = q - q % (2 * w);  // the pair of runs holding output q
        const uint32_t na = min(w, L - p0), nb = min(w, L - min(L, p0 + w));
        const uint32_t qe = min(q1, p0 + na + nb);
        merge_path(src, p0, na, p0 + na, nb, dst, p0, q - p0, qe - p0);
        q = qe;
      }
      __syncthreads();  // the round's outputs are written before the next reads them
      unsigned long long* t = src;
      src = dst;
      dst = t;
    }
    for (uint32_t i = threadIdx.x; i < L; i += kMgT) out[s + i] = (uint32_t)src[i];
    __syncthreads();
  }
}

}  // namespace

const uint32_t* sorted_instances(const Layout& L, const char* ws) { return (const uint32_t*)(ws + L.ivals); }

// grids of the scatter, the per-tile sort and the merge; each loops over
// the work the device counts call for
constexpr uint32_t kScatGrid = 152 * 6, kSortGrid = 152 * 8, kMergeGrid = 152 * 2;
constexpr uint32_t kWalkChunksPerWarp = 2;

uint32_t walk_chunk(const Layout& L) {
  const uint32_t chunk = L.mask_words / (kWalkChunksPerWarp * kScatGrid * kScatW);
  return chunk < 1 ? 1 : (chunk > 32 ? 32 : chunk);
}

uint32_t walk_blocks(const Layout& L) {
  const uint32_t chunk = walk_chunk(L);
  const uint32_t n_chunks = (L.mask_words + chunk - 1) / chunk;
  const uint32_t blocks = (n_chunks + kScatW - 1) / kScatW;
  return blocks < kScatGrid ? blocks : kScatGrid;
}

cudaError_t launch_bin_sort(const Layout& L, const CfgDev& cfg, char* ws, cudaStream_t st) {
  (void)cfg;
  Header* hdr = (Header*)(ws + L.header);
  uint32_t* tstart = (uint32_t*)(ws + L.tstart);
  if (L.R == 0)  // no records: every list is empty (and the tiles keep their order)
    return cudaMemsetAsync(tstart, 0, (size_t)(L.NT + 1) * 4, st);
  const uint32_t* tcount = (const uint32_t*)(ws + L.tcount);  // zeroed by ubs_preprocess
  uint32_t* cursor = (uint32_t*)(ws + L.cursor);
  uint2* items = (uint2*)(ws + L.items);
  // the tile order's bucket totals and cursors: zero here (zeroed by
  // ubs_preprocess with the counts, and again by the scatter once used)
  uint32_t* order_count = (uint32_t*)(ws + L.order_count);
  uint32_t* order = order_possible(L) ? (uint32_t*)(ws + L.tile_order) : nullptr;
  // the visibility walk: chunks of mask words sized so that every warp of
  // the grid has a few (between 1 and 32 words a chunk)
  const uint32_t chunk = walk_chunk(L);
  const dim3 walk_grid(walk_blocks(L));
  launch_dependent(count_kernel, walk_grid, dim3(kScatT), 0, st, (const uint32_t*)(ws + L.tiles),
                   (const uint2*)(ws + L.rect), (const uint32_t*)(ws + L.vis_mask), L.mask_words, chunk,
                   (const ViewDev*)(ws + L.views), L.V, L.NT, (uint32_t*)(ws + L.tcount),
                   (uint32_t*)(ws + L.vis_part));
  static_assert(kVisBlocks >= kScatGrid, "a visible-record count per walk block");
  const uint32_t nb = L.n_scan_blocks;
  ScanPart* part = (ScanPart*)(ws + L.scan_part);
  launch_dependent(scan_part_kernel, dim3(nb), dim3(kScT), 0, st, tcount, L.NT, part,
                   order_count, order != nullptr);
  ScanPart* pre = nullptr;
  ScanPart* tot = nullptr;
  if (nb > kFusePrefixMax) {
    pre = part + nb;
    tot = part + 2 * nb;
    launch_dependent(scan_mid_kernel, dim3(1), dim3(kScT), 0, st, (const ScanPart*)part, nb, pre, tot);
  }
  launch_dependent(scan_place_kernel, dim3(nb), dim3(kScT), 0, st, tcount, L.NT, L.cap, (const ScanPart*)part, nb,
                   (const ScanPart*)pre, (const ScanPart*)tot, hdr, tstart, cursor, items, order_count, order);
  uint32_t* bucket = (uint32_t*)(ws + L.bucket);
  launch_dependent(scatter_kernel, walk_grid, dim3(kScatT), 0, st, (const uint32_t*)(ws + L.tiles),
                   (const uint2*)(ws + L.rect), (const uint32_t*)(ws + L.vis_mask), L.mask_words, chunk,
                   (const ViewDev*)(ws + L.views), L.V, L.NT, L.cap, (const Header*)hdr, cursor, bucket,
                   (uint32_t*)(ws + L.tcount), order_count);
  uint32_t* out = (uint32_t*)(ws + L.ivals);
  unsigned long long* chunk64 = (unsigned long long*)(ws + L.chunk64);
  const uint32_t ts_blocks = (L.max_items + kTsW - 1) / kTsW;
  launch_dependent(tile_sort_kernel, dim3(ts_blocks < kSortGrid ? ts_blocks : kSortGrid), dim3(kTsW * 32), 0, st,
                   (const uint2*)items, (const uint32_t*)tstart, (const uint32_t*)(ws + L.key), L.R,
                   (const uint32_t*)bucket, out, chunk64, hdr);
  launch_dependent(tile_merge_kernel, dim3(kMergeGrid), dim3(kMgT), 0, st, (const uint2*)items,
                   (const uint32_t*)tstart, chunk64, (unsigned long long*)(ws + L.tmp64), out, hdr);
  return cudaGetLastError();
}

}  // namespace ubs
