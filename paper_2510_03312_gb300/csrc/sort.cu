// sort.cu -- B1-B3: tile binning, front-to-back order and tile ranges.
//
// The instance order is (global tile, float32 depth, record index).  It is
// produced as two stable LSD radix sorts instead of one sort of 64-bit
// (tile, depth) keys over all instances:
//   1. compact the visible records (order-preserving, so ties stay in record
//      order) and sort them by depth (4 passes of 8 bits over records);
//   2. emit the instances of the depth-sorted records in that order (every
//      record's tiles row-major in its rectangle);
//   3. sort the instances by tile id (ceil(log2 tiles / 8) passes);
//   4. find each tile's range from the boundaries of the sorted tile keys.
// Because both sorts are stable, each tile's list ends up in (depth, record)
// order: the same order as a single sort by the 64-bit key, at roughly half
// the bytes (depth passes touch records, not instances).
//
// No kernel waits on another block: every step that needs the offsets of
// earlier blocks is split at a kernel boundary (count, then scan, then
// place).  The counts a step needs are made by the kernel before it, while
// it writes that step's input: the preprocess kernel counts visible records
// per compaction block; the compaction counts the first depth pass's digits
// per (pass block, digit); each radix pass counts the next pass's digits for
// the positions it writes (the last depth pass counts instances per
// emission block instead); the emission counts the first tile pass's
// digits.  A column scan turns counts into each block's exclusive offsets
// (and digit totals), and the pass then ranks its items locally (stable)
// and places them.
#include "kernels.cuh"

namespace ubs {

namespace {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ void set_status(Header* h, uint32_t s) { atomicCAS(&h->status, 0u, s); }

__device__ __forceinline__ uint32_t lane_id() { return threadIdx.x & 31; }

// Lanes of the warp holding the same 9-bit value d (digits < 256, 0x100 for
// "no item"): one ballot per bit, each lane keeping the lanes that agree.
__device__ __forceinline__ uint32_t peer_mask(uint32_t d) {
  uint32_t peers = kFull;
#pragma unroll
  for (int b = 0; b < 9; ++b) {
    const bool bit = (d >> b) & 1u;
    const uint32_t bal = __ballot_sync(kFull, bit);
    peers &= bit ? bal : ~bal;
  }
  return peers;
}

__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t v) {
  const uint32_t lane = lane_id();
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t t = __shfl_up_sync(kFull, v, o);
    if (lane >= (uint32_t)o) v += t;
  }
  return v;
}

// Exclusive scan of one value per thread over a block of NT threads.
// s_w must hold NT/32 + 1 words.  Must be called by every thread.
template <int NT>
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t& total, uint32_t* s_w) {
  constexpr int NW = NT / 32;
  const uint32_t lane = lane_id(), warp = threadIdx.x >> 5;
  const uint32_t incl = warp_incl_scan(v);
  if (lane == 31) s_w[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    uint32_t w = lane < NW ? s_w[lane] : 0;
    uint32_t wi = warp_incl_scan(w);
    if (lane < NW) s_w[lane] = wi - w;
    if (lane == NW - 1) s_w[NW] = wi;
  }
  __syncthreads();
  total = s_w[NW];
  const uint32_t out = s_w[warp] + incl - v;
  __syncthreads();
  return out;
}

// ---------------------------------------------------------------- column scan

constexpr int kScT = 256, kScI = 8;

// Exclusive scan down each column of a row-major [rows][cols] matrix (out
// may equal in); one block per column; the column sums go to totals (if
// non-null).  With n_ptr, only the first ceil(min(*n_ptr, cap) / per_row)
// rows are scanned: the rows that can hold counts of n items.
__global__ void __launch_bounds__(kScT) col_scan_kernel(const uint32_t* in, uint32_t* out, uint32_t rows,
                                                        uint32_t cols, uint32_t* totals, const uint64_t* n_ptr,
                                                        uint32_t cap, uint32_t per_row) {
  wait_prior_grid();
  __shared__ uint32_t s_w[kScT / 32 + 1];
  const uint32_t c = blockIdx.x;
  if (n_ptr) {
    const uint64_t n = *n_ptr < cap ? *n_ptr : cap;
    const uint64_t used = (n + per_row - 1) / per_row;
    if (used < rows) rows = (uint32_t)used;
  }
  uint32_t carry = 0;
  for (uint32_t r0 = 0; r0 < rows; r0 += kScT * kScI) {
    uint32_t v[kScI], sum = 0;
    const uint32_t rb = r0 + threadIdx.x * kScI;
#pragma unroll
    for (int i = 0; i < kScI; ++i) {
      v[i] = (rb + i < rows) ? in[(size_t)(rb + i) * cols + c] : 0u;
      sum += v[i];
    }
    uint32_t total;
    uint32_t ex = block_excl_scan<kScT>(sum, total, s_w);
#pragma unroll
    for (int i = 0; i < kScI; ++i) {
      if (rb + i < rows) out[(size_t)(rb + i) * cols + c] = carry + ex;
      ex += v[i];
    }
    carry += total;
  }
  if (totals && threadIdx.x == 0) totals[c] = carry;
}

// ---------------------------------------------------------------- compaction

constexpr int kCmpT = 256, kCmpI = kCmpTile / kCmpT;
// depth pass blocks that kCmpTile consecutive output positions can fall in
constexpr int kCmpSpan = (kCmpTile + kDsTile - 1) / kDsTile + 1;

// The sum of v[0 .. n) over a block of NT threads (every thread calls it).
template <int NT>
__device__ __forceinline__ uint32_t block_sum_prefix(const uint32_t* __restrict__ v, uint32_t n, uint32_t* s_w) {
  uint32_t part = 0;
  for (uint32_t i = threadIdx.x; i < n; i += NT) part += v[i];
  uint32_t total;
  block_excl_scan<NT>(part, total, s_w);
  return total;
}

// Keeps the records with tiles_touched > 0, in record order, as (depth key,
// record) pairs starting at the block's exclusive prefix of the visible
// counts, and counts the first depth pass's digits per (pass block, digit)
// into hist0.  The prefix is vis_prefix[block] (scanned by a kernel before),
// or, where there are few compaction blocks (vis_count non-null), the sum of
// the earlier blocks' counts, taken here: one launch fewer.
constexpr uint32_t kFusePrefixMax = 2048;  // blocks up to which a block sums the earlier blocks' counts itself
__global__ void __launch_bounds__(kCmpT) compact_kernel(const uint32_t* __restrict__ tiles,
                                                        const uint32_t* __restrict__ key, uint32_t R,
                                                        const uint32_t* __restrict__ vis_prefix,
                                                        const uint32_t* __restrict__ vis_count,
                                                        uint32_t* __restrict__ okey, uint32_t* __restrict__ oval,
                                                        uint32_t* __restrict__ hist0, Header* hdr) {
  wait_prior_grid();
  __shared__ uint32_t s_w[kCmpT / 32 + 1];
  const uint32_t t = blockIdx.x;
  const uint32_t excl = vis_count ? block_sum_prefix<kCmpT>(vis_count, t, s_w) : vis_prefix[t];
  const uint32_t base = t * kCmpTile + threadIdx.x * kCmpI;
  bool f[kCmpI];
  uint32_t k[kCmpI];
  uint32_t cnt = 0;
#pragma unroll
  for (int i = 0; i < kCmpI; ++i) {
    const uint32_t idx = base + i;
    f[i] = idx < R && __ldg(tiles + idx) > 0;
    k[i] = f[i] ? __ldg(key + idx) : 0u;
    cnt += f[i];
  }
  uint32_t total;
  uint32_t pos = excl + block_excl_scan<kCmpT>(cnt, total, s_w);
  __shared__ uint32_t s_h[kCmpSpan][256];
  for (int i = threadIdx.x; i < kCmpSpan * 256; i += kCmpT) (&s_h[0][0])[i] = 0;
  __syncthreads();
  const uint32_t ob0 = excl / kDsTile;
#pragma unroll
  for (int i = 0; i < kCmpI; ++i)
    if (f[i]) {
      if (pos < R) {  // holds by construction (counts made by preprocess)
        okey[pos] = k[i];
        oval[pos] = base + i;
        atomicAdd(&s_h[min(pos / kDsTile - ob0, (uint32_t)kCmpSpan - 1u)][k[i] & 255u], 1u);
      }
      ++pos;
    }
  __syncthreads();
  // first depth pass: counts per (pass block, digit)
  for (int i = threadIdx.x; i < kCmpSpan * 256; i += kCmpT) {
    const uint32_t c = (&s_h[0][0])[i];
    if (c) atomicAdd(hist0 + (size_t)(ob0 + i / 256) * 256 + (i & 255), c);
  }
  if (t == gridDim.x - 1 && threadIdx.x == 0) hdr->n_visible = excl + total;
}

// ---------------------------------------------------------------- radix pass

constexpr int kOsT = 256, kOsW = kOsT / 32;

// One stable pass of the LSD radix sort over the 8 bits at `shift`: local
// ranking, placement at (exclusive prefix of ghist) + hprefix[block][digit]
// + rank, and, while placing, the counts the following step needs:
//   ghist:   digit totals of this pass over all n items
//   hprefix: [blocks][256] exclusive column prefix of this pass's
//            per-(block, digit) counts
//   hnext:   if non-null, counts of the next pass's digit (at shift + 8) per
//            (output block, digit)
//   icount:  if non-null, instances (tiles_touched of each placed record)
//            per emission block of the output
// The counts are summed over lanes with equal (block, digit) before one
// atomic add per group.  A block ranks TILE items.
template <int TILE>
__global__ void __launch_bounds__(kOsT, 5) downsweep_kernel(const uint32_t* __restrict__ kin,
                                                         const uint32_t* __restrict__ vin, uint32_t* __restrict__ kout,
                                                         uint32_t* __restrict__ vout, const uint64_t* n_ptr,
                                                         uint32_t cap, int shift, const uint32_t* __restrict__ ghist,
                                                         const uint32_t* __restrict__ hprefix, uint32_t* hnext,
                                                         uint32_t* icount, const uint32_t* __restrict__ tiles_touched) {
  wait_prior_grid();
  constexpr int kOsI = TILE / kOsT;
  __shared__ uint32_t s_keys[TILE];
  __shared__ uint32_t s_vals[TILE];
  __shared__ uint32_t s_hist[kOsW][256];
  __shared__ uint32_t s_boff[256];
  __shared__ uint32_t s_goff[256];
  __shared__ uint32_t s_w[kOsT / 32 + 1];
  const uint64_t n64 = *n_ptr;
  const uint32_t n = (uint32_t)(n64 < cap ? n64 : cap);
  // grid-stride over the pass's tiles (the grid is sized by the capacity,
  // the work by the count found on the device)
  for (uint32_t t = blockIdx.x; (uint64_t)t * TILE < n; t += gridDim.x) {
    __syncthreads();  // the shared arrays of the previous tile are free
    const uint32_t tile_base = t * TILE;
    for (int i = threadIdx.x; i < kOsW * 256; i += kOsT) (&s_hist[0][0])[i] = 0;
    __syncthreads();
    const uint32_t lane = lane_id(), warp = threadIdx.x >> 5;
    const uint32_t lt_mask = (1u << lane) - 1u;
    const uint32_t wbase = tile_base + warp * (kOsI * 32);
    uint32_t k[kOsI], v[kOsI], rank[kOsI];
#pragma unroll
    for (int i = 0; i < kOsI; ++i) {
      const uint32_t idx = wbase + i * 32 + lane;
      const bool ok = idx < n;
      k[i] = ok ? kin[idx] : 0u;
      v[i] = ok ? vin[idx] : 0u;
    }
#pragma unroll
    for (int i = 0; i < kOsI; ++i) {
      const uint32_t idx = wbase + i * 32 + lane;
      const bool ok = idx < n;
      const uint32_t d = ok ? (k[i] >> shift) & 255u : 0x100u;
      const uint32_t peers = peer_mask(d);
      uint32_t cnt = 0;
      if (d < 256) cnt = s_hist[warp][d];
      __syncwarp();
      rank[i] = ok ? cnt + __popc(peers & lt_mask) : 0xffffffffu;
      if (d < 256 && lane == (uint32_t)(__ffs(peers) - 1)) s_hist[warp][d] = cnt + __popc(peers);
      __syncwarp();
    }
    __syncthreads();
    const uint32_t d = threadIdx.x;  // one digit per thread
    uint32_t acc = 0;
#pragma unroll
    for (int w = 0; w < kOsW; ++w) {
      const uint32_t c = s_hist[w][d];
      s_hist[w][d] = acc;
      acc += c;
    }
    uint32_t gtot;
    const uint32_t gbase = block_excl_scan<kOsT>(ghist[d], gtot, s_w);
    uint32_t btot;
    const uint32_t boff = block_excl_scan<kOsT>(acc, btot, s_w);
    s_boff[d] = boff;
    s_goff[d] = gbase + hprefix[(size_t)t * 256 + d] - boff;
    __syncthreads();
#pragma unroll
    for (int i = 0; i < kOsI; ++i) {
      if (rank[i] != 0xffffffffu) {
        const uint32_t dd = (k[i] >> shift) & 255u;
        const uint32_t pos = s_boff[dd] + s_hist[warp][dd] + rank[i];
        s_keys[pos] = k[i];
        s_vals[pos] = v[i];
      }
    }
    __syncthreads();
    const uint32_t cnt_tile = (n - tile_base) < (uint32_t)TILE ? (n - tile_base) : (uint32_t)TILE;
#pragma unroll 4
    for (int it = 0; it < kOsI; ++it) {
      const uint32_t j = it * kOsT + threadIdx.x;
      bool valid = j < cnt_tile;
      uint32_t key = 0, val = 0, g = 0;
      if (valid) {
        key = s_keys[j];
        val = s_vals[j];
        g = s_goff[(key >> shift) & 255u] + j;
        valid = g < n;  // holds by construction (consistent digit counts)
        if (valid) {
          kout[g] = key;
          vout[g] = val;
        }
      }
      if (hnext) {
        const uint32_t grp = valid ? ((g / TILE) << 8) | ((key >> (shift + 8)) & 255u) : 0xffffffffu;
        const uint32_t peers = __match_any_sync(kFull, grp);
        if (valid && lane == (uint32_t)(__ffs(peers) - 1))
          atomicAdd(hnext + (size_t)(grp >> 8) * 256 + (grp & 255u), (uint32_t)__popc(peers));
      }
      if (icount) {
        const uint32_t grp = valid ? g / kEmTile : 0xffffffffu;
        const uint32_t peers = __match_any_sync(kFull, grp);
        const uint32_t sum = __reduce_add_sync(peers, valid ? tiles_touched[val] : 0u);
        if (valid && lane == (uint32_t)(__ffs(peers) - 1)) atomicAdd(icount + grp, sum);
      }
    }
  }
}

// ---------------------------------------------------------------- emission

constexpr int kEmT = 256, kEmI = kEmTile / kEmT;

// First instance of each depth-sorted record: ioff[i] = the block's
// exclusive prefix of the instance counts + the exclusive scan of
// tiles_touched within the block.  The prefix is icount[block], scanned in
// place by a kernel before, or, with `summed` (few blocks), the sum of the
// earlier blocks' raw counts, taken here.  The last block records the
// instance total and flags an instance capacity overflow.
__global__ void __launch_bounds__(kEmT) emit_offsets_kernel(const uint32_t* __restrict__ srec,
                                                            const uint32_t* __restrict__ tiles,
                                                            const uint32_t* __restrict__ icount, bool summed,
                                                            uint32_t* __restrict__ ioff, uint32_t cap, Header* hdr) {
  wait_prior_grid();
  __shared__ uint32_t s_w[kEmT / 32 + 1];
  __shared__ uint32_t s_pre;
  const uint32_t n = (uint32_t)hdr->n_visible;
  const uint32_t n_blocks = (n + kEmTile - 1) / kEmTile;
  for (uint32_t t = blockIdx.x; t < n_blocks; t += gridDim.x) {
    if (summed) {
      const uint32_t pre = block_sum_prefix<kEmT>(icount, t, s_w);
      if (threadIdx.x == 0) s_pre = pre;
    } else if (threadIdx.x == 0) {
      s_pre = icount[t];
    }
    __syncthreads();
    const uint32_t prefix = s_pre;
    const uint32_t base = t * kEmTile + threadIdx.x * kEmI;
    uint32_t c[kEmI], sum = 0;
#pragma unroll
    for (int i = 0; i < kEmI; ++i) {
      c[i] = base + i < n ? tiles[srec[base + i]] : 0u;
      sum += c[i];
    }
    uint32_t total;
    uint32_t ex = prefix + block_excl_scan<kEmT>(sum, total, s_w);
#pragma unroll
    for (int i = 0; i < kEmI; ++i) {
      if (base + i < n) ioff[base + i] = ex;
      ex += c[i];
    }
    if (t == n_blocks - 1 && threadIdx.x == 0) {
      const uint64_t n_inst = (uint64_t)prefix + total;
      hdr->n_inst = n_inst;
      if (n_inst > cap) set_status(hdr, kDevCapacity);
    }
  }
}

constexpr int kFlT = 256, kFlI = kIsTile / kFlT;
static_assert(kFlI == 8, "a thread's instances are written as two 16-byte vectors per array");
static_assert(kMaxViews <= 256, "view indices are staged as bytes");

// Instances [b K, (b + 1) K) of the depth-sorted order, K = kIsTile: block b
// of the first tile-key pass, so that every block does the same work however
// unevenly the instances fall over the records.  Instance j belongs to the
// sorted record i with ioff[i] <= j < ioff[i + 1] and is that record's
// (j - ioff[i])-th tile, row-major in its rectangle; it is written as
// (global tile, record).  ioff strictly increases (every visible record
// touches a tile), so the block's instances lie in at most K records from
// the one holding its first instance.  The block first stages those
// records (id, rectangle, view) in shared memory, all gathers in flight at
// once; each thread then walks its kFlI consecutive instances from shared
// memory and writes them as 16-byte vectors.  Writes the first tile pass's
// digit counts of the block.
__global__ void __launch_bounds__(kFlT) emit_fill_kernel(const uint32_t* __restrict__ srec,
                                                         const uint32_t* __restrict__ ioff,
                                                         const uint2* __restrict__ rect,
                                                         const ViewDev* __restrict__ views, int V, uint32_t cap,
                                                         uint32_t* __restrict__ ikey, uint32_t* __restrict__ ival,
                                                         uint32_t* __restrict__ hist0, const Header* hdr) {
  wait_prior_grid();
  __shared__ uint32_t s_off[kIsTile + 1];
  __shared__ uint32_t s_rec[kIsTile];
  __shared__ uint2 s_rect[kIsTile];
  __shared__ uint8_t s_view[kIsTile];
  __shared__ uint32_t s_h[256];
  __shared__ uint32_t s_recoff[kMaxViews], s_tileoff[kMaxViews], s_tilesx[kMaxViews];
  __shared__ uint32_t s_r0, s_nr;
  const uint32_t nv = (uint32_t)hdr->n_visible;
  const uint64_t ni64 = hdr->n_inst;
  const uint32_t n_inst = (uint32_t)(ni64 < cap ? ni64 : cap);
  if (nv == 0) return;
  for (int i = threadIdx.x; i < V; i += kFlT) {
    s_recoff[i] = views[i].rec_off;
    s_tileoff[i] = views[i].tile_off;
    s_tilesx[i] = (uint32_t)views[i].tiles_x;
  }
  for (uint32_t b = blockIdx.x; (uint64_t)b * kIsTile < n_inst; b += gridDim.x) {
    const uint32_t s = b * kIsTile;
    __syncthreads();  // the shared arrays of the previous block are free
    for (int i = threadIdx.x; i < 256; i += kFlT) s_h[i] = 0;
    if (threadIdx.x == 0) s_nr = 0;
    if (threadIdx.x < 32) {
      // the last sorted record with ioff <= s, by a 32-way search: each round
      // samples 32 offsets of [lo, hi) and keeps the span after the last one
      // <= s (ioff[0] = 0 <= s, so lane 0's sample always qualifies)
      const uint32_t lane = threadIdx.x;
      uint32_t lo = 0, hi = nv;
      while (hi - lo > 32) {
        const uint32_t step = (hi - lo + 31) / 32;
        const uint32_t idx = lo + lane * step;
        const uint32_t m = __ballot_sync(kFull, idx < hi && ioff[idx] <= s);
        lo += (31u - __clz(m)) * step;
        hi = min(hi, lo + step);
      }
      const uint32_t idx = lo + lane;
      const uint32_t m = __ballot_sync(kFull, idx < hi && ioff[idx] <= s);
      if (lane == 0) s_r0 = lo + 31u - __clz(m);
    }
    __syncthreads();
    const uint32_t r0 = s_r0;
    // the offsets of records r0 .. r0 + K, and the number of those records
    // that start inside the block (the records holding its instances)
    uint32_t starts = 0;
    for (uint32_t i = threadIdx.x; i <= (uint32_t)kIsTile; i += kFlT) {
      const uint32_t o = r0 + i < nv ? ioff[r0 + i] : 0xffffffffu;
      s_off[i] = o;
      starts += (i < (uint32_t)kIsTile && o < s + (uint32_t)kIsTile);
    }
    if (starts) atomicAdd(&s_nr, starts);
    __syncthreads();
    const uint32_t nr = min(s_nr, (uint32_t)kIsTile);
    // stage those records (id, rectangle and view), a thread's ids loaded
    // together and then its rectangles
    {
      uint32_t rk[kFlI];
      uint2 rc[kFlI];
#pragma unroll
      for (int k = 0; k < kFlI; ++k) {
        const uint32_t i = threadIdx.x + k * kFlT;
        rk[k] = i < nr ? srec[r0 + i] : 0u;
      }
#pragma unroll
      for (int k = 0; k < kFlI; ++k) {
        const uint32_t i = threadIdx.x + k * kFlT;
        if (i < nr) rc[k] = rect[rk[k]];
      }
#pragma unroll
      for (int k = 0; k < kFlI; ++k) {
        const uint32_t i = threadIdx.x + k * kFlT;
        if (i < nr) {
          int vlo = 0, vhi = V - 1;  // view of the record: last view with rec_off <= rec
          while (vlo < vhi) {
            const int mid = (vlo + vhi + 1) >> 1;
            if (s_recoff[mid] <= rk[k]) vlo = mid; else vhi = mid - 1;
          }
          s_rec[i] = rk[k];
          s_rect[i] = rc[k];
          s_view[i] = (uint8_t)vlo;
        }
      }
    }
    __syncthreads();
    // kFlI consecutive instances per thread, walking the staged records
    const uint32_t j0 = s + threadIdx.x * kFlI;
    if (j0 < n_inst) {
      int lo = 0, hi = (int)nr - 1;  // last i with s_off[i] <= j0 (s_off[0] <= s)
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (s_off[mid] <= j0) lo = mid; else hi = mid - 1;
      }
      uint32_t i = (uint32_t)lo;
      uint32_t kk[kFlI], vv[kFlI];
      uint32_t rec = 0, x0 = 0, x1 = 0, tx = 0, ty = 0, vt = 0, vx = 0;
      bool fresh = true;
#pragma unroll
      for (int k = 0; k < kFlI; ++k) {
        const uint32_t j = j0 + k;
        kk[k] = vv[k] = 0;
        if (j < n_inst) {
          while (s_off[i + 1] <= j) {  // stays below nr: s_off[nr] > j
            ++i;
            fresh = true;
          }
          if (fresh) {
            fresh = false;
            rec = s_rec[i];
            const uint2 rc = s_rect[i];
            x0 = rc.x & 0xFFFFu;
            x1 = rc.y & 0xFFFFu;
            const uint32_t w = x1 - x0, local = j - s_off[i];
            tx = x0 + local % w;
            ty = (rc.x >> 16) + local / w;
            vt = s_tileoff[s_view[i]];
            vx = s_tilesx[s_view[i]];
          }
          const uint32_t gt = vt + ty * vx + tx;
          kk[k] = gt;
          vv[k] = rec;
          atomicAdd(&s_h[gt & 255u], 1u);
          if (++tx == x1) {
            tx = x0;
            ++ty;
          }
        }
      }
      if (j0 + kFlI <= n_inst) {  // j0 is a multiple of 8: 32-byte aligned
        uint4* kd = reinterpret_cast<uint4*>(ikey + j0);
        uint4* vd = reinterpret_cast<uint4*>(ival + j0);
        kd[0] = make_uint4(kk[0], kk[1], kk[2], kk[3]);
        kd[1] = make_uint4(kk[4], kk[5], kk[6], kk[7]);
        vd[0] = make_uint4(vv[0], vv[1], vv[2], vv[3]);
        vd[1] = make_uint4(vv[4], vv[5], vv[6], vv[7]);
      } else {
#pragma unroll
        for (int k = 0; k < kFlI; ++k)
          if (j0 + k < n_inst) {
            ikey[j0 + k] = kk[k];
            ival[j0 + k] = vv[k];
          }
      }
    }
    __syncthreads();
    // this block is block b of the first tile pass: its counts are
    // written whole (no pass and no counts when the problem has one tile)
    if (hist0)
      for (int d = threadIdx.x; d < 256; d += kFlT) hist0[(size_t)b * 256 + d] = s_h[d];
  }
}

// ---------------------------------------------------------------- ranges

// Position i of the sorted tile keys starts the ranges of every tile g with
// key[i-1] < g <= key[i] (key[-1] = -1, key[n] = NT), so tstart[g] is the
// first position whose key is >= g, and tstart[NT] = n.
__global__ void ranges_kernel(const uint32_t* __restrict__ skeys, const uint64_t* n_ptr, uint32_t cap, uint32_t NT,
                              uint32_t* __restrict__ tstart) {
  wait_prior_grid();
  const uint64_t n64 = *n_ptr;
  const uint32_t n = (uint32_t)(n64 < cap ? n64 : cap);
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i <= n; i += gridDim.x * blockDim.x) {
    const int64_t prev = i > 0 ? (int64_t)skeys[i - 1] : -1;
    const int64_t cur = i < n ? (int64_t)min(skeys[i], NT) : (int64_t)NT;
    for (int64_t g = prev + 1; g <= cur; ++g) tstart[g] = i;
  }
}

// ---------------------------------------------------------------- tile order

constexpr int kOrdT = 1024, kOrdBuckets = 4 * 33;

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

// The tiles in the order the blend kernels take them.  Where lists are long
// on average, by list length, longest first (to a quarter octave; the order
// within a bucket is arbitrary), so that long tiles start early and do not
// trail the grid; where they are short, the blend kernels keep the tiles'
// own order (neighbouring tiles share records) and nothing here runs.
// Every tile appears once, so the order changes no result.
//
// Up to kOrdSingle tiles: one block counts the tiles per bucket, scans the
// counts and places the tiles.
constexpr uint32_t kOrdSingle = 16384;
__global__ void __launch_bounds__(kOrdT) tile_order_single_kernel(const uint32_t* __restrict__ tstart, uint32_t NT,
                                                                 uint32_t cap, const Header* hdr,
                                                                 uint32_t* __restrict__ order) {
  wait_prior_grid();
  if (!order_dense(hdr, NT, cap)) return;
  __shared__ uint32_t s_n[kOrdBuckets];
  for (int i = threadIdx.x; i < kOrdBuckets; i += kOrdT) s_n[i] = 0;
  __syncthreads();
  // every tile's bucket in registers first: the loads are all in flight at once
  constexpr int PER_T = kOrdSingle / kOrdT;
  int bk[PER_T];
#pragma unroll
  for (int k = 0; k < PER_T; ++k) {
    const uint32_t t = k * kOrdT + threadIdx.x;
    bk[k] = t < NT ? length_bucket(tstart[t + 1] - tstart[t]) : -1;
  }
#pragma unroll
  for (int k = 0; k < PER_T; ++k)
    if (k * kOrdT < NT) bucket_add(s_n, bk[k]);  // uniform over the block: whole warps
  __syncthreads();
  if (threadIdx.x < 32) {  // exclusive scan of the counts: five buckets a lane
    constexpr int PER = (kOrdBuckets + 31) / 32;
    const int lane = threadIdx.x;
    uint32_t c[PER], sum = 0;
#pragma unroll
    for (int j = 0; j < PER; ++j) {
      const int i = lane * PER + j;
      c[j] = i < kOrdBuckets ? s_n[i] : 0u;
      sum += c[j];
    }
    uint32_t incl = sum;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const uint32_t o = __shfl_up_sync(0xffffffffu, incl, d);
      if (lane >= d) incl += o;
    }
    uint32_t run = incl - sum;
#pragma unroll
    for (int j = 0; j < PER; ++j) {
      const int i = lane * PER + j;
      if (i < kOrdBuckets) s_n[i] = run;
      run += c[j];
    }
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < PER_T; ++k)
    if (k * kOrdT < NT) {
      const uint32_t pos = bucket_add(s_n, bk[k]);
      if (bk[k] >= 0) order[pos] = k * kOrdT + threadIdx.x;
    }
}

// More tiles, pass 1: the tiles per bucket, one block per kOrdT tiles.
__global__ void __launch_bounds__(kOrdT) tile_order_count_kernel(const uint32_t* __restrict__ tstart, uint32_t NT,
                                                                uint32_t cap, const Header* hdr,
                                                                uint32_t* __restrict__ totals) {
  wait_prior_grid();
  if (!order_dense(hdr, NT, cap)) return;
  __shared__ uint32_t s_n[kOrdBuckets];
  for (int i = threadIdx.x; i < kOrdBuckets; i += kOrdT) s_n[i] = 0;
  __syncthreads();
  const uint32_t t = blockIdx.x * kOrdT + threadIdx.x;
  bucket_add(s_n, t < NT ? length_bucket(tstart[t + 1] - tstart[t]) : -1);
  __syncthreads();
  for (int i = threadIdx.x; i < kOrdBuckets; i += kOrdT)
    if (s_n[i]) atomicAdd(totals + i, s_n[i]);
}

// Pass 2: each block reserves a range per bucket (after the longer buckets'
// totals) and places its tiles there.
__global__ void __launch_bounds__(kOrdT) tile_order_place_kernel(const uint32_t* __restrict__ tstart, uint32_t NT,
                                                                uint32_t cap, const Header* hdr,
                                                                const uint32_t* __restrict__ totals,
                                                                uint32_t* __restrict__ cursor,
                                                                uint32_t* __restrict__ order) {
  wait_prior_grid();
  if (!order_dense(hdr, NT, cap)) return;
  const uint32_t t = blockIdx.x * kOrdT + threadIdx.x;
  __shared__ uint32_t s_n[kOrdBuckets], s_base[kOrdBuckets];
  for (int i = threadIdx.x; i < kOrdBuckets; i += kOrdT) s_n[i] = 0;
  __syncthreads();
  const int b = t < NT ? length_bucket(tstart[t + 1] - tstart[t]) : -1;
  const uint32_t rank = bucket_add(s_n, b);
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t start = 0;  // the bucket's first position: the longer buckets' totals
    for (int i = 0; i < kOrdBuckets; ++i) {
      if (s_n[i]) s_base[i] = start + atomicAdd(cursor + i, s_n[i]);
      start += totals[i];
    }
  }
  __syncthreads();
  if (b >= 0) order[s_base[b] + rank] = t;
}

}  // namespace

const uint32_t* sorted_instances(const Layout& L, const char* ws) {
  return (const uint32_t*)(ws + ((L.tile_passes & 1) ? L.ivB : L.ivA));
}

// grids of the radix passes (5 resident CTAs per SM: the pass is held to 48
// registers for it, against 4 CTAs at 64 -- the 64-job mix's sort 1676 ->
// 1622 us; 6 spilled) and of the emission kernels; each loops over the
// blocks of work the device counts call for
constexpr uint32_t kPassGrid = 152 * 5, kEmitGrid = 152 * 8;

cudaError_t launch_tile_order(const Layout& L, char* ws, const Header* hdr, cudaStream_t st) {
  if (!order_possible(L)) return cudaSuccess;  // the lists cannot be dense: the tiles keep their order
  const uint32_t* tstart = (const uint32_t*)(ws + L.tstart);
  uint32_t* order = (uint32_t*)(ws + L.tile_order);
  if (L.NT <= kOrdSingle) {
    launch_dependent(tile_order_single_kernel, dim3(1), dim3(kOrdT), 0, st, tstart, L.NT, L.cap, hdr, order);
    return cudaGetLastError();
  }
  uint32_t* totals = (uint32_t*)(ws + L.order_count);  // zeroed at the start of bin_sort
  const unsigned blocks = (L.NT + kOrdT - 1) / kOrdT;
  launch_dependent(tile_order_count_kernel, dim3(blocks), dim3(kOrdT), 0, st, tstart, L.NT, L.cap, hdr, totals);
  launch_dependent(tile_order_place_kernel, dim3(blocks), dim3(kOrdT), 0, st, tstart, L.NT, L.cap, hdr,
                   (const uint32_t*)totals, totals + kOrdBuckets, order);
  return cudaGetLastError();
}

cudaError_t launch_bin_sort(const Layout& L, const CfgDev& cfg, char* ws, cudaStream_t st) {
  (void)cfg;
  Header* hdr = (Header*)(ws + L.header);
  if (L.R == 0)  // no records: every list is empty (and the tiles keep their order)
    return cudaMemsetAsync(ws + L.tstart, 0, (size_t)(L.NT + 1) * 4, st);
  // the per-pass counts are accumulated with atomics: start them at zero
  cudaError_t e = cudaMemsetAsync(ws + L.hist_d, 0, L.Tfin - L.hist_d, st);
  if (e != cudaSuccess) return e;
  const uint32_t* vis = (const uint32_t*)(ws + L.vis_count);
  uint32_t* vis_prefix = (uint32_t*)(ws + L.vis_prefix);
  uint32_t* hd = (uint32_t*)(ws + L.hist_d);
  uint32_t* hi = (uint32_t*)(ws + L.hist_i);
  uint32_t* icount = (uint32_t*)(ws + L.icount);
  uint32_t* ghist = (uint32_t*)(ws + L.ghist);  // [4 depth + 3 tile][256]
  const uint32_t* tiles = (const uint32_t*)(ws + L.tiles);
  uint32_t* ckA = (uint32_t*)(ws + L.ckA);
  uint32_t* cvA = (uint32_t*)(ws + L.cvA);
  uint32_t* ckB = (uint32_t*)(ws + L.ckB);
  uint32_t* cvB = (uint32_t*)(ws + L.cvB);
  const bool fuse_vis = L.n_cmp_tiles <= kFusePrefixMax;
  if (!fuse_vis)
    launch_dependent(col_scan_kernel, dim3(1), dim3(kScT), 0, st, vis, vis_prefix, L.n_cmp_tiles, 1, nullptr,
                     nullptr, 0u, 1u);
  const size_t hd_stride = (size_t)L.n_dsort_tiles * 256;
  launch_dependent(compact_kernel, dim3(L.n_cmp_tiles), dim3(kCmpT), 0, st, tiles, (const uint32_t*)(ws + L.key), L.R,
                   (const uint32_t*)vis_prefix, fuse_vis ? vis : nullptr, ckA, cvA, hd, hdr);
  // depth sort: 4 passes A->B->A->B->A; the last one counts instances per
  // emission block
  for (int p = 0; p < 4; ++p) {
    const bool even = (p & 1) == 0;
    uint32_t* hp = hd + p * hd_stride;
    const bool last = p == 3;
    launch_dependent(col_scan_kernel, dim3(256), dim3(kScT), 0, st, hp, hp, L.n_dsort_tiles, 256, ghist + 256 * p,
                     (const uint64_t*)&hdr->n_visible, L.R, (uint32_t)kDsTile);
    launch_dependent(downsweep_kernel<kDsTile>, dim3(min(L.n_dsort_tiles, kPassGrid)), dim3(kOsT), 0, st, even ? ckA : ckB, even ? cvA : cvB, even ? ckB : ckA,
                                                       even ? cvB : cvA, &hdr->n_visible, L.R, 8 * p, ghist + 256 * p,
                                                       hp, last ? nullptr : hp + hd_stride, last ? icount : nullptr,
                                                       tiles);
  }
  uint32_t* ikA = (uint32_t*)(ws + L.ikA);
  uint32_t* ivA = (uint32_t*)(ws + L.ivA);
  uint32_t* ikB = (uint32_t*)(ws + L.ikB);
  uint32_t* ivB = (uint32_t*)(ws + L.ivB);
  const ViewDev* views = (const ViewDev*)(ws + L.views);
  const bool fuse_icount = L.n_emit_tiles <= kFusePrefixMax;
  if (!fuse_icount)
    launch_dependent(col_scan_kernel, dim3(1), dim3(kScT), 0, st, icount, icount, L.n_emit_tiles, 1, nullptr,
                     (const uint64_t*)&hdr->n_visible, L.R, (uint32_t)kEmTile);
  uint32_t* ioff = (uint32_t*)(ws + L.ioff);
  launch_dependent(emit_offsets_kernel, dim3(min(L.n_emit_tiles, kEmitGrid)), dim3(kEmT), 0, st, cvA, tiles,
                   (const uint32_t*)icount, fuse_icount, ioff, L.cap, hdr);
  launch_dependent(emit_fill_kernel, dim3(min(L.n_isort_tiles, kEmitGrid)), dim3(kFlT), 0, st, cvA, ioff, (const uint2*)(ws + L.rect), views, L.V, L.cap,
                                                     ikA, ivA, L.tile_passes > 0 ? hi : nullptr, hdr);
  uint32_t* gh_tile = ghist + 4 * 256;
  const size_t hi_stride = (size_t)L.n_isort_tiles * 256;
  for (int p = 0; p < L.tile_passes; ++p) {
    const bool even = (p & 1) == 0;
    uint32_t* hp = hi + p * hi_stride;
    const bool last = p == L.tile_passes - 1;
    launch_dependent(col_scan_kernel, dim3(256), dim3(kScT), 0, st, hp, hp, L.n_isort_tiles, 256, gh_tile + 256 * p,
                     (const uint64_t*)&hdr->n_inst, L.cap, (uint32_t)kIsTile);
    launch_dependent(downsweep_kernel<kIsTile>, dim3(min(L.n_isort_tiles, kPassGrid)), dim3(kOsT), 0, st, even ? ikA : ikB, even ? ivA : ivB, even ? ikB : ikA,
                                                       even ? ivB : ivA, &hdr->n_inst, L.cap, 8 * p,
                                                       gh_tile + 256 * p, hp, last ? nullptr : hp + hi_stride,
                                                       nullptr, nullptr);
  }
  const uint32_t* skeys = (const uint32_t*)(ws + ((L.tile_passes & 1) ? L.ikB : L.ikA));
  launch_dependent(ranges_kernel, dim3(592), dim3(256), 0, st, skeys, &hdr->n_inst, L.cap, L.NT, (uint32_t*)(ws + L.tstart));
  return launch_tile_order(L, ws, hdr, st);
}

void sort_tile_sizes(uint32_t R, uint32_t cap, uint32_t* n_cmp, uint32_t* n_emit, uint32_t* n_dsort,
                     uint32_t* n_isort) {
  *n_cmp = (R + kCmpTile - 1) / kCmpTile;
  *n_emit = (R + kEmTile - 1) / kEmTile;
  *n_dsort = (R + kDsTile - 1) / kDsTile;
  *n_isort = (cap + kIsTile - 1) / kIsTile;
}

}  // namespace ubs
