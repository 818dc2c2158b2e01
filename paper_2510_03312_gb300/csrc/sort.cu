// sort.cu -- B1-B3: tile binning, front-to-back order and tile ranges.
//
// The instance order is (global tile, float32 depth, record index).  It is
// produced as two stable LSD radix sorts instead of one sort of 64-bit
// (tile, depth) keys over all instances:
//   1. compact the visible records (order-preserving, so ties stay in record
//      order) and sort them by depth (4 passes of 8 bits over records);
//   2. emit the instances of the depth-sorted records in that order (every
//      record's tiles row-major in its rectangle), counting instances per tile;
//   3. sort the instances by tile id (ceil(log2 tiles / 8) passes).
// Because both sorts are stable, each tile's list ends up in (depth, record)
// order: the same order as a single sort by the 64-bit key, at roughly half
// the bytes (depth passes touch records, not instances).
//
// Every pass is a single-pass kernel with decoupled look-back: the onesweep
// radix sort (Adinets & Merrill 2022) and single-pass prefix scans (Merrill &
// Garland 2016), written here from those descriptions.  Each block takes its
// tile index from an atomic counter, so a block only ever waits on tiles
// already taken by running blocks.  Every wait is bounded (kSpinLimit polls);
// a wait that gives up records UBS_ERR_TIMEOUT in the header and continues
// with a zero contribution, so the kernel always finishes.
#include "kernels.cuh"

namespace ubs {

namespace {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ uint64_t ld_acq64(const uint64_t* p) {
  uint64_t v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_rel64(uint64_t* p, uint64_t v) {
  asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ uint32_t ld_acq32(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_rel32(uint32_t* p, uint32_t v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ void set_status(Header* h, uint32_t s) { atomicCAS(&h->status, 0u, s); }

#ifndef UBS_PEERS_BALLOT
#define UBS_PEERS_BALLOT 1
#endif

// Lanes of the warp holding the same 9-bit value d (digits < 256, 0x100 for
// "no item"): one ballot per bit, each lane keeping the lanes that agree.
__device__ __forceinline__ uint32_t peer_mask(uint32_t d) {
#if UBS_PEERS_BALLOT
  uint32_t peers = 0xffffffffu;
#pragma unroll
  for (int b = 0; b < 9; ++b) {
    const bool bit = (d >> b) & 1u;
    const uint32_t bal = __ballot_sync(0xffffffffu, bit);
    peers &= bit ? bal : ~bal;
  }
  return peers;
#else
  return __match_any_sync(0xffffffffu, d);
#endif
}

__device__ __forceinline__ uint32_t lane_id() { return threadIdx.x & 31; }

__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t v) {
  const uint32_t lane = lane_id();
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t t = __shfl_up_sync(kFull, v, o);
    if (lane >= (uint32_t)o) v += t;
  }
  return v;
}

__device__ __forceinline__ uint64_t warp_sum64(uint64_t v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
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

// Decoupled look-back over 64-bit tile status words (flag in the top two
// bits).  Called uniformly by warp 0; returns the tile's exclusive prefix.
__device__ uint64_t lookback64(uint64_t* stat, uint32_t tile, uint64_t agg, Header* hdr) {
  const uint32_t lane = lane_id();
  if (tile == 0) {
    if (lane == 0) st_rel64(stat, kFlagInc | agg);
    return 0;
  }
  if (lane == 0) st_rel64(stat + tile, kFlagAgg | agg);
  uint64_t excl = 0;
  int64_t pred = (int64_t)tile - 1;
  while (true) {
    const int64_t idx = pred - (int64_t)lane;
    uint64_t s = kFlagInc;  // before the first tile: inclusive prefix 0
    if (idx >= 0) {
      s = ld_acq64(stat + idx);
      uint32_t spins = 0;
      while ((s >> 62) == 0) {
        if (++spins >= kSpinLimit) {
          set_status(hdr, kDevTimeout);
          s = kFlagAgg;
          break;
        }
        s = ld_acq64(stat + idx);
      }
    }
    const uint32_t inc = __ballot_sync(kFull, (s >> 62) == 2);
    uint64_t v = s & kValMask;
    if (inc) {
      const uint32_t first = __ffs(inc) - 1;
      if (lane > first) v = 0;
      excl += warp_sum64(v);
      break;
    }
    excl += warp_sum64(v);
    pred -= 32;
  }
  if (lane == 0) st_rel64(stat + tile, kFlagInc | (excl + agg));
  return excl;
}

// ---------------------------------------------------------------- compaction

constexpr int kCmpT = 256, kCmpI = 8, kCmpTile = kCmpT * kCmpI;

// Keeps the records with tiles_touched > 0, in record order, as (depth key,
// record) pairs, and accumulates the 4 digit histograms of their depth keys.
__global__ void __launch_bounds__(kCmpT) compact_kernel(const uint32_t* __restrict__ tiles,
                                                        const uint32_t* __restrict__ key, uint32_t R,
                                                        uint32_t* __restrict__ okey, uint32_t* __restrict__ oval,
                                                        uint64_t* stat, uint32_t* ghist, Header* hdr,
                                                        uint32_t n_tiles) {
  __shared__ uint32_t s_tile, s_w[kCmpT / 32 + 1];
  __shared__ uint64_t s_excl;
  __shared__ uint32_t s_h[4][256];
  for (int i = threadIdx.x; i < 4 * 256; i += kCmpT) (&s_h[0][0])[i] = 0;
  if (threadIdx.x == 0) s_tile = atomicAdd(&hdr->ctr[0], 1u);
  __syncthreads();
  const uint32_t tile = s_tile;
  const uint32_t base = tile * kCmpTile + threadIdx.x * kCmpI;
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
  // digit histograms of the kept keys (warp-aggregated)
  const uint32_t lane = lane_id();
#pragma unroll
  for (int i = 0; i < kCmpI; ++i) {
#pragma unroll
    for (int p = 0; p < 4; ++p) {
      const uint32_t d = f[i] ? (k[i] >> (8 * p)) & 255u : 0x100u;
      const uint32_t peers = __match_any_sync(kFull, d);
      if (d < 256 && lane == (uint32_t)(__ffs(peers) - 1)) atomicAdd(&s_h[p][d], (uint32_t)__popc(peers));
    }
  }
  uint32_t total;
  const uint32_t ex = block_excl_scan<kCmpT>(cnt, total, s_w);
  if ((threadIdx.x >> 5) == 0) {
    const uint64_t e = lookback64(stat, tile, total, hdr);
    if (lane == 0) s_excl = e;
  }
  __syncthreads();
  uint64_t pos = s_excl + ex;
#pragma unroll
  for (int i = 0; i < kCmpI; ++i)
    if (f[i]) {
      if (pos < R) {  // always true unless a bounded wait gave up (status is then set)
        okey[pos] = k[i];
        oval[pos] = base + i;
      }
      ++pos;
    }
  for (int i = threadIdx.x; i < 4 * 256; i += kCmpT) {
    const uint32_t c = (&s_h[0][0])[i];
    if (c) atomicAdd(ghist + i, c);
  }
  if (tile == n_tiles - 1 && threadIdx.x == 0) hdr->n_visible = s_excl + total;
}

// ---------------------------------------------------------------- onesweep

constexpr int kOsT = 256, kOsI = 16, kOsW = kOsT / 32, kOsTile = kOsT * kOsI;
constexpr int kLbW = 1;  // look-back window (predecessor statuses loaded at once)

// One stable pass of the LSD radix sort over 8 bits at `shift`.
// ghist: global counts of this pass's digits over all n items.
__global__ void __launch_bounds__(kOsT) onesweep_kernel(const uint32_t* __restrict__ kin,
                                                        const uint32_t* __restrict__ vin, uint32_t* __restrict__ kout,
                                                        uint32_t* __restrict__ vout, const uint64_t* n_ptr,
                                                        uint32_t cap, int shift, const uint32_t* __restrict__ ghist,
                                                        uint32_t* stat, Header* hdr, int ctr) {
  __shared__ uint32_t s_keys[kOsTile];
  __shared__ uint32_t s_vals[kOsTile];
  __shared__ uint32_t s_hist[kOsW][256];
  __shared__ uint32_t s_boff[256];
  __shared__ uint32_t s_goff[256];
  __shared__ uint32_t s_tile, s_w[kOsT / 32 + 1];
  const uint64_t n64 = *n_ptr;
  const uint32_t n = (uint32_t)(n64 < cap ? n64 : cap);
  if (threadIdx.x == 0) s_tile = atomicAdd(&hdr->ctr[ctr], 1u);
  for (int i = threadIdx.x; i < kOsW * 256; i += kOsT) (&s_hist[0][0])[i] = 0;
  __syncthreads();
  const uint32_t tile = s_tile;
  const uint32_t tile_base = tile * kOsTile;
  if (tile_base >= n) return;
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
    const uint32_t d = ok ? (k[i] >> shift) & 255u : 0x100u;
    const uint32_t peers = peer_mask(d);
    uint32_t cnt = 0;
    if (d < 256) cnt = s_hist[warp][d];
    __syncwarp();
    rank[i] = cnt + __popc(peers & lt_mask);
    if (d < 256 && lane == (uint32_t)(__ffs(peers) - 1)) s_hist[warp][d] = cnt + __popc(peers);
    __syncwarp();
    if (!ok) rank[i] = 0xffffffffu;
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
  // decoupled look-back for digit d: the statuses of a window of kLbW
  // predecessors are loaded together (independent loads in flight), then
  // summed nearest-first up to the first inclusive prefix
  uint32_t excl = 0;
  uint32_t* st = stat + (size_t)tile * 256 + d;
  if (tile == 0) {
    st_rel32(st, kFlagInc32 | acc);
  } else {
    st_rel32(st, kFlagAgg32 | acc);
    int64_t t = (int64_t)tile - 1;
    bool found = false;
    while (!found) {
      uint32_t s[kLbW];
#pragma unroll
      for (int k = 0; k < kLbW; ++k) s[k] = (t - k >= 0) ? ld_acq32(stat + (size_t)(t - k) * 256 + d) : kFlagInc32;
#pragma unroll
      for (int k = 0; k < kLbW; ++k) {
        if (!found) {
          uint32_t spins = 0;
          while ((s[k] >> 30) == 0) {
            if (++spins >= kSpinLimit) {
              set_status(hdr, kDevTimeout);
              s[k] = kFlagAgg32;
              break;
            }
            s[k] = ld_acq32(stat + (size_t)(t - k) * 256 + d);
          }
          excl += s[k] & kValMask32;
          found = (s[k] >> 30) == 2;
        }
      }
      t -= kLbW;
    }
    st_rel32(st, kFlagInc32 | (excl + acc));
  }
  uint32_t gtot;
  const uint32_t gbase = block_excl_scan<kOsT>(ghist[d], gtot, s_w);
  uint32_t btot;
  const uint32_t boff = block_excl_scan<kOsT>(acc, btot, s_w);
  s_boff[d] = boff;
  s_goff[d] = gbase + excl - boff;
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
  const uint32_t cnt_tile = (n - tile_base) < (uint32_t)kOsTile ? (n - tile_base) : (uint32_t)kOsTile;
  for (uint32_t j = threadIdx.x; j < cnt_tile; j += kOsT) {
    const uint32_t key = s_keys[j];
    const uint32_t g = s_goff[(key >> shift) & 255u] + j;
    if (g < n) {  // always true unless a bounded wait gave up (status is then set)
      kout[g] = key;
      vout[g] = s_vals[j];
    }
  }
}

// ---------------------------------------------------------------- emission

constexpr int kEmT = 256, kEmI = 4, kEmTile = kEmT * kEmI;

// For the depth-sorted visible records, writes each record's tiles (row-major
// within its rectangle) as (global tile, record) instances at the positions of
// an exclusive scan of tiles_touched, and counts instances per tile.
__global__ void __launch_bounds__(kEmT) emit_kernel(const uint32_t* __restrict__ srec,
                                                    const uint32_t* __restrict__ tiles,
                                                    const uint2* __restrict__ rect,
                                                    const ViewDev* __restrict__ views, int V, uint32_t cap,
                                                    uint32_t* __restrict__ ikey, uint32_t* __restrict__ ival,
                                                    uint32_t* tcount, uint64_t* stat, Header* hdr) {
  __shared__ uint32_t s_rec[kEmTile];
  __shared__ uint32_t s_off[kEmTile + 1];
  __shared__ uint2 s_rect[kEmTile];
  __shared__ uint32_t s_vtile[kEmTile];
  __shared__ uint32_t s_vtx[kEmTile];
  __shared__ uint32_t s_recoff[kMaxViews], s_tileoff[kMaxViews], s_tilesx[kMaxViews];
  __shared__ uint32_t s_tile, s_w[kEmT / 32 + 1];
  __shared__ uint64_t s_excl;
  const uint64_t n = hdr->n_visible;
  for (int i = threadIdx.x; i < V; i += kEmT) {
    s_recoff[i] = views[i].rec_off;
    s_tileoff[i] = views[i].tile_off;
    s_tilesx[i] = (uint32_t)views[i].tiles_x;
  }
  if (threadIdx.x == 0) s_tile = atomicAdd(&hdr->ctr[5], 1u);
  __syncthreads();
  const uint32_t tile = s_tile;
  const uint64_t n_tiles = (n + kEmTile - 1) / kEmTile;
  if ((uint64_t)tile >= n_tiles) return;
  const uint32_t base = tile * kEmTile + threadIdx.x * kEmI;
  uint32_t c[kEmI];
  uint32_t tsum = 0;
#pragma unroll
  for (int i = 0; i < kEmI; ++i) {
    const uint32_t idx = base + i;
    const uint32_t slot = threadIdx.x * kEmI + i;
    uint32_t r = 0;
    c[i] = 0;
    if (idx < n) {
      r = srec[idx];
      c[i] = tiles[r];
      s_rect[slot] = rect[r];
      int lo = 0, hi = V - 1;  // view of record r: last view with rec_off <= r
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (s_recoff[mid] <= r) lo = mid; else hi = mid - 1;
      }
      s_vtile[slot] = s_tileoff[lo];
      s_vtx[slot] = s_tilesx[lo];
    }
    s_rec[slot] = r;
    tsum += c[i];
  }
  uint32_t total;
  uint32_t ex = block_excl_scan<kEmT>(tsum, total, s_w);
#pragma unroll
  for (int i = 0; i < kEmI; ++i) {
    s_off[threadIdx.x * kEmI + i] = ex;
    ex += c[i];
  }
  if (threadIdx.x == 0) s_off[kEmTile] = total;
  if ((threadIdx.x >> 5) == 0) {
    const uint64_t e = lookback64(stat, tile, total, hdr);
    if (lane_id() == 0) s_excl = e;
  }
  __syncthreads();
  const uint64_t excl = s_excl;
  bool overflow = false;
  for (uint32_t j = threadIdx.x; j < total; j += kEmT) {
    int lo = 0, hi = kEmTile - 1;  // last item with s_off <= j
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (s_off[mid] <= j) lo = mid; else hi = mid - 1;
    }
    const uint32_t local = j - s_off[lo];
    const uint2 rc = s_rect[lo];
    const uint32_t x0 = rc.x & 0xFFFFu, y0 = rc.x >> 16, x1 = rc.y & 0xFFFFu;
    const uint32_t w = x1 - x0;
    const uint32_t tx = x0 + local % w, ty = y0 + local / w;
    const uint32_t gt = s_vtile[lo] + ty * s_vtx[lo] + tx;
    const uint64_t pos = excl + j;
    if (pos < cap) {
      ikey[pos] = gt;
      ival[pos] = s_rec[lo];
      atomicAdd(tcount + gt, 1u);
    } else {
      overflow = true;
    }
  }
  if (overflow) set_status(hdr, kDevCapacity);
  if ((uint64_t)tile == n_tiles - 1 && threadIdx.x == 0) hdr->n_inst = excl + total;
}

// ---------------------------------------------------------------- ranges

constexpr int kRgT = 256, kRgI = 8, kRgTile = kRgT * kRgI;

// Exclusive scan of per-tile instance counts into tile starts (tstart[NT] =
// total), plus the digit histograms of the instances' tile keys.
__global__ void __launch_bounds__(kRgT) range_kernel(const uint32_t* __restrict__ tcount, uint32_t NT,
                                                     uint32_t* __restrict__ tstart, uint64_t* stat, Header* hdr,
                                                     int passes, uint32_t* ghist, uint32_t n_tiles) {
  __shared__ uint32_t s_tile, s_w[kRgT / 32 + 1];
  __shared__ uint64_t s_excl;
  __shared__ uint32_t s_h[3][256];
  for (int i = threadIdx.x; i < 3 * 256; i += kRgT) (&s_h[0][0])[i] = 0;
  if (threadIdx.x == 0) s_tile = atomicAdd(&hdr->ctr[6], 1u);
  __syncthreads();
  const uint32_t tile = s_tile;
  const uint32_t base = tile * kRgTile + threadIdx.x * kRgI;
  uint32_t c[kRgI], sum = 0;
#pragma unroll
  for (int i = 0; i < kRgI; ++i) {
    c[i] = (base + i < NT) ? tcount[base + i] : 0u;
    sum += c[i];
  }
  // pass 0 digits differ per item (distinct addresses across the warp);
  // higher digits are shared by the thread's 8 consecutive tiles
  if (passes > 0) {
#pragma unroll
    for (int i = 0; i < kRgI; ++i)
      if (c[i]) atomicAdd(&s_h[0][(base + i) & 255u], c[i]);
  }
  const uint32_t lane = lane_id();
  for (int p = 1; p < passes; ++p) {
    const uint32_t d = sum ? (base >> (8 * p)) & 255u : 0x100u;
    const uint32_t peers = __match_any_sync(kFull, d);
    uint32_t s = sum;
    // sum over peers
    uint32_t tot = 0;
    for (int l = 0; l < 32; ++l) {
      const uint32_t sv = __shfl_sync(kFull, s, l);
      if (peers & (1u << l)) tot += sv;
    }
    if (d < 256 && lane == (uint32_t)(__ffs(peers) - 1)) atomicAdd(&s_h[p][d], tot);
  }
  uint32_t total;
  uint32_t ex = block_excl_scan<kRgT>(sum, total, s_w);
  if ((threadIdx.x >> 5) == 0) {
    const uint64_t e = lookback64(stat, tile, total, hdr);
    if (lane == 0) s_excl = e;
  }
  __syncthreads();
  uint32_t pos = (uint32_t)s_excl + ex;
#pragma unroll
  for (int i = 0; i < kRgI; ++i) {
    if (base + i < NT) tstart[base + i] = pos;
    pos += c[i];
  }
  if (tile == n_tiles - 1 && threadIdx.x == 0) tstart[NT] = (uint32_t)(s_excl + total);
  for (int i = threadIdx.x; i < passes * 256; i += kRgT) {
    const uint32_t v = (&s_h[0][0])[i];
    if (v) atomicAdd(ghist + i, v);
  }
}

}  // namespace

const uint32_t* sorted_instances(const Layout& L, const char* ws) {
  return (const uint32_t*)(ws + ((L.tile_passes & 1) ? L.ivB : L.ivA));
}

cudaError_t launch_bin_sort(const Layout& L, const CfgDev& cfg, char* ws, cudaStream_t st) {
  (void)cfg;
  Header* hdr = (Header*)(ws + L.header);
  cudaError_t e;
  // reset counters, look-back status words, histograms and tile counts
  e = cudaMemsetAsync(hdr->ctr, 0, sizeof(hdr->ctr), st);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(ws + L.scan_stat, 0, L.Tfin - L.scan_stat, st);
  if (e != cudaSuccess) return e;
  if (L.R == 0) return cudaMemsetAsync(ws + L.tstart, 0, (size_t)(L.NT + 1) * 4, st);
  uint64_t* scan_stat = (uint64_t*)(ws + L.scan_stat);
  uint64_t* st_cmp = scan_stat;
  uint64_t* st_emit = st_cmp + L.n_cmp_tiles;
  uint64_t* st_rng = st_emit + L.n_emit_tiles;
  uint32_t* sort_stat = (uint32_t*)(ws + L.sort_stat);
  uint32_t* ghist = (uint32_t*)(ws + L.ghist);  // [4 depth + 3 tile][256]
  uint32_t* tcount = (uint32_t*)(ws + L.tcount);
  uint32_t* ckA = (uint32_t*)(ws + L.ckA);
  uint32_t* cvA = (uint32_t*)(ws + L.cvA);
  uint32_t* ckB = (uint32_t*)(ws + L.ckB);
  uint32_t* cvB = (uint32_t*)(ws + L.cvB);
  compact_kernel<<<L.n_cmp_tiles, kCmpT, 0, st>>>((const uint32_t*)(ws + L.tiles), (const uint32_t*)(ws + L.key),
                                                  L.R, ckA, cvA, st_cmp, ghist, hdr, L.n_cmp_tiles);
  // depth sort: 4 passes A->B->A->B->A
  for (int p = 0; p < 4; ++p) {
    const bool even = (p & 1) == 0;
    onesweep_kernel<<<L.n_dsort_tiles, kOsT, 0, st>>>(even ? ckA : ckB, even ? cvA : cvB, even ? ckB : ckA,
                                                      even ? cvB : cvA, &hdr->n_visible, L.R, 8 * p,
                                                      ghist + 256 * p,
                                                      sort_stat + (size_t)p * L.n_dsort_tiles * 256, hdr, 1 + p);
  }
  uint32_t* ikA = (uint32_t*)(ws + L.ikA);
  uint32_t* ivA = (uint32_t*)(ws + L.ivA);
  uint32_t* ikB = (uint32_t*)(ws + L.ikB);
  uint32_t* ivB = (uint32_t*)(ws + L.ivB);
  const ViewDev* views = (const ViewDev*)(ws + L.views);
  emit_kernel<<<L.n_emit_tiles, kEmT, 0, st>>>(cvA, (const uint32_t*)(ws + L.tiles), (const uint2*)(ws + L.rect),
                                               views, L.V, L.cap, ikA, ivA, tcount, st_emit, hdr);
  uint32_t* gh_tile = ghist + 4 * 256;
  range_kernel<<<L.n_rng_tiles, kRgT, 0, st>>>(tcount, L.NT, (uint32_t*)(ws + L.tstart), st_rng, hdr, L.tile_passes,
                                               gh_tile, L.n_rng_tiles);
  uint32_t* istat = sort_stat + (size_t)4 * L.n_dsort_tiles * 256;
  for (int p = 0; p < L.tile_passes; ++p) {
    const bool even = (p & 1) == 0;
    onesweep_kernel<<<L.n_isort_tiles, kOsT, 0, st>>>(even ? ikA : ikB, even ? ivA : ivB, even ? ikB : ikA,
                                                      even ? ivB : ivA, &hdr->n_inst, L.cap, 8 * p, gh_tile + 256 * p,
                                                      istat + (size_t)p * L.n_isort_tiles * 256, hdr, 7 + p);
  }
  return cudaGetLastError();
}

size_t sort_tile_sizes(uint32_t R, uint32_t NT, uint32_t cap, uint32_t* n_cmp, uint32_t* n_emit, uint32_t* n_rng,
                       uint32_t* n_dsort, uint32_t* n_isort) {
  *n_cmp = (R + kCmpTile - 1) / kCmpTile;
  *n_emit = (R + kEmTile - 1) / kEmTile;
  *n_rng = (NT + kRgTile - 1) / kRgTile;
  *n_dsort = (R + kOsTile - 1) / kOsTile;
  *n_isort = (cap + kOsTile - 1) / kOsTile;
  return 0;
}

}  // namespace ubs
