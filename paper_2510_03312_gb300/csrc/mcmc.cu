// mcmc.cu -- MCMC relocation of dead primitives (Sec. 4.5, primitive
// management after Deformable Beta Splatting): ubs_mcmc_relocate.
//
// A primitive is dead when its opacity is at most a threshold.  Each dead
// slot j is moved onto a live source drawn with probability proportional to
// opacity, exactly: the weight of a live primitive is the integer
// floor(o 2^24) (the float32 product is exact), the cumulative weights are
// 64-bit integers, and the source is the first primitive whose inclusive
// cumulative weight exceeds rand[j] mod (total weight).  A source drawn n
// times and its n copies take o' = 1 - (1 - o)^(1/(n+1)), which keeps their
// composited density; every other parameter of a copy is the source's, and
// the Adam moments of all touched primitives are reset.
//
// Kernels (one launch each, in order):
//   mcmc_weights_kernel  weights, per-1024-block inclusive scans, block sums;
//                        clears the per-primitive counts and sources
//   mcmc_scan_kernel     exclusive scan of the block sums (one block)
//   mcmc_sample_kernel   each dead slot's source (two binary searches:
//                        over the block offsets, then within the block);
//                        per-source copy counts by integer atomics (exact)
//   mcmc_copy_kernel     copies of the sources into the dead slots
//   mcmc_sources_kernel  the sources' new opacity and reset moments
// The copy kernel reads each source before the sources kernel updates it.
#include <math.h>

#include "ubs.h"
#include "kernels.cuh"

namespace ubs {
namespace {

constexpr int kMcBlock = 1024;  // elements per scan block
constexpr int kMcThreads = 256;
constexpr int kMcMaxPlanes = 64;

inline size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

struct McLayout {
  size_t cdf, boff, counts, src, header, total;
  uint32_t nb;
};

McLayout mc_layout(int64_t P) {
  McLayout L;
  L.nb = (uint32_t)((P + kMcBlock - 1) / kMcBlock);
  size_t o = 0;
  L.header = o;
  o += 256;  // total weight (u64), relocated count (i64)
  L.cdf = o;
  o += align256((size_t)P * 8);
  L.boff = o;
  o += align256((size_t)L.nb * 8);
  L.counts = o;
  o += align256((size_t)P * 4);
  L.src = o;
  o += align256((size_t)P * 4);
  L.total = o;
  return L;
}

struct McHeader {
  unsigned long long total;
  long long relocated;
};

__device__ __forceinline__ bool is_dead(float o, float thr) { return o <= thr; }
__device__ __forceinline__ uint32_t weight_of(float o, float thr) {
  return is_dead(o, thr) ? 0u : (uint32_t)(o * 16777216.0f);  // floor for o >= 0
}

__global__ void __launch_bounds__(kMcThreads)
    mcmc_weights_kernel(const float* __restrict__ op, int64_t P, float thr, unsigned long long* __restrict__ cdf,
                        unsigned long long* __restrict__ bsum, uint32_t* __restrict__ counts,
                        int32_t* __restrict__ src, McHeader* hdr) {
  wait_prior_grid();
  __shared__ unsigned long long warp_tot[kMcThreads / 32];
  constexpr int E = kMcBlock / kMcThreads;  // 4 consecutive elements per thread
  const int64_t base = (int64_t)blockIdx.x * kMcBlock + (int64_t)threadIdx.x * E;
  unsigned long long v[E], run = 0;
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const int64_t i = base + e;
    uint32_t w = 0;
    if (i < P) {
      w = weight_of(op[i], thr);
      counts[i] = 0;
      src[i] = -1;
    }
    run += w;
    v[e] = run;  // thread-local inclusive
  }
  // inclusive scan of the thread totals over the block
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned long long x = run;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const unsigned long long y = __shfl_up_sync(0xffffffffu, x, d);
    if (lane >= d) x += y;
  }
  if (lane == 31) warp_tot[warp] = x;
  __syncthreads();
  unsigned long long woff = 0;
  for (int w = 0; w < warp; ++w) woff += warp_tot[w];
  const unsigned long long excl = woff + x - run;
#pragma unroll
  for (int e = 0; e < E; ++e)
    if (base + e < P) cdf[base + e] = excl + v[e];
  if (threadIdx.x == kMcThreads - 1) bsum[blockIdx.x] = woff + x;
  if (blockIdx.x == 0 && threadIdx.x == 0) hdr->relocated = 0;
}

// exclusive scan of the block sums in place (one block, sequential chunks)
__global__ void __launch_bounds__(1024) mcmc_scan_kernel(unsigned long long* __restrict__ bsum, uint32_t nb,
                                                         McHeader* hdr) {
  wait_prior_grid();
  __shared__ unsigned long long wt[32];
  __shared__ unsigned long long carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (uint32_t b0 = 0; b0 < nb; b0 += 1024) {
    const uint32_t i = b0 + threadIdx.x;
    const unsigned long long a = i < nb ? bsum[i] : 0ull;
    unsigned long long x = a;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const unsigned long long y = __shfl_up_sync(0xffffffffu, x, d);
      if (lane >= d) x += y;
    }
    if (lane == 31) wt[warp] = x;
    __syncthreads();
    unsigned long long woff = 0;
    for (int w = 0; w < warp; ++w) woff += wt[w];
    const unsigned long long c = carry;
    if (i < nb) bsum[i] = c + woff + x - a;
    __syncthreads();
    if (threadIdx.x == 1023) carry = c + woff + x;
    __syncthreads();
  }
  if (threadIdx.x == 0) hdr->total = carry;
}

__global__ void __launch_bounds__(kMcThreads)
    mcmc_sample_kernel(const float* __restrict__ op, int64_t P, float thr, const unsigned long long* __restrict__ rnd,
                       const unsigned long long* __restrict__ cdf, const unsigned long long* __restrict__ boff,
                       uint32_t nb, uint32_t* __restrict__ counts, int32_t* __restrict__ src, McHeader* hdr) {
  wait_prior_grid();
  const int64_t j = (int64_t)blockIdx.x * kMcThreads + threadIdx.x;
  const unsigned long long total = hdr->total;
  if (j >= P || total == 0 || !is_dead(op[j], thr)) return;
  const unsigned long long r = rnd[j] % total;
  // the last block whose offset is <= r, then the first element of it whose
  // inclusive cumulative weight exceeds r
  uint32_t lo = 0, hi = nb - 1;
  while (lo < hi) {
    const uint32_t mid = (lo + hi + 1) >> 1;
    if (boff[mid] <= r) lo = mid; else hi = mid - 1;
  }
  const unsigned long long rr = r - boff[lo];
  int64_t a = (int64_t)lo * kMcBlock, b = a + kMcBlock - 1;
  if (b > P - 1) b = P - 1;
  while (a < b) {
    const int64_t mid = (a + b) >> 1;
    if (cdf[mid] > rr) b = mid; else a = mid + 1;
  }
  src[j] = (int32_t)a;
  atomicAdd(&counts[a], 1u);
  atomicAdd((unsigned long long*)&hdr->relocated, 1ull);
}

struct McPlanes {
  int32_t K, op_row;
};

__device__ __forceinline__ float cloned_opacity(float o, uint32_t n) {
  return 1.0f - powf(1.0f - o, 1.0f / (float)(n + 1));
}

__global__ void __launch_bounds__(kMcThreads)
    mcmc_copy_kernel(McPlanes pl, int64_t P, float* __restrict__ act, float* __restrict__ raw,
                     float* __restrict__ m, float* __restrict__ v, const uint32_t* __restrict__ counts,
                     const int32_t* __restrict__ src) {
  wait_prior_grid();
  const int64_t j = (int64_t)blockIdx.x * kMcThreads + threadIdx.x;
  if (j >= P) return;
  const int32_t s = src[j];
  if (s < 0) return;
  for (int k = 0; k < pl.K; ++k) {
    const size_t d = (size_t)k * P + j, o = (size_t)k * P + s;
    if (k == pl.op_row) {
      const float op = cloned_opacity(act[o], counts[s]);
      act[d] = op;
      raw[d] = logf(op / (1.0f - op));
    } else {
      act[d] = act[o];
      raw[d] = raw[o];
    }
    m[d] = 0.0f;
    v[d] = 0.0f;
  }
}

__global__ void __launch_bounds__(kMcThreads)
    mcmc_sources_kernel(McPlanes pl, int64_t P, float* __restrict__ act, float* __restrict__ raw,
                        float* __restrict__ m, float* __restrict__ v, const uint32_t* __restrict__ counts) {
  wait_prior_grid();
  const int64_t s = (int64_t)blockIdx.x * kMcThreads + threadIdx.x;
  if (s >= P) return;
  const uint32_t n = counts[s];
  if (n == 0) return;
  const size_t o = (size_t)pl.op_row * P + s;
  const float op = cloned_opacity(act[o], n);
  act[o] = op;
  raw[o] = logf(op / (1.0f - op));
  for (int k = 0; k < pl.K; ++k) {
    m[(size_t)k * P + s] = 0.0f;
    v[(size_t)k * P + s] = 0.0f;
  }
}

__global__ void mcmc_export_kernel(const int32_t* __restrict__ src, int64_t P, int32_t* __restrict__ out,
                                   const McHeader* hdr, long long* __restrict__ n_out) {
  wait_prior_grid();
  const int64_t j = (int64_t)blockIdx.x * kMcThreads + threadIdx.x;
  if (out && j < P) out[j] = src[j];
  if (n_out && j == 0) *n_out = hdr->relocated;
}

}  // namespace
}  // namespace ubs

using namespace ubs;

extern "C" size_t ubs_mcmc_workspace_size(int64_t P) {
  if (P < 1 || P > (int64_t)0x7fffffff) return 0;
  return mc_layout(P).total;
}

extern "C" ubs_status ubs_mcmc_relocate(int32_t K, int64_t P, int32_t opacity_row, float dead_threshold,
                                        float* act, float* raw, float* m, float* v, const uint64_t* rand,
                                        int32_t* sources, int64_t* n_relocated, void* workspace,
                                        size_t workspace_bytes, cudaStream_t stream) {
  ubs::TraceRange trace_("ubs_mcmc_relocate");
  if (K < 1 || K > kMcMaxPlanes || P < 1 || P > (int64_t)0x7fffffff) return UBS_ERR_INVALID_ARG;
  if (opacity_row < 0 || opacity_row >= K || !(dead_threshold >= 0.0f && dead_threshold < 1.0f))
    return UBS_ERR_INVALID_ARG;
  if (!act || !raw || !m || !v || !rand || !workspace) return UBS_ERR_INVALID_ARG;
  if (((uintptr_t)act | (uintptr_t)raw | (uintptr_t)m | (uintptr_t)v | (uintptr_t)sources) & 3u)
    return UBS_ERR_ALIGNMENT;
  if ((((uintptr_t)rand | (uintptr_t)n_relocated) & 7u) || ((uintptr_t)workspace & 255u)) return UBS_ERR_ALIGNMENT;
  const McLayout L = mc_layout(P);
  if (workspace_bytes < L.total) return UBS_ERR_WORKSPACE;
  char* ws = (char*)workspace;
  McHeader* hdr = (McHeader*)(ws + L.header);
  unsigned long long* cdf = (unsigned long long*)(ws + L.cdf);
  unsigned long long* boff = (unsigned long long*)(ws + L.boff);
  uint32_t* counts = (uint32_t*)(ws + L.counts);
  int32_t* src = (int32_t*)(ws + L.src);
  const float* op = act + (size_t)opacity_row * P;
  const unsigned grid = (unsigned)((P + kMcThreads - 1) / kMcThreads);
  McPlanes pl{K, opacity_row};
  cudaError_t e = launch_dependent(mcmc_weights_kernel, dim3(L.nb), dim3(kMcThreads), 0, stream, op, P,
                                   dead_threshold, cdf, boff, counts, src, hdr);
  if (e == cudaSuccess) e = launch_dependent(mcmc_scan_kernel, dim3(1), dim3(1024), 0, stream, boff, L.nb, hdr);
  if (e == cudaSuccess)
    e = launch_dependent(mcmc_sample_kernel, dim3(grid), dim3(kMcThreads), 0, stream, op, P, dead_threshold,
                         (const unsigned long long*)rand, (const unsigned long long*)cdf,
                         (const unsigned long long*)boff, L.nb, counts, src, hdr);
  if (e == cudaSuccess)
    e = launch_dependent(mcmc_copy_kernel, dim3(grid), dim3(kMcThreads), 0, stream, pl, P, act, raw, m, v,
                         (const uint32_t*)counts, (const int32_t*)src);
  if (e == cudaSuccess)
    e = launch_dependent(mcmc_sources_kernel, dim3(grid), dim3(kMcThreads), 0, stream, pl, P, act, raw, m, v,
                         (const uint32_t*)counts);
  if (e == cudaSuccess && (sources || n_relocated))
    e = launch_dependent(mcmc_export_kernel, dim3(grid), dim3(kMcThreads), 0, stream, (const int32_t*)src, P,
                         sources, (const McHeader*)hdr, (long long*)n_relocated);
  return e == cudaSuccess ? UBS_OK : UBS_ERR_CUDA;
}
