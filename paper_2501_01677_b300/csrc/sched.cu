// Longest-processing-time-first order of the active tiles for the persistent
// render launches: uneven sub-regions and views (Sec. 4.1 grouping, parallel
// groups in Sec. 5.1) give tiles whose work (rendered pixels x Gaussians in the
// tile's list) differs by orders of magnitude; handing the costliest tiles out
// first keeps the tail of a persistent launch short.  Tiles are bucketed by
// floor(log2(cost)) and emitted in descending bucket order (counting sort; the
// order inside a bucket is unspecified).
#include "common.cuh"

namespace pgsag {

constexpr int kBuckets = 33;  // floor(log2(cost)) for cost in [1, 2^32), bucket 0 for cost 0

__device__ __forceinline__ int cost_bucket(const uint2* __restrict__ ranges, const uint4* __restrict__ act_tiles,
                                           uint32_t t) {
  const uint2 r = __ldg(ranges + t);
  const uint32_t npix = __ldg(&act_tiles[t].w);
  const unsigned long long c = (unsigned long long)npix * (unsigned long long)(r.y - r.x + 1);
  const uint32_t c32 = c > 0xffffffffull ? 0xffffffffu : (uint32_t)c;
  return c32 ? 32 - __clz(c32) : 0;  // 1..32
}

__global__ void k_lpt_hist(uint32_t n, const uint2* __restrict__ ranges, const uint4* __restrict__ act_tiles,
                           uint32_t* __restrict__ hist, const int32_t* status) {
  __shared__ uint32_t h[kBuckets];
  if (threadIdx.x < kBuckets) h[threadIdx.x] = 0;
  __syncthreads();
  if (status_bad(status)) return;
  for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x)
    atomicAdd(&h[cost_bucket(ranges, act_tiles, t)], 1u);
  __syncthreads();
  if (threadIdx.x < kBuckets && h[threadIdx.x]) atomicAdd(hist + threadIdx.x, h[threadIdx.x]);
}

// Descending bucket order: slot base of bucket b = number of tiles in buckets > b.
__global__ void k_lpt_scan(uint32_t* __restrict__ hist, const int32_t* status) {
  if (status_bad(status)) return;
  if (threadIdx.x != 0) return;
  uint32_t run = 0;
  for (int b = kBuckets - 1; b >= 0; --b) {
    const uint32_t c = hist[b];
    hist[b] = run;
    run += c;
  }
}

__global__ void k_lpt_scatter(uint32_t n, const uint2* __restrict__ ranges, const uint4* __restrict__ act_tiles,
                              uint32_t* __restrict__ hist, uint32_t* __restrict__ order, const int32_t* status) {
  if (status_bad(status)) return;
  for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
    const uint32_t slot = atomicAdd(hist + cost_bucket(ranges, act_tiles, t), 1u);
    if (slot < n) order[slot] = t;
  }
}

}  // namespace pgsag

using namespace pgsag;

extern "C" int pgsag_schedule_lpt(uint32_t n_active_total, const void* ranges, const void* act_tiles,
                                  uint32_t* ws, uint32_t* order, int32_t* status, void* stream) {
  if (!status) return PGSAG_ERR_ARG;
  if (n_active_total == 0) return PGSAG_OK;
  if (!ranges || !act_tiles || !ws || !order) return PGSAG_ERR_ARG;
  if (((uintptr_t)act_tiles & 15u) || ((uintptr_t)ranges & 7u)) return PGSAG_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  PGSAG_CUDA(cudaMemsetAsync(ws, 0, kBuckets * sizeof(uint32_t), s));
  const unsigned blocks = min(pgsag_div_up(n_active_total, 256), 148u * 8u);
  k_lpt_hist<<<blocks, 256, 0, s>>>(n_active_total, (const uint2*)ranges, (const uint4*)act_tiles, ws, status);
  PGSAG_CHECK_LAUNCH();
  k_lpt_scan<<<1, 32, 0, s>>>(ws, status);
  PGSAG_CHECK_LAUNCH();
  k_lpt_scatter<<<blocks, 256, 0, s>>>(n_active_total, (const uint2*)ranges, (const uint4*)act_tiles, ws, order,
                                       status);
  PGSAG_CHECK_LAUNCH();
  return PGSAG_OK;
}
