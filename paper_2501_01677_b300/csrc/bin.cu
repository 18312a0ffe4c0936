// Tile binning and ordering (Sec. 3.1: 2D Gaussians "projected onto different
// image tiles" and "sorted").  All pairs are first ordered by depth key with a
// stable LSD radix sort, duplicated once per active tile in that order, then
// stably sorted by active tile: each tile's list ends up in ascending
// (depth key, Gaussian index) order, identical to sorting 64-bit (tile, depth)
// keys, with N-sized instead of K-sized depth passes.
//
// The radix sort is a reduce-then-scan design with no inter-block waits:
// per pass (8-bit digit) one histogram kernel, one row-parallel scan of the
// digit-major histogram table (a block per digit), and one scatter kernel that
// scans the 256 digit totals, then ranks keys stably inside each block with
// warp match/popc.
#include "common.cuh"

namespace pgsag {

constexpr int kRsThreads = 256;
constexpr int kRsWarps = kRsThreads / 32;
constexpr int kRsIpt = 8;
constexpr int kRsTile = kRsThreads * kRsIpt;  // 2048 keys per block iteration
constexpr int kRsBlocks = 592;                // 4 blocks per SM on 148 SMs
constexpr int kScanBlocks = 592;
constexpr int kScanThreads = 256;

__device__ __forceinline__ uint64_t umin64(uint64_t a, uint64_t b) { return a < b ? a : b; }

__device__ __forceinline__ void block_range(uint64_t n, uint32_t b, uint32_t nb, uint32_t& lo,
                                            uint32_t& hi) {
  const uint64_t per = (n + nb - 1) / nb;
  const uint64_t l = umin64(n, (uint64_t)b * per);
  lo = (uint32_t)l;
  hi = (uint32_t)umin64(n, l + per);
}

__device__ __forceinline__ uint32_t load_n(const uint64_t* n_dev, uint64_t n_const, uint64_t cap) {
  return (uint32_t)(n_dev ? umin64(*n_dev, cap) : n_const);
}

__device__ __forceinline__ uint32_t lanemask_lt() {
  uint32_t m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// drop != 0: keys equal to kDropKey are left out (counted nowhere, not written).
constexpr uint32_t kDropKey = 0xffffffffu;

__global__ void __launch_bounds__(kRsThreads) k_radix_hist(const uint32_t* __restrict__ keys,
                                                           const uint64_t* n_dev, uint64_t n_const,
                                                           uint64_t cap, int shift, int drop,
                                                           uint32_t* __restrict__ hist,
                                                           const int32_t* status) {
  __shared__ uint32_t h[256];
  h[threadIdx.x] = 0;
  __syncthreads();
  if (status_bad(status)) return;
  const uint32_t n = load_n(n_dev, n_const, cap);
  uint32_t lo, hi;
  block_range(n, blockIdx.x, gridDim.x, lo, hi);
  const int lane = threadIdx.x & 31;
  for (uint32_t base = lo; base < hi; base += kRsThreads) {
    const uint32_t i = base + threadIdx.x;
    const uint32_t key = i < hi ? __ldg(keys + i) : kDropKey;
    const bool valid = i < hi && !(drop && key == kDropKey);
    const uint32_t d = valid ? ((key >> shift) & 255u) : 256u;
    const uint32_t peers = __match_any_sync(kFull, d);
    if (valid && lane == __ffs(peers) - 1) atomicAdd(&h[d], (uint32_t)__popc(peers));
  }
  __syncthreads();
  hist[threadIdx.x * gridDim.x + blockIdx.x] = h[threadIdx.x];
}

// One block per digit d: exclusive scan (in place) of row d of the digit-major
// histogram table (the counts of digit d in blocks 0..G-1) and the row total.
__global__ void __launch_bounds__(1024) k_radix_rowscan(uint32_t* __restrict__ hist, uint32_t G,
                                                        uint32_t* __restrict__ dtot, const int32_t* status) {
  __shared__ uint32_t wsum[32];
  __shared__ uint32_t carry;
  if (status_bad(status)) return;
  uint32_t* row = hist + (size_t)blockIdx.x * G;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (uint32_t base = 0; base < G; base += 1024) {
    const uint32_t i = base + threadIdx.x;
    const uint32_t s = i < G ? row[i] : 0u;
    uint32_t x = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(kFull, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) wsum[warp] = x;
    __syncthreads();
    if (warp == 0) {
      uint32_t w = wsum[lane];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(kFull, w, o);
        if (lane >= o) w += y;
      }
      wsum[lane] = w;
    }
    __syncthreads();
    const uint32_t c = carry;
    if (i < G) row[i] = c + x - s + (warp > 0 ? wsum[warp - 1] : 0u);
    __syncthreads();
    if (threadIdx.x == 0) carry = c + wsum[31];
    __syncthreads();
  }
  if (threadIdx.x == 0) dtot[blockIdx.x] = carry;
}

__global__ void __launch_bounds__(kRsThreads) k_radix_scatter(
    const uint32_t* __restrict__ keys_in, const uint32_t* __restrict__ vals_in,
    uint32_t* __restrict__ keys_out, uint32_t* __restrict__ vals_out, const uint64_t* n_dev,
    uint64_t n_const, uint64_t cap, int shift, int drop, const uint32_t* __restrict__ hist,
    const uint32_t* __restrict__ dtot, uint64_t* __restrict__ n_kept, const int32_t* status) {
  __shared__ uint32_t run[256];
  __shared__ uint32_t tot[256];
  __shared__ uint32_t wcnt[kRsWarps][256];
  if (status_bad(status)) return;
  const uint32_t n = load_n(n_dev, n_const, cap);
  uint32_t lo, hi;
  block_range(n, blockIdx.x, gridDim.x, lo, hi);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  {
    // digit bases: exclusive scan of the 256 digit totals
    const uint32_t t = dtot[threadIdx.x];
    uint32_t x = t;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(kFull, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) tot[warp] = x;
    __syncthreads();
    uint32_t pre = 0;
    for (int w = 0; w < warp; ++w) pre += tot[w];
    run[threadIdx.x] = pre + x - t + hist[threadIdx.x * gridDim.x + blockIdx.x];
    // number of keys this pass keeps (all of them unless dropping)
    if (n_kept != nullptr && blockIdx.x == 0 && threadIdx.x == kRsThreads - 1) *n_kept = pre + x;
    __syncthreads();
  }
  const uint32_t lt = lanemask_lt();
  for (uint32_t tile = lo; tile < hi; tile += kRsTile) {
#pragma unroll
    for (int w = 0; w < kRsWarps; ++w) wcnt[w][threadIdx.x] = 0;
    uint32_t k[kRsIpt], v[kRsIpt], rk[kRsIpt], dg[kRsIpt];
#pragma unroll
    for (int j = 0; j < kRsIpt; ++j) {
      const uint32_t idx = tile + warp * (32 * kRsIpt) + j * 32 + lane;
      k[j] = idx < hi ? __ldg(keys_in + idx) : kDropKey;
      const bool valid = idx < hi && !(drop && k[j] == kDropKey);
      v[j] = valid ? (vals_in ? __ldg(vals_in + idx) : idx) : 0u;
      dg[j] = valid ? ((k[j] >> shift) & 255u) : 256u;
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < kRsIpt; ++j) {
      const uint32_t peers = __match_any_sync(kFull, dg[j]);
      uint32_t base = 0;
      if (dg[j] < 256u) base = wcnt[warp][dg[j]];
      rk[j] = base + __popc(peers & lt);
      __syncwarp();
      if (dg[j] < 256u && lane == __ffs(peers) - 1) wcnt[warp][dg[j]] = base + __popc(peers);
      __syncwarp();
    }
    __syncthreads();
    {
      uint32_t s = 0;
#pragma unroll
      for (int w = 0; w < kRsWarps; ++w) {
        const uint32_t t = wcnt[w][threadIdx.x];
        wcnt[w][threadIdx.x] = s;
        s += t;
      }
      tot[threadIdx.x] = s;
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < kRsIpt; ++j) {
      if (dg[j] < 256u) {
        const uint32_t dst = run[dg[j]] + wcnt[warp][dg[j]] + rk[j];
        keys_out[dst] = k[j];
        vals_out[dst] = v[j];
      }
    }
    __syncthreads();
    run[threadIdx.x] += tot[threadIdx.x];
    __syncthreads();
  }
}

// ---------------------------------------------------------------- scan + emit

__device__ __forceinline__ uint32_t block_excl_scan(uint32_t x, uint32_t& total, uint32_t* sh) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t inc = x;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(kFull, inc, o);
    if (lane >= o) inc += y;
  }
  if (lane == 31) sh[warp] = inc;
  __syncthreads();
  uint32_t pre = 0, tot = 0;
#pragma unroll
  for (int w = 0; w < kScanThreads / 32; ++w) {
    const uint32_t t = sh[w];
    if (w < warp) pre += t;
    tot += t;
  }
  __syncthreads();
  total = tot;
  return pre + inc - x;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_reduce(const uint32_t* __restrict__ order,
                                                              const uint4* __restrict__ bininfo,
                                                              const uint64_t* n_dev, uint64_t cap,
                                                              uint64_t* __restrict__ partial,
                                                              const int32_t* status) {
  __shared__ unsigned long long ws[kScanThreads / 32];
  if (status_bad(status)) return;
  const uint32_t n = load_n(n_dev, 0, cap);
  uint32_t lo, hi;
  block_range(n, blockIdx.x, gridDim.x, lo, hi);
  unsigned long long s = 0;
  for (uint32_t i = lo + threadIdx.x; i < hi; i += kScanThreads) s += __ldg(&bininfo[__ldg(order + i)].w);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(kFull, s, o);
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long t = 0;
    for (int w = 0; w < kScanThreads / 32; ++w) t += ws[w];
    partial[blockIdx.x] = t;
  }
}

__global__ void __launch_bounds__(1024) k_scan_partials(uint64_t* __restrict__ partial, uint32_t nb,
                                                        uint64_t* __restrict__ k_out, uint64_t capacity,
                                                        int32_t* status) {
  __shared__ unsigned long long wsum[32];
  if (status_bad(status)) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned long long s = threadIdx.x < nb ? partial[threadIdx.x] : 0ull;
  unsigned long long x = s;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned long long y = __shfl_up_sync(kFull, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) wsum[warp] = x;
  __syncthreads();
  if (warp == 0) {
    unsigned long long w = wsum[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned long long y = __shfl_up_sync(kFull, w, o);
      if (lane >= o) w += y;
    }
    wsum[lane] = w;
  }
  __syncthreads();
  const unsigned long long pre = x - s + (warp > 0 ? wsum[warp - 1] : 0ull);
  if (threadIdx.x < nb) partial[threadIdx.x] = pre;
  if (threadIdx.x == 1023) {
    const unsigned long long total = pre + s;
    *k_out = total;
    if (total > capacity) status_set(status, PGSAG_DEV_CAPACITY);
  }
}

__global__ void __launch_bounds__(kScanThreads) k_scan_emit(
    const uint32_t* __restrict__ order, const uint4* __restrict__ bininfo, const uint64_t* n_dev, uint64_t cap,
    const uint64_t* __restrict__ partial, const pgsag_view* __restrict__ views,
    const int32_t* __restrict__ tile_act, const float4* __restrict__ rec, uint32_t* __restrict__ keys_out,
    uint32_t* __restrict__ vals_out, int32_t* status) {
  __shared__ uint32_t sh[kScanThreads / 32];
  if (status_bad(status)) return;
  const uint32_t n = load_n(n_dev, 0, cap);
  uint32_t lo, hi;
  block_range(n, blockIdx.x, gridDim.x, lo, hi);
  uint32_t carry = (uint32_t)partial[blockIdx.x];
  for (uint32_t base = lo; base < hi; base += kScanThreads) {
    const uint32_t i = base + threadIdx.x;
    const bool valid = i < hi;
    uint32_t p = 0;
    uint4 bi = make_uint4(0, 0, 0, 0);
    if (valid) {
      p = __ldg(order + i);
      bi = __ldg(&bininfo[p]);
    }
    uint32_t total;
    const uint32_t off = block_excl_scan(bi.w, total, sh);
    if (bi.w) {
      const pgsag_view* V = views + bi.z;
      const int tiles_x = __ldg(&V->tiles_x);
      const int32_t* ta = tile_act + __ldg(&V->tile_base);
      const uint32_t x0 = bi.x & 0xffffu, y0 = bi.x >> 16, x1 = bi.y & 0xffffu, y1 = bi.y >> 16;
      const bool exact = (x1 - x0 + 1) * (y1 - y0 + 1) <= (uint32_t)kExactTileMax;
      float4 r0 = make_float4(0.f, 0.f, 0.f, 0.f), r3 = r0;
      float l22 = 0.f;
      int tw = 0, th = 0, W = 0, H = 0;
      if (exact) {
        r0 = __ldg(rec + 4ull * p);
        l22 = __ldg(&rec[4ull * p + 1].x);
        r3 = __ldg(rec + 4ull * p + 3);
        tw = __ldg(&V->tile_w);
        th = __ldg(&V->tile_h);
        W = __ldg(&V->width);
        H = __ldg(&V->height);
      }
      uint32_t o = carry + off;
      const uint32_t oend = o + bi.w;
      for (uint32_t ty = y0; ty <= y1; ++ty) {
        const int32_t* row = ta + (size_t)ty * tiles_x;
        for (uint32_t tx = x0; tx <= x1; ++tx) {
          const int32_t a = __ldg(row + tx);
          if (a >= 0 && (!exact || tile_hit(r0.x, r0.y, r3.z, r3.w, r0.z, r0.w, l22, r3.y, (int)tx, (int)ty, tw, th, W, H))) {
            if (o < oend) {
              keys_out[o] = (uint32_t)a;
              vals_out[o] = p;
            }
            ++o;
          }
        }
      }
      if (o != oend) status_set(status, PGSAG_DEV_BOUNDS);
    }
    carry += total;
  }
}

__global__ void k_ranges(const uint32_t* __restrict__ keys, const uint64_t* n_dev, uint64_t cap,
                         uint2* __restrict__ ranges, uint32_t n_active, int32_t* status) {
  if (status_bad(status)) return;
  const uint32_t n = (uint32_t)umin64(*n_dev, cap);
  for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    const uint32_t t = __ldg(keys + k);
    if (t >= n_active) {
      status_set(status, PGSAG_DEV_BOUNDS);
      continue;
    }
    if (k == 0 || __ldg(keys + k - 1) != t) ranges[t].x = k;
    if (k == n - 1 || __ldg(keys + k + 1) != t) ranges[t].y = k + 1;
  }
}

}  // namespace pgsag

using namespace pgsag;

namespace {
struct BinWs {
  uint32_t *kA, *kB, *vA, *vB;  // depth sort (n_pairs)
  uint32_t *dkA, *dkB, *dvW;    // tile sort (capacity)
  uint32_t* hist;               // 256 * kRsBlocks counts, then 256 digit totals
  uint64_t* partial;            // kScanBlocks + 1
  uint64_t* n_bin;              // pairs kept by the depth sort (touching an active tile)
  size_t bytes;
};
size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }
BinWs carve(void* base, uint32_t np, uint64_t cap) {
  BinWs w;
  size_t o = 0;
  char* b = (char*)base;
  auto take = [&](size_t bytes) {
    char* p = b ? b + o : nullptr;
    o += align256(bytes);
    return p;
  };
  const size_t npb = (size_t)(np ? np : 1) * 4, capb = (size_t)(cap ? cap : 1) * 4;
  w.kA = (uint32_t*)take(npb);
  w.kB = (uint32_t*)take(npb);
  w.vA = (uint32_t*)take(npb);
  w.vB = (uint32_t*)take(npb);
  w.dkA = (uint32_t*)take(capb);
  w.dkB = (uint32_t*)take(capb);
  w.dvW = (uint32_t*)take(capb);
  w.hist = (uint32_t*)take((size_t)256 * (kRsBlocks + 1) * 4);
  w.partial = (uint64_t*)take((size_t)(kScanBlocks + 1) * 8);
  w.n_bin = (uint64_t*)take(8);
  w.bytes = o;
  return w;
}

int radix_pass(const uint32_t* kin, const uint32_t* vin, uint32_t* kout, uint32_t* vout,
               const uint64_t* n_dev, uint64_t n_const, uint64_t cap, int shift, uint32_t* hist,
               uint64_t* n_kept, int32_t* status, cudaStream_t s) {
  const int drop = n_kept != nullptr;
  k_radix_hist<<<kRsBlocks, kRsThreads, 0, s>>>(kin, n_dev, n_const, cap, shift, drop, hist, status);
  PGSAG_CHECK_LAUNCH();
  k_radix_rowscan<<<256, 1024, 0, s>>>(hist, kRsBlocks, hist + 256 * kRsBlocks, status);
  PGSAG_CHECK_LAUNCH();
  k_radix_scatter<<<kRsBlocks, kRsThreads, 0, s>>>(kin, vin, kout, vout, n_dev, n_const, cap, shift, drop, hist,
                                                   hist + 256 * kRsBlocks, n_kept, status);
  PGSAG_CHECK_LAUNCH();
  return PGSAG_OK;
}
}  // namespace

extern "C" size_t pgsag_bin_workspace_size(uint32_t n_pairs, uint64_t capacity) {
  return carve(nullptr, n_pairs, capacity).bytes;
}

extern "C" int pgsag_bin(uint32_t n_pairs, uint32_t n_views, const pgsag_view* views,
                         uint32_t n_active_total, const int32_t* tile_act, const float* rec, const void* bininfo,
                         const uint32_t* depth_key, uint64_t capacity, void* ws, size_t ws_bytes,
                         uint32_t* dup_pairs, void* ranges, uint64_t* k_out, int32_t* status,
                         void* stream) {
  if (n_views == 0 || n_views > PGSAG_MAX_VIEWS) return PGSAG_ERR_UNSUPPORTED;
  if (!views || !k_out || !status || !ws) return PGSAG_ERR_ARG;
  if (capacity > 0xffffffffull) return PGSAG_ERR_UNSUPPORTED;
  if (n_pairs && (!bininfo || !depth_key || !tile_act || !rec)) return PGSAG_ERR_ARG;
  if (((uintptr_t)rec | (uintptr_t)bininfo) & 15u) return PGSAG_ERR_ARG;
  if (n_active_total && !ranges) return PGSAG_ERR_ARG;
  if (capacity && !dup_pairs) return PGSAG_ERR_ARG;
  const BinWs w = carve(ws, n_pairs, capacity);
  if (ws_bytes < w.bytes) return PGSAG_ERR_CAPACITY;
  cudaStream_t s = (cudaStream_t)stream;
  PGSAG_CUDA(cudaMemsetAsync(k_out, 0, sizeof(uint64_t), s));
  if (n_active_total) PGSAG_CUDA(cudaMemsetAsync(ranges, 0, (size_t)n_active_total * sizeof(uint2), s));
  if (n_pairs == 0) return PGSAG_OK;

  // 1. stable sort of pairs by depth key (4 x 8-bit digits).  The first pass
  // leaves out the culled pairs (key 0xffffffff: outside the image or touching
  // no active tile) and counts the rest into n_bin; later passes and the scan
  // run on those only.
  const uint32_t* kin = depth_key;
  const uint32_t* vin = nullptr;
  uint32_t* kb[2] = {w.kA, w.kB};
  uint32_t* vb[2] = {w.vA, w.vB};
  for (int pass = 0; pass < 4; ++pass) {
    const int r = radix_pass(kin, vin, kb[pass & 1], vb[pass & 1], pass ? w.n_bin : nullptr, n_pairs, n_pairs,
                             8 * pass, w.hist, pass ? nullptr : w.n_bin, status, s);
    if (r) return r;
    kin = kb[pass & 1];
    vin = vb[pass & 1];
  }
  const uint32_t* order = vin;  // pair indices in (depth key, pair index) order

  // 2-3. scan of touched in that order, K, emission of (active tile, pair)
  int tile_passes = 0;
  if (n_active_total > 1) {
    const int bits = 32 - __builtin_clz(n_active_total - 1);
    tile_passes = (bits + 7) / 8;
  }
  // buffers: pass i reads X_i, writes X_{i+1}; X_P must be dup_pairs
  uint32_t* keysX[5];
  uint32_t* valsX[5];
  for (int i = 0; i <= tile_passes; ++i) {
    const int from_end = tile_passes - i;
    keysX[i] = (from_end & 1) ? w.dkA : w.dkB;
    valsX[i] = (from_end & 1) ? w.dvW : dup_pairs;
  }
  const uint32_t nsb = kScanBlocks;
  k_scan_reduce<<<nsb, kScanThreads, 0, s>>>(order, (const uint4*)bininfo, w.n_bin, n_pairs, w.partial, status);
  PGSAG_CHECK_LAUNCH();
  k_scan_partials<<<1, 1024, 0, s>>>(w.partial, nsb, k_out, capacity, status);
  PGSAG_CHECK_LAUNCH();
  k_scan_emit<<<nsb, kScanThreads, 0, s>>>(order, (const uint4*)bininfo, w.n_bin, n_pairs, w.partial, views,
                                           tile_act, (const float4*)rec, keysX[0], valsX[0], status);
  PGSAG_CHECK_LAUNCH();

  // 4. stable sort of the duplicates by active tile
  for (int pass = 0; pass < tile_passes; ++pass) {
    const int r = radix_pass(keysX[pass], valsX[pass], keysX[pass + 1], valsX[pass + 1], k_out, 0, capacity,
                             8 * pass, w.hist, nullptr, status, s);
    if (r) return r;
  }
  // 5. ranges
  if (n_active_total) {
    k_ranges<<<592, 256, 0, s>>>(keysX[tile_passes], k_out, capacity, (uint2*)ranges, n_active_total, status);
    PGSAG_CHECK_LAUNCH();
  }
  return PGSAG_OK;
}
