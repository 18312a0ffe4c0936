// Depth-map mean fusion and TSDF integration (Sec. 4.4).
//
// Integration is voxel-parallel: each thread owns kTsdfVPT voxels (consecutive
// threads take consecutive x, so grid reads and writes are coalesced), keeps
// their running sums and counts in registers while it sweeps a chunk of views,
// and touches the grids once per chunk.  A voxel's samples of one view are
// spread over the whole depth map (the rays of a column of voxels meet the same
// pixels), so each map is re-read about as often as voxels project into it; the
// views are therefore taken in chunks whose maps fit in the L2 together (one
// launch per chunk, later chunks merged into the running mean): inside a launch
// the CTAs drift over at most one chunk of views, and a map comes from HBM a few
// times at most.  On the 32-view bench workload (20 MB maps, 126 MB L2) a
// single launch over all views read 97 GB from HBM and took 17.3 ms; chunks of
// 6 / 3 / 1 views take 7.8 / 8.7 / 12.8 ms (more chunks: more grid passes).  The camera table is a
// __grid_constant__ kernel parameter (constant-cache broadcast).  The
// projection, the pixel choice and the sdf >= -trunc test are a fixed sequence
// of correctly rounded float32 operations (reproducible off the GPU).
#include <math.h>

#include "common.cuh"

namespace pgsag {

constexpr int kTsdfThreads = 256;
#ifndef PGSAG_TSDF_L2_DIV
#define PGSAG_TSDF_L2_DIV 1  // depth maps of one launch: at most L2 / this many bytes
#endif
constexpr int kTsdfVPT = 4;  // voxels per thread

template <int kMaxViews>
struct DepthTable {
  pgsag_depth_view v[kMaxViews];
};

__device__ __forceinline__ void fuse_add(float d, float& s, float& n) {
  if (d > 0.f && d < INFINITY) {
    s += d;
    n += 1.f;
  }
}

// kVec: 4 pixels per thread and iteration through 16-byte loads and stores (maps
// and out 16-byte aligned, n_pix a multiple of 4), all maps' loads in flight
// before the sums.
template <bool kVec>
__global__ void __launch_bounds__(256) k_depth_fuse(uint32_t n_maps, const float* __restrict__ maps, uint64_t n_pix,
                                                    float* __restrict__ out) {
  if constexpr (kVec) {
    const uint64_t n4 = n_pix / 4;
    const float4* m4 = reinterpret_cast<const float4*>(maps);
    for (uint64_t p = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n4; p += (uint64_t)gridDim.x * blockDim.x) {
      float4 v[8];
#pragma unroll
      for (int m = 0; m < 8; ++m)
        if (m < (int)n_maps) v[m] = __ldg(m4 + (uint64_t)m * n4 + p);
      float4 s = make_float4(0.f, 0.f, 0.f, 0.f), n = s;
#pragma unroll
      for (int m = 0; m < 8; ++m) {
        if (m >= (int)n_maps) break;
        fuse_add(v[m].x, s.x, n.x);
        fuse_add(v[m].y, s.y, n.y);
        fuse_add(v[m].z, s.z, n.z);
        fuse_add(v[m].w, s.w, n.w);
      }
      reinterpret_cast<float4*>(out)[p] = make_float4(n.x > 0.f ? s.x / n.x : 0.f, n.y > 0.f ? s.y / n.y : 0.f,
                                                      n.z > 0.f ? s.z / n.z : 0.f, n.w > 0.f ? s.w / n.w : 0.f);
    }
  } else {
    for (uint64_t p = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n_pix;
         p += (uint64_t)gridDim.x * blockDim.x) {
      float s = 0.f, n = 0.f;
      for (uint32_t m = 0; m < n_maps; ++m) fuse_add(__ldg(maps + (uint64_t)m * n_pix + p), s, n);
      out[p] = n > 0.f ? s / n : 0.f;
    }
  }
}

#ifndef PGSAG_TSDF_MINB
#define PGSAG_TSDF_MINB 1
#endif
template <int kMaxViews>
__global__ void __launch_bounds__(kTsdfThreads, PGSAG_TSDF_MINB) k_tsdf(pgsag_tsdf_grid G, uint32_t n_views,
                                                       const __grid_constant__ DepthTable<kMaxViews> T,
                                                       const float* __restrict__ depth, int accumulate,
                                                       float* __restrict__ tsdf, float* __restrict__ weight,
                                                       const int32_t* status) {
  if (status_bad(status)) return;
  const uint32_t nvox = G.nx * G.ny * G.nz;
  constexpr uint32_t kGroup = (uint32_t)(kTsdfThreads * kTsdfVPT);
  const uint32_t n_groups = (nvox + kGroup - 1) / kGroup;
  const float nmu = -G.trunc, imu = 1.f / G.trunc;  // the value sdf / trunc is taken as sdf * (1 / trunc)
  for (uint32_t grp = blockIdx.x; grp < n_groups; grp += gridDim.x) {
    const uint32_t base = grp * kGroup + threadIdx.x;
    float X[kTsdfVPT], Y[kTsdfVPT], Z[kTsdfVPT], sum[kTsdfVPT];
    uint32_t cnt[kTsdfVPT];
#pragma unroll
    for (int k = 0; k < kTsdfVPT; ++k) {
      const uint32_t i = min(base + (uint32_t)(k * kTsdfThreads), nvox - 1);
      const uint32_t ix = i % G.nx, r = i / G.nx, iy = r % G.ny, iz = r / G.ny;
      // centre = origin + (index + 1/2) voxel
      X[k] = __fadd_rn(G.origin[0], __fmul_rn(__fadd_rn((float)ix, 0.5f), G.voxel));
      Y[k] = __fadd_rn(G.origin[1], __fmul_rn(__fadd_rn((float)iy, 0.5f), G.voxel));
      Z[k] = __fadd_rn(G.origin[2], __fmul_rn(__fadd_rn((float)iz, 0.5f), G.voxel));
      sum[k] = 0.f;
      cnt[k] = 0u;
    }
    for (uint32_t v = 0; v < n_views; ++v) {
      const pgsag_depth_view& V = T.v[v];
      const float r0 = V.R[0], r1 = V.R[1], r2 = V.R[2], r3 = V.R[3], r4 = V.R[4], r5 = V.R[5];
      const float r6 = V.R[6], r7 = V.R[7], r8 = V.R[8];
      const float t0 = V.t[0], t1 = V.t[1], t2 = V.t[2];
      const float fx = V.fx, fy = V.fy, cx = V.cx, cy = V.cy, zn = V.znear;
      const float Wf = (float)V.width, Hf = (float)V.height;
      const uint32_t W = (uint32_t)V.width;
      const float* dm = depth + V.depth_offset;
      bool in[kTsdfVPT];
      float zc[kTsdfVPT];
      uint32_t pix[kTsdfVPT];
#pragma unroll
      for (int k = 0; k < kTsdfVPT; ++k) {
        const float xc = __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(r0, X[k]), __fmul_rn(r1, Y[k])), __fmul_rn(r2, Z[k])), t0);
        const float yc = __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(r3, X[k]), __fmul_rn(r4, Y[k])), __fmul_rn(r5, Z[k])), t1);
        zc[k] = __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(r6, X[k]), __fmul_rn(r7, Y[k])), __fmul_rn(r8, Z[k])), t2);
        const float iz = __frcp_rn(zc[k]);
        const float u = __fadd_rn(__fmul_rn(fx, __fmul_rn(xc, iz)), cx);
        const float w = __fadd_rn(__fmul_rn(fy, __fmul_rn(yc, iz)), cy);
        in[k] = zc[k] > zn && u >= 0.f && u < Wf && w >= 0.f && w < Hf;  // false for NaN
        pix[k] = in[k] ? (uint32_t)w * W + (uint32_t)u : 0u;               // floor: u, w >= 0
      }
      float d[kTsdfVPT];
#pragma unroll
      for (int k = 0; k < kTsdfVPT; ++k) d[k] = in[k] ? __ldg(dm + pix[k]) : 0.f;
#pragma unroll
      for (int k = 0; k < kTsdfVPT; ++k) {
        const float sdf = __fsub_rn(d[k], zc[k]);
        if (in[k] && d[k] > 0.f && d[k] < INFINITY && sdf >= nmu) {
          sum[k] += fminf(1.f, __fmul_rn(sdf, imu));
          cnt[k] += 1u;
        }
      }
    }
#pragma unroll
    for (int k = 0; k < kTsdfVPT; ++k) {
      const uint32_t i = base + (uint32_t)(k * kTsdfThreads);
      if (i >= nvox) continue;
      if (accumulate) {
        if (cnt[k] == 0u) continue;
        const float w0 = weight[i], t0 = tsdf[i];
        const float w = w0 + (float)cnt[k];
        tsdf[i] = (t0 * w0 + sum[k]) / w;
        weight[i] = w;
      } else {
        tsdf[i] = cnt[k] ? sum[k] / (float)cnt[k] : 1.f;
        weight[i] = (float)cnt[k];
      }
    }
  }
}

}  // namespace pgsag

using namespace pgsag;

extern "C" int pgsag_depth_fuse(uint32_t n_maps, const float* maps, uint64_t n_pix, float* out, void* stream) {
  if (n_maps == 0 || n_maps > 8) return PGSAG_ERR_UNSUPPORTED;
  if (n_pix == 0) return PGSAG_OK;
  if (!maps || !out) return PGSAG_ERR_ARG;
  const bool vec = (n_pix % 4 == 0) && !(((uintptr_t)maps | (uintptr_t)out) & 15u);
  const uint64_t items = vec ? n_pix / 4 : n_pix;
  const uint64_t want = (items + 255) / 256;
  const unsigned blocks = (unsigned)(want < 148ull * 16ull ? want : 148ull * 16ull);
  if (vec)
    k_depth_fuse<true><<<blocks, 256, 0, (cudaStream_t)stream>>>(n_maps, maps, n_pix, out);
  else
    k_depth_fuse<false><<<blocks, 256, 0, (cudaStream_t)stream>>>(n_maps, maps, n_pix, out);
  PGSAG_CHECK_LAUNCH();
  return PGSAG_OK;
}

template <int kMaxViews>
static int launch_tsdf(const pgsag_tsdf_grid& G, uint32_t nv, const pgsag_depth_view* views, const float* depth,
                       int acc, float* tsdf, float* weight, int32_t* status, cudaStream_t s) {
  DepthTable<kMaxViews> T;
  for (uint32_t v = 0; v < nv; ++v) T.v[v] = views[v];
  for (uint32_t v = nv; v < (uint32_t)kMaxViews; ++v) T.v[v] = pgsag_depth_view{};
  static int occ = 0, sms = 0;
  if (occ <= 0) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return PGSAG_ERR_CUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return PGSAG_ERR_CUDA;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, (const void*)k_tsdf<kMaxViews>, kTsdfThreads, 0) !=
        cudaSuccess)
      return PGSAG_ERR_CUDA;
    if (occ <= 0) occ = 1;
  }
  const uint64_t nvox = (uint64_t)G.nx * G.ny * G.nz;
  const uint64_t groups = (nvox + (uint64_t)kTsdfThreads * kTsdfVPT - 1) / ((uint64_t)kTsdfThreads * kTsdfVPT);
  const uint64_t wave = (uint64_t)sms * occ;
  const unsigned blocks = (unsigned)(groups < wave ? groups : wave);
  k_tsdf<kMaxViews><<<blocks, kTsdfThreads, 0, s>>>(G, nv, T, depth, acc, tsdf, weight, status);
  PGSAG_CHECK_LAUNCH();
  return PGSAG_OK;
}

extern "C" int pgsag_tsdf_integrate(const pgsag_tsdf_grid* grid, uint32_t n_views, const pgsag_depth_view* views,
                                    const float* depth, int accumulate, float* tsdf, float* weight, int32_t* status,
                                    void* stream) {
  if (n_views > PGSAG_TSDF_MAX_VIEWS) return PGSAG_ERR_UNSUPPORTED;
  if (!grid || !status) return PGSAG_ERR_ARG;
  const pgsag_tsdf_grid G = *grid;
  if (!(G.voxel > 0.f) || !(G.trunc > 0.f)) return PGSAG_ERR_ARG;
  const uint64_t nvox = (uint64_t)G.nx * G.ny * G.nz;
  if (nvox >= (1ull << 32)) return PGSAG_ERR_UNSUPPORTED;
  if (nvox == 0) return PGSAG_OK;
  if (!tsdf || !weight) return PGSAG_ERR_ARG;
  if (n_views > 0 && (!views || !depth)) return PGSAG_ERR_ARG;
  for (uint32_t v = 0; v < n_views; ++v)
    if (views[v].width <= 0 || views[v].height <= 0) return PGSAG_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  if (n_views == 0)
    return launch_tsdf<32>(G, 0, views, depth, accumulate, tsdf, weight, status, s);
  static int l2 = -1;
  if (l2 < 0) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return PGSAG_ERR_CUDA;
    if (cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev) != cudaSuccess) return PGSAG_ERR_CUDA;
  }
  const uint64_t budget = (uint64_t)(l2 > 0 ? l2 : (64 << 20)) / PGSAG_TSDF_L2_DIV;
  uint32_t v0 = 0;
  int acc = accumulate;
  while (v0 < n_views) {
    // the longest run of views (at least one, at most 32) whose maps fit the budget
    uint32_t n = 0;
    uint64_t bytes = 0;
    while (v0 + n < n_views && n < 32) {
      const uint64_t b = 4ull * (uint64_t)views[v0 + n].width * (uint64_t)views[v0 + n].height;
      if (n > 0 && bytes + b > budget) break;
      bytes += b;
      ++n;
    }
    const int r = launch_tsdf<32>(G, n, views + v0, depth, acc, tsdf, weight, status, s);
    if (r) return r;
    v0 += n;
    acc = 1;
  }
  return PGSAG_OK;
}
