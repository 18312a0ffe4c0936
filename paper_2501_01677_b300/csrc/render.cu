// Masked tile rendering, forward (Sec. 3.1 Eq. 1-4) and adjoint.
//
// Work item = chunk: up to 32 rendered (mask-dilated) pixels of one active tile,
// handled by one warp, one pixel per lane.  Warps are independent: each stages
// its tile's sorted Gaussians through its own shared-memory slot in batches of
// 32 (one 64-byte record per lane, coalesced), then every lane walks the batch
// reading the records as broadcasts.  A ballot stops the walk once every lane
// has terminated.
#include "common.cuh"

namespace pgsag {

constexpr int kRenderWarps = 8;
constexpr int kRenderThreads = kRenderWarps * 32;

struct ChunkInfo {
  uint32_t act, view, px_first, count;
  uint32_t rbeg, rend;
};

__device__ __forceinline__ ChunkInfo load_chunk(uint32_t c, const uint2* __restrict__ chunks,
                                                const uint4* __restrict__ act_tiles,
                                                const uint2* __restrict__ ranges) {
  ChunkInfo ci;
  const uint2 ch = __ldg(chunks + c);
  const uint4 at = __ldg(act_tiles + ch.x);
  const uint2 rg = __ldg(ranges + ch.x);
  ci.act = ch.x;
  ci.view = at.x;
  ci.px_first = ch.y;
  ci.count = min(32u, at.z + at.w - ch.y);
  ci.rbeg = rg.x;
  ci.rend = rg.y;
  return ci;
}

// Next chunk for this warp: plain grid (one chunk per warp) or a persistent
// loop over an atomic work counter, optionally through a processing order.
struct Sched {
  const uint32_t* order;
  uint32_t* counter;
};

__device__ __forceinline__ uint32_t next_chunk(const Sched& s, uint32_t& iter, uint32_t n_chunks, int lane) {
  uint32_t c;
  if (s.counter) {
    uint32_t t = 0;
    if (lane == 0) t = atomicAdd(s.counter, 1u);
    t = __shfl_sync(kFull, t, 0);
    c = t;
  } else {
    c = (iter == 0) ? (blockIdx.x * kRenderWarps + (threadIdx.x >> 5)) : n_chunks;
  }
  ++iter;
  if (c < n_chunks && s.order) c = __ldg(s.order + c);
  return c;
}

__global__ void __launch_bounds__(kRenderThreads) k_render_fwd(
    const pgsag_view* __restrict__ views, const float4* __restrict__ rec,
    const uint32_t* __restrict__ dup_pairs, const uint2* __restrict__ ranges,
    const uint4* __restrict__ act_tiles, uint32_t n_chunks, const uint2* __restrict__ chunks,
    const uint32_t* __restrict__ px_list, Sched sched, float4* __restrict__ out8,
    float* __restrict__ depth, uint4* __restrict__ aux, const int32_t* status) {
  __shared__ float4 sm[kRenderWarps][32][4];
  if (status_bad(status)) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float4(*S)[4] = sm[warp];
  uint32_t iter = 0;
  for (;;) {
    const uint32_t c = next_chunk(sched, iter, n_chunks, lane);
    if (c >= n_chunks) break;
    const ChunkInfo ci = load_chunk(c, chunks, act_tiles, ranges);
    const ViewLite V = load_view_lite(views + ci.view);
    const bool has = (uint32_t)lane < ci.count;
    const uint32_t pix = has ? __ldg(px_list + ci.px_first + lane) : 0u;
    const uint32_t py_i = pix / (uint32_t)V.width;
    const float px = (float)(pix - py_i * (uint32_t)V.width) + 0.5f;
    const float py = (float)py_i + 0.5f;

    float T = 1.f, C0 = 0.f, C1 = 0.f, C2 = 0.f, D = 0.f, N0 = 0.f, N1 = 0.f, N2 = 0.f;
    uint32_t last = 0, cnt = 0;
    bool done = !has;
    for (uint32_t base = ci.rbeg; base < ci.rend; base += 32) {
      if (__all_sync(kFull, done)) break;
      const uint32_t nb = min(32u, ci.rend - base);
      __syncwarp();
      if ((uint32_t)lane < nb) {
        const uint32_t p = __ldg(dup_pairs + base + lane);
        const float4* r = rec + 4ull * p;
        S[lane][0] = __ldg(r + 0);
        S[lane][1] = __ldg(r + 1);
        S[lane][2] = __ldg(r + 2);
        S[lane][3] = __ldg(r + 3);
      }
      __syncwarp();
      if (!done) {
        for (uint32_t j = 0; j < nb; ++j) {
          const float4 r0 = S[j][0];
          const float4 r1 = S[j][1];
          float dx, dy;
          const float pw = gauss_power(px, py, r0, r1.x, dx, dy);
          const float raw = __fmul_rn(r1.y, __expf(pw));
          if (raw < kAlphaMin) continue;
          const float alpha = fminf(raw, kAlphaMax);
          const float test = __fmul_rn(T, __fsub_rn(1.f, alpha));
          if (test < kTMin) {
            done = true;
            break;
          }
          const float4 r2 = S[j][2];
          const float4 r3 = S[j][3];
          const float w = __fmul_rn(alpha, T);
          C0 = fmaf(w, r1.z, C0);
          C1 = fmaf(w, r1.w, C1);
          C2 = fmaf(w, r2.x, C2);
          D = fmaf(w, r2.y, D);
          N0 = fmaf(w, r2.z, N0);
          N1 = fmaf(w, r2.w, N1);
          N2 = fmaf(w, r3.x, N2);
          T = test;
          last = base + j;
          ++cnt;
        }
      }
    }
    if (has) {
      const uint64_t gp = V.pix_base + pix;
      out8[2 * gp + 0] = make_float4(C0, C1, C2, D);
      out8[2 * gp + 1] = make_float4(N0, N1, N2, 1.f - T);
      // Eq. 4: ray-plane depth
      const float rx = (px - V.cx) / V.fx, ry = (py - V.cy) / V.fy;
      const float sdot = -(N0 * rx + N1 * ry + N2);
      const bool valid = cnt > 0 && sdot > kRayDotMin && D > 0.f;
      depth[gp] = valid ? D / sdot : 0.f;
      aux[gp] = make_uint4(__float_as_uint(T), last, cnt, 0u);
    }
  }
}

// Reduce 16 per-lane values over the warp; afterwards lane l holds the warp total
// of value (l >> 1) (lanes l and l^1 hold the same total).  16 shuffles.
__device__ __forceinline__ float warp_reduce_scatter16(float v[16], int lane) {
  float a8[8];
  {
    const bool hi = lane & 16;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const float send = hi ? v[i] : v[i + 8];
      const float keep = hi ? v[i + 8] : v[i];
      a8[i] = keep + __shfl_xor_sync(kFull, send, 16);
    }
  }
  float a4[4];
  {
    const bool hi = lane & 8;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const float send = hi ? a8[i] : a8[i + 4];
      const float keep = hi ? a8[i + 4] : a8[i];
      a4[i] = keep + __shfl_xor_sync(kFull, send, 8);
    }
  }
  float a2[2];
  {
    const bool hi = lane & 4;
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      const float send = hi ? a4[i] : a4[i + 2];
      const float keep = hi ? a4[i + 2] : a4[i];
      a2[i] = keep + __shfl_xor_sync(kFull, send, 4);
    }
  }
  float a1;
  {
    const bool hi = lane & 2;
    const float send = hi ? a2[0] : a2[1];
    const float keep = hi ? a2[1] : a2[0];
    a1 = keep + __shfl_xor_sync(kFull, send, 2);
  }
  return a1 + __shfl_xor_sync(kFull, a1, 1);
}

__global__ void __launch_bounds__(kRenderThreads) k_render_bwd(
    const pgsag_view* __restrict__ views, const float4* __restrict__ rec,
    const uint32_t* __restrict__ dup_pairs, const uint2* __restrict__ ranges,
    const uint4* __restrict__ act_tiles, uint32_t n_chunks, const uint2* __restrict__ chunks,
    const uint32_t* __restrict__ px_list, Sched sched, const float4* __restrict__ out8,
    const uint4* __restrict__ aux, const float4* __restrict__ dout8, const float* __restrict__ ddepth,
    const float* __restrict__ dout_scale, float* __restrict__ grad2d, const int32_t* status) {
  __shared__ float4 sm[kRenderWarps][32][4];
  __shared__ uint32_t sp[kRenderWarps][32];
  if (status_bad(status)) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float4(*S)[4] = sm[warp];
  uint32_t* SP = sp[warp];
  const float gscale = dout_scale ? __ldg(dout_scale) : 1.f;
  uint32_t iter = 0;
  for (;;) {
    const uint32_t c = next_chunk(sched, iter, n_chunks, lane);
    if (c >= n_chunks) break;
    const ChunkInfo ci = load_chunk(c, chunks, act_tiles, ranges);
    const ViewLite V = load_view_lite(views + ci.view);
    const bool has = (uint32_t)lane < ci.count;
    const uint32_t pix = has ? __ldg(px_list + ci.px_first + lane) : 0u;
    const uint32_t py_i = pix / (uint32_t)V.width;
    const float px = (float)(pix - py_i * (uint32_t)V.width) + 0.5f;
    const float py = (float)py_i + 0.5f;
    const uint64_t gp = V.pix_base + pix;

    float T = 1.f, Tfin = 1.f;
    int lane_last = -1;
    float dC0 = 0.f, dC1 = 0.f, dC2 = 0.f, dD = 0.f, dN0 = 0.f, dN1 = 0.f, dN2 = 0.f, dA = 0.f;
    if (has) {
      const uint4 ax = __ldg(aux + gp);
      Tfin = __uint_as_float(ax.x);
      T = Tfin;
      lane_last = ax.z > 0 ? (int)ax.y : -1;
      const float4 g0 = __ldg(dout8 + 2 * gp), g1 = __ldg(dout8 + 2 * gp + 1);
      dC0 = g0.x;
      dC1 = g0.y;
      dC2 = g0.z;
      dD = g0.w;
      dN0 = g1.x;
      dN1 = g1.y;
      dN2 = g1.z;
      dA = g1.w;
      dC0 *= gscale;
      dC1 *= gscale;
      dC2 *= gscale;
      dD *= gscale;
      dN0 *= gscale;
      dN1 *= gscale;
      dN2 *= gscale;
      dA *= gscale;
      if (ddepth != nullptr && ax.z > 0) {
        // Eq. 4: Depth = D / s, s = -N . r
        const float gd = gscale * __ldg(ddepth + gp);
        if (gd != 0.f) {
          const float4 o0 = __ldg(out8 + 2 * gp), o1 = __ldg(out8 + 2 * gp + 1);
          const float rx = (px - V.cx) / V.fx, ry = (py - V.cy) / V.fy;
          const float sdot = -(o1.x * rx + o1.y * ry + o1.z);
          if (sdot > kRayDotMin && o0.w > 0.f) {
            const float is = 1.f / sdot;
            dD += gd * is;
            const float k = gd * o0.w * is * is;
            dN0 += k * rx;
            dN1 += k * ry;
            dN2 += k;
          }
        }
      }
    }
    const int max_last = warp_max_i(lane_last);
    if (max_last < (int)ci.rbeg) continue;
    // suffix accumulators (colour, normal, distance behind the current Gaussian)
    float SC0 = 0.f, SC1 = 0.f, SC2 = 0.f, SN0 = 0.f, SN1 = 0.f, SN2 = 0.f, SD = 0.f;
    float pa = 0.f, pc0 = 0.f, pc1 = 0.f, pc2 = 0.f, pn0 = 0.f, pn1 = 0.f, pn2 = 0.f, pd = 0.f;
    for (int hi = max_last; hi >= (int)ci.rbeg; hi -= 32) {
      const int lo = max((int)ci.rbeg, hi - 31);
      const int nb = hi - lo + 1;
      __syncwarp();
      if (lane < nb) {
        const uint32_t p = __ldg(dup_pairs + lo + lane);
        const float4* r = rec + 4ull * p;
        S[lane][0] = __ldg(r + 0);
        S[lane][1] = __ldg(r + 1);
        S[lane][2] = __ldg(r + 2);
        S[lane][3] = __ldg(r + 3);
        SP[lane] = p;
      }
      __syncwarp();
      for (int j = nb - 1; j >= 0; --j) {
        const int idx = lo + j;
        float g[16];
#pragma unroll
        for (int k = 0; k < 16; ++k) g[k] = 0.f;
        bool contrib = false;
        if (idx <= lane_last) {
          const float4 r0 = S[j][0];
          const float4 r1 = S[j][1];
          float dx, dy;
          const float pw = gauss_power(px, py, r0, r1.x, dx, dy);
          const float G = __expf(pw);
          const float raw = __fmul_rn(r1.y, G);
          if (raw >= kAlphaMin) {
            contrib = true;
            const float4 r2 = S[j][2];
            const float4 r3 = S[j][3];
            const float alpha = fminf(raw, kAlphaMax);
            const float oma = 1.f - alpha;
            T = T / oma;  // transmittance in front of this Gaussian
            const float w = alpha * T;
            // S_i = a_{i+1} x_{i+1} + (1 - a_{i+1}) S_{i+1}
            SC0 = pa * pc0 + (1.f - pa) * SC0;
            SC1 = pa * pc1 + (1.f - pa) * SC1;
            SC2 = pa * pc2 + (1.f - pa) * SC2;
            SN0 = pa * pn0 + (1.f - pa) * SN0;
            SN1 = pa * pn1 + (1.f - pa) * SN1;
            SN2 = pa * pn2 + (1.f - pa) * SN2;
            SD = pa * pd + (1.f - pa) * SD;
            const float c0 = r1.z, c1 = r1.w, c2 = r2.x, d = r2.y, n0 = r2.z, n1 = r2.w, n2 = r3.x;
            float dalpha = T * ((c0 - SC0) * dC0 + (c1 - SC1) * dC1 + (c2 - SC2) * dC2 + (d - SD) * dD +
                                (n0 - SN0) * dN0 + (n1 - SN1) * dN1 + (n2 - SN2) * dN2);
            dalpha += dA * Tfin / oma;
            pa = alpha;
            pc0 = c0;
            pc1 = c1;
            pc2 = c2;
            pd = d;
            pn0 = n0;
            pn1 = n1;
            pn2 = n2;
            // colour, distance, normal
            g[6] = w * dC0;
            g[7] = w * dC1;
            g[8] = w * dC2;
            g[9] = w * dD;
            g[10] = w * dN0;
            g[11] = w * dN1;
            g[12] = w * dN2;
            if (raw < kAlphaMax) {
              g[5] = dalpha * G;                 // d alpha / d o
              const float dp = dalpha * alpha;   // d alpha / d power
              g[0] = dp * (r0.z * dx + r0.w * dy);
              g[1] = dp * (r0.w * dx + r1.x * dy);
              g[2] = -0.5f * dp * dx * dx;
              g[3] = -dp * dx * dy;
              g[4] = -0.5f * dp * dy * dy;
            }
          }
        }
        if (__any_sync(kFull, contrib)) {
          const float tot = warp_reduce_scatter16(g, lane);
          const int k = lane >> 1;
          if (!(lane & 1) && k < 13) atomicAdd(grad2d + 16ull * SP[j] + k, tot);
        }
      }
    }
  }
}

}  // namespace pgsag

using namespace pgsag;

static int launch_cfg(const pgsag_sched* sched, uint32_t n_chunks, Sched& s, unsigned& blocks) {
  s.order = sched ? sched->order : nullptr;
  s.counter = sched ? sched->counter : nullptr;
  if (s.counter) {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return PGSAG_ERR_CUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return PGSAG_ERR_CUDA;
    const int per = sched->ctas_per_sm > 0 ? sched->ctas_per_sm : 8;
    blocks = (unsigned)(sms * per);
  } else {
    blocks = pgsag_div_up(n_chunks, kRenderWarps);
  }
  return PGSAG_OK;
}

extern "C" int pgsag_render_fwd(uint32_t n_views, const pgsag_view* views, const float* rec,
                                const uint32_t* dup_pairs, const void* ranges, const void* act_tiles,
                                uint32_t n_chunks, const void* chunks, const uint32_t* px_list,
                                const pgsag_sched* sched, float* out8, float* depth, void* aux,
                                int32_t* status, void* stream) {
  if (n_views == 0 || n_views > PGSAG_MAX_VIEWS) return PGSAG_ERR_UNSUPPORTED;
  if (!views || !status) return PGSAG_ERR_ARG;
  if (n_chunks == 0) return PGSAG_OK;
  if (!rec || !ranges || !act_tiles || !chunks || !px_list || !out8 || !depth || !aux) return PGSAG_ERR_ARG;
  if (((uintptr_t)rec | (uintptr_t)out8 | (uintptr_t)aux | (uintptr_t)act_tiles) & 15u) return PGSAG_ERR_ARG;
  Sched s;
  unsigned blocks;
  int r = launch_cfg(sched, n_chunks, s, blocks);
  if (r) return r;
  cudaStream_t st = (cudaStream_t)stream;
  if (s.counter) PGSAG_CUDA(cudaMemsetAsync(s.counter, 0, sizeof(uint32_t), st));
  k_render_fwd<<<blocks, kRenderThreads, 0, st>>>(
      views, (const float4*)rec, dup_pairs, (const uint2*)ranges, (const uint4*)act_tiles, n_chunks,
      (const uint2*)chunks, px_list, s, (float4*)out8, depth, (uint4*)aux, status);
  PGSAG_CHECK_LAUNCH();
  return PGSAG_OK;
}

extern "C" int pgsag_render_bwd(uint32_t n_views, const pgsag_view* views, const float* rec,
                                const uint32_t* dup_pairs, const void* ranges, const void* act_tiles,
                                uint32_t n_chunks, const void* chunks, const uint32_t* px_list,
                                const pgsag_sched* sched, const float* out8, const void* aux,
                                const float* dout8, const float* ddepth, const float* dout_scale,
                                uint32_t n_pairs, float* grad2d, int32_t* status, void* stream) {
  if (n_views == 0 || n_views > PGSAG_MAX_VIEWS) return PGSAG_ERR_UNSUPPORTED;
  if (!views || !status) return PGSAG_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  if (n_pairs) {
    if (!grad2d) return PGSAG_ERR_ARG;
    PGSAG_CUDA(cudaMemsetAsync(grad2d, 0, (size_t)n_pairs * PGSAG_GRAD2D_FLOATS * sizeof(float), st));
  }
  if (n_chunks == 0) return PGSAG_OK;
  if (!rec || !ranges || !act_tiles || !chunks || !px_list || !out8 || !aux || !dout8 || !grad2d)
    return PGSAG_ERR_ARG;
  if (((uintptr_t)rec | (uintptr_t)out8 | (uintptr_t)aux | (uintptr_t)dout8 | (uintptr_t)act_tiles) & 15u)
    return PGSAG_ERR_ARG;
  Sched s;
  unsigned blocks;
  int r = launch_cfg(sched, n_chunks, s, blocks);
  if (r) return r;
  if (s.counter) PGSAG_CUDA(cudaMemsetAsync(s.counter, 0, sizeof(uint32_t), st));
  k_render_bwd<<<blocks, kRenderThreads, 0, st>>>(
      views, (const float4*)rec, dup_pairs, (const uint2*)ranges, (const uint4*)act_tiles, n_chunks,
      (const uint2*)chunks, px_list, s, (const float4*)out8, (const uint4*)aux, (const float4*)dout8, ddepth,
      dout_scale, grad2d, status);
  PGSAG_CHECK_LAUNCH();
  return PGSAG_OK;
}
