// Masked tile rendering, forward (Sec. 3.1 Eq. 1-4) and adjoint.
//
// Work item = one active tile, handled by one CTA of 4 warps.  The tile's
// rendered (mask-dilated) pixels are compacted; each lane takes 2 of them (more
// rounds for tiles larger than 256 pixels).  The tile's depth-sorted Gaussians
// are staged through shared memory in batches of 256 (64-byte records,
// coalesced), then each warp walks the batch, skipping -- as a warp-uniform
// branch -- every Gaussian whose alpha >= 1/255 box misses the bounding box of
// the warp's pixels.  A pair is rejected before the exponential when the
// exponent is below the Gaussian's threshold -ln(255 o) (alpha < 1/255).  The forward stops a batch loop when every warp of the
// CTA has terminated (__syncthreads_or).  The adjoint re-walks the list back to
// front from the CTA's last blended Gaussian, recovers T by division, reduces
// each Gaussian's 13 gradient values across the warp with 16 shuffles, sums the
// warps in shared memory and issues one float4 atomic per 4 values per tile.
#include "common.cuh"

namespace pgsag {

// Launch shape (compile-time; the defaults are the best measured on B300 for the
// 5472x3648 aerial workload): warps per CTA (one CTA per active tile), pixels
// per lane, Gaussians staged per batch, the number of resident CTAs per SM the
// register allocation must allow (forward 10, adjoint 7), and the largest number
// of contributing lanes for which the adjoint adds a Gaussian's gradient to
// shared memory lane by lane instead of reducing across the warp (0: always
// reduce).
#ifndef PGSAG_FWD_WARPS
#define PGSAG_FWD_WARPS 4
#endif
#ifndef PGSAG_FWD_PPT
#define PGSAG_FWD_PPT 2
#endif
#ifndef PGSAG_BWD_WARPS
#define PGSAG_BWD_WARPS 4
#endif
#ifndef PGSAG_BWD_PPT
#define PGSAG_BWD_PPT 2
#endif
#ifndef PGSAG_BWD_DIRECT
#define PGSAG_BWD_DIRECT 0
#endif
#ifndef PGSAG_BATCH
#define PGSAG_BATCH 128
#endif
#ifndef PGSAG_FWD_MINB
#define PGSAG_FWD_MINB 10  // resident CTAs per SM the register budget must allow
#endif
#ifndef PGSAG_BWD_MINB
#define PGSAG_BWD_MINB 7
#endif
constexpr int kBatch = PGSAG_BATCH;  // Gaussians staged per batch

struct TileInfo {
  uint32_t view, tx, ty, px_first, npix, rbeg, rend;
};

__device__ __forceinline__ TileInfo load_tile(uint32_t t, const uint4* __restrict__ act_tiles,
                                              const uint2* __restrict__ ranges) {
  TileInfo ti;
  const uint4 at = __ldg(act_tiles + t);
  const uint2 rg = __ldg(ranges + t);
  ti.view = at.x;
  ti.tx = at.y & 0xffffu;
  ti.ty = at.y >> 16;
  ti.px_first = at.z;
  ti.npix = at.w;
  ti.rbeg = rg.x;
  ti.rend = rg.y;
  return ti;
}

// Next tile for this CTA: plain grid (one tile per CTA) or a persistent loop over
// an atomic work counter, optionally through a processing order.  Called by all
// threads; thread 0 fetches.
struct Sched {
  const uint32_t* order;
  uint32_t* counter;
};

__device__ __forceinline__ uint32_t next_tile(const Sched& s, uint32_t& iter, uint32_t n_items,
                                              uint32_t* s_item) {
  if (threadIdx.x == 0) {
    uint32_t c;
    if (s.counter)
      c = atomicAdd(s.counter, 1u);
    else
      c = iter == 0 ? blockIdx.x : n_items;
    if (c < n_items && s.order) c = __ldg(s.order + c);
    *s_item = c;
  }
  __syncthreads();
  const uint32_t c = *s_item;
  __syncthreads();
  ++iter;
  return c;
}

// Pixels of lane `lane` in warp `warp` for the round starting at r0: entries
// r0 + (warp * kPPT + k) * 32 + lane of the tile's compacted pixel list, so a
// warp covers kPPT consecutive 32-pixel runs.  Pixel centres are kept relative
// to an origin (ox, oy) near the tile, exactly, like the staged Gaussian
// centres, so that offsets do not lose precision to the image size.
template <int kPPT>
struct Pix {
  bool has[kPPT];
  uint32_t q[kPPT];          // compact index (position in px_list): per-pixel arrays
  float px[kPPT], py[kPPT];  // centre minus tile origin
};

template <int kPPT>
__device__ __forceinline__ Pix<kPPT> load_pixels(const TileInfo& ti, uint32_t r0, int warp, int lane, int width,
                                                 int ox, int oy, const uint32_t* __restrict__ px_list) {
  Pix<kPPT> P;
#pragma unroll
  for (int k = 0; k < kPPT; ++k) {
    const uint32_t li = r0 + (uint32_t)((warp * kPPT + k) * 32 + lane);
    P.has[k] = li < ti.npix;
    P.q[k] = ti.px_first + li;
    const uint32_t pix = P.has[k] ? __ldg(px_list + P.q[k]) : 0u;
    const uint32_t yy = pix / (uint32_t)width;
    P.px[k] = (float)((int)(pix - yy * (uint32_t)width) - ox) + 0.5f;
    P.py[k] = (float)((int)yy - oy) + 0.5f;
  }
  return P;
}

// Bounding box of the warp's valid pixel centres (warp-uniform result).
template <int kPPT>
__device__ __forceinline__ float4 warp_pixel_box(const Pix<kPPT>& P) {
  float x0 = 3.0e38f, x1 = -3.0e38f, y0 = 3.0e38f, y1 = -3.0e38f;
#pragma unroll
  for (int k = 0; k < kPPT; ++k) {
    if (P.has[k]) {
      x0 = fminf(x0, P.px[k]);
      x1 = fmaxf(x1, P.px[k]);
      y0 = fminf(y0, P.py[k]);
      y1 = fmaxf(y1, P.py[k]);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    x0 = fminf(x0, __shfl_xor_sync(kFull, x0, o));
    x1 = fmaxf(x1, __shfl_xor_sync(kFull, x1, o));
    y0 = fminf(y0, __shfl_xor_sync(kFull, y0, o));
    y1 = fmaxf(y1, __shfl_xor_sync(kFull, y1, o));
  }
  return make_float4(x0, x1, y0, y1);
}

// Shared-memory image of a batch of staged Gaussians, packed by use:
// g0 = {mx, my, l11, l21}, g1 = {l22, o, thr, -}, g2 = {r, g, b, d}, g3 = {nx, ny, nz, -}
// (l11, l21, l22: Cholesky factor of the conic).
struct Stage {
  float4 g0[kBatch], g1[kBatch], g2[kBatch], g3[kBatch];
};

// The centre is staged relative to the origin (ox, oy): (integer part - origin)
// is exact, then the fraction is added.
__device__ __forceinline__ void stage(uint32_t i, int slot, const uint32_t* __restrict__ dup_pairs,
                                      const float4* __restrict__ rec, float ox, float oy, Stage& S,
                                      uint32_t* spair) {
  const uint32_t p = __ldg(dup_pairs + i);
  const float4* r = rec + 4ull * p;
  const float4 r0 = __ldg(r + 0), r1 = __ldg(r + 1), r2 = __ldg(r + 2), r3 = __ldg(r + 3);
  S.g0[slot] = make_float4(__fadd_rn(__fsub_rn(r0.x, ox), r3.z), __fadd_rn(__fsub_rn(r0.y, oy), r3.w), r0.z, r0.w);
  S.g1[slot] = make_float4(r1.x, r1.y, r3.y, 0.f);
  S.g2[slot] = make_float4(r1.z, r1.w, r2.x, r2.y);
  S.g3[slot] = make_float4(r2.z, r2.w, r3.x, 0.f);
  if (spair) spair[slot] = p;
}

// Relevance of staged Gaussians c*32 + lane (c < kBatch/32) to the warp's pixel
// rectangle: one ellipse-rectangle test per lane, one ballot per 32 Gaussians.
// Bits beyond `limit` (exclusive) are cleared.
__device__ __forceinline__ void warp_relevance(const Stage& S, int limit, float4 cbox, int lane,
                                               uint32_t rel[kBatch / 32]) {
#pragma unroll
  for (int c = 0; c < kBatch / 32; ++c) {
    const int j = c * 32 + lane;
    bool hit = false;
    if (j < limit) {
      const float4 a = S.g0[j];
      const float4 b = S.g1[j];
      hit = factor_rect_hit(a.z, a.w, b.x, b.z, cbox.x - a.x, cbox.y - a.x, cbox.z - a.y, cbox.w - a.y);
    }
    rel[c] = __ballot_sync(kFull, hit);
  }
}

template <int kWarps, int kPPT>
__global__ void __launch_bounds__(kWarps * 32, PGSAG_FWD_MINB) k_render_fwd(
    const pgsag_view* __restrict__ views, const float4* __restrict__ rec,
    const uint32_t* __restrict__ dup_pairs, const uint2* __restrict__ ranges,
    const uint4* __restrict__ act_tiles, uint32_t n_items, const uint32_t* __restrict__ px_list,
    Sched sched, float4* __restrict__ out8, float* __restrict__ depth, uint4* __restrict__ aux,
    const int32_t* status) {
  constexpr int kRenderThreads = kWarps * 32;
  constexpr int kTilePix = kRenderThreads * kPPT;
  constexpr int kStagePerThread = kBatch / kRenderThreads;
  static_assert(kBatch % kRenderThreads == 0 && kStagePerThread >= 1, "batch must be a multiple of the CTA size");
  __shared__ Stage S;
  __shared__ uint32_t s_item;
  if (status_bad(status)) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t iter = 0;
  for (;;) {
    const uint32_t t = next_tile(sched, iter, n_items, &s_item);
    if (t >= n_items) break;
    const TileInfo ti = load_tile(t, act_tiles, ranges);
    const ViewLite V = load_view_lite(views + ti.view);
    for (uint32_t r0 = 0; r0 < ti.npix; r0 += kTilePix) {
      // coordinate origin: the 32-pixel-aligned corner of the 32x32 cell holding
      // the tile (every supported tile lies in one cell), so offsets round the
      // same way whatever the tile size
      const int ox = ((int)ti.tx * V.tile_w) & ~31, oy = ((int)ti.ty * V.tile_h) & ~31;
      const Pix<kPPT> P = load_pixels<kPPT>(ti, r0, warp, lane, V.width, ox, oy, px_list);
      const float4 cbox = warp_pixel_box(P);
      float T[kPPT], C0[kPPT], C1[kPPT], C2[kPPT], D[kPPT], N0[kPPT], N1[kPPT], N2[kPPT];
      uint32_t last[kPPT], cnt[kPPT];
      bool done[kPPT];
      bool all_done = true;
#pragma unroll
      for (int k = 0; k < kPPT; ++k) {
        T[k] = 1.f;
        C0[k] = C1[k] = C2[k] = D[k] = N0[k] = N1[k] = N2[k] = 0.f;
        last[k] = 0;
        cnt[k] = 0;
        done[k] = !P.has[k];
        all_done = all_done && done[k];
      }
      for (uint32_t base = ti.rbeg; base < ti.rend; base += kBatch) {
        if (!__syncthreads_or(!all_done)) break;
        const uint32_t nb = min((uint32_t)kBatch, ti.rend - base);
#pragma unroll
        for (int u = 0; u < kStagePerThread; ++u) {
          const uint32_t slot = threadIdx.x + u * kRenderThreads;
          if (slot < nb) stage(base + slot, slot, dup_pairs, rec, (float)ox, (float)oy, S, nullptr);
        }
        __syncthreads();
        if (!__any_sync(kFull, !all_done)) continue;
        uint32_t rel[kBatch / 32];
        warp_relevance(S, (int)nb, cbox, lane, rel);
        if (all_done) continue;
#pragma unroll 1
        for (int c = 0; c < kBatch / 32; ++c) {
          uint32_t m = rel[c];
          while (m) {
            const int j = c * 32 + __ffs(m) - 1;
            m &= m - 1;
            const float4 q0 = S.g0[j];
            const float4 q1 = S.g1[j];
#pragma unroll
            for (int k = 0; k < kPPT; ++k) {
              if (done[k]) continue;
              float dx, dy, u, w2;
              const float pw = gauss_power(P.px[k], P.py[k], q0, q1.x, dx, dy, u, w2);
              if (!(pw >= q1.z)) continue;  // alpha < 1/255
              const float alpha = fminf(__fmul_rn(q1.y, __expf(pw)), kAlphaMax);
              const float test = __fmul_rn(T[k], __fsub_rn(1.f, alpha));
              if (test < kTMin) {
                done[k] = true;
                continue;
              }
              const float4 q2 = S.g2[j];
              const float4 q3 = S.g3[j];
              const float w = __fmul_rn(alpha, T[k]);
              C0[k] = fmaf(w, q2.x, C0[k]);
              C1[k] = fmaf(w, q2.y, C1[k]);
              C2[k] = fmaf(w, q2.z, C2[k]);
              D[k] = fmaf(w, q2.w, D[k]);
              N0[k] = fmaf(w, q3.x, N0[k]);
              N1[k] = fmaf(w, q3.y, N1[k]);
              N2[k] = fmaf(w, q3.z, N2[k]);
              T[k] = test;
              last[k] = base + j;
              ++cnt[k];
            }
            bool ad = true;
#pragma unroll
            for (int k = 0; k < kPPT; ++k) ad = ad && done[k];
            if (ad) {
              all_done = true;
              c = kBatch / 32;
              break;
            }
          }
        }
      }
#pragma unroll
      for (int k = 0; k < kPPT; ++k) {
        if (!P.has[k]) continue;
        const uint64_t gp = P.q[k];
        out8[2 * gp + 0] = make_float4(C0[k], C1[k], C2[k], D[k]);
        out8[2 * gp + 1] = make_float4(N0[k], N1[k], N2[k], 1.f - T[k]);
        // Eq. 4: ray-plane depth
        const float rx = (P.px[k] + (float)ox - V.cx) / V.fx, ry = (P.py[k] + (float)oy - V.cy) / V.fy;
        const float sdot = -(N0[k] * rx + N1[k] * ry + N2[k]);
        const bool valid = cnt[k] > 0 && sdot > kRayDotMin && D[k] > 0.f;
        depth[gp] = valid ? D[k] / sdot : 0.f;
        aux[gp] = make_uint4(__float_as_uint(T[k]), last[k], cnt[k], 0u);
      }
    }
  }
}

// Reduce 16 per-lane values over the warp; afterwards lane l holds the warp total
// of value (l >> 1) (lanes l and l^1 hold the same total).  16 shuffles.
__device__ __forceinline__ float warp_reduce_scatter16(const float v[16], int lane) {
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

// Per-pixel adjoint state.  S* hold the suffix sums S_i = sum_{j>i} x_j a_j
// prod_{i<l<j} (1 - a_l) of the channels behind the Gaussian being processed;
// they are advanced eagerly (S <- a x + (1 - a) S) after each contributor.
struct BwdPix {
  float T;
  int last;
  float dC0, dC1, dC2, dD, dN0, dN1, dN2, dATf;  // dATf = dL/dA * T_final
  float SC0, SC1, SC2, SN0, SN1, SN2, SD;
};

template <int kWarps, int kPPT, int kDirect>
__global__ void __launch_bounds__(kWarps * 32, PGSAG_BWD_MINB) k_render_bwd(
    const pgsag_view* __restrict__ views, const float4* __restrict__ rec,
    const uint32_t* __restrict__ dup_pairs, const uint2* __restrict__ ranges,
    const uint4* __restrict__ act_tiles, uint32_t n_items, const uint32_t* __restrict__ px_list,
    Sched sched, const float4* __restrict__ out8, const uint4* __restrict__ aux,
    const float4* __restrict__ dout8, const float* __restrict__ ddepth, const float* __restrict__ dout_scale,
    float* __restrict__ grad2d, const int32_t* status) {
  constexpr int kRenderThreads = kWarps * 32;
  constexpr int kTilePix = kRenderThreads * kPPT;
  constexpr int kStagePerThread = kBatch / kRenderThreads;
  static_assert(kBatch % kRenderThreads == 0 && kStagePerThread >= 1, "batch must be a multiple of the CTA size");
  __shared__ Stage S;
  __shared__ uint32_t spair[kBatch];
  __shared__ float4 sacc[kBatch][4];
  __shared__ uint32_t s_item;
  __shared__ int s_max;
  if (status_bad(status)) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const float gscale = dout_scale ? __ldg(dout_scale) : 1.f;
  for (int i = threadIdx.x; i < kBatch; i += kRenderThreads)
    sacc[i][0] = sacc[i][1] = sacc[i][2] = sacc[i][3] = make_float4(0.f, 0.f, 0.f, 0.f);
  uint32_t iter = 0;
  for (;;) {
    const uint32_t t = next_tile(sched, iter, n_items, &s_item);
    if (t >= n_items) break;
    const TileInfo ti = load_tile(t, act_tiles, ranges);
    const ViewLite V = load_view_lite(views + ti.view);
    for (uint32_t r0 = 0; r0 < ti.npix; r0 += kTilePix) {
      // coordinate origin: the 32-pixel-aligned corner of the 32x32 cell holding
      // the tile (every supported tile lies in one cell), so offsets round the
      // same way whatever the tile size
      const int ox = ((int)ti.tx * V.tile_w) & ~31, oy = ((int)ti.ty * V.tile_h) & ~31;
      const Pix<kPPT> P = load_pixels<kPPT>(ti, r0, warp, lane, V.width, ox, oy, px_list);
      const float4 cbox = warp_pixel_box(P);
      BwdPix B[kPPT];
      int lane_last = -1;
#pragma unroll
      for (int k = 0; k < kPPT; ++k) {
        BwdPix& b = B[k];
        b.T = 1.f;
        b.last = -1;
        b.dC0 = b.dC1 = b.dC2 = b.dD = b.dN0 = b.dN1 = b.dN2 = b.dATf = 0.f;
        b.SC0 = b.SC1 = b.SC2 = b.SN0 = b.SN1 = b.SN2 = b.SD = 0.f;
        if (!P.has[k]) continue;
        const uint64_t gp = P.q[k];
        const uint4 ax = __ldg(aux + gp);
        b.T = __uint_as_float(ax.x);
        b.last = ax.z > 0 ? (int)ax.y : -1;
        const float4 g0 = __ldg(dout8 + 2 * gp), g1 = __ldg(dout8 + 2 * gp + 1);
        b.dC0 = gscale * g0.x;
        b.dC1 = gscale * g0.y;
        b.dC2 = gscale * g0.z;
        b.dD = gscale * g0.w;
        b.dN0 = gscale * g1.x;
        b.dN1 = gscale * g1.y;
        b.dN2 = gscale * g1.z;
        b.dATf = gscale * g1.w * b.T;
        if (ddepth != nullptr && ax.z > 0) {
          // Eq. 4: Depth = D / s, s = -N . r
          const float gd = gscale * __ldg(ddepth + gp);
          if (gd != 0.f) {
            const float4 o0 = __ldg(out8 + 2 * gp), o1 = __ldg(out8 + 2 * gp + 1);
            const float rx = (P.px[k] + (float)ox - V.cx) / V.fx, ry = (P.py[k] + (float)oy - V.cy) / V.fy;
            const float sdot = -(o1.x * rx + o1.y * ry + o1.z);
            if (sdot > kRayDotMin && o0.w > 0.f) {
              const float is = 1.f / sdot;
              b.dD += gd * is;
              const float kk = gd * o0.w * is * is;
              b.dN0 += kk * rx;
              b.dN1 += kk * ry;
              b.dN2 += kk;
            }
          }
        }
        lane_last = max(lane_last, b.last);
      }
      const int warp_last = warp_max_i(lane_last);
      if (threadIdx.x == 0) s_max = -1;
      __syncthreads();
      if (lane == 0) atomicMax(&s_max, warp_last);
      __syncthreads();
      const int cta_last = s_max;
      __syncthreads();
      for (int hi = cta_last; hi >= (int)ti.rbeg; hi -= kBatch) {
        const int lo = max((int)ti.rbeg, hi - kBatch + 1);
        const int nb = hi - lo + 1;
#pragma unroll
        for (int u = 0; u < kStagePerThread; ++u) {
          const int slot = threadIdx.x + u * kRenderThreads;
          if (slot < nb) stage(lo + slot, slot, dup_pairs, rec, (float)ox, (float)oy, S, spair);
        }
        __syncthreads();
        uint32_t rel[kBatch / 32];
        warp_relevance(S, min(nb, warp_last - lo + 1), cbox, lane, rel);
#pragma unroll 1
        for (int c = kBatch / 32 - 1; c >= 0; --c) {
         uint32_t m = rel[c];
         while (m) {
          const int bit = 31 - __clz(m);
          m &= ~(1u << bit);
          const int j = c * 32 + bit;
          const int idx = lo + j;
          const float4 q0 = S.g0[j];
          const float4 q1 = S.g1[j];
          const float thr = q1.z;
          float g[16];
#pragma unroll
          for (int k = 0; k < 16; ++k) g[k] = 0.f;
          int ncontrib = 0;
#pragma unroll
          for (int k = 0; k < kPPT; ++k) {
            BwdPix& b = B[k];
            if (idx > b.last) continue;
            float dx, dy, u, wq;
            const float pw = gauss_power(P.px[k], P.py[k], q0, q1.x, dx, dy, u, wq);
            if (!(pw >= thr)) continue;  // alpha < 1/255: not blended
            ++ncontrib;
            const float4 q2 = S.g2[j];
            const float4 q3 = S.g3[j];
            const float G = __expf(pw);
            const float raw = __fmul_rn(q1.y, G);
            const float alpha = fminf(raw, kAlphaMax);
            const float oma = 1.f - alpha;
            const float roma = __fdividef(1.f, oma);  // 1 <= 1/(1-alpha) <= 100
            b.T *= roma;                              // transmittance in front of this Gaussian
            const float w = alpha * b.T;
            const float c0 = q2.x, c1 = q2.y, c2 = q2.z, d = q2.w, n0 = q3.x, n1 = q3.y, n2 = q3.z;
            float dalpha = b.T * ((c0 - b.SC0) * b.dC0 + (c1 - b.SC1) * b.dC1 + (c2 - b.SC2) * b.dC2 +
                                  (d - b.SD) * b.dD + (n0 - b.SN0) * b.dN0 + (n1 - b.SN1) * b.dN1 +
                                  (n2 - b.SN2) * b.dN2);
            dalpha += b.dATf * roma;
            // advance the suffix sums past this Gaussian: S <- a x + (1 - a) S
            b.SC0 = fmaf(alpha, c0 - b.SC0, b.SC0);
            b.SC1 = fmaf(alpha, c1 - b.SC1, b.SC1);
            b.SC2 = fmaf(alpha, c2 - b.SC2, b.SC2);
            b.SN0 = fmaf(alpha, n0 - b.SN0, b.SN0);
            b.SN1 = fmaf(alpha, n1 - b.SN1, b.SN1);
            b.SN2 = fmaf(alpha, n2 - b.SN2, b.SN2);
            b.SD = fmaf(alpha, d - b.SD, b.SD);
            g[6] += w * b.dC0;
            g[7] += w * b.dC1;
            g[8] += w * b.dC2;
            g[9] += w * b.dD;
            g[10] += w * b.dN0;
            g[11] += w * b.dN1;
            g[12] += w * b.dN2;
            if (raw < kAlphaMax) {
              g[5] += dalpha * G;                // d alpha / d o
              const float dp = dalpha * alpha;   // d alpha / d power
              // power = -1/2 (u^2 + w^2), u = l11 dx + l21 dy, w = l22 dy, d = p - m
              g[0] += dp * u * q0.z;
              g[1] += dp * (u * q0.w + wq * q1.x);
              g[2] -= dp * u * dx;
              g[3] -= dp * u * dy;
              g[4] -= dp * wq * dy;
            }
          }
          const uint32_t cm = __ballot_sync(kFull, ncontrib > 0);
          if (cm) {
            float* acc = reinterpret_cast<float*>(sacc[j]);
            if (__popc(cm) <= kDirect) {
              // few contributing lanes: add their values directly
              if (ncontrib > 0) {
#pragma unroll
                for (int k = 0; k < 13; ++k) atomicAdd(acc + k, g[k]);
              }
            } else {
              const float tot = warp_reduce_scatter16(g, lane);
              const int k = lane >> 1;
              if (!(lane & 1) && k < 13) atomicAdd(acc + k, tot);
            }
          }
         }
        }
        __syncthreads();
        // one float4 atomic per 4 gradient values per Gaussian for the whole tile
#pragma unroll
        for (int u = 0; u < kStagePerThread; ++u) {
          const int slot = threadIdx.x + u * kRenderThreads;
          if (slot < nb) {
            float* gdst = grad2d + 16ull * spair[slot];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              const float4 a = sacc[slot][q];
              if (a.x != 0.f || a.y != 0.f || a.z != 0.f || a.w != 0.f) {
                atomicAdd(reinterpret_cast<float4*>(gdst) + q, a);
                sacc[slot][q] = make_float4(0.f, 0.f, 0.f, 0.f);
              }
            }
          }
        }
        __syncthreads();
      }
    }
  }
}

}  // namespace pgsag

using namespace pgsag;

static int launch_cfg(const pgsag_sched* sched, uint32_t n_items, Sched& s, unsigned& blocks) {
  s.order = sched ? sched->order : nullptr;
  s.counter = sched ? sched->counter : nullptr;
  if (s.counter) {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return PGSAG_ERR_CUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return PGSAG_ERR_CUDA;
    const int per = sched->ctas_per_sm > 0 ? sched->ctas_per_sm : 4;
    blocks = (unsigned)(sms * per);
  } else {
    blocks = n_items;
  }
  return PGSAG_OK;
}

extern "C" int pgsag_render_fwd(uint32_t n_views, const pgsag_view* views, const float* rec,
                                const uint32_t* dup_pairs, const void* ranges, const void* act_tiles,
                                uint32_t n_active, const uint32_t* px_list, const pgsag_sched* sched,
                                float* out8, float* depth, void* aux, int32_t* status, void* stream) {
  if (n_views == 0 || n_views > PGSAG_MAX_VIEWS) return PGSAG_ERR_UNSUPPORTED;
  if (!views || !status) return PGSAG_ERR_ARG;
  if (n_active == 0) return PGSAG_OK;
  if (!rec || !ranges || !act_tiles || !px_list || !out8 || !depth || !aux) return PGSAG_ERR_ARG;
  if (((uintptr_t)rec | (uintptr_t)out8 | (uintptr_t)aux | (uintptr_t)act_tiles) & 15u) return PGSAG_ERR_ARG;
  Sched s;
  unsigned blocks;
  int r = launch_cfg(sched, n_active, s, blocks);
  if (r) return r;
  cudaStream_t st = (cudaStream_t)stream;
  if (s.counter) PGSAG_CUDA(cudaMemsetAsync(s.counter, 0, sizeof(uint32_t), st));
  k_render_fwd<PGSAG_FWD_WARPS, PGSAG_FWD_PPT><<<blocks, PGSAG_FWD_WARPS * 32, 0, st>>>(views, (const float4*)rec, dup_pairs, (const uint2*)ranges,
                                                  (const uint4*)act_tiles, n_active, px_list, s, (float4*)out8, depth,
                                                  (uint4*)aux, status);
  PGSAG_CHECK_LAUNCH();
  return PGSAG_OK;
}

extern "C" int pgsag_render_bwd(uint32_t n_views, const pgsag_view* views, const float* rec,
                                const uint32_t* dup_pairs, const void* ranges, const void* act_tiles,
                                uint32_t n_active, const uint32_t* px_list, const pgsag_sched* sched,
                                const float* out8, const void* aux, const float* dout8, const float* ddepth,
                                const float* dout_scale, uint32_t n_pairs, float* grad2d, int32_t* status,
                                void* stream) {
  if (n_views == 0 || n_views > PGSAG_MAX_VIEWS) return PGSAG_ERR_UNSUPPORTED;
  if (!views || !status) return PGSAG_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  if (n_pairs) {
    if (!grad2d || ((uintptr_t)grad2d & 15u)) return PGSAG_ERR_ARG;
    PGSAG_CUDA(cudaMemsetAsync(grad2d, 0, (size_t)n_pairs * PGSAG_GRAD2D_FLOATS * sizeof(float), st));
  }
  if (n_active == 0) return PGSAG_OK;
  if (!rec || !ranges || !act_tiles || !px_list || !out8 || !aux || !dout8 || !grad2d) return PGSAG_ERR_ARG;
  if (((uintptr_t)rec | (uintptr_t)out8 | (uintptr_t)aux | (uintptr_t)dout8 | (uintptr_t)act_tiles) & 15u)
    return PGSAG_ERR_ARG;
  Sched s;
  unsigned blocks;
  int r = launch_cfg(sched, n_active, s, blocks);
  if (r) return r;
  if (s.counter) PGSAG_CUDA(cudaMemsetAsync(s.counter, 0, sizeof(uint32_t), st));
  k_render_bwd<PGSAG_BWD_WARPS, PGSAG_BWD_PPT, PGSAG_BWD_DIRECT><<<blocks, PGSAG_BWD_WARPS * 32, 0, st>>>(views, (const float4*)rec, dup_pairs, (const uint2*)ranges,
                                                  (const uint4*)act_tiles, n_active, px_list, s, (const float4*)out8,
                                                  (const uint4*)aux, (const float4*)dout8, ddepth, dout_scale, grad2d,
                                                  status);
  PGSAG_CHECK_LAUNCH();
  return PGSAG_OK;
}
