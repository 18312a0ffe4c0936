// Masked tile rendering, forward (Sec. 3.1 Eq. 1-4) and adjoint.
//
// Work item = one active tile, handled by one CTA of 4 warps.  The tile's
// rendered (mask-dilated) pixels are compacted; each lane takes 2 of them (more
// rounds for tiles larger than 256 pixels) and evaluates both with packed
// two-lane FP32 instructions (fma/add/mul .f32x2).  The tile's depth-sorted Gaussians
// are staged through shared memory in batches of 128 (64-byte records,
// coalesced), then each warp walks the batch, skipping -- as a warp-uniform
// branch -- every Gaussian whose alpha >= 1/255 box misses the bounding box of
// the warp's pixels.  A pair is rejected before the exponential when the
// exponent is below the Gaussian's threshold -ln(255 o) (alpha < 1/255).  The
// forward stops a batch loop when every warp of the CTA has terminated
// (__syncthreads_or).  The adjoint re-walks the list back to front from the
// CTA's last blended Gaussian, recovers T by division, carries one suffix
// scalar per pixel (see BwdPix), reduces each Gaussian's 13 gradient values
// across the warp with 16 shuffles, sums the warps in shared memory and issues
// one float4 atomic per 4 values per tile; its prologue does the loss's
// deferred Eq. 8 gather and the Eq. 4 chain from the depth output.
#include "common.cuh"

namespace pgsag {

// Launch shape (compile-time; the defaults are the best measured on B300 for the
// 5472x3648 aerial workload): warps per CTA (one CTA per active tile), Gaussians
// staged per batch and the number of resident CTAs per SM the register
// allocation must allow (forward 10, adjoint 9).  Each lane renders 2 pixels.
#ifndef PGSAG_FWD_WARPS
#define PGSAG_FWD_WARPS 4
#endif
#ifndef PGSAG_BWD_WARPS
#define PGSAG_BWD_WARPS 4
#endif
#ifndef PGSAG_BATCH
#define PGSAG_BATCH 128
#endif
#ifndef PGSAG_FWD_MINB
#define PGSAG_FWD_MINB 9  // resident CTAs per SM the register budget must allow (56 registers)
#endif
#ifndef PGSAG_BWD_MINB
#define PGSAG_BWD_MINB 9
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

// Next tile for this CTA (adjoint): plain grid (one tile per CTA, known to every thread)
// or a persistent loop over an atomic work counter (thread 0 fetches, one
// barrier publishes; the slot alternates between calls so that it is written
// again only after every thread has passed the next call's barrier), optionally
// through a processing order.  Called by all threads.
struct Sched {
  const uint32_t* order;
  uint32_t* counter;
};

__device__ __forceinline__ uint32_t next_tile(const Sched& s, uint32_t& iter, uint32_t n_items,
                                              uint32_t* s_item) {
  if (!s.counter) {
    const uint32_t c = iter++ == 0 ? blockIdx.x : n_items;
    return (c < n_items && s.order) ? __ldg(s.order + c) : c;
  }
  uint32_t* slot = s_item + (iter & 1u);
  if (threadIdx.x == 0) {
    uint32_t c = atomicAdd(s.counter, 1u);
    if (c < n_items && s.order) c = __ldg(s.order + c);
    *slot = c;
  }
  __syncthreads();
  ++iter;
  return *slot;
}

// The same with the tile index always broadcast through shared memory by thread
// 0 (two barriers): the forward uses this form, which keeps the scheduling state
// out of the other threads' registers (the per-thread form makes the forward
// spill at its 48-register budget: 0.300 -> 0.324 ms at config 1).
__device__ __forceinline__ uint32_t next_tile_bcast(const Sched& s, uint32_t& iter, uint32_t n_items,
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
// r0 + (2 warp + k) * 32 + lane (k = 0, 1) of the tile's compacted pixel list,
// so a warp covers two consecutive 32-pixel runs.  The two pixels of a lane are
// processed together with packed two-lane FP32 instructions (x = pixel 0,
// y = pixel 1).  Pixel centres are kept relative to an origin (ox, oy) near the
// tile, exactly, like the staged Gaussian centres, so that offsets do not lose
// precision to the image size.
struct Pix {
  bool has0, has1;
  uint32_t q0, q1;  // compact index (position in px_list): per-pixel arrays
  float2 px, py;    // centres minus tile origin
};

__device__ __forceinline__ Pix load_pixels(const TileInfo& ti, uint32_t r0, int warp, int lane, int width, int ox,
                                           int oy, const uint32_t* __restrict__ px_list) {
  Pix P;
  float c[2][2];
  bool has[2];
  uint32_t q[2];
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const uint32_t li = r0 + (uint32_t)((warp * 2 + k) * 32 + lane);
    has[k] = li < ti.npix;
    q[k] = ti.px_first + li;
    const uint32_t pix = has[k] ? __ldg(px_list + q[k]) : 0u;
    const uint32_t yy = pix / (uint32_t)width;
    c[k][0] = (float)((int)(pix - yy * (uint32_t)width) - ox) + 0.5f;
    c[k][1] = (float)((int)yy - oy) + 0.5f;
  }
  P.has0 = has[0];
  P.has1 = has[1];
  P.q0 = q[0];
  P.q1 = q[1];
  P.px = make_float2(c[0][0], c[1][0]);
  P.py = make_float2(c[0][1], c[1][1]);
  return P;
}

// Bounding box of the warp's valid pixel centres (warp-uniform result).
__device__ __forceinline__ float4 warp_pixel_box(const Pix& P) {
  float x0 = 3.0e38f, x1 = -3.0e38f, y0 = 3.0e38f, y1 = -3.0e38f;
  if (P.has0) {
    x0 = fminf(x0, P.px.x);
    x1 = fmaxf(x1, P.px.x);
    y0 = fminf(y0, P.py.x);
    y1 = fmaxf(y1, P.py.x);
  }
  if (P.has1) {
    x0 = fminf(x0, P.px.y);
    x1 = fmaxf(x1, P.px.y);
    y0 = fminf(y0, P.py.y);
    y1 = fmaxf(y1, P.py.y);
  }
  return make_float4(warp_min_f(x0), warp_max_f(x1), warp_min_f(y0), warp_max_f(y1));
}

__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }

// gauss_power for the lane's two pixels with packed instructions.  Each half is
// the same sequence of correctly rounded operations as the scalar form (x - m
// is x + (-m)), so forward and adjoint obtain identical exponents.
__device__ __forceinline__ float2 gauss_power2(float2 px, float2 py, float4 r0, float l22, float2& dx, float2& dy,
                                               float2& u, float2& w) {
  dx = __fadd2_rn(px, f2(-r0.x));
  dy = __fadd2_rn(py, f2(-r0.y));
  u = __ffma2_rn(f2(r0.z), dx, __fmul2_rn(f2(r0.w), dy));
  w = __fmul2_rn(f2(l22), dy);
  return __fmul2_rn(f2(-0.5f), __ffma2_rn(u, u, __fmul2_rn(w, w)));
}

// Shared-memory image of a batch of staged Gaussians, packed by use:
// g0 = {mx, my, l11, l21}, g1 = {l22, o, thr, -}, g2 = {r, g, b, d}, g3 = {nx, ny, nz, -}
// (l11, l21, l22: Cholesky factor of the conic); for the warps' relevance test
// q = {qa, qb, qc, bound}, c = {mx, my, 1/qa, 1/qc} (see EllipseTest).
struct Stage {
  float4 g0[kBatch], g1[kBatch], g2[kBatch], g3[kBatch], q[kBatch], c[kBatch];
};

// The centre is staged relative to the origin (ox, oy): (integer part - origin)
// is exact, then the fraction is added.
__device__ __forceinline__ void stage(uint32_t i, int slot, const uint32_t* __restrict__ dup_pairs,
                                      const float4* __restrict__ rec, float ox, float oy, Stage& S,
                                      uint32_t* spair) {
  const uint32_t p = __ldg(dup_pairs + i);
  const float4* r = rec + 4ull * p;
  const float4 r0 = __ldg(r + 0), r1 = __ldg(r + 1), r2 = __ldg(r + 2), r3 = __ldg(r + 3);
  const float mx = __fadd_rn(__fsub_rn(r0.x, ox), r3.z), my = __fadd_rn(__fsub_rn(r0.y, oy), r3.w);
  S.g0[slot] = make_float4(mx, my, r0.z, r0.w);
  S.g1[slot] = make_float4(r1.x, r1.y, r3.y, 0.f);
  S.g2[slot] = make_float4(r1.z, r1.w, r2.x, r2.y);
  S.g3[slot] = make_float4(r2.z, r2.w, r3.x, 0.f);
  const EllipseTest e = ellipse_test(r0.z, r0.w, r1.x, r3.y);
  S.q[slot] = make_float4(e.qa, e.qb, e.qc, e.bound);
  S.c[slot] = make_float4(mx, my, e.iqa, e.iqc);
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
      const float4 q = S.q[j], c = S.c[j];
      const EllipseTest e = {q.x, q.y, q.z, c.z, c.w, q.w};
      hit = ellipse_rect_hit(e, cbox.x - c.x, cbox.y - c.x, cbox.z - c.y, cbox.w - c.y);
    }
    rel[c] = __ballot_sync(kFull, hit);
  }
}

// Forward outputs of one pixel: {C, D}, {N, A = 1 - T}, the Eq. 4 depth and
// {T, last blended, count, soft count (kSoft) or the ray-plane dot s of Eq. 4}.
// (x, y) is the pixel centre in image coordinates.
template <bool kSoft>
__device__ __forceinline__ void write_pixel(uint64_t gp, float4 cd, float4 nt, uint32_t last, uint32_t cnt,
                                            float soft, float x, float y, const ViewLite& V,
                                            float4* __restrict__ out8, float* __restrict__ depth,
                                            uint4* __restrict__ aux) {
  out8[2 * gp + 0] = cd;
  out8[2 * gp + 1] = make_float4(nt.x, nt.y, nt.z, 1.f - nt.w);
  // Eq. 4: ray-plane depth
  const float rx = (x - V.cx) * V.ifx, ry = (y - V.cy) * V.ify;
  const float sdot = -(nt.x * rx + nt.y * ry + nt.z);
  const bool valid = cnt > 0 && sdot > kRayDotMin && cd.w > 0.f;
  depth[gp] = valid ? cd.w / sdot : 0.f;
  aux[gp] = make_uint4(__float_as_uint(nt.w), last, cnt, __float_as_uint(kSoft ? soft : sdot));
}

// kSoft: also sum the blended alphas per pixel (the soft count g~ of Eq. 9's
// differentiable form) into aux.w.
template <int kWarps, bool kSoft>
__global__ void __launch_bounds__(kWarps * 32, PGSAG_FWD_MINB) k_render_fwd(
    const pgsag_view* __restrict__ views, const float4* __restrict__ rec,
    const uint32_t* __restrict__ dup_pairs, const uint2* __restrict__ ranges,
    const uint4* __restrict__ act_tiles, uint32_t n_items, const uint32_t* __restrict__ px_list,
    Sched sched, float4* __restrict__ out8, float* __restrict__ depth, uint4* __restrict__ aux,
    const int32_t* status) {
  constexpr int kRenderThreads = kWarps * 32;
  constexpr int kTilePix = kRenderThreads * 2;
  constexpr int kStagePerThread = kBatch / kRenderThreads;
  static_assert(kBatch % kRenderThreads == 0 && kStagePerThread >= 1, "batch must be a multiple of the CTA size");
  __shared__ Stage S;
  __shared__ uint32_t s_item;
  if (status_bad(status)) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t iter = 0;
  for (;;) {
    const uint32_t t = next_tile_bcast(sched, iter, n_items, &s_item);
    if (t >= n_items) break;
    const TileInfo ti = load_tile(t, act_tiles, ranges);
    const ViewLite V = load_view_lite(views + ti.view);
    // coordinate origin: the 32-pixel-aligned corner of the 32x32 cell holding
    // the tile (every supported tile lies in one cell), so offsets round the
    // same way whatever the tile size
    const int ox = ((int)ti.tx * V.tile_w) & ~31, oy = ((int)ti.ty * V.tile_h) & ~31;
    // the first batch is staged before the pixels are loaded, so that the two
    // dependent global-load chains overlap; `staged` = S holds the batch at rbeg
    bool staged = false;
    if (ti.rbeg < ti.rend) {
      const uint32_t nb = min((uint32_t)kBatch, ti.rend - ti.rbeg);
#pragma unroll
      for (int u = 0; u < kStagePerThread; ++u) {
        const uint32_t slot = threadIdx.x + u * kRenderThreads;
        if (slot < nb) stage(ti.rbeg + slot, slot, dup_pairs, rec, (float)ox, (float)oy, S, nullptr);
      }
      staged = true;
    }
    for (uint32_t r0 = 0; r0 < ti.npix; r0 += kTilePix) {
      const Pix P = load_pixels(ti, r0, warp, lane, V.width, ox, oy, px_list);
      const float4 cbox = warp_pixel_box(P);
      float2 T = f2(1.f), C0 = f2(0.f), C1 = f2(0.f), C2 = f2(0.f), D = f2(0.f), N0 = f2(0.f), N1 = f2(0.f),
             N2 = f2(0.f);
      uint32_t last0 = 0, last1 = 0, cnt0 = 0, cnt1 = 0;
      float2 Gs = f2(0.f);  // soft count (kSoft)
      bool done0 = !P.has0, done1 = !P.has1;
      bool all_done = done0 && done1;
      for (uint32_t base = ti.rbeg; base < ti.rend; base += kBatch) {
        // this barrier also publishes an early-staged first batch
        if (!__syncthreads_or(!all_done)) break;
        const uint32_t nb = min((uint32_t)kBatch, ti.rend - base);
        if (!(staged && base == ti.rbeg)) {
#pragma unroll
          for (int u = 0; u < kStagePerThread; ++u) {
            const uint32_t slot = threadIdx.x + u * kRenderThreads;
            if (slot < nb) stage(base + slot, slot, dup_pairs, rec, (float)ox, (float)oy, S, nullptr);
          }
          staged = base == ti.rbeg;
          __syncthreads();
        }
        if (!__any_sync(kFull, !all_done)) continue;
        uint32_t rel[kBatch / 32];
        warp_relevance(S, (int)nb, cbox, lane, rel);
        // the whole warp walks the relevant Gaussians; lanes that are done take
        // no part through their masks (the 4 chunks unrolled: rel stays in
        // registers; 2% faster than a rolled loop here, not in the adjoint)
#pragma unroll
        for (int c = 0; c < kBatch / 32; ++c) {
          uint32_t m = rel[c];
          while (m) {
            const int j = c * 32 + __ffs(m) - 1;
            m &= m - 1;
            const float4 q0 = S.g0[j];
            const float4 q1 = S.g1[j];
            float2 dx, dy, u, w2;
            const float2 pw = gauss_power2(P.px, P.py, q0, q1.x, dx, dy, u, w2);
            bool a0 = !done0 && pw.x >= q1.z;  // alpha >= 1/255
            bool a1 = !done1 && pw.y >= q1.z;
            // warp-uniform: the blend runs for the whole warp with masked weights
            // (also when no lane enters -- 1% of the events: a vote per event
            // cost more than it saved)
            const float2 alpha = make_float2(fminf(__fmul_rn(q1.y, __expf(pw.x)), kAlphaMax),
                                             fminf(__fmul_rn(q1.y, __expf(pw.y)), kAlphaMax));
            const float2 test = __fmul2_rn(T, __ffma2_rn(alpha, f2(-1.f), f2(1.f)));  // T (1 - alpha)
            if (a0 && test.x < kTMin) {
              done0 = true;
              a0 = false;
            }
            if (a1 && test.y < kTMin) {
              done1 = true;
              a1 = false;
            }
            float2 w = __fmul2_rn(alpha, T);
            w.x = a0 ? w.x : 0.f;
            w.y = a1 ? w.y : 0.f;
            const float4 q2 = S.g2[j];
            const float4 q3 = S.g3[j];
            C0 = __ffma2_rn(w, f2(q2.x), C0);
            C1 = __ffma2_rn(w, f2(q2.y), C1);
            C2 = __ffma2_rn(w, f2(q2.z), C2);
            D = __ffma2_rn(w, f2(q2.w), D);
            N0 = __ffma2_rn(w, f2(q3.x), N0);
            N1 = __ffma2_rn(w, f2(q3.y), N1);
            N2 = __ffma2_rn(w, f2(q3.z), N2);
            if constexpr (kSoft) Gs = __fadd2_rn(Gs, make_float2(a0 ? alpha.x : 0.f, a1 ? alpha.y : 0.f));
            if (a0) {
              T.x = test.x;
              last0 = base + j;
              ++cnt0;
            }
            if (a1) {
              T.y = test.y;
              last1 = base + j;
              ++cnt1;
            }
          }
          // leave the batch once every pixel of the warp has terminated (checked
          // per 32 Gaussians: a vote per Gaussian cost more than the Gaussians a
          // finished warp still walks; terminated lanes take part with zero weight)
          if (__all_sync(kFull, done0 && done1)) {
            all_done = true;
            break;
          }
        }
      }
      if (P.has0)
        write_pixel<kSoft>(P.q0, make_float4(C0.x, C1.x, C2.x, D.x), make_float4(N0.x, N1.x, N2.x, T.x), last0, cnt0,
                    Gs.x, P.px.x + (float)ox, P.py.x + (float)oy, V, out8, depth, aux);
      if (P.has1)
        write_pixel<kSoft>(P.q1, make_float4(C0.y, C1.y, C2.y, D.y), make_float4(N0.y, N1.y, N2.y, T.y), last1, cnt1,
                    Gs.y, P.px.y + (float)ox, P.py.y + (float)oy, V, out8, depth, aux);
    }
  }
}

// Reduce 16 per-lane values over the warp; afterwards lane l holds the warp total
// of value (l >> 1) (lanes l and l^1 hold the same total).  16 shuffles; the
// additions of the first three levels run in pairs (add.f32x2).
__device__ __forceinline__ float warp_reduce_scatter16(const float v[16], int lane) {
  float a8[8];
  {
    const bool hi = lane & 16;
#pragma unroll
    for (int i = 0; i < 8; i += 2) {
      const float2 send = hi ? make_float2(v[i], v[i + 1]) : make_float2(v[i + 8], v[i + 9]);
      const float2 keep = hi ? make_float2(v[i + 8], v[i + 9]) : make_float2(v[i], v[i + 1]);
      const float2 got = make_float2(__shfl_xor_sync(kFull, send.x, 16), __shfl_xor_sync(kFull, send.y, 16));
      const float2 sum = __fadd2_rn(keep, got);
      a8[i] = sum.x;
      a8[i + 1] = sum.y;
    }
  }
  float a4[4];
  {
    const bool hi = lane & 8;
#pragma unroll
    for (int i = 0; i < 4; i += 2) {
      const float2 send = hi ? make_float2(a8[i], a8[i + 1]) : make_float2(a8[i + 4], a8[i + 5]);
      const float2 keep = hi ? make_float2(a8[i + 4], a8[i + 5]) : make_float2(a8[i], a8[i + 1]);
      const float2 got = make_float2(__shfl_xor_sync(kFull, send.x, 8), __shfl_xor_sync(kFull, send.y, 8));
      const float2 sum = __fadd2_rn(keep, got);
      a4[i] = sum.x;
      a4[i + 1] = sum.y;
    }
  }
  float a2[2];
  {
    const bool hi = lane & 4;
    const float2 send = hi ? make_float2(a4[0], a4[1]) : make_float2(a4[2], a4[3]);
    const float2 keep = hi ? make_float2(a4[2], a4[3]) : make_float2(a4[0], a4[1]);
    const float2 got = make_float2(__shfl_xor_sync(kFull, send.x, 4), __shfl_xor_sync(kFull, send.y, 4));
    const float2 sum = __fadd2_rn(keep, got);
    a2[0] = sum.x;
    a2[1] = sum.y;
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

// Adjoint state of the lane's two pixels (x = pixel 0, y = pixel 1).  For a
// blended Gaussian i, dL/dalpha_i needs sum_ch (x_ch,i - S_ch,i) dL/dX_ch with the
// suffix sums S_ch,i = sum_{j>i} x_ch,j a_j prod_{i<l<j} (1 - a_l) of the 7
// channels (colour, plane distance, normal) behind it.  The upstream gradients
// dL/dX_ch are constant along the pixel's list, so only Q = sum_ch S_ch dL/dX_ch
// is needed, and it obeys the same recurrence as each S_ch:
// Q <- Q + a (P - Q), P = sum_ch x_ch dL/dX_ch of the Gaussian just passed.
struct BwdPix {
  float2 T;
  int last0, last1;
  float2 dC0, dC1, dC2, dD, dN0, dN1, dN2, dATf;  // dATf = dL/dA * T_final
  float2 Q;
  float2 dG;  // dL/d(soft count) (objective Eq. 11)
};

// Deferred Eq. 8 adjoint (the loss's second pass, run here): dL/dP of the pixel's
// back-projected point P = Depth r, gathered from the 4 neighbours whose central
// differences used it (their dL/da, dL/db in the loss scratch), as dL/dDepth;
// the rendered-normal gradient from the loss is scaled by lambda / |V|
// (`scale`, ban_scale of the pixel's view).
// Returns dL/dDepth; scales gn (dL/dN) in place.  q: the pixel's compact index.
__device__ __forceinline__ float ban_scale(const pgsag_ban_gather& bg, uint32_t view) {
  const double nV = bg.acc[8 * view + 2];
  return nV > 0.0 ? (float)((double)bg.lambda_ban / nV) : 0.f;
}

__device__ __forceinline__ float ban_gather(const pgsag_ban_gather& bg, float scale, uint64_t q, float rx, float ry,
                                            float3& gn) {
  gn.x *= scale;
  gn.y *= scale;
  gn.z *= scale;
  // this pixel is P[y+1] of its up neighbour, P[y-1] of the down one, P[x+1] of
  // the left one, P[x-1] of the right one; every rendered neighbour's scratch row
  // is written by the loss (zero off the mask), so no flag test is needed
  const uint4 nb = __ldg(reinterpret_cast<const uint4*>(bg.nbr) + q);
  const uint32_t qn[4] = {nb.x, nb.y, nb.z, nb.w};
  const float sg[4] = {1.f, -1.f, 1.f, -1.f};
  const int off[4] = {0, 0, 3, 3};
  bool mk[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) mk[k] = qn[k] != 0xffffffffu;
  float dP0 = 0.f, dP1 = 0.f, dP2 = 0.f;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    if (!mk[k]) continue;
    const float* sc = bg.scratch + 6ull * qn[k] + off[k];
    dP0 += sg[k] * __ldg(sc + 0);
    dP1 += sg[k] * __ldg(sc + 1);
    dP2 += sg[k] * __ldg(sc + 2);
  }
  return scale * (dP0 * rx + dP1 * ry + dP2);  // P = Depth r, r = (rx, ry, 1)
}

// Upstream gradient of one pixel (scaled), with the depth output's gradient
// (given, or gathered from the Eq. 8 loss) folded into dD and dN through Eq. 4
// (Depth = D / s, s = -N . r).
__device__ __forceinline__ void load_upstream(uint64_t gp, float px, float py, int ox, int oy, const ViewLite& V,
                                              uint32_t view, float gscale, const uint4* __restrict__ aux,
                                              const float4* __restrict__ dout8, const float* __restrict__ ddepth,
                                              bool use_ban, const pgsag_ban_gather& ban, float bscale,
                                              const float4* __restrict__ out8, float v[10], int& last,
                                              bool soft, float gscale_gc) {
  const uint4 ax = __ldg(aux + gp);
  // Eq. 4 chain from the depth output and the ray-plane dot s: aux.w holds s
  // under the default objective; under Eq. 11 (aux.w = soft count) s comes from
  // the rendered normal, the second half of the pixel's out8 record
  const bool dep_route = ban.depth != nullptr;
  const float dep = dep_route ? __ldg(ban.depth + gp) : 0.f;
  const float4 nrm = (dep_route && soft) ? __ldg(out8 + 2 * gp + 1) : make_float4(0.f, 0.f, 0.f, 0.f);
  v[9] = 0.f;
  if (soft) {
    // Eq. 9 with the soft count: L_GC = std_i(x_i), x_i = g~_i / w_i over the
    // view's rendered pixels; dL/dg~_i = (lambda / (n sigma)) (x_i - mean) / w_i,
    // with {lambda / (n sigma), mean} per view from the loss pass
    const float2 cm = *reinterpret_cast<const float2*>(ban.acc + 8 * view + 3);
    const float iw = __fdividef(1.f, __ldg(ban.gc_weight + gp));  // w >= 1
    v[9] = gscale_gc * cm.x * (__uint_as_float(ax.w) * iw - cm.y) * iw;
  }
  const float T = __uint_as_float(ax.x);
  last = ax.z > 0 ? (int)ax.y : -1;
  const float4 g0 = __ldg(dout8 + 2 * gp), g1 = __ldg(dout8 + 2 * gp + 1);
  const float rx = (px + (float)ox - V.cx) * V.ifx, ry = (py + (float)oy - V.cy) * V.ify;
  float3 gn = make_float3(g1.x, g1.y, g1.z);
  float gd = ddepth != nullptr ? __ldg(ddepth + gp) : 0.f;
  if (use_ban) {
    gd += ban_gather(ban, bscale, gp, rx, ry, gn);
  }
  v[0] = gscale * g0.x;
  v[1] = gscale * g0.y;
  v[2] = gscale * g0.z;
  v[3] = gscale * g0.w;
  v[4] = gscale * gn.x;
  v[5] = gscale * gn.y;
  v[6] = gscale * gn.z;
  v[7] = gscale * g1.w * T;
  v[8] = T;
  if (ax.z > 0) {
    gd *= gscale;
    if (gd != 0.f && dep_route) {
      // Depth = D / s > 0 exactly when the pixel is valid; dDepth/dD = 1 / s,
      // dDepth/dN = D / s^2 r = Depth / s r (1 / s by the fast reciprocal:
      // s is in (1e-8, 2] on a valid pixel, and the exact division's
      // multi-instruction sequence cost the adjoint 8 us)
      if (dep > 0.f) {
        const float is = __fdividef(1.f, soft ? -(nrm.x * rx + nrm.y * ry + nrm.z) : __uint_as_float(ax.w));
        v[3] += gd * is;
        const float kk = gd * dep * is;
        v[4] += kk * rx;
        v[5] += kk * ry;
        v[6] += kk;
      }
    } else if (gd != 0.f) {
      const float4 o0 = __ldg(out8 + 2 * gp), o1 = __ldg(out8 + 2 * gp + 1);
      const float sdot = -(o1.x * rx + o1.y * ry + o1.z);
      if (sdot > kRayDotMin && o0.w > 0.f) {
        const float is = __fdividef(1.f, sdot);
        v[3] += gd * is;
        const float kk = gd * o0.w * is * is;
        v[4] += kk * rx;
        v[5] += kk * ry;
        v[6] += kk;
      }
    }
  }
}

// kSoft: objective Eq. 11 -- the loss gradients get the (1 - lambda) factor and
// every blended alpha the soft-count GC-load gradient dL/dg~ of its pixel.
// Buffers the adjoint's CTAs set to zero on the side (pgsag_clear): their
// float4 bodies, laid end to end (buffer i holds units [start[i], start[i+1])),
// are cut into one share of `per` units per CTA (32-bit: the host checks the
// range); the at most 3 trailing floats of a buffer are cleared by CTA 0.
struct ClearJob {
  float4* p[PGSAG_CLEAR_MAX];
  uint32_t start[PGSAG_CLEAR_MAX + 1];
  uint32_t per;
  float* tail[PGSAG_CLEAR_MAX];
  uint32_t n_tail[PGSAG_CLEAR_MAX];
  bool on;
};

// Streaming stores (evict-first in L2): they drain while the CTA renders and
// leave the lists and records the adjoint re-reads in L2.
__device__ __forceinline__ void clear_share(const ClearJob& cj) {
  if (blockIdx.x == 0 && threadIdx.x < 3) {
#pragma unroll
    for (int i = 0; i < PGSAG_CLEAR_MAX; ++i)
      if (threadIdx.x < cj.n_tail[i]) cj.tail[i][threadIdx.x] = 0.f;
  }
  const uint32_t lo = blockIdx.x * cj.per, hi = min(cj.start[PGSAG_CLEAR_MAX], lo + cj.per);
#pragma unroll
  for (int i = 0; i < PGSAG_CLEAR_MAX; ++i) {
    const uint32_t b = min(hi, cj.start[i + 1]);
    for (uint32_t k = max(lo, cj.start[i]) + threadIdx.x; k < b; k += blockDim.x)
      __stcs(cj.p[i] + (k - cj.start[i]), make_float4(0.f, 0.f, 0.f, 0.f));
  }
}

template <int kWarps, bool kSoft>
__global__ void __launch_bounds__(kWarps * 32, PGSAG_BWD_MINB) k_render_bwd(
    const pgsag_view* __restrict__ views, const float4* __restrict__ rec,
    const uint32_t* __restrict__ dup_pairs, const uint2* __restrict__ ranges,
    const uint4* __restrict__ act_tiles, uint32_t n_items, const uint32_t* __restrict__ px_list,
    Sched sched, const float4* __restrict__ out8, const uint4* __restrict__ aux,
    const float4* __restrict__ dout8, const float* __restrict__ ddepth, const pgsag_ban_gather ban, bool use_ban,
    const float* __restrict__ dout_scale, float* __restrict__ grad2d, const ClearJob clear,
    const int32_t* status) {
  constexpr int kRenderThreads = kWarps * 32;
  constexpr int kTilePix = kRenderThreads * 2;
  constexpr int kStagePerThread = kBatch / kRenderThreads;
  static_assert(kBatch % kRenderThreads == 0 && kStagePerThread >= 1, "batch must be a multiple of the CTA size");
  __shared__ Stage S;
  __shared__ uint32_t spair[kBatch];
  __shared__ float4 sacc[kBatch][4];
  __shared__ uint32_t s_item[2];
  __shared__ int s_wmax[2][kWarps];
  uint32_t round = 0;
  if (status_bad(status)) return;
  if (clear.on) clear_share(clear);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const float gscale_in = dout_scale ? __ldg(dout_scale) : 1.f;
  // Eq. 11: the photometric / normal-loss gradients are scaled by (1 - lambda)
  const float gscale = kSoft ? gscale_in * (1.f - ban.lambda_gc) : gscale_in;
  for (int i = threadIdx.x; i < kBatch; i += kRenderThreads)
    sacc[i][0] = sacc[i][1] = sacc[i][2] = sacc[i][3] = make_float4(0.f, 0.f, 0.f, 0.f);
  uint32_t iter = 0;
  for (;;) {
    const uint32_t t = next_tile(sched, iter, n_items, s_item);
    if (t >= n_items) break;
    const TileInfo ti = load_tile(t, act_tiles, ranges);
    const ViewLite V = load_view_lite(views + ti.view);
    // the Eq. 8 scale lambda / |V| of the tile's view (once per tile, not per pixel)
    const float bscale = use_ban ? ban_scale(ban, ti.view) : 0.f;
    // coordinate origin: the 32-pixel-aligned corner of the 32x32 cell holding
    // the tile (every supported tile lies in one cell), so offsets round the
    // same way whatever the tile size
    const int ox = ((int)ti.tx * V.tile_w) & ~31, oy = ((int)ti.ty * V.tile_h) & ~31;
    // a list of at most one batch is staged whole before the pixels' upstream
    // gradients are loaded (the two dependent global-load chains overlap) and
    // serves every pixel round; slot j holds entry rbeg + j, as in the batch loop
    const bool one_batch = ti.rend - ti.rbeg <= (uint32_t)kBatch;
    if (one_batch) {
      const uint32_t nb = ti.rend - ti.rbeg;
#pragma unroll
      for (int u = 0; u < kStagePerThread; ++u) {
        const uint32_t slot = threadIdx.x + u * kRenderThreads;
        if (slot < nb) stage(ti.rbeg + slot, slot, dup_pairs, rec, (float)ox, (float)oy, S, spair);
      }
    }
    for (uint32_t r0 = 0; r0 < ti.npix; r0 += kTilePix) {
      const Pix P = load_pixels(ti, r0, warp, lane, V.width, ox, oy, px_list);
      const float4 cbox = warp_pixel_box(P);
      BwdPix B;
      {
        float v0[10] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 1.f, 0.f},
              v1[10] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 1.f, 0.f};
        B.last0 = B.last1 = -1;
        {
          // both pixels' loads in one basic block (a missing pixel reads the tile's
          // first row and its results are discarded)
          float w0[10], w1[10];
          int l0, l1;
          load_upstream(P.has0 ? P.q0 : ti.px_first, P.px.x, P.py.x, ox, oy, V, ti.view, gscale, aux, dout8, ddepth,
                        use_ban, ban, bscale, out8, w0, l0, kSoft, gscale_in);
          load_upstream(P.has1 ? P.q1 : ti.px_first, P.px.y, P.py.y, ox, oy, V, ti.view, gscale, aux, dout8, ddepth,
                        use_ban, ban, bscale, out8, w1, l1, kSoft, gscale_in);
#pragma unroll
          for (int k = 0; k < 10; ++k) {
            v0[k] = P.has0 ? w0[k] : v0[k];
            v1[k] = P.has1 ? w1[k] : v1[k];
          }
          B.last0 = P.has0 ? l0 : -1;
          B.last1 = P.has1 ? l1 : -1;
        }
        B.dC0 = make_float2(v0[0], v1[0]);
        B.dC1 = make_float2(v0[1], v1[1]);
        B.dC2 = make_float2(v0[2], v1[2]);
        B.dD = make_float2(v0[3], v1[3]);
        B.dN0 = make_float2(v0[4], v1[4]);
        B.dN1 = make_float2(v0[5], v1[5]);
        B.dN2 = make_float2(v0[6], v1[6]);
        B.dATf = make_float2(v0[7], v1[7]);
        B.T = make_float2(v0[8], v1[8]);
        B.dG = make_float2(v0[9], v1[9]);
        B.Q = f2(0.f);
      }
      // CTA maximum of the last blended entry: one slot per warp, double-buffered
      // by round so that one barrier suffices (the slots of a round are written
      // again two rounds later, past this round's barrier and the next one's)
      const int warp_last = warp_max_i(max(B.last0, B.last1));
      int* wmax = s_wmax[round & 1];
      if (lane == 0) wmax[warp] = warp_last;
      __syncthreads();  // also publishes an early-staged list
      int cta_last = wmax[0];
#pragma unroll
      for (int w = 1; w < kWarps; ++w) cta_last = max(cta_last, wmax[w]);
      ++round;
      for (int hi = cta_last; hi >= (int)ti.rbeg; hi -= kBatch) {
        const int lo = max((int)ti.rbeg, hi - kBatch + 1);
        const int nb = hi - lo + 1;
        if (!one_batch) {
#pragma unroll
          for (int u = 0; u < kStagePerThread; ++u) {
            const int slot = threadIdx.x + u * kRenderThreads;
            if (slot < nb) stage(lo + slot, slot, dup_pairs, rec, (float)ox, (float)oy, S, spair);
          }
          __syncthreads();
        }
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
          float2 dx, dy, u, wq;
          const float2 pw = gauss_power2(P.px, P.py, q0, q1.x, dx, dy, u, wq);
          const bool a0 = idx <= B.last0 && pw.x >= q1.z;  // blended by the forward
          const bool a1 = idx <= B.last1 && pw.y >= q1.z;
          // warp-uniform: the whole warp runs the adjoint with masked inputs, so a
          // lane with no contribution produces zeros (all terms are finite); run
          // for every relevant Gaussian (1% have no contributing lane: a vote per
          // event cost more than it saved)
          {
            float g[16];
            g[13] = g[14] = g[15] = 0.f;
            const float4 q2 = S.g2[j];
            const float4 q3 = S.g3[j];
            const float2 G = make_float2(__expf(pw.x), __expf(pw.y));
            const float2 raw = __fmul2_rn(f2(q1.y), G);
            const float2 alpha = make_float2(fminf(raw.x, kAlphaMax), fminf(raw.y, kAlphaMax));
            const float2 oma = __ffma2_rn(alpha, f2(-1.f), f2(1.f));
            const float2 roma = make_float2(__fdividef(1.f, oma.x), __fdividef(1.f, oma.y));  // in [1, 100]
            const float2 Tn = __fmul2_rn(B.T, roma);  // transmittance in front of this Gaussian
            B.T.x = a0 ? Tn.x : B.T.x;
            B.T.y = a1 ? Tn.y : B.T.y;
            const float2 am = make_float2(a0 ? alpha.x : 0.f, a1 ? alpha.y : 0.f);
            const float2 w = __fmul2_rn(am, B.T);
            // dL/dalpha = T (P - Q) + dL/dA T_final / (1 - alpha), P = sum_ch x_ch dL/dX_ch;
            // Q then advances past this Gaussian (unchanged where a = 0)
            float2 Pc = __fmul2_rn(f2(q2.x), B.dC0);
            Pc = __ffma2_rn(f2(q2.y), B.dC1, Pc);
            Pc = __ffma2_rn(f2(q2.z), B.dC2, Pc);
            Pc = __ffma2_rn(f2(q2.w), B.dD, Pc);
            Pc = __ffma2_rn(f2(q3.x), B.dN0, Pc);
            Pc = __ffma2_rn(f2(q3.y), B.dN1, Pc);
            Pc = __ffma2_rn(f2(q3.z), B.dN2, Pc);
            const float2 acc = __ffma2_rn(B.Q, f2(-1.f), Pc);
            B.Q = __ffma2_rn(am, acc, B.Q);
            float2 dal = __ffma2_rn(B.dATf, roma, __fmul2_rn(B.T, acc));
            if constexpr (kSoft) dal = __fadd2_rn(dal, B.dG);  // d g~ / d alpha = 1
            g[6] = fmaf(w.y, B.dC0.y, w.x * B.dC0.x);
            g[7] = fmaf(w.y, B.dC1.y, w.x * B.dC1.x);
            g[8] = fmaf(w.y, B.dC2.y, w.x * B.dC2.x);
            g[9] = fmaf(w.y, B.dD.y, w.x * B.dD.x);
            g[10] = fmaf(w.y, B.dN0.y, w.x * B.dN0.x);
            g[11] = fmaf(w.y, B.dN1.y, w.x * B.dN1.x);
            g[12] = fmaf(w.y, B.dN2.y, w.x * B.dN2.x);
            // through alpha = o G (not clamped): d/do and d/dpower, power = -1/2 (u^2 + w^2),
            // u = l11 dx + l21 dy, w = l22 dy, d = p - m
            const float2 dam = make_float2(a0 && raw.x < kAlphaMax ? dal.x : 0.f,
                                           a1 && raw.y < kAlphaMax ? dal.y : 0.f);
            g[5] = fmaf(dam.y, G.y, dam.x * G.x);
            const float2 dp = __fmul2_rn(dam, alpha);
            const float2 du = __fmul2_rn(dp, u), dw = __fmul2_rn(dp, wq);
            g[0] = q0.z * (du.x + du.y);
            const float2 t1 = __ffma2_rn(du, f2(q0.w), __fmul2_rn(dw, f2(q1.x)));
            g[1] = t1.x + t1.y;
            g[2] = -fmaf(du.y, dx.y, du.x * dx.x);
            g[3] = -fmaf(du.y, dy.y, du.x * dy.x);
            g[4] = -fmaf(dw.y, dy.y, dw.x * dy.x);
            float* sa = reinterpret_cast<float*>(sacc[j]);
            const float tot = warp_reduce_scatter16(g, lane);
            const int k = lane >> 1;
            if (!(lane & 1) && k < 13) atomicAdd(sa + k, tot);
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
        // the slots are staged and accumulated again only by a following batch of
        // this round; the next round or tile reaches them past a barrier of its own
        if (hi - kBatch >= (int)ti.rbeg) __syncthreads();
      }
    }
  }
}

}  // namespace pgsag

using namespace pgsag;

// Grid of a render launch: one CTA per active tile, or for a persistent launch
// ctas_per_sm x SMs CTAs (ctas_per_sm <= 0: as many as the kernel's occupancy
// allows, so the queue never leaves SM slots empty).  `occ` caches the
// occupancy query (the same on every device of this architecture); the first
// persistent call should come before any stream capture.
static int launch_cfg(const pgsag_sched* sched, uint32_t n_items, const void* kernel, int threads, int* occ,
                      Sched& s, unsigned& blocks) {
  s.order = sched ? sched->order : nullptr;
  s.counter = sched ? sched->counter : nullptr;
  if (s.counter) {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return PGSAG_ERR_CUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return PGSAG_ERR_CUDA;
    int per = sched->ctas_per_sm;
    if (per <= 0) {
      if (*occ <= 0 && cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, kernel, threads, 0) != cudaSuccess)
        return PGSAG_ERR_CUDA;
      per = *occ;
    }
    blocks = (unsigned)(sms * (per > 0 ? per : 1));
  } else {
    blocks = n_items;
  }
  return PGSAG_OK;
}

template <bool kSoft>
static int launch_fwd(const pgsag_sched* sched, uint32_t n_active, const pgsag_view* views, const float* rec,
                      const uint32_t* dup_pairs, const void* ranges, const void* act_tiles, const uint32_t* px_list,
                      float* out8, float* depth, void* aux, int32_t* status, cudaStream_t st) {
  Sched s;
  unsigned blocks;
  static int occ = 0;
  int r = launch_cfg(sched, n_active, (const void*)k_render_fwd<PGSAG_FWD_WARPS, kSoft>, PGSAG_FWD_WARPS * 32, &occ,
                     s, blocks);
  if (r) return r;
  if (s.counter) PGSAG_CUDA(cudaMemsetAsync(s.counter, 0, sizeof(uint32_t), st));
  k_render_fwd<PGSAG_FWD_WARPS, kSoft><<<blocks, PGSAG_FWD_WARPS * 32, 0, st>>>(
      views, (const float4*)rec, dup_pairs, (const uint2*)ranges, (const uint4*)act_tiles, n_active, px_list, s,
      (float4*)out8, depth, (uint4*)aux, status);
  PGSAG_CHECK_LAUNCH();
  return PGSAG_OK;
}

extern "C" int pgsag_render_fwd(uint32_t n_views, const pgsag_view* views, const float* rec,
                                const uint32_t* dup_pairs, const void* ranges, const void* act_tiles,
                                uint32_t n_active, const uint32_t* px_list, const pgsag_sched* sched, uint32_t flags,
                                float* out8, float* depth, void* aux, int32_t* status, void* stream) {
  if (n_views == 0 || n_views > PGSAG_MAX_VIEWS) return PGSAG_ERR_UNSUPPORTED;
  if (!views || !status) return PGSAG_ERR_ARG;
  if (flags & ~PGSAG_RENDER_SOFT_COUNT) return PGSAG_ERR_UNSUPPORTED;
  if (n_active == 0) return PGSAG_OK;
  if (!rec || !ranges || !act_tiles || !px_list || !out8 || !depth || !aux) return PGSAG_ERR_ARG;
  if (((uintptr_t)rec | (uintptr_t)out8 | (uintptr_t)aux | (uintptr_t)act_tiles) & 15u) return PGSAG_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  if (flags & PGSAG_RENDER_SOFT_COUNT)
    return launch_fwd<true>(sched, n_active, views, rec, dup_pairs, ranges, act_tiles, px_list, out8, depth, aux,
                            status, st);
  return launch_fwd<false>(sched, n_active, views, rec, dup_pairs, ranges, act_tiles, px_list, out8, depth, aux,
                           status, st);
}

template <bool kSoft>
static int launch_bwd(const pgsag_sched* sched, uint32_t n_active, const pgsag_view* views, const float* rec,
                      const uint32_t* dup_pairs, const void* ranges, const void* act_tiles, const uint32_t* px_list,
                      const float* out8, const void* aux, const float* dout8, const float* ddepth,
                      const pgsag_ban_gather& bg, bool use_ban, const float* dout_scale, float* grad2d,
                      const ClearJob& cj, int32_t* status, cudaStream_t st) {
  Sched s;
  unsigned blocks;
  static int occ = 0;
  int r = launch_cfg(sched, n_active, (const void*)k_render_bwd<PGSAG_BWD_WARPS, kSoft>, PGSAG_BWD_WARPS * 32, &occ,
                     s, blocks);
  if (r) return r;
  if (s.counter) PGSAG_CUDA(cudaMemsetAsync(s.counter, 0, sizeof(uint32_t), st));
  ClearJob job = cj;
  job.per = (uint32_t)(((uint64_t)job.start[PGSAG_CLEAR_MAX] + blocks - 1) / blocks);
  k_render_bwd<PGSAG_BWD_WARPS, kSoft><<<blocks, PGSAG_BWD_WARPS * 32, 0, st>>>(
      views, (const float4*)rec, dup_pairs, (const uint2*)ranges, (const uint4*)act_tiles, n_active, px_list, s,
      (const float4*)out8, (const uint4*)aux, (const float4*)dout8, ddepth, bg, use_ban, dout_scale, grad2d, job,
      status);
  PGSAG_CHECK_LAUNCH();
  return PGSAG_OK;
}

extern "C" int pgsag_render_bwd(uint32_t n_views, const pgsag_view* views, const float* rec,
                                const uint32_t* dup_pairs, const void* ranges, const void* act_tiles,
                                uint32_t n_active, const uint32_t* px_list, const pgsag_sched* sched,
                                const float* out8, const void* aux, const float* dout8, const float* ddepth,
                                const pgsag_ban_gather* ban, const float* dout_scale, uint32_t n_pairs,
                                float* grad2d, const pgsag_clear* clear, int32_t* status, void* stream) {
  if (n_views == 0 || n_views > PGSAG_MAX_VIEWS) return PGSAG_ERR_UNSUPPORTED;
  if (!views || !status) return PGSAG_ERR_ARG;
  if (ban && ban->objective != PGSAG_OBJ_PG && ban->objective != PGSAG_OBJ_EQ11) return PGSAG_ERR_UNSUPPORTED;
  const bool soft = ban && ban->objective == PGSAG_OBJ_EQ11;
  cudaStream_t st = (cudaStream_t)stream;
  ClearJob cj{};
  bool clear_by_memset = false;
  if (clear) {
    uint64_t total = 0;
    for (int i = 0; i < PGSAG_CLEAR_MAX; ++i) {
      const uint64_t n = clear->n[i];
      cj.start[i] = (uint32_t)total;
      if (n == 0) continue;
      if (!clear->ptr[i] || ((uintptr_t)clear->ptr[i] & 15u)) return PGSAG_ERR_ARG;
      cj.p[i] = reinterpret_cast<float4*>(clear->ptr[i]);
      cj.tail[i] = clear->ptr[i] + 4 * (n / 4);
      cj.n_tail[i] = (uint32_t)(n % 4);
      cj.on = true;
      total += n / 4;
    }
    // shares are indexed in 32 bits (with a CTA's share added): beyond 2^31
    // float4 units (32 GiB) the buffers are cleared by memsets instead
    if (total >= (1ull << 31)) {
      clear_by_memset = true;
      cj = ClearJob{};
    } else {
      cj.start[PGSAG_CLEAR_MAX] = (uint32_t)total;
    }
  }
  if (n_pairs) {
    if (!grad2d || ((uintptr_t)grad2d & 15u)) return PGSAG_ERR_ARG;
    PGSAG_CUDA(cudaMemsetAsync(grad2d, 0, (size_t)n_pairs * PGSAG_GRAD2D_FLOATS * sizeof(float), st));
  }
  if (n_active == 0 || clear_by_memset) {
    // no CTA runs (or the buffers are too large for its shares): memsets
    if (clear)
      for (int i = 0; i < PGSAG_CLEAR_MAX; ++i)
        if (clear->n[i]) PGSAG_CUDA(cudaMemsetAsync(clear->ptr[i], 0, clear->n[i] * sizeof(float), st));
    if (n_active == 0) return PGSAG_OK;
  }
  if (!rec || !ranges || !act_tiles || !px_list || !out8 || !aux || !dout8 || !grad2d) return PGSAG_ERR_ARG;
  if (ban && !(ban->nbr && ban->scratch && ban->acc)) return PGSAG_ERR_ARG;
  if (ban && ((uintptr_t)ban->nbr & 15u)) return PGSAG_ERR_ARG;
  if (soft && (!ban->gc_weight || ((uintptr_t)ban->acc & 7u))) return PGSAG_ERR_ARG;
  pgsag_ban_gather bg{};
  if (ban) bg = *ban;
  if (((uintptr_t)rec | (uintptr_t)out8 | (uintptr_t)aux | (uintptr_t)dout8 | (uintptr_t)act_tiles) & 15u)
    return PGSAG_ERR_ARG;
  if (soft)
    return launch_bwd<true>(sched, n_active, views, rec, dup_pairs, ranges, act_tiles, px_list, out8, aux, dout8,
                            ddepth, bg, true, dout_scale, grad2d, cj, status, st);
  return launch_bwd<false>(sched, n_active, views, rec, dup_pairs, ranges, act_tiles, px_list, out8, aux, dout8,
                           ddepth, bg, ban != nullptr, dout_scale, grad2d, cj, status, st);
}
