// Photometric L1 term and boundary-aware normal loss (Sec. 4.2, Eq. 8) with
// their gradient on the rendered channels; per-tile / per-pixel Gaussian
// counts and the GC-load statistic (Sec. 4.3, Eq. 9).
//
// The kernels walk the compacted pixel lists chunk by chunk (one warp, one pixel
// per lane); per-pixel arrays are compact (indexed by px_list position) and a
// pixel's 4 neighbours and flags come from the compact tables of mask
// preparation (pgsag_prep_neighbours), so every per-pixel load is coalesced or
// one indirection away.  Pass A
// (loss, own-pixel gradient, neighbour scratch, optionally the GC-load sums)
// is followed either by pass B here or by the same gather in the render
// adjoint's prologue.
#include <float.h>
#include <mutex>

#include "common.cuh"

namespace pgsag {

constexpr int kLossThreads = 256;
#ifndef PGSAG_LOSS_MINB
#define PGSAG_LOSS_MINB 8  // resident loss blocks per SM the register budget must allow (full occupancy)
#endif
constexpr float kWBoundary = 0.1f;  // Eq. 8: boundary weight
#ifndef PGSAG_REDUCE_BLOCKS
#define PGSAG_REDUCE_BLOCKS 148  // one per SM: 64 left SMs idle (loss stage 0.263 -> 0.253 ms at config 1)
#endif
constexpr int kReduceBlocks = PGSAG_REDUCE_BLOCKS;  // blocks per view for the per-view sums

struct PixCtx {
  bool has;
  uint32_t view;
  ViewLite V;
  int x, y;
  uint64_t q;  // compact index (position in px_list)
};

// A chunk record is {view, first px_list entry, pixel count, active tile}.
__device__ __forceinline__ PixCtx pix_ctx(uint32_t c, int lane, const uint4* __restrict__ chunks,
                                          const uint32_t* __restrict__ px_list,
                                          const pgsag_view* __restrict__ views) {
  PixCtx P;
  const uint4 ch = __ldg(chunks + c);
  P.view = ch.x;
  P.V = load_view_lite(views + ch.x);
  P.has = (uint32_t)lane < ch.z;
  P.q = ch.y + lane;
  const uint32_t pix = P.has ? __ldg(px_list + P.q) : 0u;
  P.y = (int)(pix / (uint32_t)P.V.width);
  P.x = (int)(pix - (uint32_t)P.y * (uint32_t)P.V.width);
  return P;
}

__device__ __forceinline__ void ray(const ViewLite& V, int x, int y, float r[3]) {
  r[0] = ((float)x + 0.5f - V.cx) * V.ifx;
  r[1] = ((float)y + 0.5f - V.cy) * V.ify;
  r[2] = 1.f;
}

// Pass A: per rendered pixel.  L1 term and its gradient; for interior valid
// mask pixels with valid neighbours, the Eq. 8 term, the gradient on the own
// rendered normal (unscaled) and dL/da, dL/db of the two central differences
// (stored in `scratch` for the neighbours to gather).
__global__ void __launch_bounds__(kLossThreads, PGSAG_LOSS_MINB) k_loss_a(
    const pgsag_view* __restrict__ views, uint32_t n_chunks, const uint4* __restrict__ chunks,
    const uint32_t* __restrict__ px_list, const uint8_t* __restrict__ flags_c, const uint4* __restrict__ nbr,
    const float4* __restrict__ out8, const float* __restrict__ depth, const float* __restrict__ target,
    const uint4* __restrict__ aux,
    const float* __restrict__ gc_weight, bool soft, float l1_scale, float* __restrict__ scratch,
    float4* __restrict__ partial,
    float4* __restrict__ dout8, double* __restrict__ acc, uint32_t n_acc, const int32_t* status) {
  // the per-view accumulators the reduction after this pass adds into (a memset
  // node costs more than these few stores)
  if (blockIdx.x == 0)
    for (uint32_t i = threadIdx.x; i < n_acc; i += blockDim.x) acc[i] = 0.0;
  if (status_bad(status)) return;
  const int lane = threadIdx.x & 31;
  const uint32_t c = blockIdx.x * (kLossThreads / 32) + (threadIdx.x >> 5);
  if (c >= n_chunks) return;
  const PixCtx P = pix_ctx(c, lane, chunks, px_list, views);
  {
    // the chunk's target (3 lines), neighbour-table (4 lines) and depth (1 line)
    // rows are read only after the flag and depth tests: ask L2 for them now
    // (only lines that start inside the chunk's rows)
    const uint32_t n = __popc(__ballot_sync(0xffffffffu, P.has));
    const uint64_t q0 = P.q - (uint64_t)lane;
    const char* a = nullptr;
    if (lane < 3 && 128u * lane < 12u * n) a = reinterpret_cast<const char*>(target + 3 * q0) + 128 * lane;
    else if (lane >= 3 && lane < 7 && 128u * (lane - 3) < 16u * n) a = reinterpret_cast<const char*>(nbr + q0) + 128 * (lane - 3);
    else if (lane == 7 && n > 0) a = reinterpret_cast<const char*>(depth + q0);
    if (a) asm volatile("prefetch.global.L2 [%0];" ::"l"(a));
  }
  float l1 = 0.f, lb = 0.f, nv = 0.f, gn = 0.f, gx = 0.f;
  if (P.has) {
    // the flags and outputs are loaded before the Eq. 9 division waits on the count
    const uint8_t f = __ldg(flags_c + P.q);
    const float4 o0 = __ldg(out8 + 2 * P.q), o1 = __ldg(out8 + 2 * P.q + 1);
    if (gc_weight != nullptr) {
      // Eq. 9 term of this rendered pixel: g / w (g = Gaussians blended, or the
      // soft count g~ = sum of their alphas)
      const float g = soft ? __uint_as_float(__ldg(&aux[P.q].w)) : (float)__ldg(&aux[P.q].z);
      gx = __fdividef(g, __ldg(gc_weight + P.q));  // w >= 1
      gn = 1.f;
    }
    float dC[3] = {0.f, 0.f, 0.f}, dNo[3] = {0.f, 0.f, 0.f};
    if (f & PGSAG_PIX_MASK) {
      const uint32_t nm = __ldg(&views[P.view].n_mask);
      const float inv3m = nm ? __fdividef(l1_scale, 3.f * (float)nm) : 0.f;
      const float C[3] = {o0.x, o0.y, o0.z};
#pragma unroll
      for (int ch = 0; ch < 3; ++ch) {
        const float d = C[ch] - __ldg(target + 3 * P.q + ch);
        l1 += fabsf(d);
        dC[ch] = d > 0.f ? inv3m : (d < 0.f ? -inv3m : 0.f);
      }
      float ga[3] = {0.f, 0.f, 0.f}, gb[3] = {0.f, 0.f, 0.f};
      const int W = P.V.width, H = P.V.height;
      const float dep = __ldg(depth + P.q);
      bool inV = P.x >= 1 && P.x <= W - 2 && P.y >= 1 && P.y <= H - 2 && dep > 0.f;
      // central differences of the back-projected points P = Depth r, r = ((x + 1/2 - cx) / fx,
      // (y + 1/2 - cy) / fy, 1): a = P[y+1] - P[y-1], b = P[x+1] - P[x-1]
      float a[3] = {0.f, 0.f, 0.f}, b[3] = {0.f, 0.f, 0.f};
      if (inV) {
        // up, down, left, right neighbours (~0: not rendered)
        const uint4 nb = __ldg(nbr + P.q);
        const uint32_t qn[4] = {nb.x, nb.y, nb.z, nb.w};
        float dq[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) dq[k] = qn[k] != 0xffffffffu ? __ldg(depth + qn[k]) : 0.f;
#pragma unroll
        for (int k = 0; k < 4; ++k) inV = inV && qn[k] != 0xffffffffu && dq[k] > 0.f;
        // d1 r1 - d0 r0 = (d1 - d0) r1 + d0 (r1 - r0): the depth difference is exact
        // for depths within a factor 2 of each other and the two rays differ by two
        // pixel pitches along one axis, so the difference carries no cancellation
        // (forming d1 r1 and d0 r0 first loses ~depth / footprint ulps: ~1e3 at
        // aerial range)
        float r[3], rd[3], rr[3];
        ray(P.V, P.x, P.y, r);
        ray(P.V, P.x, P.y + 1, rd);
        ray(P.V, P.x + 1, P.y, rr);
        const float dv = dq[1] - dq[0], du = dq[3] - dq[2];
        a[0] = dv * r[0];
        a[1] = fmaf(dv, rd[1], dq[0] * (2.f * P.V.ify));
        a[2] = dv;
        b[0] = fmaf(du, rr[0], dq[2] * (2.f * P.V.ifx));
        b[1] = du * r[1];
        b[2] = du;
      }
      if (inV) {
        const float cr[3] = {a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0]};
        // unit vectors by reciprocal square roots of the squared norms (a norm
        // this side of the smallest normal float is taken as zero)
        const float c2 = cr[0] * cr[0] + cr[1] * cr[1] + cr[2] * cr[2];
        const float n2 = o1.x * o1.x + o1.y * o1.y + o1.z * o1.z;
        if (c2 >= FLT_MIN && n2 >= FLT_MIN) {
          const float icn = rsqrtf(c2), iNn = rsqrtf(n2);
          const float nd[3] = {cr[0] * icn, cr[1] * icn, cr[2] * icn};
          const float nr[3] = {o1.x * iNn, o1.y * iNn, o1.z * iNn};
          const float w = (f & PGSAG_PIX_EDGE) ? kWBoundary : 1.f;
          const float df[3] = {nd[0] - nr[0], nd[1] - nr[1], nd[2] - nr[2]};
          lb = w * (df[0] * df[0] + df[1] * df[1] + df[2] * df[2]);
          nv = 1.f;
          // d/d nd = 2 w df, d/d nr = -2 w df
          const float gnd[3] = {2.f * w * df[0], 2.f * w * df[1], 2.f * w * df[2]};
          const float pnd = nd[0] * gnd[0] + nd[1] * gnd[1] + nd[2] * gnd[2];
          const float gc[3] = {(gnd[0] - nd[0] * pnd) * icn, (gnd[1] - nd[1] * pnd) * icn,
                               (gnd[2] - nd[2] * pnd) * icn};
          const float pnr = -(nr[0] * gnd[0] + nr[1] * gnd[1] + nr[2] * gnd[2]);
#pragma unroll
          for (int k = 0; k < 3; ++k) dNo[k] = (-gnd[k] - nr[k] * pnr) * iNn;
          // c = a x b: dL/da = b x gc, dL/db = gc x a
          ga[0] = b[1] * gc[2] - b[2] * gc[1];
          ga[1] = b[2] * gc[0] - b[0] * gc[2];
          ga[2] = b[0] * gc[1] - b[1] * gc[0];
          gb[0] = gc[1] * a[2] - gc[2] * a[1];
          gb[1] = gc[2] * a[0] - gc[0] * a[2];
          gb[2] = gc[0] * a[1] - gc[1] * a[0];
        }
      }
      float* sc = scratch + 6ull * P.q;
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        sc[k] = ga[k];
        sc[3 + k] = gb[k];
      }
    } else {
      // rendered pixels off the mask have no Eq. 8 term: zero rows, so that a
      // neighbour's gather needs no flag test
      float* sc = scratch + 6ull * P.q;
#pragma unroll
      for (int k = 0; k < 6; ++k) sc[k] = 0.f;
    }
    dout8[2 * P.q] = make_float4(dC[0], dC[1], dC[2], 0.f);
    dout8[2 * P.q + 1] = make_float4(dNo[0], dNo[1], dNo[2], 0.f);
  }
  // per-chunk partial sums (8 per chunk), reduced per view by k_view_reduce
  const float s1 = warp_sum(l1), s2 = warp_sum(lb), s3 = warp_sum(nv);
  float s4 = 0.f, s5 = 0.f, s6 = 0.f;
  if (gc_weight != nullptr) {
    s4 = warp_sum(gn);
    s5 = warp_sum(gx);
    s6 = warp_sum(gx * gx);
  }
  if (lane == 0) {
    partial[2 * c] = make_float4(s1, s2, s3, 0.f);
    partial[2 * c + 1] = make_float4(s4, s5, s6, 0.f);
  }
}

// Grid (blocks, views): each block sums a slice of the view's per-chunk partials
// (pstride floats per chunk, the first ncomp <= 8 used) in double and adds them
// into acc[stride * v + 0 .. ncomp) (acc zeroed before).  n_rows = partial rows
// available: a view whose chunk range leaves them sets PGSAG_DEV_BOUNDS and is
// skipped.
__global__ void __launch_bounds__(256) k_view_reduce(const pgsag_view* __restrict__ views,
                                                     const float* __restrict__ partial, int pstride, int ncomp,
                                                     int stride, double* __restrict__ acc, uint32_t n_rows,
                                                     int32_t* status) {
  __shared__ double sh[8][8];
  if (status_bad(status)) return;
  const pgsag_view* V = views + blockIdx.y;
  const uint32_t b = __ldg(&V->chunk_base), n = __ldg(&V->n_chunks);
  if ((uint64_t)b + n > n_rows) {
    if (blockIdx.x == 0 && threadIdx.x == 0) status_set(status, PGSAG_DEV_BOUNDS);
    return;
  }
  const uint32_t per = (n + gridDim.x - 1) / gridDim.x;
  const uint32_t lo = min(n, blockIdx.x * per), hi = min(n, lo + per);
  if (lo >= hi) return;
  double a[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  for (uint32_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
    const float* p = partial + (size_t)(b + i) * pstride;
#pragma unroll
    for (int k = 0; k < 8; ++k)
      if (k < ncomp) a[k] += __ldg(p + k);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    if (k < ncomp) {
      const double t = warp_sum_d(a[k]);
      if (lane == 0) sh[warp][k] = t;
    }
  }
  __syncthreads();
  if (threadIdx.x < ncomp) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += sh[w][threadIdx.x];
    atomicAdd(acc + stride * blockIdx.y + threadIdx.x, t);
  }
}

// Pass B: per rendered pixel, gather dL/dP from the neighbours whose central
// differences used this pixel, map it to D and N through Eq. 4, scale.
__global__ void __launch_bounds__(kLossThreads) k_loss_b(
    const pgsag_view* __restrict__ views, uint32_t n_chunks, const uint4* __restrict__ chunks,
    const uint32_t* __restrict__ px_list, const uint4* __restrict__ nbr,
    const float4* __restrict__ out8, const float* __restrict__ depth, const float* __restrict__ scratch,
    const double* __restrict__ acc,
    float lambda_ban, float4* __restrict__ dout8, const int32_t* status) {
  if (status_bad(status)) return;
  const int lane = threadIdx.x & 31;
  const uint32_t c = blockIdx.x * (kLossThreads / 32) + (threadIdx.x >> 5);
  if (c >= n_chunks) return;
  const PixCtx P = pix_ctx(c, lane, chunks, px_list, views);
  if (!P.has) return;
  const double nV = acc[8 * P.view + 2];
  const float scale = nV > 0.0 ? (float)(lambda_ban / nV) : 0.f;
  float dP[3] = {0.f, 0.f, 0.f};
  // this pixel is P[y+1] of (x, y-1) (up), P[y-1] of (x, y+1) (down), P[x+1] of
  // (x-1, y) (left), P[x-1] of (x+1, y) (right); only mask neighbours wrote scratch
  const float sg[4] = {1.f, -1.f, 1.f, -1.f};
  const int off[4] = {0, 0, 3, 3};
  const uint4 nb = __ldg(nbr + P.q);
  const uint32_t qn[4] = {nb.x, nb.y, nb.z, nb.w};
  bool mk[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) mk[k] = qn[k] != 0xffffffffu;  // off-mask rows are zero
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    if (!mk[k]) continue;
    const float* sc = scratch + 6ull * qn[k] + off[k];
    dP[0] += sg[k] * __ldg(sc + 0);
    dP[1] += sg[k] * __ldg(sc + 1);
    dP[2] += sg[k] * __ldg(sc + 2);
  }
  float4 g1 = dout8[2 * P.q + 1];
  float dD = 0.f, dN[3] = {0.f, 0.f, 0.f};
  const float dep = __ldg(depth + P.q);
  if (dep > 0.f && (dP[0] != 0.f || dP[1] != 0.f || dP[2] != 0.f)) {
    const float4 o0 = __ldg(out8 + 2 * P.q), o1 = __ldg(out8 + 2 * P.q + 1);
    float r[3];
    ray(P.V, P.x, P.y, r);
    const float sdot = -(o1.x * r[0] + o1.y * r[1] + o1.z * r[2]);
    const float gdep = dP[0] * r[0] + dP[1] * r[1] + dP[2] * r[2];  // P = Depth r
    const float is = 1.f / sdot;
    dD = gdep * is;
    const float k = gdep * o0.w * is * is;
    dN[0] = k * r[0];
    dN[1] = k * r[1];
    dN[2] = k * r[2];
  }
  float4 g0 = dout8[2 * P.q];
  g0.w = scale * dD;
  g1.x = scale * (g1.x + dN[0]);
  g1.y = scale * (g1.y + dN[1]);
  g1.z = scale * (g1.z + dN[2]);
  g1.w = 0.f;
  dout8[2 * P.q] = g0;
  dout8[2 * P.q + 1] = g1;
}

// One thread: per-view losses and their sum (views are few); with gc_load, the
// per-view GC-load (Eq. 9: population std of g / w over the rendered pixels).
__device__ __forceinline__ float gc_std(double n, double s, double q) {
  double var = 0.0;
  if (n > 0.0) {
    const double m = s / n;
    var = q / n - m * m;
  }
  return (float)sqrt(var > 0.0 ? var : 0.0);
}

// Per view: L_rgb, L_ban, the view's loss and the GC-load; the sum over views.
// Objective Eq. 11: the view's loss is (1 - lambda)(L_rgb + lambda_4 L_ban) +
// lambda GC-load_v, the total adds (1 - lambda) lambda_3 L_s (L_s = the
// flattening sum in acc[8 n_views] over n_gauss), and slot 3 of each view's
// accumulators receives {lambda / (n sigma), mean} (two floats), the
// coefficients of the soft-count gradient dL/dg~_i = c (x_i - mean) / w_i.
// With D-SSIM (lambda_d > 0) L_rgb = (1 - lambda_d) L1 + lambda_d (1 - SSIM_M),
// SSIM_M from the sum in slot 7.
__global__ void k_loss_final(const pgsag_view* __restrict__ views, uint32_t n_views, double* __restrict__ acc,
                             float lambda_ban, uint32_t objective, uint32_t n_gauss, float lambda_d,
                             float* __restrict__ loss, float* __restrict__ gc_load, const int32_t* status) {
  if (status_bad(status)) return;
  if (threadIdx.x != 0) return;
  const bool eq11 = objective == PGSAG_OBJ_EQ11;
  const double lam = (double)PGSAG_LAMBDA_GC;
  double total = 0.0;
  for (uint32_t v = 0; v < n_views; ++v) {
    double* a = acc + 8 * v;
    const uint32_t nm = views[v].n_mask;
    double lr = nm ? a[0] / (3.0 * nm) : 0.0;
    if (lambda_d > 0.f && nm)
      lr = (1.0 - (double)lambda_d) * lr + (double)lambda_d * (1.0 - a[7] / (3.0 * nm));
    const double lb = a[2] > 0.0 ? a[1] / a[2] : 0.0;
    const float gc = gc_load ? gc_std(a[4], a[5], a[6]) : 0.f;
    double lv = lr + (double)lambda_ban * lb;
    if (eq11) {
      lv = (1.0 - lam) * lv + lam * (double)gc;
      const double n = a[4];
      float2 cm = make_float2(0.f, 0.f);
      if (n > 0.0) {
        cm.y = (float)(a[5] / n);
        if (gc > 0.f) cm.x = (float)(lam / (n * (double)gc));
      }
      *reinterpret_cast<float2*>(a + 3) = cm;
    }
    loss[3 * v + 0] = (float)lr;
    loss[3 * v + 1] = (float)lb;
    loss[3 * v + 2] = (float)lv;
    total += lv;
    if (gc_load) gc_load[v] = gc;
  }
  if (eq11 && n_gauss > 0)
    total += (1.0 - lam) * (double)PGSAG_LAMBDA_FLAT * acc[8 * n_views] / (double)n_gauss;
  loss[3 * n_views] = (float)total;
}

// Flattening loss (Eq. 11's L_s): sum over the Gaussians of min(exp(log_scales)).
__global__ void __launch_bounds__(256) k_flat_sum(uint32_t n, const float* __restrict__ log_scales,
                                                  double* __restrict__ out, const int32_t* status) {
  if (status_bad(status)) return;
  __shared__ double s_w[8];
  double acc = 0.0;
  for (uint32_t g = blockIdx.x * blockDim.x + threadIdx.x; g < n; g += gridDim.x * blockDim.x) {
    const float a = __ldg(log_scales + 3ull * g), b = __ldg(log_scales + 3ull * g + 1),
                c = __ldg(log_scales + 3ull * g + 2);
    acc += (double)expf(fminf(a, fminf(b, c)));
  }
  acc = warp_sum_d(acc);
  if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += s_w[w];
    atomicAdd(out, t);
  }
}

// ------------------------------------------------------------------ Eq. 9

__global__ void k_tile_counts(uint32_t n_active, const uint2* __restrict__ ranges,
                              uint32_t* __restrict__ counts, const int32_t* status) {
  if (status_bad(status)) return;
  const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n_active) return;
  const uint2 r = __ldg(ranges + t);
  counts[t] = r.y - r.x;
}

__global__ void __launch_bounds__(kLossThreads) k_gc_accum(
    const pgsag_view* __restrict__ views, uint32_t n_chunks, const uint4* __restrict__ chunks,
    const uint32_t* __restrict__ px_list, const uint4* __restrict__ aux, const float* __restrict__ weight,
    float4* __restrict__ partial,
    const int32_t* status) {
  if (status_bad(status)) return;
  const int lane = threadIdx.x & 31;
  const uint32_t c = blockIdx.x * (kLossThreads / 32) + (threadIdx.x >> 5);
  if (c >= n_chunks) return;
  const PixCtx P = pix_ctx(c, lane, chunks, px_list, views);
  float x = 0.f, n = 0.f;
  if (P.has) {
    const uint32_t g = __ldg(&aux[P.q].z);
    x = (float)g / __ldg(weight + P.q);
    n = 1.f;
  }
  const float s0 = warp_sum(n), s1 = warp_sum(x), s2 = warp_sum(x * x);
  if (lane == 0) partial[c] = make_float4(s0, s1, s2, 0.f);
}

__global__ void k_gc_final(uint32_t n_views, const double* __restrict__ acc, float* __restrict__ out,
                           const int32_t* status) {
  if (status_bad(status)) return;
  const uint32_t v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n_views) return;
  out[v] = gc_std(acc[3 * v], acc[3 * v + 1], acc[3 * v + 2]);
}

// Per rendered pixel of one view (compact index px_base + i): the target colour
// gathered from the dense image, and w = 1 + |Sobel(Y)| with replicated borders.
__global__ void k_gc_weight(int W, int H, uint32_t n, const uint32_t* __restrict__ px,
                            const float* __restrict__ target, float* __restrict__ target_c,
                            float* __restrict__ weight) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint32_t pix = __ldg(px + i);
  const int y = (int)(pix / (uint32_t)W), x = (int)(pix - (uint32_t)y * (uint32_t)W);
  float Y[3][3];
#pragma unroll
  for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
    for (int dx = -1; dx <= 1; ++dx) {
      const int xx = min(max(x + dx, 0), W - 1), yy = min(max(y + dy, 0), H - 1);
      const float* t = target + 3 * ((size_t)yy * W + xx);
      Y[dy + 1][dx + 1] = 0.299f * t[0] + 0.587f * t[1] + 0.114f * t[2];
    }
  const float gx = (Y[0][2] + 2.f * Y[1][2] + Y[2][2]) - (Y[0][0] + 2.f * Y[1][0] + Y[2][0]);
  const float gy = (Y[2][0] + 2.f * Y[2][1] + Y[2][2]) - (Y[0][0] + 2.f * Y[0][1] + Y[0][2]);
  weight[i] = 1.f + sqrtf(gx * gx + gy * gy);
  const float* t = target + 3 * (size_t)pix;
  target_c[3 * (size_t)i + 0] = t[0];
  target_c[3 * (size_t)i + 1] = t[1];
  target_c[3 * (size_t)i + 2] = t[2];
}

}  // namespace pgsag

using namespace pgsag;

extern "C" int pgsag_loss_ban(uint32_t n_views, const pgsag_view* views, uint32_t n_chunks,
                              const void* chunks, const void* act_tiles, const uint32_t* px_list,
                              const uint8_t* flags_c, const void* nbr, const float* out8, const float* depth,
                              const void* aux, const float* target, float lambda_ban, const float* gc_weight,
                              int gather, float* scratch, double* acc, float* chunk_scratch, float* loss,
                              float* gc_load, float* dout8, uint32_t objective, uint32_t n_gauss,
                              const float* log_scales, const pgsag_dssim* dssim, int32_t* status, void* stream) {
  if (n_views == 0 || n_views > PGSAG_MAX_VIEWS) return PGSAG_ERR_UNSUPPORTED;
  if (objective != PGSAG_OBJ_PG && objective != PGSAG_OBJ_EQ11) return PGSAG_ERR_UNSUPPORTED;
  if (!views || !status || !acc || !loss) return PGSAG_ERR_ARG;
  if ((gc_weight == nullptr) != (gc_load == nullptr)) return PGSAG_ERR_ARG;
  const bool eq11 = objective == PGSAG_OBJ_EQ11;
  if (eq11 && (!gc_weight || gather || (n_gauss && !log_scales))) return PGSAG_ERR_ARG;
  if (dssim && (!dssim->pidx || !dssim->scratch || !act_tiles || ((uintptr_t)act_tiles & 15u) ||
                !(dssim->lambda >= 0.f && dssim->lambda <= 1.f) || dssim->tile_w <= 0 || dssim->tile_h <= 0))
    return PGSAG_ERR_ARG;
  const float lambda_d = dssim ? dssim->lambda : 0.f;
  cudaStream_t s = (cudaStream_t)stream;
  const uint32_t n_acc = (n_views + (eq11 ? 1u : 0u)) * 8u;
  if (n_chunks == 0) PGSAG_CUDA(cudaMemsetAsync(acc, 0, (size_t)n_acc * sizeof(double), s));
  if (n_chunks) {
    if (!chunks || !px_list || !flags_c || !nbr || !out8 || !depth || !target || !scratch || !dout8 ||
        !chunk_scratch || (gc_weight && !aux))
      return PGSAG_ERR_ARG;
    if (((uintptr_t)out8 | (uintptr_t)dout8 | (uintptr_t)chunks | (uintptr_t)nbr | (uintptr_t)chunk_scratch |
         (uintptr_t)aux) & 15u)
      return PGSAG_ERR_ARG;
    const unsigned blocks = pgsag_div_up(n_chunks, kLossThreads / 32);
    k_loss_a<<<blocks, kLossThreads, 0, s>>>(views, n_chunks, (const uint4*)chunks, px_list, flags_c,
                                             (const uint4*)nbr, (const float4*)out8, depth, target,
                                             (const uint4*)aux, gc_weight, eq11, 1.f - lambda_d, scratch,
                                             (float4*)chunk_scratch, (float4*)dout8, acc, n_acc, status);
    PGSAG_CHECK_LAUNCH();
    k_view_reduce<<<dim3(kReduceBlocks, n_views), 256, 0, s>>>(views, chunk_scratch, 8, gc_weight ? 7 : 3, 8,
                                                                acc, n_chunks, status);
    PGSAG_CHECK_LAUNCH();
    if (dssim && dssim->n_active_total) {
      const int r = launch_dssim(dssim->n_active_total, dssim->tile_w, dssim->tile_h, views, act_tiles, dssim->pidx,
                                 flags_c, out8, target, dssim->scratch, acc, dssim->lambda, dout8, status, s);
      if (r) return r;
    }
    if (gather) {
      k_loss_b<<<blocks, kLossThreads, 0, s>>>(views, n_chunks, (const uint4*)chunks, px_list,
                                               (const uint4*)nbr, (const float4*)out8, depth, scratch, acc,
                                               lambda_ban, (float4*)dout8, status);
      PGSAG_CHECK_LAUNCH();
    }
  }
  if (eq11 && n_gauss) {
    const unsigned fb = pgsag_div_up(n_gauss, 256) < 148u * 8u ? pgsag_div_up(n_gauss, 256) : 148u * 8u;
    k_flat_sum<<<fb, 256, 0, s>>>(n_gauss, log_scales, acc + 8 * (size_t)n_views, status);
    PGSAG_CHECK_LAUNCH();
  }
  k_loss_final<<<1, 32, 0, s>>>(views, n_views, acc, lambda_ban, objective, n_gauss, lambda_d, loss, gc_load,
                                status);
  PGSAG_CHECK_LAUNCH();
  return PGSAG_OK;
}

extern "C" int pgsag_tile_stats(uint32_t n_views, const pgsag_view* views, uint32_t n_active_total,
                                const void* ranges, uint32_t n_chunks, const void* chunks,
                                const void* act_tiles, const uint32_t* px_list, const void* aux,
                                const float* gc_weight, uint32_t* tile_counts, double* acc,
                                float* chunk_scratch, float* gc_load, int32_t* status, void* stream) {
  if (n_views == 0 || n_views > PGSAG_MAX_VIEWS) return PGSAG_ERR_UNSUPPORTED;
  if (!views || !status) return PGSAG_ERR_ARG;
  const bool gc = gc_load != nullptr;  // NULL: per-tile counts only
  if (gc && !acc) return PGSAG_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  if (gc) PGSAG_CUDA(cudaMemsetAsync(acc, 0, (size_t)n_views * 3 * sizeof(double), s));
  if (n_active_total) {
    if (!ranges || !tile_counts) return PGSAG_ERR_ARG;
    k_tile_counts<<<pgsag_div_up(n_active_total, 256), 256, 0, s>>>(n_active_total, (const uint2*)ranges,
                                                                    tile_counts, status);
    PGSAG_CHECK_LAUNCH();
  }
  if (!gc) return PGSAG_OK;
  if (n_chunks) {
    if (!chunks || !px_list || !aux || !gc_weight || !chunk_scratch) return PGSAG_ERR_ARG;
    if (((uintptr_t)chunk_scratch | (uintptr_t)aux | (uintptr_t)chunks) & 15u) return PGSAG_ERR_ARG;
    k_gc_accum<<<pgsag_div_up(n_chunks, kLossThreads / 32), kLossThreads, 0, s>>>(
        views, n_chunks, (const uint4*)chunks, px_list, (const uint4*)aux, gc_weight,
        (float4*)chunk_scratch, status);
    PGSAG_CHECK_LAUNCH();
    k_view_reduce<<<dim3(kReduceBlocks, n_views), 256, 0, s>>>(views, chunk_scratch, 4, 3, 3, acc, n_chunks,
                                                                status);
    PGSAG_CHECK_LAUNCH();
  }
  k_gc_final<<<pgsag_div_up(n_views, 128), 128, 0, s>>>(n_views, acc, gc_load, status);
  PGSAG_CHECK_LAUNCH();
  return PGSAG_OK;
}

extern "C" int pgsag_prep_gc_weight(const pgsag_view* view, const float* target, const uint32_t* px_list,
                                    uint32_t px_base, uint32_t n_px, float* target_c, float* weight,
                                    void* stream) {
  if (!view || !target || !px_list || !target_c || !weight) return PGSAG_ERR_ARG;
  if (view->width <= 0 || view->height <= 0) return PGSAG_ERR_ARG;
  if (n_px == 0) return PGSAG_OK;
  k_gc_weight<<<pgsag_div_up(n_px, 256), 256, 0, (cudaStream_t)stream>>>(
      view->width, view->height, n_px, px_list + px_base, target, target_c + 3ull * px_base, weight + px_base);
  PGSAG_CHECK_LAUNCH();
  return PGSAG_OK;
}

// ---------------------------------------------------------------------------
// Allocation-free variant of pgsag_tile_stats.
//
// Some callers cannot allocate device memory: a host application or plug-in
// that must take every device buffer from its own memory manager, or a
// latency-critical loop where a cudaMalloc (which can synchronise the device)
// is not acceptable.  This entry point keeps its scratch -- the per-view double
// accumulators and the per-chunk partial sums -- in a fixed array below, so it
// needs no workspace from the caller and allocates nothing.
//
// The array is a file-scope __device__ variable: every GPU that loads this
// library holds it (kNoAllocScratchBytes) until the process exits.  Host code
// cannot use its name as a device address, so its address is looked up once per
// device with cudaGetSymbolAddress, on that device's first call (with the device
// current).  Make that first call before any stream capture.  The address is
// kept for the process, so it is stale after a cudaDeviceReset (the entry point
// must not be called on that device again).  All calls share the array and it
// keeps the last call's contents: the accumulators are cleared at the start of
// every call, and calls that overlap on the GPU (different streams, or host
// threads on the same device) race on it.
// ---------------------------------------------------------------------------
namespace {
constexpr uint32_t kNoAllocMaxChunks = PGSAG_NOALLOC_MAX_CHUNKS;
constexpr size_t kNoAllocAccBytes = (size_t)PGSAG_MAX_VIEWS * 3 * sizeof(double);
constexpr size_t kNoAllocScratchBytes = kNoAllocAccBytes + (size_t)kNoAllocMaxChunks * 4 * sizeof(float);
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kNoAllocMaxDevices = 64;
std::mutex g_noalloc_mutex;
void* g_noalloc_ptr[kNoAllocMaxDevices] = {};

// Device address of g_noalloc_scratch on the current device (looked up once).
int noalloc_scratch(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return PGSAG_ERR_CUDA;
  if (dev < 0 || dev >= kNoAllocMaxDevices) return PGSAG_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || p == nullptr) {
      cudaGetLastError();
      return PGSAG_ERR_CUDA;
    }
    g_noalloc_ptr[dev] = p;
  }
  *out = g_noalloc_ptr[dev];
  return PGSAG_OK;
}
}  // namespace

extern "C" int pgsag_tile_stats_noalloc(uint32_t n_views, const pgsag_view* views, uint32_t n_active_total,
                                        const void* ranges, uint32_t n_chunks, const void* chunks,
                                        const void* act_tiles, const uint32_t* px_list, const void* aux,
                                        const float* gc_weight, uint32_t* tile_counts, float* gc_load,
                                        int32_t* status, void* stream) {
  if (n_views == 0 || n_views > PGSAG_MAX_VIEWS) return PGSAG_ERR_UNSUPPORTED;
  if (n_chunks > kNoAllocMaxChunks) return PGSAG_ERR_CAPACITY;
  void* base = nullptr;
  const int r = noalloc_scratch(&base);
  if (r) return r;
  double* acc = reinterpret_cast<double*>(base);
  float* chunk_scratch = reinterpret_cast<float*>(static_cast<unsigned char*>(base) + kNoAllocAccBytes);
  return pgsag_tile_stats(n_views, views, n_active_total, ranges, n_chunks, chunks, act_tiles, px_list, aux,
                          gc_weight, tile_counts, acc, chunk_scratch, gc_load, status, stream);
}
