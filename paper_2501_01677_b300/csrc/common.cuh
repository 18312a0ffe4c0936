// Shared device helpers for libpgsag (sm_103a).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "pgsag.h"

namespace pgsag {

constexpr float kAlphaMin = 1.0f / 255.0f;  // 3DGS alpha cutoff (Sec. 3.1 by citation)
constexpr float kAlphaMax = 0.99f;          // alpha clamp
constexpr float kTMin = 1e-4f;              // transmittance termination
constexpr float kCovDilation = 0.3f;        // low-pass dilation of Sigma' (px^2)
constexpr float kJacClamp = 1.3f;           // x/z, y/z clamp in units of half-FOV
constexpr float kShOffset = 0.5f;           // SH colour offset
constexpr float kRayDotMin = 1e-8f;         // Eq. 4 validity: -N.r > 1e-8
constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ bool status_bad(const int32_t* st) {
  return *((volatile const int32_t*)st) != 0;
}
__device__ __forceinline__ void status_set(int32_t* st, unsigned flag) {
  atomicOr((int*)st, (int)flag);
}

// Camera / view fields needed per chunk, read from the device view table.
struct ViewLite {
  float fx, fy, cx, cy;
  float ifx, ify;  // 1 / fx, 1 / fy: a pixel's ray (u + 1/2 - cx) / fx is taken as (u + 1/2 - cx) * ifx
  int width, height, tile_w, tile_h;
  uint64_t pix_base;
};
__device__ __forceinline__ ViewLite load_view_lite(const pgsag_view* v) {
  ViewLite r;
  r.fx = __ldg(&v->fx);
  r.fy = __ldg(&v->fy);
  r.cx = __ldg(&v->cx);
  r.cy = __ldg(&v->cy);
  r.ifx = 1.f / r.fx;
  r.ify = 1.f / r.fy;
  r.width = __ldg(&v->width);
  r.height = __ldg(&v->height);
  r.tile_w = __ldg(&v->tile_w);
  r.tile_h = __ldg(&v->tile_h);
  r.pix_base = __ldg((const unsigned long long*)&v->pix_base);
  return r;
}

// The Gaussian's exponent at a pixel, -1/2 d^T Q d, from the Cholesky factor
// Q = L L^T, L = [[l11, 0], [l21, l22]]:  -1/2 ((l11 dx + l21 dy)^2 + (l22 dy)^2),
// a sum of squares (no cancellation for elongated Gaussians).  Evaluated in a
// fixed sequence of correctly rounded operations so that the forward and the
// adjoint kernel obtain identical bits (the alpha >= 1/255 and termination
// decisions must agree between them).  r0 = {mx, my, l11, l21}.
__device__ __forceinline__ float gauss_power(float px, float py, float4 r0, float l22, float& dx, float& dy,
                                             float& u, float& w) {
  dx = __fsub_rn(px, r0.x);
  dy = __fsub_rn(py, r0.y);
  u = __fmaf_rn(r0.z, dx, __fmul_rn(r0.w, dy));
  w = __fmul_rn(l22, dy);
  return __fmul_rn(-0.5f, __fmaf_rn(u, u, __fmul_rn(w, w)));
}

// Does the region {d : -1/2 d^T Q d >= thr} of a 2D Gaussian (conic
// Q = [[qa, qb], [qb, qc]]) meet the axis-aligned rectangle [dx0, dx1] x
// [dy0, dy1] of pixel-centre offsets from its centre?  The quadratic is
// minimised over the rectangle (centre inside, else each edge's 1D minimum
// clamped to the edge).  Conservative: the bound is widened by the float32
// error of evaluating the quadratic at any pixel, which grows with the conic's
// condition number, so every pixel whose float32 exponent passes the threshold
// lies in a rectangle this test accepts (the rounding of the edge minimisers is
// far inside that margin).  The per-Gaussian part is computed once
// (ellipse_test) and reused for every rectangle.
struct EllipseTest {
  float qa, qb, qc;  // conic Q = L L^T
  float iqa, iqc;    // 1 / qa, 1 / qc
  float bound;       // d^T Q d <= bound  <=>  the region reaches d (with margin)
};

__device__ __forceinline__ EllipseTest ellipse_test(float l11, float l21, float l22, float thr) {
  EllipseTest e;
  e.qa = l11 * l11;
  e.qb = l11 * l21;
  e.qc = fmaf(l21, l21, l22 * l22);
  e.iqa = __frcp_rn(e.qa);
  e.iqc = __frcp_rn(e.qc);
  const float hm = 0.5f * (e.qa + e.qc);
  const float dq = e.qa - e.qc;
  const float rt = sqrtf(fmaf(0.25f * dq, dq, e.qb * e.qb));
  const float lmin = fmaxf(hm - rt, 1e-30f);
  const float kappa = (hm + rt) / lmin;
  e.bound = fmaf(-2.f * thr, 1.001f + 1e-6f * kappa, 1e-3f);
  return e;
}

__device__ __forceinline__ bool ellipse_rect_hit(const EllipseTest& e, float dx0, float dx1, float dy0, float dy1) {
  if (dx0 <= 0.f && dx1 >= 0.f && dy0 <= 0.f && dy1 >= 0.f) return true;
  const float ex[2] = {dx0, dx1}, ey[2] = {dy0, dy1};
  float f = 3.0e38f;
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const float dx = ex[i];
    const float dy = fminf(fmaxf(-e.qb * dx * e.iqc, dy0), dy1);
    f = fminf(f, fmaf(e.qa * dx, dx, fmaf(2.f * e.qb * dx, dy, e.qc * dy * dy)));
  }
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const float dy = ey[i];
    const float dx = fminf(fmaxf(-e.qb * dy * e.iqa, dx0), dx1);
    f = fminf(f, fmaf(e.qa * dx, dx, fmaf(2.f * e.qb * dx, dy, e.qc * dy * dy)));
  }
  return f <= e.bound;
}

// Tile binning rule (pgsag_preprocess): a pair whose tile rectangle spans at
// most kExactTileMax tiles is binned to the active tiles its alpha >= 1/255
// region meets (on the tile's pixel centres); a larger rectangle goes to all its
// active tiles.  The 2D mean is given as integer part (mi, ni) + fraction
// (mf, nf), so the offsets are exact up to one rounding.
constexpr int kExactTileMax = 64;

__device__ __forceinline__ bool tile_hit(const EllipseTest& e, float mi, float ni, float mf, float nf, int tx, int ty,
                                         int tw, int th, int W, int H) {
  const float x0 = (float)(tx * tw) + 0.5f, x1 = (float)min((tx + 1) * tw, W) - 0.5f;
  const float y0 = (float)(ty * th) + 0.5f, y1 = (float)min((ty + 1) * th, H) - 0.5f;
  return ellipse_rect_hit(e, (x0 - mi) - mf, (x1 - mi) - mf, (y0 - ni) - nf, (y1 - ni) - nf);
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}
__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}
__device__ __forceinline__ int warp_max_i(int v) { return __reduce_max_sync(kFull, v); }
// Warp-wide float minimum / maximum in one instruction (redux.sync .f32,
// Blackwell); exact, so every lane obtains the same value a shuffle tree would.
__device__ __forceinline__ float warp_min_f(float v) {
  float r;
  asm volatile("redux.sync.min.f32 %0, %1, 0xffffffff;" : "=f"(r) : "f"(v));
  return r;
}
__device__ __forceinline__ float warp_max_f(float v) {
  float r;
  asm volatile("redux.sync.max.f32 %0, %1, 0xffffffff;" : "=f"(r) : "f"(v));
  return r;
}

// Masked D-SSIM passes (ssim.cu), launched by pgsag_loss_ban.
int launch_dssim(uint32_t n_active, int tw, int th, const pgsag_view* views, const void* act_tiles,
                 const uint32_t* pidx, const uint8_t* flags_c, const float* out8, const float* target,
                 float* scratch, double* acc, float lambda, float* dout8, int32_t* status, cudaStream_t s);

}  // namespace pgsag

#define PGSAG_CHECK_LAUNCH()                          \
  do {                                                \
    if (cudaPeekAtLastError() != cudaSuccess) {       \
      cudaGetLastError();                             \
      return PGSAG_ERR_CUDA;                          \
    }                                                 \
  } while (0)

#define PGSAG_CUDA(call)                              \
  do {                                                \
    if ((call) != cudaSuccess) {                      \
      cudaGetLastError();                             \
      return PGSAG_ERR_CUDA;                          \
    }                                                 \
  } while (0)

static inline unsigned pgsag_div_up(unsigned long long a, unsigned long long b) {
  return (unsigned)((a + b - 1) / b);
}
