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
  int width, height;
  uint64_t pix_base;
};
__device__ __forceinline__ ViewLite load_view_lite(const pgsag_view* v) {
  ViewLite r;
  r.fx = __ldg(&v->fx);
  r.fy = __ldg(&v->fy);
  r.cx = __ldg(&v->cx);
  r.cy = __ldg(&v->cy);
  r.width = __ldg(&v->width);
  r.height = __ldg(&v->height);
  r.pix_base = __ldg((const unsigned long long*)&v->pix_base);
  return r;
}

// The Gaussian's exponent at a pixel, -1/2 d^T Q d, evaluated in a fixed
// sequence of correctly rounded operations so that the forward and the adjoint
// kernel obtain identical bits (the alpha >= 1/255 and termination decisions
// must agree between them).  r0 = {mx, my, Qxx, Qxy}, qyy = Qyy.
__device__ __forceinline__ float gauss_power(float px, float py, float4 r0, float qyy,
                                             float& dx, float& dy) {
  dx = __fsub_rn(px, r0.x);
  dy = __fsub_rn(py, r0.y);
  float t = __fmul_rn(r0.z, __fmul_rn(dx, dx));
  t = __fmaf_rn(qyy, __fmul_rn(dy, dy), t);
  t = __fmul_rn(-0.5f, t);
  return __fmaf_rn(-r0.w, __fmul_rn(dx, dy), t);
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
__device__ __forceinline__ int warp_max_i(int v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(kFull, v, o));
  return v;
}

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
