// Masked D-SSIM term of L_rgb (3DGS's L_rgb = (1 - 0.2) L1 + 0.2 (1 - SSIM),
// restricted to the building mask): SSIM per mask pixel and channel with the
// 11 x 11 Gaussian window (sigma 1.5) restricted to the rendered set R and
// renormalised over it, C1 = 0.01^2, C2 = 0.03^2.
//
// One CTA per active tile.  The tile and a 5-pixel halo are gathered into
// shared memory through the dense pixel map (rendered colour, target, and the
// indicator of R); the window is separable (the 2D Gaussian is an outer
// product and R enters as a factor of every image), so each of the 16 windowed
// sums per pixel (the weight, and per channel the sums of x, y, x^2, y^2, x y)
// is a horizontal 11-tap pass into shared memory followed by a vertical one.
//
// Gradient: with a_ik = G(k - i) [k in R] / W_i the window weights of pixel i,
// dSSIM_i/dx_k = a_ik (S_mu + 2 S_var (x_k - mu_x) + S_cov (y_k - mu_y)), so
//   dL/dx_k = [k in R] (G * P + 2 x_k G * Q + y_k G * Rc)(k)
// with P = (S_mu - 2 S_var mu_x - S_cov mu_y) / W, Q = S_var / W, Rc = S_cov / W
// stored per mask pixel by the forward kernel (zero elsewhere): the backward is
// the same separable blur of those 9 images.
#include <math.h>

#include "common.cuh"

namespace pgsag {

constexpr int kSsimR = 5;         // window radius
constexpr int kSsimThreads = 256;
constexpr float kSsimC1 = 0.01f * 0.01f, kSsimC2 = 0.03f * 0.03f;

__device__ __forceinline__ void ssim_weights(float* s_g) {
  if (threadIdx.x < 2 * kSsimR + 1) {
    const float d = (float)((int)threadIdx.x - kSsimR);
    s_g[threadIdx.x] = expf(-d * d / (2.f * 1.5f * 1.5f));
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.f;
    for (int k = 0; k <= 2 * kSsimR; ++k) t += s_g[k];
    s_g[2 * kSsimR + 1] = 1.f / t;
  }
  __syncthreads();
  if (threadIdx.x < 2 * kSsimR + 1) s_g[threadIdx.x] *= s_g[2 * kSsimR + 1];
  __syncthreads();
}

// Forward: SSIM of every mask pixel of the tile (summed over channels into the
// view's accumulator acc[8 v + 7]) and the 9 gradient coefficients per rendered
// pixel (zero off the mask).
__global__ void __launch_bounds__(kSsimThreads) k_ssim_fwd(const pgsag_view* __restrict__ views,
                                                           const uint4* __restrict__ act_tiles,
                                                           const uint32_t* __restrict__ pidx,
                                                           const uint8_t* __restrict__ flags_c,
                                                           const float4* __restrict__ out8,
                                                           const float* __restrict__ target,
                                                           float* __restrict__ scratch, double* __restrict__ acc,
                                                           const int32_t* status) {
  extern __shared__ __align__(16) float smem[];
  __shared__ float s_g[2 * kSsimR + 2];
  __shared__ float s_w[kSsimThreads / 32];
  if (status_bad(status)) return;
  const uint4 at = __ldg(act_tiles + blockIdx.x);
  const pgsag_view* vp = views + at.x;
  const int W = __ldg(&vp->width), H = __ldg(&vp->height);
  const int tw = __ldg(&vp->tile_w), th = __ldg(&vp->tile_h);
  const uint64_t pix_base = __ldg((const unsigned long long*)&vp->pix_base);
  const int x0 = (int)(at.y & 0xffffu) * tw, y0 = (int)(at.y >> 16) * th;
  const int RW = tw + 2 * kSsimR, RH = th + 2 * kSsimR, NR = RW * RH;
  float* sv = smem;                                  // [7][NR]: r, x0..2, y0..2 (planes: no bank conflicts)
  float* hs = smem + 7 * NR;                         // [16][RH * tw]
  ssim_weights(s_g);
  for (int i = threadIdx.x; i < NR; i += kSsimThreads) {
    const int X = x0 - kSsimR + i % RW, Y = y0 - kSsimR + i / RW;
    float v[7] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (X >= 0 && X < W && Y >= 0 && Y < H) {
      const uint32_t q = __ldg(pidx + pix_base + (uint64_t)Y * W + X);
      if (q != 0xffffffffu) {
        const float4 c = __ldg(out8 + 2ull * q);
        v[0] = 1.f;
        v[1] = c.x;
        v[2] = c.y;
        v[3] = c.z;
        v[4] = __ldg(target + 3ull * q);
        v[5] = __ldg(target + 3ull * q + 1);
        v[6] = __ldg(target + 3ull * q + 2);
      }
    }
#pragma unroll
    for (int k = 0; k < 7; ++k) sv[k * NR + i] = v[k];
  }
  __syncthreads();
  // horizontal pass: 16 windowed sums for every region row and tile column
  for (int it = threadIdx.x; it < RH * tw; it += kSsimThreads) {
    const int ry = it / tw, cx = it % tw;
    float h[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) h[k] = 0.f;
    for (int d = 0; d <= 2 * kSsimR; ++d) {
      const float* p = sv + (ry * RW + cx + d);
      const float g = s_g[d];
      h[0] += g * p[0];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const float x = p[(1 + c) * NR], y = p[(4 + c) * NR];  // zero off R
        h[1 + 5 * c] += g * x;
        h[2 + 5 * c] += g * y;
        h[3 + 5 * c] += g * x * x;
        h[4 + 5 * c] += g * y * y;
        h[5 + 5 * c] += g * x * y;
      }
    }
#pragma unroll
    for (int k = 0; k < 16; ++k) hs[k * RH * tw + it] = h[k];
  }
  __syncthreads();
  float ssum = 0.f;
  for (int it = threadIdx.x; it < tw * th; it += kSsimThreads) {
    const int oy = it / tw, ox = it % tw;
    const int X = x0 + ox, Y = y0 + oy;
    if (X >= W || Y >= H) continue;
    const uint32_t q = __ldg(pidx + pix_base + (uint64_t)Y * W + X);
    if (q == 0xffffffffu) continue;
    float* sc = scratch + 9ull * q;
    if (!(__ldg(flags_c + q) & PGSAG_PIX_MASK)) {
#pragma unroll
      for (int k = 0; k < 9; ++k) sc[k] = 0.f;
      continue;
    }
    float v[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) v[k] = 0.f;
    for (int d = 0; d <= 2 * kSsimR; ++d) {
      const float* p = hs + (oy + d) * tw + ox;
      const float g = s_g[d];
#pragma unroll
      for (int k = 0; k < 16; ++k) v[k] += g * p[k * RH * tw];
    }
    const float iw = 1.f / v[0];  // > 0: the pixel itself is rendered
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const float mx = v[1 + 5 * c] * iw, my = v[2 + 5 * c] * iw;
      const float vx = v[3 + 5 * c] * iw - mx * mx, vy = v[4 + 5 * c] * iw - my * my;
      const float cxy = v[5 + 5 * c] * iw - mx * my;
      const float A1 = 2.f * mx * my + kSsimC1, A2 = 2.f * cxy + kSsimC2;
      const float B1 = mx * mx + my * my + kSsimC1, B2 = vx + vy + kSsimC2;
      const float S = (A1 * A2) / (B1 * B2);
      ssum += S;
      const float s_mu = S * (2.f * my / A1 - 2.f * mx / B1);
      const float s_var = -S / B2;
      const float s_cov = 2.f * S / A2;
      sc[3 * c + 0] = (s_mu - 2.f * s_var * mx - s_cov * my) * iw;
      sc[3 * c + 1] = s_var * iw;
      sc[3 * c + 2] = s_cov * iw;
    }
  }
  ssum = warp_sum(ssum);
  if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = ssum;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.f;
    for (int w = 0; w < kSsimThreads / 32; ++w) t += s_w[w];
    if (t != 0.f) atomicAdd(acc + 8ull * at.x + 7, (double)t);
  }
}

// Backward: dL/dC of every rendered pixel of the tile, added to dout8's colour:
// scale_v (G * P + 2 x G * Q + y G * Rc), scale_v = -lambda / (3 |M_v|).
__global__ void __launch_bounds__(kSsimThreads) k_ssim_bwd(const pgsag_view* __restrict__ views,
                                                           const uint4* __restrict__ act_tiles,
                                                           const uint32_t* __restrict__ pidx,
                                                           const float4* __restrict__ out8,
                                                           const float* __restrict__ target,
                                                           const float* __restrict__ scratch, float lambda,
                                                           float4* __restrict__ dout8, const int32_t* status) {
  extern __shared__ __align__(16) float smem[];
  __shared__ float s_g[2 * kSsimR + 2];
  if (status_bad(status)) return;
  const uint4 at = __ldg(act_tiles + blockIdx.x);
  const pgsag_view* vp = views + at.x;
  const int W = __ldg(&vp->width), H = __ldg(&vp->height);
  const int tw = __ldg(&vp->tile_w), th = __ldg(&vp->tile_h);
  const uint64_t pix_base = __ldg((const unsigned long long*)&vp->pix_base);
  const uint32_t nm = __ldg(&vp->n_mask);
  const float scale = nm ? -lambda / (3.f * (float)nm) : 0.f;
  const int x0 = (int)(at.y & 0xffffu) * tw, y0 = (int)(at.y >> 16) * th;
  const int RW = tw + 2 * kSsimR, RH = th + 2 * kSsimR, NR = RW * RH;
  float* sv = smem;              // [9][NR]
  float* hs = smem + 9 * NR;     // [9][RH * tw]
  ssim_weights(s_g);
  for (int i = threadIdx.x; i < NR; i += kSsimThreads) {
    const int X = x0 - kSsimR + i % RW, Y = y0 - kSsimR + i / RW;
    float v[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (X >= 0 && X < W && Y >= 0 && Y < H) {
      const uint32_t q = __ldg(pidx + pix_base + (uint64_t)Y * W + X);
      if (q != 0xffffffffu) {
#pragma unroll
        for (int k = 0; k < 9; ++k) v[k] = __ldg(scratch + 9ull * q + k);
      }
    }
#pragma unroll
    for (int k = 0; k < 9; ++k) sv[k * NR + i] = v[k];
  }
  __syncthreads();
  for (int it = threadIdx.x; it < RH * tw; it += kSsimThreads) {
    const int ry = it / tw, cx = it % tw;
    float h[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) h[k] = 0.f;
    for (int d = 0; d <= 2 * kSsimR; ++d) {
      const float* p = sv + (ry * RW + cx + d);
      const float g = s_g[d];
#pragma unroll
      for (int k = 0; k < 9; ++k) h[k] += g * p[k * NR];
    }
#pragma unroll
    for (int k = 0; k < 9; ++k) hs[k * RH * tw + it] = h[k];
  }
  __syncthreads();
  for (int it = threadIdx.x; it < tw * th; it += kSsimThreads) {
    const int oy = it / tw, ox = it % tw;
    const int X = x0 + ox, Y = y0 + oy;
    if (X >= W || Y >= H) continue;
    const uint32_t q = __ldg(pidx + pix_base + (uint64_t)Y * W + X);
    if (q == 0xffffffffu) continue;
    float b[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) b[k] = 0.f;
    for (int d = 0; d <= 2 * kSsimR; ++d) {
      const float* p = hs + (oy + d) * tw + ox;
      const float g = s_g[d];
#pragma unroll
      for (int k = 0; k < 9; ++k) b[k] += g * p[k * RH * tw];
    }
    const float4 c = __ldg(out8 + 2ull * q);
    const float x[3] = {c.x, c.y, c.z};
    float gr[3];
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) {
      const float y = __ldg(target + 3ull * q + ch);
      gr[ch] = scale * (b[3 * ch] + 2.f * x[ch] * b[3 * ch + 1] + y * b[3 * ch + 2]);
    }
    float4 d = dout8[2ull * q];
    d.x += gr[0];
    d.y += gr[1];
    d.z += gr[2];
    dout8[2ull * q] = d;
  }
}

size_t ssim_fwd_smem(int tw, int th) {
  const size_t NR = (size_t)(tw + 2 * kSsimR) * (th + 2 * kSsimR);
  return sizeof(float) * (7 * NR + (size_t)(th + 2 * kSsimR) * tw * 16);
}

size_t ssim_bwd_smem(int tw, int th) {
  const size_t NR = (size_t)(tw + 2 * kSsimR) * (th + 2 * kSsimR);
  return sizeof(float) * (9 * NR + (size_t)(th + 2 * kSsimR) * tw * 9);
}

// Launch both passes over n_active tiles whose views all have tile_w x tile_h
// tiles (the dynamic shared memory is sized for them).
int launch_dssim(uint32_t n_active, int tw, int th, const pgsag_view* views, const void* act_tiles,
                 const uint32_t* pidx, const uint8_t* flags_c, const float* out8, const float* target,
                 float* scratch, double* acc, float lambda, float* dout8, int32_t* status, cudaStream_t s) {
  const size_t sf = ssim_fwd_smem(tw, th), sb = ssim_bwd_smem(tw, th);
  if (sf > 227 * 1024 || sb > 227 * 1024) return PGSAG_ERR_UNSUPPORTED;
  if (cudaFuncSetAttribute(k_ssim_fwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sf) != cudaSuccess ||
      cudaFuncSetAttribute(k_ssim_bwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sb) != cudaSuccess)
    return PGSAG_ERR_CUDA;
  k_ssim_fwd<<<n_active, kSsimThreads, sf, s>>>(views, (const uint4*)act_tiles, pidx, flags_c, (const float4*)out8,
                                                target, scratch, acc, status);
  PGSAG_CHECK_LAUNCH();
  k_ssim_bwd<<<n_active, kSsimThreads, sb, s>>>(views, (const uint4*)act_tiles, pidx, (const float4*)out8, target,
                                                scratch, lambda, (float4*)dout8, status);
  PGSAG_CHECK_LAUNCH();
  return PGSAG_OK;
}

}  // namespace pgsag
