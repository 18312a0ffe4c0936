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
// pixel (zero off the mask).  The 16 windowed sums travel as 8 pairs through
// packed two-lane FP32 instructions: (W, xy_2), (x_0, x_1), (y_0, y_1),
// (x_0^2, x_1^2), (y_0^2, y_1^2), (x_0 y_0, x_1 y_1), (x_2, y_2), (x_2^2, y_2^2).
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
  // tile sides are multiples of 8, so NR and every plane offset below are even
  const int RW = tw + 2 * kSsimR, RH = th + 2 * kSsimR, NR = RW * RH, NH = RH * tw;
  float2* sx = reinterpret_cast<float2*>(smem);           // [NR] (x_0, x_1)
  float2* sy = sx + NR;                                   // [NR] (y_0, y_1)
  float2* s2 = sy + NR;                                   // [NR] (x_2, y_2)
  float* sr = smem + 6 * NR;                              // [NR] indicator of R
  float2* hs = reinterpret_cast<float2*>(smem + 7 * NR);  // [8][NH] pairs of sums
  ssim_weights(s_g);
  for (int i = threadIdx.x; i < NR; i += kSsimThreads) {
    const int X = x0 - kSsimR + i % RW, Y = y0 - kSsimR + i / RW;
    float2 a = make_float2(0.f, 0.f), b = a, c = a;
    float r = 0.f;
    if (X >= 0 && X < W && Y >= 0 && Y < H) {
      const uint32_t q = __ldg(pidx + pix_base + (uint64_t)Y * W + X);
      if (q != 0xffffffffu) {
        const float4 col = __ldg(out8 + 2ull * q);
        r = 1.f;
        a = make_float2(col.x, col.y);
        b = make_float2(__ldg(target + 3ull * q), __ldg(target + 3ull * q + 1));
        c = make_float2(col.z, __ldg(target + 3ull * q + 2));
      }
    }
    sx[i] = a;
    sy[i] = b;
    s2[i] = c;
    sr[i] = r;
  }
  __syncthreads();
  // horizontal pass: the 8 pairs of windowed sums for every region row and tile column
  for (int it = threadIdx.x; it < NH; it += kSsimThreads) {
    const int ry = it / tw, cx = it % tw;
    float2 h[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) h[k] = make_float2(0.f, 0.f);
    const int i0 = ry * RW + cx;
    for (int d = 0; d <= 2 * kSsimR; ++d) {
      const float2 g = make_float2(s_g[d], s_g[d]);
      const float2 a = sx[i0 + d], b = sy[i0 + d], c = s2[i0 + d];
      h[0] = __ffma2_rn(g, make_float2(sr[i0 + d], c.x * c.y), h[0]);
      h[1] = __ffma2_rn(g, a, h[1]);
      h[2] = __ffma2_rn(g, b, h[2]);
      h[3] = __ffma2_rn(g, __fmul2_rn(a, a), h[3]);
      h[4] = __ffma2_rn(g, __fmul2_rn(b, b), h[4]);
      h[5] = __ffma2_rn(g, __fmul2_rn(a, b), h[5]);
      h[6] = __ffma2_rn(g, c, h[6]);
      h[7] = __ffma2_rn(g, __fmul2_rn(c, c), h[7]);
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) hs[k * NH + it] = h[k];
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
    float2 v[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) v[k] = make_float2(0.f, 0.f);
    for (int d = 0; d <= 2 * kSsimR; ++d) {
      const float2 g = make_float2(s_g[d], s_g[d]);
      const float2* p = hs + (oy + d) * tw + ox;
#pragma unroll
      for (int k = 0; k < 8; ++k) v[k] = __ffma2_rn(g, p[k * NH], v[k]);
    }
    const float iw = 1.f / v[0].x;  // > 0: the pixel itself is rendered
    const float sxs[3] = {v[1].x, v[1].y, v[6].x}, sys[3] = {v[2].x, v[2].y, v[6].y};
    const float sxx[3] = {v[3].x, v[3].y, v[7].x}, syy[3] = {v[4].x, v[4].y, v[7].y};
    const float sxy[3] = {v[5].x, v[5].y, v[0].y};
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const float mx = sxs[c] * iw, my = sys[c] * iw;
      const float vx = sxx[c] * iw - mx * mx, vy = syy[c] * iw - my * my;
      const float cxy = sxy[c] * iw - mx * my;
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
// scale_v (G * P + 2 x G * Q + y G * Rc), scale_v = -lambda / (3 |M_v|).  The 9
// coefficient images blur as 4 packed pairs (P_0, P_1), (Q_0, Q_1), (Rc_0, Rc_1),
// (P_2, Q_2) and Rc_2.
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
  const int RW = tw + 2 * kSsimR, RH = th + 2 * kSsimR, NR = RW * RH, NH = RH * tw;
  float2* sv = reinterpret_cast<float2*>(smem);            // [4][NR] pairs
  float* s8 = smem + 8 * NR;                               // [NR] Rc_2
  float2* hs = reinterpret_cast<float2*>(smem + 9 * NR);   // [4][NH]
  float* h8 = smem + 9 * NR + 8 * NH;                      // [NH]
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
    // v = {P0, Q0, R0, P1, Q1, R1, P2, Q2, R2}
    sv[i] = make_float2(v[0], v[3]);
    sv[NR + i] = make_float2(v[1], v[4]);
    sv[2 * NR + i] = make_float2(v[2], v[5]);
    sv[3 * NR + i] = make_float2(v[6], v[7]);
    s8[i] = v[8];
  }
  __syncthreads();
  for (int it = threadIdx.x; it < NH; it += kSsimThreads) {
    const int ry = it / tw, cx = it % tw;
    float2 h[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) h[k] = make_float2(0.f, 0.f);
    float h1 = 0.f;
    const int i0 = ry * RW + cx;
    for (int d = 0; d <= 2 * kSsimR; ++d) {
      const float2 g = make_float2(s_g[d], s_g[d]);
#pragma unroll
      for (int k = 0; k < 4; ++k) h[k] = __ffma2_rn(g, sv[k * NR + i0 + d], h[k]);
      h1 = fmaf(g.x, s8[i0 + d], h1);
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) hs[k * NH + it] = h[k];
    h8[it] = h1;
  }
  __syncthreads();
  for (int it = threadIdx.x; it < tw * th; it += kSsimThreads) {
    const int oy = it / tw, ox = it % tw;
    const int X = x0 + ox, Y = y0 + oy;
    if (X >= W || Y >= H) continue;
    const uint32_t q = __ldg(pidx + pix_base + (uint64_t)Y * W + X);
    if (q == 0xffffffffu) continue;
    float2 b[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) b[k] = make_float2(0.f, 0.f);
    float b8 = 0.f;
    const int j0 = oy * tw + ox;
    for (int d = 0; d <= 2 * kSsimR; ++d) {
      const float2 g = make_float2(s_g[d], s_g[d]);
#pragma unroll
      for (int k = 0; k < 4; ++k) b[k] = __ffma2_rn(g, hs[k * NH + j0 + d * tw], b[k]);
      b8 = fmaf(g.x, h8[j0 + d * tw], b8);
    }
    const float P[3] = {b[0].x, b[0].y, b[3].x}, Q[3] = {b[1].x, b[1].y, b[3].y}, Rc[3] = {b[2].x, b[2].y, b8};
    const float4 c = __ldg(out8 + 2ull * q);
    const float x[3] = {c.x, c.y, c.z};
    float gr[3];
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) {
      const float y = __ldg(target + 3ull * q + ch);
      gr[ch] = scale * (P[ch] + 2.f * x[ch] * Q[ch] + y * Rc[ch]);
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
