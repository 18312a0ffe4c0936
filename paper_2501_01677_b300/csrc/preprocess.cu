// Per-(view, Gaussian) projection (Sec. 3.1: EWA splatting and SH colour of 3DGS by
// citation; Eq. 2-3 flattened-Gaussian normal and plane distance) and its adjoint.
#include <math.h>

#include "common.cuh"

namespace pgsag {

// Real spherical harmonics up to degree 3 (orthonormal, no Condon-Shortley
// phase), index l*l + l + m, written as polynomials of the unit direction.
// Normalisations K_lm = sqrt((2l+1)/(4 pi) (l-|m|)!/(l+|m|)!) times the
// polynomial's own factor, evaluated here from their closed forms.
#define PGSAG_PI 3.14159265358979323846
__device__ __constant__ float kSH[10] = {
    (float)(0.5 * 0.56418958354775628695),  // 1/2 sqrt(1/pi)          Y00
    (float)(0.48860251190291992159),        // sqrt(3/(4 pi))          Y1m
    (float)(1.09254843059207907054),        // 1/2 sqrt(15/pi)         Y2-2, Y2-1, Y21
    (float)(0.31539156525252000603),        // 1/4 sqrt(5/pi)          Y20 (3z^2-1)
    (float)(0.54627421529603953527),        // 1/4 sqrt(15/pi)         Y22 (x^2-y^2)
    (float)(0.59004358992664351035),        // 1/4 sqrt(35/(2 pi))     Y3+-3
    (float)(2.89061144264055405538),        // 1/2 sqrt(105/pi)        Y3-2 xyz
    (float)(0.45704579946446573616),        // 1/4 sqrt(21/(2 pi))     Y3+-1 (5z^2-1)
    (float)(0.37317633259011539141),        // 1/4 sqrt(7/pi)          Y30 z(5z^2-3)
    (float)(1.44530572132027702769)};       // 1/4 sqrt(105/pi)        Y32 z(x^2-y^2)

__device__ __forceinline__ void sh_eval(float x, float y, float z, float Y[16]) {
  const float xx = x * x, yy = y * y, zz = z * z;
  Y[0] = kSH[0];
  Y[1] = kSH[1] * y;
  Y[2] = kSH[1] * z;
  Y[3] = kSH[1] * x;
  Y[4] = kSH[2] * x * y;
  Y[5] = kSH[2] * y * z;
  Y[6] = kSH[3] * (3.f * zz - 1.f);
  Y[7] = kSH[2] * x * z;
  Y[8] = kSH[4] * (xx - yy);
  Y[9] = kSH[5] * y * (3.f * xx - yy);
  Y[10] = kSH[6] * x * y * z;
  Y[11] = kSH[7] * y * (5.f * zz - 1.f);
  Y[12] = kSH[8] * z * (5.f * zz - 3.f);
  Y[13] = kSH[7] * x * (5.f * zz - 1.f);
  Y[14] = kSH[9] * z * (xx - yy);
  Y[15] = kSH[5] * x * (xx - 3.f * yy);
}

// Gradient of each polynomial above with respect to (x, y, z), contracted with
// per-coefficient weights c[k]: returns sum_k c[k] grad Y_k.
__device__ __forceinline__ void sh_grad(float x, float y, float z, const float c[16], float& gx,
                                        float& gy, float& gz) {
  const float xx = x * x, yy = y * y, zz = z * z;
  gx = 0.f;
  gy = 0.f;
  gz = 0.f;
  gy += c[1] * kSH[1];
  gz += c[2] * kSH[1];
  gx += c[3] * kSH[1];
  gx += c[4] * kSH[2] * y;
  gy += c[4] * kSH[2] * x;
  gy += c[5] * kSH[2] * z;
  gz += c[5] * kSH[2] * y;
  gz += c[6] * kSH[3] * 6.f * z;
  gx += c[7] * kSH[2] * z;
  gz += c[7] * kSH[2] * x;
  gx += c[8] * kSH[4] * 2.f * x;
  gy -= c[8] * kSH[4] * 2.f * y;
  gx += c[9] * kSH[5] * 6.f * x * y;
  gy += c[9] * kSH[5] * 3.f * (xx - yy);
  gx += c[10] * kSH[6] * y * z;
  gy += c[10] * kSH[6] * x * z;
  gz += c[10] * kSH[6] * x * y;
  gy += c[11] * kSH[7] * (5.f * zz - 1.f);
  gz += c[11] * kSH[7] * 10.f * y * z;
  gz += c[12] * kSH[8] * (15.f * zz - 3.f);
  gx += c[13] * kSH[7] * (5.f * zz - 1.f);
  gz += c[13] * kSH[7] * 10.f * x * z;
  gx += c[14] * kSH[9] * 2.f * x * z;
  gy -= c[14] * kSH[9] * 2.f * y * z;
  gz += c[14] * kSH[9] * (xx - yy);
  gx += c[15] * kSH[5] * 3.f * (xx - yy);
  gy -= c[15] * kSH[5] * 6.f * x * y;
}

// Rotation matrix of the unit quaternion (w, x, y, z), row-major.
__device__ __forceinline__ void quat_rot(float w, float x, float y, float z, float R[9]) {
  R[0] = 1.f - 2.f * (y * y + z * z);
  R[1] = 2.f * (x * y - w * z);
  R[2] = 2.f * (x * z + w * y);
  R[3] = 2.f * (x * y + w * z);
  R[4] = 1.f - 2.f * (x * x + z * z);
  R[5] = 2.f * (y * z - w * x);
  R[6] = 2.f * (x * z - w * y);
  R[7] = 2.f * (y * z + w * x);
  R[8] = 1.f - 2.f * (x * x + y * y);
}

// Camera centre -R^T t of every view, written into the shared-memory copy of
// the view table (reserved0) by the first threads of the block.
__device__ __forceinline__ void set_campos(pgsag_view* sv, uint32_t n_views) {
  for (uint32_t v = threadIdx.x; v < n_views; v += blockDim.x) {
    const float* R = sv[v].R;
    const float* t = sv[v].t;
#pragma unroll
    for (int j = 0; j < 3; ++j)
      sv[v].reserved0[j] = -(R[0 * 3 + j] * t[0] + R[1 * 3 + j] * t[1] + R[2 * 3 + j] * t[2]);
  }
}

struct GaussIn {
  float m[3], ls[3], q[4], ol;
  bool finite;
};

__device__ __forceinline__ GaussIn load_gauss(uint32_t g, const float* __restrict__ means,
                                              const float* __restrict__ log_scales,
                                              const float* __restrict__ quats,
                                              const float* __restrict__ opacity_logit) {
  GaussIn G;
  bool fin = true;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    G.m[i] = __ldg(means + 3ull * g + i);
    G.ls[i] = __ldg(log_scales + 3ull * g + i);
    fin &= isfinite(G.m[i]) && isfinite(G.ls[i]);
  }
  const float4 q = __ldg(reinterpret_cast<const float4*>(quats) + g);
  G.q[0] = q.x;
  G.q[1] = q.y;
  G.q[2] = q.z;
  G.q[3] = q.w;
  fin &= isfinite(q.x) && isfinite(q.y) && isfinite(q.z) && isfinite(q.w);
  G.ol = __ldg(opacity_logit + g);
  fin &= isfinite(G.ol);
  G.finite = fin;
  return G;
}

// Camera-space z in float32 without FMA: ((R20 x + R21 y) + R22 z) + t2.  This
// value orders the Gaussians and decides the near-plane cull.
__device__ __forceinline__ float depth_key_z(const pgsag_view& V, const float m[3]) {
  float a = __fmul_rn(V.R[6], m[0]);
  float b = __fmul_rn(V.R[7], m[1]);
  float c = __fmul_rn(V.R[8], m[2]);
  return __fadd_rn(__fadd_rn(__fadd_rn(a, b), c), V.t[2]);
}

// Error-free transformations: a + b = s + e (Knuth), a * b = p + e (FMA).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
__device__ __forceinline__ void two_prod(float a, float b, float& p, float& e) {
  p = __fmul_rn(a, b);
  e = __fmaf_rn(a, b, -p);
}

// Compensated R_row . m + t (hi + lo).
__device__ __forceinline__ void dot3_comp(const float* R, const float m[3], float t, float& hi, float& lo) {
  hi = t;
  lo = 0.f;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    float p, pe, s, se;
    two_prod(R[i], m[i], p, pe);
    two_sum(hi, p, s, se);
    hi = s;
    lo = __fadd_rn(lo, __fadd_rn(pe, se));
  }
}

// One pixel coordinate of the 2D mean, f (x/z) + c, in compensated float32
// (about 1e-10 relative), split into an integer part ip and a fraction fp so
// that pixel offsets (p - ip) - fp lose nothing to the magnitude of p.
__device__ __forceinline__ void mean2d_coord(float xh, float xl, float zh, float zl, float f, float c, float& ip,
                                             float& fp) {
  const float qh = __fdiv_rn(xh, zh);
  float p, pe;
  two_prod(qh, zh, p, pe);
  const float r = __fsub_rn(__fadd_rn(__fsub_rn(__fsub_rn(xh, p), pe), xl), __fmul_rn(qh, zl));
  const float ql = __fdiv_rn(r, zh);
  float m, me, s, se;
  two_prod(f, qh, m, me);
  two_sum(m, c, s, se);
  const float lo = __fadd_rn(__fadd_rn(me, __fmul_rn(f, ql)), se);
  ip = rintf(s);
  fp = __fadd_rn(__fsub_rn(s, ip), lo);
}

// Everything the forward computes for one pair that the adjoint reuses.
struct PairFwd {
  float mc[3];      // camera-frame mean
  float Rq[9];      // rotation of the normalised quaternion
  float s[3];       // scales
  float qn[4];      // normalised quaternion
  float qinv;       // 1/|q|
  float o;          // opacity
  float T2[6];      // J W (2x3)
  float M[9];       // Rq diag(s)
  float V[6];       // T2 M (2x3)
  float a, b, c;    // Sigma' (dilated)
  float det;        // det Sigma' (Lagrange identity, no cancellation)
  float l11, l21, l22;  // Cholesky factor of the conic Sigma'^-1
  bool clampx, clampy;
  float txz, tyz;   // clamped x/z, y/z
  float J00, J02, J11, J12;
  int axis;         // argmin log-scale
  float sign;       // +-1 normal flip
  float nc[3];      // camera-facing normal
  float dist;
};

// Returns false if the pair is culled.
__device__ __forceinline__ bool pair_forward(const pgsag_view& V, const GaussIn& G, PairFwd& P) {
  if (!G.finite) return false;
  const float z = depth_key_z(V, G.m);
  if (!(z > V.znear)) return false;
  P.mc[0] = fmaf(V.R[0], G.m[0], fmaf(V.R[1], G.m[1], fmaf(V.R[2], G.m[2], V.t[0])));
  P.mc[1] = fmaf(V.R[3], G.m[0], fmaf(V.R[4], G.m[1], fmaf(V.R[5], G.m[2], V.t[1])));
  P.mc[2] = z;
  // activations
  P.o = 1.f / (1.f + expf(-G.ol));
  if (!(P.o >= kAlphaMin)) return false;
#pragma unroll
  for (int i = 0; i < 3; ++i) P.s[i] = expf(G.ls[i]);
  const float qq = G.q[0] * G.q[0] + G.q[1] * G.q[1] + G.q[2] * G.q[2] + G.q[3] * G.q[3];
  if (!(qq > 0.f)) return false;
  P.qinv = rsqrtf(qq);
#pragma unroll
  for (int i = 0; i < 4; ++i) P.qn[i] = G.q[i] * P.qinv;
  quat_rot(P.qn[0], P.qn[1], P.qn[2], P.qn[3], P.Rq);
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int k = 0; k < 3; ++k) P.M[i * 3 + k] = P.Rq[i * 3 + k] * P.s[k];
  // EWA: J = d(pinhole)/d(mu_c) with clamped x/z, y/z
  const float iz = 1.f / z;
  const float limx = kJacClamp * 0.5f * (float)V.width / V.fx;
  const float limy = kJacClamp * 0.5f * (float)V.height / V.fy;
  const float xz = P.mc[0] * iz, yz = P.mc[1] * iz;
  P.clampx = (xz < -limx) || (xz > limx);
  P.clampy = (yz < -limy) || (yz > limy);
  P.txz = fminf(fmaxf(xz, -limx), limx);
  P.tyz = fminf(fmaxf(yz, -limy), limy);
  P.J00 = V.fx * iz;
  P.J11 = V.fy * iz;
  P.J02 = -V.fx * P.txz * iz;
  P.J12 = -V.fy * P.tyz * iz;
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    P.T2[j] = P.J00 * V.R[j] + P.J02 * V.R[6 + j];
    P.T2[3 + j] = P.J11 * V.R[3 + j] + P.J12 * V.R[6 + j];
  }
  // V = T2 M; Sigma' = V V^T + 0.3 I
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int k = 0; k < 3; ++k)
      P.V[i * 3 + k] = P.T2[i * 3 + 0] * P.M[0 * 3 + k] + P.T2[i * 3 + 1] * P.M[1 * 3 + k] +
                       P.T2[i * 3 + 2] * P.M[2 * 3 + k];
  const float a0 = P.V[0] * P.V[0] + P.V[1] * P.V[1] + P.V[2] * P.V[2];
  const float c0 = P.V[3] * P.V[3] + P.V[4] * P.V[4] + P.V[5] * P.V[5];
  P.a = a0 + kCovDilation;
  P.b = P.V[0] * P.V[3] + P.V[1] * P.V[4] + P.V[2] * P.V[5];
  P.c = c0 + kCovDilation;
  // det = a c - b^2 = |V0 x V1|^2 + 0.3 (|V0|^2 + |V1|^2) + 0.09 (Lagrange identity)
  const float x0 = P.V[1] * P.V[5] - P.V[2] * P.V[4];
  const float x1 = P.V[2] * P.V[3] - P.V[0] * P.V[5];
  const float x2 = P.V[0] * P.V[4] - P.V[1] * P.V[3];
  P.det = x0 * x0 + x1 * x1 + x2 * x2 + kCovDilation * (a0 + c0) + kCovDilation * kCovDilation;
  if (!(P.det > 0.f) || !isfinite(P.det)) return false;
  // conic Q = Sigma'^-1 = L L^T: l11 = sqrt(c/det), l21 = -b / sqrt(c det), l22 = 1/sqrt(c)
  const float sq = rsqrtf(P.c * P.det);
  P.l11 = P.c * sq;
  P.l21 = -P.b * sq;
  P.l22 = rsqrtf(P.c);
  // flattened-Gaussian normal: axis of the smallest log-scale (ties -> lowest)
  int k = 0;
  if (G.ls[1] < G.ls[k]) k = 1;
  if (G.ls[2] < G.ls[k]) k = 2;
  P.axis = k;
  const float nw0 = k == 0 ? P.Rq[0] : (k == 1 ? P.Rq[1] : P.Rq[2]);
  const float nw1 = k == 0 ? P.Rq[3] : (k == 1 ? P.Rq[4] : P.Rq[5]);
  const float nw2 = k == 0 ? P.Rq[6] : (k == 1 ? P.Rq[7] : P.Rq[8]);
  float nc0 = V.R[0] * nw0 + V.R[1] * nw1 + V.R[2] * nw2;
  float nc1 = V.R[3] * nw0 + V.R[4] * nw1 + V.R[5] * nw2;
  float nc2 = V.R[6] * nw0 + V.R[7] * nw1 + V.R[8] * nw2;
  const float dot = nc0 * P.mc[0] + nc1 * P.mc[1] + nc2 * P.mc[2];
  P.sign = dot > 0.f ? -1.f : 1.f;
  P.nc[0] = P.sign * nc0;
  P.nc[1] = P.sign * nc1;
  P.nc[2] = P.sign * nc2;
  P.dist = -(P.nc[0] * P.mc[0] + P.nc[1] * P.mc[1] + P.nc[2] * P.mc[2]);
  return true;
}

// SH coefficients are read per pair, only for pairs that are binned (a thread
// reads its Gaussian's 192-byte row as 12 float4, whole sectors): most
// Gaussians of a view touch no active tile and their colour is never needed.
// The adjoint's SH gradients are summed in a shared-memory slab (row stride 49
// floats, conflict-free) and written out as coalesced float4.
constexpr int kPreThreads = 128;
#ifndef PGSAG_PRE_MINB
#define PGSAG_PRE_MINB 8  // resident projection blocks per SM the register budget must allow
#endif
#ifndef PGSAG_PRE_BWD_MINB
#define PGSAG_PRE_BWD_MINB 4  // resident adjoint blocks per SM the register budget must allow
#endif
constexpr int kShStride = 49;
constexpr size_t kShSlabBytes = (size_t)kPreThreads * kShStride * sizeof(float);
constexpr int kPreBwdSlice = 2 * kPreThreads;  // Gaussians per adjoint block

__host__ __device__ __forceinline__ size_t views_bytes(uint32_t n_views) {
  return ((size_t)n_views * sizeof(pgsag_view) + 15) & ~(size_t)15;
}

// raw colour (before the clamp at 0) sum_k Y_k sh[k][ch] + 1/2 of one Gaussian
__device__ __forceinline__ void sh_colour(const float* __restrict__ sh, uint32_t g, const float Y[16],
                                          float col[3]) {
  const float4* row = reinterpret_cast<const float4*>(sh + 48ull * g);
  col[0] = col[1] = col[2] = kShOffset;
#pragma unroll
  for (int i = 0; i < 12; ++i) {
    const float4 v = __ldg(row + i);
    const float e[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int f = 4 * i + j;  // flat index 3 k + ch
      col[f % 3] += Y[f / 3] * e[j];
    }
  }
}

__global__ void __launch_bounds__(kPreThreads, PGSAG_PRE_MINB) k_preprocess(uint32_t n, const float* __restrict__ means,
                             const float* __restrict__ log_scales, const float* __restrict__ quats,
                             const float* __restrict__ opacity_logit, const float* __restrict__ sh,
                             uint32_t n_views, const pgsag_view* __restrict__ views,
                             const int32_t* __restrict__ tile_act, const uint32_t* __restrict__ sat,
                             float4* __restrict__ rec, uint32_t* __restrict__ dkey,
                             uint4* __restrict__ bininfo, unsigned long long* __restrict__ tmask,
                             float4* __restrict__ grad2d, int32_t* status) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  pgsag_view* sv = reinterpret_cast<pgsag_view*>(smem_raw);
  {
    const uint32_t words = n_views * (uint32_t)(sizeof(pgsag_view) / 4);
    const uint32_t* src = reinterpret_cast<const uint32_t*>(views);
    uint32_t* dst = reinterpret_cast<uint32_t*>(smem_raw);
    for (uint32_t i = threadIdx.x; i < words; i += blockDim.x) dst[i] = src[i];
  }
  // the step's device status starts here: this kernel sets no flag, so the
  // reset (one store) needs no memset node before it
  if (blockIdx.x == 0 && threadIdx.x == 0) *status = 0;
  __syncthreads();
  set_campos(sv, n_views);
  __syncthreads();
  const uint32_t g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= n) return;
  const GaussIn G = load_gauss(g, means, log_scales, quats, opacity_logit);
  for (uint32_t vi = 0; vi < n_views; ++vi) {
    const pgsag_view& V = sv[vi];
    if (g < V.g_begin || g >= V.g_end) continue;
    const uint32_t p = V.pair_base + (g - V.g_begin);
    PairFwd P;
    bool vis = pair_forward(V, G, P);
    float mx = 0.f, my = 0.f, ex = 0.f, ey = 0.f;
    int x0 = 0, y0 = 0, x1 = -1, y1 = -1;
    uint32_t touched = 0;
    unsigned long long mask = 0ull;  // tiles binned to, bit (ty - y0) * width + (tx - x0) of the rect
    float mi = 0.f, mf = 0.f, ni = 0.f, nf = 0.f;
    if (vis) {
      // the SH row (192 B) is read only if the pair is binned; ask L2 for it now
      // so that the read after the tile test finds it there
      {
        const float* row = sh + 48ull * g;
        asm volatile("prefetch.global.L2 [%0];" ::"l"(row));
        asm volatile("prefetch.global.L2 [%0];" ::"l"(row + 32));
      }
      {
        float xh, xl, yh, yl, zh, zl;
        dot3_comp(V.R + 0, G.m, V.t[0], xh, xl);
        dot3_comp(V.R + 3, G.m, V.t[1], yh, yl);
        dot3_comp(V.R + 6, G.m, V.t[2], zh, zl);
        mean2d_coord(xh, xl, zh, zl, V.fx, V.cx, mi, mf);
        mean2d_coord(yh, yl, zh, zl, V.fy, V.cy, ni, nf);
      }
      mx = mi + mf;
      my = ni + nf;
      // axis-aligned box of the alpha >= 1/255 ellipse, + 1 px
      const float r2 = 2.f * logf(255.f * P.o);
      ex = sqrtf(fmaxf(r2, 0.f) * P.a) + 1.f;
      ey = sqrtf(fmaxf(r2, 0.f) * P.c) + 1.f;
      const float fu0 = ceilf(mx - ex - 0.5f), fu1 = floorf(mx + ex - 0.5f);
      const float fv0 = ceilf(my - ey - 0.5f), fv1 = floorf(my + ey - 0.5f);
      if (fu0 <= (float)(V.width - 1) && fu1 >= 0.f && fv0 <= (float)(V.height - 1) && fv1 >= 0.f) {
        const int u0 = (int)fmaxf(fu0, 0.f), u1 = (int)fminf(fu1, (float)(V.width - 1));
        const int v0 = (int)fmaxf(fv0, 0.f), v1 = (int)fminf(fv1, (float)(V.height - 1));
        x0 = u0 / V.tile_w;
        x1 = u1 / V.tile_w;
        y0 = v0 / V.tile_h;
        y1 = v1 / V.tile_h;
        const uint32_t sw = (uint32_t)V.tiles_x + 1;
        const uint32_t* S = sat + V.sat_base;
        touched = __ldg(S + (uint32_t)(y1 + 1) * sw + (uint32_t)(x1 + 1)) -
                  __ldg(S + (uint32_t)y0 * sw + (uint32_t)(x1 + 1)) -
                  __ldg(S + (uint32_t)(y1 + 1) * sw + (uint32_t)x0) + __ldg(S + (uint32_t)y0 * sw + (uint32_t)x0);
        if (touched && (x1 - x0 + 1) * (y1 - y0 + 1) <= kExactTileMax) {
          const EllipseTest et = ellipse_test(P.l11, P.l21, P.l22, -logf(255.f * P.o));
          const int32_t* ta = tile_act + V.tile_base;
          const int rw = x1 - x0 + 1;
          // every tile of the rectangle is active (the usual case inside the mask):
          // the activity map need not be read tile by tile
          const bool all_active = touched == (uint32_t)(rw * (y1 - y0 + 1));
          for (int ty = y0; ty <= y1; ++ty)
            for (int tx = x0; tx <= x1; ++tx)
              if ((all_active || __ldg(ta + ty * V.tiles_x + tx) >= 0) &&
                  tile_hit(et, mi, ni, mf, nf, tx, ty, V.tile_w, V.tile_h, V.width, V.height))
                mask |= 1ull << ((ty - y0) * rw + (tx - x0));
          touched = (uint32_t)__popcll(mask);
        }
      } else {
        vis = false;
      }
    }
    float4* R4 = rec + 4ull * p;
    if (!vis || touched == 0) {
      // culled or binned to no active tile: the record and the mask are never read
      dkey[p] = 0xffffffffu;
      bininfo[p] = make_uint4(0u, 0u, vi, 0u);
      continue;
    }
    // colour: degree-3 SH at the viewing direction (world frame)
    float dx = G.m[0] - V.reserved0[0], dy = G.m[1] - V.reserved0[1], dz = G.m[2] - V.reserved0[2];
    const float il = rsqrtf(dx * dx + dy * dy + dz * dz);
    dx *= il;
    dy *= il;
    dz *= il;
    float Y[16];
    sh_eval(dx, dy, dz, Y);
    float col[3];
    sh_colour(sh, g, Y, col);
    R4[0] = make_float4(mi, ni, P.l11, P.l21);
    R4[1] = make_float4(P.l22, P.o, fmaxf(col[0], 0.f), fmaxf(col[1], 0.f));
    R4[2] = make_float4(fmaxf(col[2], 0.f), P.dist, P.nc[0], P.nc[1]);
    R4[3] = make_float4(P.nc[2], -logf(255.f * P.o), mf, nf);
    dkey[p] = __float_as_uint(P.mc[2]);
    tmask[p] = mask;
    if (grad2d) {  // the adjoint accumulates into this row
      float4* G2 = grad2d + 4ull * p;
      G2[0] = G2[1] = G2[2] = G2[3] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    bininfo[p] = make_uint4((uint32_t)x0 | ((uint32_t)y0 << 16), (uint32_t)x1 | ((uint32_t)y1 << 16), vi,
                            touched);
  }
}

// Adjoint of pair_forward + colour, accumulating into the raw-parameter gradients.
// A Gaussian with no binned pair in any view has zero gradient and reads nothing
// but its pairs' tile counts.
// Eq. 11's flattening term of Gaussian g: d(w mean_g min_k exp(ls_gk)) / d ls_gk*
// = w exp(ls_gk*) / n at the smallest axis k* (ties: lowest axis), added to gls;
// returns whether the term is on.
__device__ __forceinline__ bool add_flatten(uint32_t g, const float* __restrict__ log_scales, uint32_t n,
                                            float flatten_weight, float sc, float gls[3]) {
  if (flatten_weight == 0.f) return false;
  const float l0 = __ldg(log_scales + 3ull * g), l1 = __ldg(log_scales + 3ull * g + 1),
              l2 = __ldg(log_scales + 3ull * g + 2);
  const int k = (l0 <= l1 && l0 <= l2) ? 0 : (l1 <= l2 ? 1 : 2);
  const float lk = k == 0 ? l0 : (k == 1 ? l1 : l2);
  const float d = flatten_weight * sc * expf(lk) / (float)n;
  gls[0] += k == 0 ? d : 0.f;
  gls[1] += k == 1 ? d : 0.f;
  gls[2] += k == 2 ? d : 0.f;
  return true;
}

// Gradients of Gaussian g's means, log-scales, quaternion and opacity logit:
// written, or added to what the buffers hold.
__device__ __forceinline__ void store_small(uint32_t g, const float gm[3], const float gls[3], const float gq[4],
                                            float gol, int accumulate, float* __restrict__ d_means,
                                            float* __restrict__ d_log_scales, float* __restrict__ d_quats,
                                            float* __restrict__ d_opac) {
  float4* q4 = reinterpret_cast<float4*>(d_quats) + g;
  if (accumulate) {
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      d_means[3ull * g + i] += gm[i];
      d_log_scales[3ull * g + i] += gls[i];
    }
    float4 o = *q4;
    o.x += gq[0];
    o.y += gq[1];
    o.z += gq[2];
    o.w += gq[3];
    *q4 = o;
    d_opac[g] += gol;
  } else {
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      d_means[3ull * g + i] = gm[i];
      d_log_scales[3ull * g + i] = gls[i];
    }
    *q4 = make_float4(gq[0], gq[1], gq[2], gq[3]);
    d_opac[g] = gol;
  }
}

__global__ void __launch_bounds__(kPreThreads, PGSAG_PRE_BWD_MINB) k_preprocess_bwd(uint32_t n, const float* __restrict__ means,
                                 const float* __restrict__ log_scales,
                                 const float* __restrict__ quats,
                                 const float* __restrict__ opacity_logit,
                                 const float* __restrict__ sh, uint32_t n_views,
                                 const pgsag_view* __restrict__ views,
                                 const uint4* __restrict__ bininfo,
                                 const float* __restrict__ grad2d, int accumulate,
                                 float* __restrict__ d_means, float* __restrict__ d_log_scales,
                                 float* __restrict__ d_quats, float* __restrict__ d_opac,
                                 float* __restrict__ d_sh, const float* __restrict__ dout_scale,
                                 float flatten_weight, const int32_t* status) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  pgsag_view* sv = reinterpret_cast<pgsag_view*>(smem_raw);
  {
    const uint32_t words = n_views * (uint32_t)(sizeof(pgsag_view) / 4);
    const uint32_t* src = reinterpret_cast<const uint32_t*>(views);
    uint32_t* dst = reinterpret_cast<uint32_t*>(smem_raw);
    for (uint32_t i = threadIdx.x; i < words; i += blockDim.x) dst[i] = src[i];
  }
  // dynamic shared memory: [view table | SH gradient slab]
  float* s_gsh = reinterpret_cast<float*>(smem_raw + views_bytes(n_views));
  // Each warp works on its own 64 consecutive Gaussians of the block's slice,
  // with its own list and its own 32 rows of the slab: no block barrier after
  // the view table is set up.
  constexpr int kPreWarps = kPreThreads / 32;
  constexpr int kPerWarp = kPreBwdSlice / kPreWarps;
  static_assert(kPerWarp == 64, "two Gaussians of a warp's share per lane");
  __shared__ uint32_t s_list[kPreWarps][kPerWarp];  // each warp's Gaussians with a binned pair, ascending
  if (status_bad(status)) return;
  __syncthreads();
  set_campos(sv, n_views);
  __syncthreads();
  const float sc = dout_scale ? __ldg(dout_scale) : 1.f;
  const float zero3[3] = {0.f, 0.f, 0.f}, zero4[4] = {0.f, 0.f, 0.f, 0.f};
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t wbase = blockIdx.x * kPreBwdSlice + warp * kPerWarp;
  uint32_t* wl = s_list[warp];

  // 1. binned flags; a Gaussian with no binned pair gets its (zero or flattening
  // only) gradient here, the others go to the warp's list
  uint32_t nl = 0, bits0 = 0, bits1 = 0;
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const uint32_t g = wbase + k * 32 + lane;
    bool binned = false;
    if (g < n) {
      for (uint32_t vi = 0; vi < n_views && !binned; ++vi) {
        const pgsag_view& V = sv[vi];
        if (g >= V.g_begin && g < V.g_end) binned = __ldg(&bininfo[V.pair_base + (g - V.g_begin)].w) != 0u;
      }
    }
    const uint32_t bal = __ballot_sync(kFull, binned);
    (k == 0 ? bits0 : bits1) = bal;
    if (binned) {
      wl[nl + __popc(bal & ((1u << lane) - 1u))] = g;
    } else if (g < n) {
      float gls[3] = {0.f, 0.f, 0.f};
      const bool flat = add_flatten(g, log_scales, n, flatten_weight, sc, gls);
      // accumulate = 2: the row holds zeros already (written only for a flattening term)
      if (accumulate == 0 || flat)
        store_small(g, zero3, gls, zero4, 0.f, accumulate == 1, d_means, d_log_scales, d_quats, d_opac);
    }
    nl += __popc(bal);
  }
  if (accumulate == 0 && wbase < n) {
    // zero SH rows of the Gaussians without a binned pair (coalesced float4)
    const uint32_t nb = min((uint32_t)kPerWarp, n - wbase);
    float4* dst = reinterpret_cast<float4*>(d_sh + 48ull * wbase);
    for (uint32_t i = lane; i < nb * 12; i += 32) {
      const uint32_t row = i / 12;
      if (!(((row < 32 ? bits0 : bits1) >> (row & 31)) & 1u)) dst[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
  }
  // the list length goes through shared memory: held in a register across the
  // per-Gaussian work below it costs some 290 B of spills per thread
  __shared__ uint32_t s_nl[kPreWarps];
  if (lane == 0) s_nl[warp] = nl;
  __syncwarp();
  nl = s_nl[warp];

  // 2. the adjoint of every binned pair of the listed Gaussians, one Gaussian per
  // lane and round, SH gradients summed in the lane's slab row
  for (uint32_t base = 0; base < nl; base += 32) {
    // the warp's 32 slab rows zeroed together before a warp barrier (a lane that
    // zeroes its own row lets the compiler hold the row's sums in registers:
    // 56 B of spills per thread)
    for (uint32_t i = threadIdx.x & 31; i < 32 * kShStride; i += 32)
      s_gsh[(threadIdx.x & ~31u) * kShStride + i] = 0.f;
    __syncwarp();
    const uint32_t li = base + (threadIdx.x & 31);
    if (li < nl) {
      float* gsh = s_gsh + threadIdx.x * kShStride;
      const uint32_t g = s_list[threadIdx.x >> 5][li];
      float gm[3] = {0.f, 0.f, 0.f}, gls[3] = {0.f, 0.f, 0.f}, gq[4] = {0.f, 0.f, 0.f, 0.f}, gol = 0.f;
      const GaussIn G = load_gauss(g, means, log_scales, quats, opacity_logit);
      for (uint32_t vi = 0; vi < n_views; ++vi) {
        const pgsag_view& V = sv[vi];
        if (g < V.g_begin || g >= V.g_end) continue;
        const uint32_t p = V.pair_base + (g - V.g_begin);
        if (__ldg(&bininfo[p].w) == 0u) continue;  // culled or off-screen: no contribution
        PairFwd P;
        if (!pair_forward(V, G, P)) continue;
        const float4* G4 = reinterpret_cast<const float4*>(grad2d) + 4ull * p;
        const float4 g0 = __ldg(G4 + 0), g1 = __ldg(G4 + 1), g2 = __ldg(G4 + 2), g3 = __ldg(G4 + 3);
        // grad2d = {dmx, dmy, dl11, dl21, dl22, do, dr, dg, db, dd, dnx, dny, dnz}
        const float dmx = g0.x, dmy = g0.y, dl11 = g0.z, dl21 = g0.w;
        const float dl22 = g1.x, dop = g1.y;
        const float drgb[3] = {g1.z, g1.w, g2.x};
        const float dd = g2.y;
        float dn[3] = {g2.z, g2.w, g3.x};

        float dmc[3] = {0.f, 0.f, 0.f};
        // opacity
        gol += dop * P.o * (1.f - P.o);

        // colour (zero gradient where the colour was clamped at 0)
        {
          float dx = G.m[0] - V.reserved0[0], dy = G.m[1] - V.reserved0[1], dz = G.m[2] - V.reserved0[2];
          const float il = rsqrtf(dx * dx + dy * dy + dz * dz);
          dx *= il;
          dy *= il;
          dz *= il;
          float Y[16];
          sh_eval(dx, dy, dz, Y);
          float raw[3];
          sh_colour(sh, g, Y, raw);
          float dc[3];
#pragma unroll
          for (int ch = 0; ch < 3; ++ch) dc[ch] = raw[ch] < 0.f ? 0.f : drgb[ch];
          // cw[k] = sum_ch dc[ch] sh[k][ch] (second read of the row, from L1/L2)
          float cw[16];
#pragma unroll
          for (int k = 0; k < 16; ++k) cw[k] = 0.f;
          {
            const float4* row = reinterpret_cast<const float4*>(sh + 48ull * g);
#pragma unroll
            for (int i = 0; i < 12; ++i) {
              const float4 v = __ldg(row + i);
              const float e[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
              for (int j = 0; j < 4; ++j) {
                const int f = 4 * i + j;
                cw[f / 3] += dc[f % 3] * e[j];
              }
            }
          }
#pragma unroll
          for (int k = 0; k < 16; ++k) {
            gsh[3 * k + 0] += dc[0] * Y[k];
            gsh[3 * k + 1] += dc[1] * Y[k];
            gsh[3 * k + 2] += dc[2] * Y[k];
          }
          float gx, gy, gz;
          sh_grad(dx, dy, dz, cw, gx, gy, gz);
          // dir = v/|v|: d v = (g - dir (dir . g)) / |v|
          const float dg = dx * gx + dy * gy + dz * gz;
          gm[0] += (gx - dx * dg) * il;
          gm[1] += (gy - dy * dg) * il;
          gm[2] += (gz - dz * dg) * il;
        }

        // plane distance d = -n_c . mu_c
#pragma unroll
        for (int i = 0; i < 3; ++i) {
          dmc[i] -= dd * P.nc[i];
          dn[i] -= dd * P.mc[i];
        }
        // n_c = sign * W n_w, n_w = column `axis` of Rq
        float dRq[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        {
          const float s = P.sign;
          const float dnw0 = s * (V.R[0] * dn[0] + V.R[3] * dn[1] + V.R[6] * dn[2]);
          const float dnw1 = s * (V.R[1] * dn[0] + V.R[4] * dn[1] + V.R[7] * dn[2]);
          const float dnw2 = s * (V.R[2] * dn[0] + V.R[5] * dn[1] + V.R[8] * dn[2]);
#pragma unroll
          for (int kk = 0; kk < 3; ++kk) {
            if (P.axis == kk) {
              dRq[0 * 3 + kk] += dnw0;
              dRq[1 * 3 + kk] += dnw1;
              dRq[2 * 3 + kk] += dnw2;
            }
          }
        }

        // 2D mean
        const float z = P.mc[2], iz = 1.f / z, iz2 = iz * iz;
        dmc[0] += dmx * V.fx * iz;
        dmc[1] += dmy * V.fy * iz;
        dmc[2] -= dmx * V.fx * P.mc[0] * iz2 + dmy * V.fy * P.mc[1] * iz2;

        // Cholesky factor of the conic -> Sigma' = (a, b, c), det = a c - b^2:
        // l11 = sqrt(c/det), l21 = -b/sqrt(c det), l22 = c^-1/2
        const float a = P.a, b = P.b, c = P.c;
        const float iD = 1.f / P.det, ic = 1.f / c;
        const float da = -0.5f * c * iD * (dl11 * P.l11 + dl21 * P.l21);
        const float db = dl11 * P.l11 * b * iD - dl21 * a * P.l11 * iD;
        const float dcc = dl11 * P.l11 * 0.5f * (ic - a * iD) - dl21 * P.l21 * 0.5f * (ic + a * iD) -
                          dl22 * 0.5f * P.l22 * ic;
        // Sigma' = V V^T: dV0 = 2 da V0 + db V1, dV1 = db V0 + 2 dc V1
        float dV[6];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          dV[k] = 2.f * da * P.V[k] + db * P.V[3 + k];
          dV[3 + k] = db * P.V[k] + 2.f * dcc * P.V[3 + k];
        }
        // V = T2 M: dT2 = dV M^T, dM = T2^T dV
        float dT2[6];
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
          for (int j = 0; j < 3; ++j)
            dT2[i * 3 + j] = dV[i * 3 + 0] * P.M[j * 3 + 0] + dV[i * 3 + 1] * P.M[j * 3 + 1] +
                             dV[i * 3 + 2] * P.M[j * 3 + 2];
        float dM[9];
#pragma unroll
        for (int j = 0; j < 3; ++j)
#pragma unroll
          for (int k = 0; k < 3; ++k) dM[j * 3 + k] = P.T2[j] * dV[k] + P.T2[3 + j] * dV[3 + k];
        // T2 = J W: dJ = dT2 W^T (entries J00, J02, J11, J12)
        const float dJ00 = dT2[0] * V.R[0] + dT2[1] * V.R[1] + dT2[2] * V.R[2];
        const float dJ02 = dT2[0] * V.R[6] + dT2[1] * V.R[7] + dT2[2] * V.R[8];
        const float dJ11 = dT2[3] * V.R[3] + dT2[4] * V.R[4] + dT2[5] * V.R[5];
        const float dJ12 = dT2[3] * V.R[6] + dT2[4] * V.R[7] + dT2[5] * V.R[8];
        dmc[2] += -dJ00 * V.fx * iz2 - dJ11 * V.fy * iz2;
        if (!P.clampx) {
          // J02 = -fx x / z^2
          dmc[0] += -dJ02 * V.fx * iz2;
          dmc[2] += dJ02 * 2.f * V.fx * P.mc[0] * iz2 * iz;
        } else {
          // J02 = -fx txz / z with txz constant
          dmc[2] += dJ02 * V.fx * P.txz * iz2;
        }
        if (!P.clampy) {
          dmc[1] += -dJ12 * V.fy * iz2;
          dmc[2] += dJ12 * 2.f * V.fy * P.mc[1] * iz2 * iz;
        } else {
          dmc[2] += dJ12 * V.fy * P.tyz * iz2;
        }
        // M = Rq diag(s)
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          const float dsk = dM[0 * 3 + k] * P.Rq[0 * 3 + k] + dM[1 * 3 + k] * P.Rq[1 * 3 + k] +
                            dM[2 * 3 + k] * P.Rq[2 * 3 + k];
          gls[k] += dsk * P.s[k];
#pragma unroll
          for (int j = 0; j < 3; ++j) dRq[j * 3 + k] += dM[j * 3 + k] * P.s[k];
        }
        // Rq(q^) -> q^
        {
          const float w = P.qn[0], x = P.qn[1], y = P.qn[2], zq = P.qn[3];
          const float* Gr = dRq;
          const float dw = 2.f * (-zq * Gr[1] + y * Gr[2] + zq * Gr[3] - x * Gr[5] - y * Gr[6] + x * Gr[7]);
          const float dx = 2.f * (y * Gr[1] + zq * Gr[2] + y * Gr[3] - 2.f * x * Gr[4] - w * Gr[5] +
                                  zq * Gr[6] + w * Gr[7] - 2.f * x * Gr[8]);
          const float dy = 2.f * (-2.f * y * Gr[0] + x * Gr[1] + w * Gr[2] + x * Gr[3] + zq * Gr[5] -
                                  w * Gr[6] + zq * Gr[7] - 2.f * y * Gr[8]);
          const float dz = 2.f * (-2.f * zq * Gr[0] - w * Gr[1] + x * Gr[2] + w * Gr[3] - 2.f * zq * Gr[4] +
                                  y * Gr[5] + x * Gr[6] + y * Gr[7]);
          // q^ = q/|q|: dq = (dq^ - q^ (q^ . dq^)) / |q|
          const float pr = w * dw + x * dx + y * dy + zq * dz;
          gq[0] += (dw - w * pr) * P.qinv;
          gq[1] += (dx - x * pr) * P.qinv;
          gq[2] += (dy - y * pr) * P.qinv;
          gq[3] += (dz - zq * pr) * P.qinv;
        }
        // mu_c = W mu + t
#pragma unroll
        for (int j = 0; j < 3; ++j) gm[j] += V.R[0 * 3 + j] * dmc[0] + V.R[1 * 3 + j] * dmc[1] + V.R[2 * 3 + j] * dmc[2];
      }

      add_flatten(g, log_scales, n, flatten_weight, sc, gls);
      store_small(g, gm, gls, gq, gol, accumulate == 1, d_means, d_log_scales, d_quats, d_opac);
    }
    __syncwarp();
    // SH gradient rows of this round: coalesced float4 stores, 12 per row
    const uint32_t nr = min(32u, nl - base);
    for (uint32_t i = threadIdx.x & 31; i < nr * 12; i += 32) {
      const uint32_t row = i / 12, c4 = i - row * 12;
      const float* sg = s_gsh + ((threadIdx.x & ~31u) + row) * kShStride + 4 * c4;
      float4 v = make_float4(sg[0], sg[1], sg[2], sg[3]);
      float4* dst = reinterpret_cast<float4*>(d_sh + 48ull * s_list[threadIdx.x >> 5][base + row]) + c4;
      if (accumulate == 1) {
        const float4 o = *dst;
        v.x += o.x;
        v.y += o.y;
        v.z += o.z;
        v.w += o.w;
      }
      *dst = v;
    }
    __syncwarp();
  }
}

}  // namespace pgsag

using namespace pgsag;

static bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

extern "C" int pgsag_preprocess(uint32_t n_gauss, const float* means, const float* log_scales,
                                const float* quats, const float* opacity_logit, const float* sh,
                                uint32_t n_views, const pgsag_view* views, const int32_t* tile_act,
                                const uint32_t* sat, float* rec, uint32_t* depth_key, void* bininfo,
                                uint64_t* tile_mask, float* grad2d, int32_t* status, void* stream) {
  if (n_views == 0 || n_views > PGSAG_MAX_VIEWS) return PGSAG_ERR_UNSUPPORTED;
  if (!views || !sat || !tile_act || !status) return PGSAG_ERR_ARG;
  if (n_gauss == 0) return cudaMemsetAsync(status, 0, sizeof(int32_t), (cudaStream_t)stream) == cudaSuccess ? PGSAG_OK : PGSAG_ERR_CUDA;
  if (!means || !log_scales || !quats || !opacity_logit || !sh || !rec || !depth_key || !bininfo || !tile_mask)
    return PGSAG_ERR_ARG;
  if (!aligned16(quats) || !aligned16(sh) || !aligned16(rec) || !aligned16(bininfo) || ((uintptr_t)tile_mask & 7u))
    return PGSAG_ERR_ARG;
  if (grad2d && !aligned16(grad2d)) return PGSAG_ERR_ARG;
  const unsigned threads = kPreThreads;
  const size_t smem = views_bytes(n_views);
  if (smem > 48 * 1024 &&
      cudaFuncSetAttribute(k_preprocess, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return PGSAG_ERR_CUDA;
  k_preprocess<<<pgsag_div_up(n_gauss, threads), threads, smem, (cudaStream_t)stream>>>(
      n_gauss, means, log_scales, quats, opacity_logit, sh, n_views, views, tile_act, sat,
      reinterpret_cast<float4*>(rec), depth_key, reinterpret_cast<uint4*>(bininfo),
      reinterpret_cast<unsigned long long*>(tile_mask), reinterpret_cast<float4*>(grad2d), status);
  PGSAG_CHECK_LAUNCH();
  return PGSAG_OK;
}

extern "C" int pgsag_preprocess_bwd(uint32_t n_gauss, const float* means, const float* log_scales,
                                    const float* quats, const float* opacity_logit, const float* sh,
                                    uint32_t n_views, const pgsag_view* views, const void* bininfo,
                                    const float* grad2d, int accumulate, float* d_means,
                                    float* d_log_scales, float* d_quats, float* d_opacity_logit,
                                    float* d_sh, const float* dout_scale, float flatten_weight,
                                    int32_t* status, void* stream) {
  if (n_views == 0 || n_views > PGSAG_MAX_VIEWS) return PGSAG_ERR_UNSUPPORTED;
  if (!views || !status || accumulate < 0 || accumulate > 2) return PGSAG_ERR_ARG;
  if (n_gauss == 0) return PGSAG_OK;
  if (!means || !log_scales || !quats || !opacity_logit || !sh || !bininfo || !grad2d || !d_means ||
      !d_log_scales || !d_quats || !d_opacity_logit || !d_sh)
    return PGSAG_ERR_ARG;
  if (!aligned16(quats) || !aligned16(sh) || !aligned16(d_quats) || !aligned16(d_sh) || !aligned16(grad2d) ||
      !aligned16(bininfo))
    return PGSAG_ERR_ARG;
  const unsigned threads = kPreThreads;
  const size_t smem = views_bytes(n_views) + kShSlabBytes;
  if (cudaFuncSetAttribute(k_preprocess_bwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return PGSAG_ERR_CUDA;
  k_preprocess_bwd<<<pgsag_div_up(n_gauss, (uint32_t)kPreBwdSlice), threads, smem, (cudaStream_t)stream>>>(
      n_gauss, means, log_scales, quats, opacity_logit, sh, n_views, views,
      reinterpret_cast<const uint4*>(bininfo), grad2d, accumulate, d_means, d_log_scales, d_quats,
      d_opacity_logit, d_sh, dout_scale, flatten_weight, status);
  PGSAG_CHECK_LAUNCH();
  return PGSAG_OK;
}
