// Fused Adam step over a flat float32 parameter buffer.  The paper does not
// name its optimiser; Adam is the 3DGS convention it builds on (Sec. 3.1).
#include <math.h>

#include "common.cuh"

namespace pgsag {

__global__ void k_adam(uint64_t n, float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, float lr, float b1, float b2, float eps, float c1, float c2) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

struct AdamTable {
  pgsag_adam_tensor t[PGSAG_ADAM_MAX_TENSORS];
  uint64_t start[PGSAG_ADAM_MAX_TENSORS + 1];  // prefix of the tensor sizes
};

// step[0] += 1; step[1], step[2] = the bias corrections 1 - b^step (float bits),
// in double as on the host path.
__global__ void k_step_advance(int32_t* step, float b1, float b2, const int32_t* status) {
  if (status_bad(status)) return;
  const int32_t st = step[0] + 1;
  step[0] = st;
  step[1] = __float_as_int((float)(1.0 - pow((double)b1, (double)st)));
  step[2] = __float_as_int((float)(1.0 - pow((double)b2, (double)st)));
}

__device__ __forceinline__ void adam1(float& p, float g, float& m, float& v, float lr, float b1, float b2, float eps,
                                      float ic1, float ic2) {
  m = b1 * m + (1.f - b1) * g;
  v = b2 * v + (1.f - b2) * g * g;
  p -= lr * (m * ic1) / (sqrtf(v * ic2) + eps);
}

// The tensors one after the other, each over the whole grid: 16-byte loads and
// stores (4 elements per thread and round) where the tensor's arrays are 16-byte
// aligned, the remainder element by element.  Bias corrections from
// k_step_advance.  HBM-bound: 28 bytes per element.
__global__ void __launch_bounds__(256) k_adam_multi(uint32_t nt, const __grid_constant__ AdamTable T, float b1,
                                                    float b2, float eps, const int32_t* __restrict__ step,
                                                    const int32_t* status) {
  if (status_bad(status)) return;
  const float ic1 = 1.f / __int_as_float(step[1]), ic2 = 1.f / __int_as_float(step[2]);
  const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint32_t k = 0; k < nt; ++k) {
    const pgsag_adam_tensor& D = T.t[k];
    const float lr = D.lr;
    uint64_t done = 0;
    if (!(((uintptr_t)D.p | (uintptr_t)D.g | (uintptr_t)D.m | (uintptr_t)D.v) & 15u)) {
      const uint64_t n4 = D.n / 4;
      float4* p4 = reinterpret_cast<float4*>(D.p);
      const float4* g4 = reinterpret_cast<const float4*>(D.g);
      float4* m4 = reinterpret_cast<float4*>(D.m);
      float4* v4 = reinterpret_cast<float4*>(D.v);
      for (uint64_t i = tid; i < n4; i += stride) {
        const float4 g = __ldg(g4 + i);
        float4 p = p4[i], m = m4[i], v = v4[i];
        adam1(p.x, g.x, m.x, v.x, lr, b1, b2, eps, ic1, ic2);
        adam1(p.y, g.y, m.y, v.y, lr, b1, b2, eps, ic1, ic2);
        adam1(p.z, g.z, m.z, v.z, lr, b1, b2, eps, ic1, ic2);
        adam1(p.w, g.w, m.w, v.w, lr, b1, b2, eps, ic1, ic2);
        p4[i] = p;
        m4[i] = m;
        v4[i] = v;
      }
      done = n4 * 4;
    }
    for (uint64_t i = done + tid; i < D.n; i += stride) {
      float p = D.p[i], m = D.m[i], v = D.v[i];
      adam1(p, D.g[i], m, v, lr, b1, b2, eps, ic1, ic2);
      D.p[i] = p;
      D.m[i] = m;
      D.v[i] = v;
    }
  }
}

}  // namespace pgsag

extern "C" int pgsag_adam_multi(uint32_t n_tensors, const pgsag_adam_tensor* tensors, float beta1, float beta2,
                                float eps, int32_t* step, int32_t* status, void* stream) {
  if (n_tensors > PGSAG_ADAM_MAX_TENSORS) return PGSAG_ERR_UNSUPPORTED;
  if (!step || !status || (n_tensors && !tensors)) return PGSAG_ERR_ARG;
  pgsag::AdamTable T{};
  uint64_t total = 0;
  for (uint32_t k = 0; k < n_tensors; ++k) {
    const pgsag_adam_tensor& D = tensors[k];
    if (D.n && (!D.p || !D.g || !D.m || !D.v)) return PGSAG_ERR_ARG;
    T.t[k] = D;
    T.start[k] = total;
    total += D.n;
  }
  T.start[n_tensors] = total;
  cudaStream_t s = (cudaStream_t)stream;
  pgsag::k_step_advance<<<1, 1, 0, s>>>(step, beta1, beta2, status);
  PGSAG_CHECK_LAUNCH();
  if (total == 0) return PGSAG_OK;
  const uint64_t want = (total + 4 * 256 - 1) / (4 * 256);
  const unsigned blocks = (unsigned)(want < 148ull * 8ull ? want : 148ull * 8ull);
  pgsag::k_adam_multi<<<blocks, 256, 0, s>>>(n_tensors, T, beta1, beta2, eps, step, status);
  PGSAG_CHECK_LAUNCH();
  return PGSAG_OK;
}

extern "C" int pgsag_adam(uint64_t n, float* p, const float* g, float* m, float* v, float lr, float beta1,
                          float beta2, float eps, int32_t step, void* stream) {
  if (n == 0) return PGSAG_OK;
  if (!p || !g || !m || !v || step < 1) return PGSAG_ERR_ARG;
  const float c1 = (float)(1.0 - pow((double)beta1, (double)step));
  const float c2 = (float)(1.0 - pow((double)beta2, (double)step));
  const unsigned blocks = (unsigned)((n + 255) / 256 < 148u * 16u ? (n + 255) / 256 : 148u * 16u);
  pgsag::k_adam<<<blocks, 256, 0, (cudaStream_t)stream>>>(n, p, g, m, v, lr, beta1, beta2, eps, c1, c2);
  PGSAG_CHECK_LAUNCH();
  return PGSAG_OK;
}
