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

}  // namespace pgsag

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
