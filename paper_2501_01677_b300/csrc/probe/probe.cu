// Arithmetic-throughput probes for the roofline of the ALU-bound render
// kernels: FP32 fused multiply-add (scalar and packed .f32x2) and the ex2
// special-function unit, each timed with CUDA events on the given stream.
// Measurement infrastructure only (libpgsag_probe.so); not part of libpgsag.
#include <cuda_runtime.h>
#include <stdint.h>

namespace {

constexpr int kChains = 8;  // independent dependency chains per thread

__global__ void __launch_bounds__(256) k_fma(float* out, int iters, float a, float b) {
  float x[kChains];
#pragma unroll
  for (int i = 0; i < kChains; ++i) x[i] = 1e-3f * (float)threadIdx.x + (float)i;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < kChains; ++i) x[i] = fmaf(x[i], a, b);
  }
  float s = 0.f;
#pragma unroll
  for (int i = 0; i < kChains; ++i) s += x[i];
  if (s == 123456.789f) out[0] = s;  // keeps the chains alive
}

__global__ void __launch_bounds__(256) k_fma2(float* out, int iters, float a, float b) {
  float2 x[kChains];
#pragma unroll
  for (int i = 0; i < kChains; ++i) x[i] = make_float2(1e-3f * (float)threadIdx.x + (float)i, (float)i);
  const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < kChains; ++i) x[i] = __ffma2_rn(x[i], a2, b2);
  }
  float s = 0.f;
#pragma unroll
  for (int i = 0; i < kChains; ++i) s += x[i].x + x[i].y;
  if (s == 123456.789f) out[0] = s;
}

__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__global__ void __launch_bounds__(256) k_ex2(float* out, int iters) {
  float x[kChains];
#pragma unroll
  for (int i = 0; i < kChains; ++i) x[i] = -1e-3f * (float)(threadIdx.x + i);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < kChains; ++i) x[i] = -ex2_approx(x[i]);  // stays in [-1, 0]
  }
  float s = 0.f;
#pragma unroll
  for (int i = 0; i < kChains; ++i) s += x[i];
  if (s == 123456.789f) out[0] = s;
}

}  // namespace

// kind 0: scalar FFMA, 1: packed FFMA2 (both in TFLOP/s, an FMA counted as 2),
// 2: ex2.approx (in Gop/s).  Launches 8 blocks of 256 threads per SM, once to
// warm up and once timed.  Returns 0 on success, -1 on a CUDA error.
extern "C" int pgsag_probe_throughput(int kind, int iters, double* result, void* stream) {
  if (!result || iters <= 0 || kind < 0 || kind > 2) return -1;
  cudaStream_t s = (cudaStream_t)stream;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return -1;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return -1;
  const unsigned blocks = (unsigned)sms * 8u, threads = 256u;
  float* out = nullptr;
  if (cudaMalloc(&out, sizeof(float)) != cudaSuccess) return -1;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float ms = 0.f;
  for (int rep = 0; rep < 2; ++rep) {
    cudaEventRecord(e0, s);
    if (kind == 0) k_fma<<<blocks, threads, 0, s>>>(out, iters, 0.99999f, 1e-6f);
    if (kind == 1) k_fma2<<<blocks, threads, 0, s>>>(out, iters, 0.99999f, 1e-6f);
    if (kind == 2) k_ex2<<<blocks, threads, 0, s>>>(out, iters);
    cudaEventRecord(e1, s);
  }
  const bool ok = cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  if (!ok || ms <= 0.f) {
    cudaGetLastError();
    return -1;
  }
  const double ops = (double)blocks * threads * (double)iters * kChains * (kind == 1 ? 2.0 : 1.0);
  *result = kind == 2 ? ops / (ms * 1e-3) / 1e9 : 2.0 * ops / (ms * 1e-3) / 1e12;
  return 0;
}
