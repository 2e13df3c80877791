// Device calibration used by the roofline report and the autotuner: the
// rate at which L2 executes 16-byte floating-point reductions (the
// operation the adjoint passes are bound by) on this device.
#include "internal.h"

namespace cs {

namespace {

__device__ __forceinline__ uint32_t mix32(uint32_t x) {
  x ^= x >> 16;
  x *= 0x7feb352du;
  x ^= x >> 15;
  x *= 0x846ca68bu;
  x ^= x >> 16;
  return x;
}

// Each thread issues `iters` v4.f32 reductions to pseudo-random 16-byte
// slots of a buffer of (mask + 1) slots.
__global__ void __launch_bounds__(256)
k_red_rate(float4* __restrict__ buf, uint32_t mask, int iters) {
  const uint32_t g = blockIdx.x * blockDim.x + threadIdx.x;
  for (int i = 0; i < iters; ++i) {
    const uint32_t q = mix32(g * 0x9E3779B1u + (uint32_t)i) & mask;
    atomicAdd(buf + q, make_float4(1.f, 1.f, 1.f, 1.f));
  }
}

}  // namespace

cudaError_t measure_red_rate(void* scratch, size_t bytes, int num_sms, cudaStream_t s,
                             double* gops) {
  // largest power-of-two slot count that fits, at most 1 Mi slots (16 MiB)
  size_t slots = 1;
  while (slots * 2 * sizeof(float4) <= bytes && slots < ((size_t)1 << 20)) slots *= 2;
  const uint32_t mask = (uint32_t)(slots - 1);
  float4* buf = static_cast<float4*>(scratch);
  const int blocks = num_sms * 8, iters = 256;
  cudaError_t e = cudaMemsetAsync(buf, 0, slots * sizeof(float4), s);
  if (e != cudaSuccess) return e;
  cudaEvent_t a, b;
  if ((e = cudaEventCreate(&a)) != cudaSuccess) return e;
  if ((e = cudaEventCreate(&b)) != cudaSuccess) {
    cudaEventDestroy(a);
    return e;
  }
  float best = 1e30f;
  for (int rep = 0; rep < 3 && e == cudaSuccess; ++rep) {
    cudaEventRecord(a, s);
    k_red_rate<<<blocks, 256, 0, s>>>(buf, mask, iters);
    count_launches(1);
    cudaEventRecord(b, s);
    e = cudaEventSynchronize(b);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
    if (e == cudaSuccess && ms < best) best = ms;
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (e != cudaSuccess) return e;
  *gops = (double)blocks * 256.0 * iters / (best * 1e-3) / 1e9;
  return cudaGetLastError();
}

}  // namespace cs
