// Microbenchmarks of the arithmetic units the rasterizers are bound by, for the roofline the
// benchmark reports: the special-function unit's base-2 exponential (ex2.approx.ftz.f32, one per
// evaluated (pixel, Gaussian) pair in the plain blend) and the FP32 fused multiply-add. Built as a
// separate library (libtgs_microbench.so) used only by the benchmark; not part of the tgs ABI.
#include <cuda_runtime.h>
#include <stdint.h>

namespace {

constexpr int kChains = 8;  // independent dependency chains per thread (hide the unit's latency)

__device__ __forceinline__ float ex2(float x) {
  float y;
  asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Each thread runs kChains chains of `iters` dependent ex2 (the argument stays in [-1, 1]: x <-
// ex2(x) - 1.5 has a fixed point near -0.9), then stores their sum so nothing is dead code.
__global__ void k_ex2(int iters, float seed, float* out) {
  float x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = seed * (float)(threadIdx.x + c) * 1e-6f;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = ex2(x[c]) - 1.5f;
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// The same structure with FFMA: x <- x * a + b (|a| < 1 keeps x bounded).
__global__ void k_ffma(int iters, float seed, float* out) {
  float x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = seed * (float)(threadIdx.x + c) * 1e-6f;
  const float a = 0.999f, b = 1e-3f;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = fmaf(x[c], a, b);
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <typename K>
int time_kernel(K kernel, int blocks, int threads, int iters, float* out, float* ms) {
  cudaEvent_t a, b;
  if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) return 2;
  kernel<<<blocks, threads>>>(iters / 8, 1.0f, out);  // warm-up
  cudaEventRecord(a);
  kernel<<<blocks, threads>>>(iters, 1.0f, out);
  cudaEventRecord(b);
  const cudaError_t e = cudaEventSynchronize(b);
  cudaEventElapsedTime(ms, a, b);
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  return e == cudaSuccess && cudaGetLastError() == cudaSuccess ? 0 : 2;
}

}  // namespace

// Measured rates on the current device: ex2 results per second and FFMA per second (not FLOP:
// one FFMA is two FLOP), and the SM count. `out` is caller-provided device scratch of at least
// 4 * blocks * 512 bytes for blocks = 8 * SM count. Returns 0 on success.
extern "C" int tgs_microbench_peaks(float* out, int sm_count, double* ex2_per_s,
                                    double* ffma_per_s) {
  const int threads = 512, blocks = 8 * sm_count, iters = 4096;
  float ms = 0.f;
  if (time_kernel(k_ex2, blocks, threads, iters, out, &ms) != 0) return 2;
  *ex2_per_s = (double)blocks * threads * iters * kChains / (ms * 1e-3);
  if (time_kernel(k_ffma, blocks, threads, iters, out, &ms) != 0) return 2;
  *ffma_per_s = (double)blocks * threads * iters * kChains / (ms * 1e-3);
  return 0;
}
