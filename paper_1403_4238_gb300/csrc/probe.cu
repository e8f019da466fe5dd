// Measured instruction-rate peaks of the GPU, the denominators of the
// roofline fractions this library reports for its arithmetic-bound kernels.
//
// Each probe kernel runs long independent dependency chains of one operation
// on every SM (4 CTAs x 256 threads per SM, 8 chains per thread) and is timed
// with CUDA events; the SM clock during the probe is derived from clock64()
// against the global nanosecond timer.
#include <cstring>

#include "inpaint_internal.cuh"
#include "inpaint_probe.h"

namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;

// One SSD evaluation of this library: byte-SIMD |a-b| then a 4-way byte dot
// product of the difference with itself (3 channels + a zero byte).
__global__ void p_ssd(uint32_t seed, int iters, uint32_t* sink) {
  uint32_t acc[kChains], a[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) {
    acc[k] = threadIdx.x + k;
    a[k] = seed ^ (k * 0x01010101u) ^ (blockIdx.x << 8);
  }
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) {
      const uint32_t d = __vabsdiffu4(a[k], acc[k]);
      acc[k] = __dp4a(d, d, acc[k]);
    }
  }
  uint32_t s = 0;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s ^= acc[k];
  if (s == 0x12345678u) sink[0] = s;
}

// The chains are coupled (each update reads its neighbour chain), so no
// iteration count can be folded into a closed form: every multiply-add and
// every three-input add below is executed.
__global__ void p_imad(uint32_t seed, int iters, uint32_t* sink) {
  uint32_t acc[kChains];
  const uint32_t c = seed >> 3;
#pragma unroll
  for (int k = 0; k < kChains; ++k) acc[k] = seed + k + threadIdx.x;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) acc[k] = acc[k] * (acc[(k + 1) % kChains] | 1u) + c;
  }
  uint32_t s = 0;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s ^= acc[k];
  if (s == 0x12345678u) sink[0] = s;
}

__global__ void p_iadd3(uint32_t seed, int iters, uint32_t* sink) {
  uint32_t acc[kChains];
  const uint32_t c = seed >> 3;
#pragma unroll
  for (int k = 0; k < kChains; ++k) acc[k] = seed + k + threadIdx.x;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) acc[k] = acc[k] + acc[(k + 1) % kChains] + c;
  }
  uint32_t s = 0;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s ^= acc[k];
  if (s == 0x12345678u) sink[0] = s;
}

__global__ void p_dadd(uint32_t seed, int iters, uint32_t* sink) {
  double acc[kChains];
  const double c = 1e-30 * (double)(seed & 7);
#pragma unroll
  for (int k = 0; k < kChains; ++k) acc[k] = (double)(k + threadIdx.x);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) acc[k] = __dadd_rn(acc[k], c);
  }
  double s = 0;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += acc[k];
  if (s == -1.0) sink[0] = 1;
}

__global__ void p_clock(int spins, unsigned long long* out) {
  unsigned long long t0, t1;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
  const long long c0 = clock64();
  long long c1 = c0;
  while (c1 - c0 < spins) c1 = clock64();
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t1));
  out[0] = (unsigned long long)(c1 - c0);
  out[1] = t1 - t0;
}

template <class K>
double rate(K kern, int blocks, int iters, uint32_t* sink, double ops_per_iter_thread) {
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  kern<<<blocks, kThreads>>>(12345u, iters / 4, sink);  // warm-up
  cudaEventRecord(e0);
  kern<<<blocks, kThreads>>>(12345u, iters, sink);
  cudaEventRecord(e1);
  cudaEventSynchronize(e1);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return (double)blocks * kThreads * iters * ops_per_iter_thread / (ms * 1e-3);
}

}  // namespace

extern "C" int inpaint_probe_peaks(inpaint_peaks* out) {
  if (!out) return INPAINT_ERR_ARG;
  memset(out, 0, sizeof *out);
  int dev = 0;
  cudaDeviceProp prop;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&prop, dev) != cudaSuccess)
    return INPAINT_ERR_CUDA;
  out->sm_count = prop.multiProcessorCount;
  uint32_t* sink = nullptr;
  unsigned long long* clk = nullptr;
  if (cudaMalloc(&sink, 16) != cudaSuccess) return INPAINT_ERR_NOMEM;
  if (cudaMalloc(&clk, 16) != cudaSuccess) {
    cudaFree(sink);
    return INPAINT_ERR_NOMEM;
  }
  const int blocks = 4 * prop.multiProcessorCount;
  out->ssd_evals_per_s = rate(p_ssd, blocks, 1 << 15, sink, kChains);
  out->imad_per_s = rate(p_imad, blocks, 1 << 15, sink, kChains);
  out->iadd3_per_s = rate(p_iadd3, blocks, 1 << 15, sink, kChains);
  out->dadd_per_s = rate(p_dadd, blocks, 1 << 11, sink, kChains);
  p_clock<<<1, 1>>>(20000000, clk);
  unsigned long long h[2] = {0, 0};
  cudaError_t e = cudaMemcpy(h, clk, sizeof h, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && h[1] > 0) out->sm_clock_mhz = (double)h[0] / (double)h[1] * 1e3;
  cudaFree(sink);
  cudaFree(clk);
  e = cudaGetLastError();
  return e == cudaSuccess ? INPAINT_OK : INPAINT_ERR_CUDA;
}
