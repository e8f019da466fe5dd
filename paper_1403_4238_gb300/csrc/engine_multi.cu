// The persistent engine kernel: one cooperative launch runs the fill loops
// of every image of every team to completion (single image: one team of all
// CTAs; batch: many teams, each with a list of images).  The per-image body
// for the image's patch radius is selected at run time.
#include "inpaint_engine.h"

namespace inp {

__device__ inline unsigned long long ld_acquire64_pub(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

// Dispatch on the image's patch radius and search rows per warp.
__device__ inline void run_by_radius(const EngineArgs& ea, int j, EngCtx& x) {
  const bool two = ea.imgs[j].srw == 2;
  switch (ea.imgs[j].r) {
#define INP_CASE(R)                                  \
  case R:                                            \
    if (two) run_image_r##R##_s2(ea, j, x);          \
    else run_image_r##R##_s1(ea, j, x);              \
    break;
    INP_CASE(1) INP_CASE(2) INP_CASE(3) INP_CASE(4) INP_CASE(5) INP_CASE(6) INP_CASE(7)
    INP_CASE(8)
#undef INP_CASE
    default:
      break;
  }
}

__global__ void __launch_bounds__(kEngThreads, 1) k_engine(EngineArgs ea) {
  extern __shared__ __align__(128) uint8_t smem_raw[];
  EngCtx x;
  x.smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
  uint32_t dyn;
  asm("mov.u32 %0, %%dynamic_smem_size;" : "=r"(dyn));
  x.smem_end = smem_raw + dyn;
  const int team = ea.cta_team[blockIdx.x];
  const int first = ea.team_first[team];
  x.rank = blockIdx.x - first;
  x.tsize = ea.team_first[team + 1] - first;
  x.tc = &ea.teams[team];
  x.tpart = ea.partials + first;
  // the two TMA completion barriers sit at the start of shared memory
  uint64_t* bars = reinterpret_cast<uint64_t*>(x.smem);
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"((uint32_t)__cvta_generic_to_shared(&bars[0])) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"((uint32_t)__cvta_generic_to_shared(&bars[1])) : "memory");
  }
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  __syncthreads();
  x.ph0 = 0;
  x.ph1 = 0;
  x.epoch = (unsigned)ld_acquire64_pub(&x.tc->pub);
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(x.t_start));
  for (int li = ea.team_img_off[team]; li < ea.team_img_off[team + 1]; ++li) {
    run_by_radius(ea, ea.team_img[li], x);
    // the leader's last publication of the image was acquired by every CTA
    // of the team, so all of them see the same flag here
    unsigned expired;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(expired) : "l"(&x.tc->expired) : "memory");
    if (expired) break;
  }
}

cudaError_t engine_occupancy(size_t smem, int* blocks_per_sm) {
  cudaError_t e = cudaFuncSetAttribute(k_engine, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_engine, kEngThreads, smem);
}

size_t engine_launch_smem() {
  static size_t cached = 0;
  if (cached) return cached;
  int dev = 0, optin = 0;
  cudaFuncAttributes fa;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess ||
      cudaFuncGetAttributes(&fa, k_engine) != cudaSuccess)
    return 0;
  cached = (size_t)optin - fa.sharedSizeBytes;
  return cached;
}

cudaError_t engine_launch(size_t smem, const EngineArgs& ea, int grid, cudaStream_t st) {
  cudaError_t e = cudaFuncSetAttribute(k_engine, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  // key slots: all ones (a tag no round carries) before the launch
  e = cudaMemsetAsync(ea.partials, 0xff, sizeof(unsigned long long) * (size_t)grid, st);
  if (e != cudaSuccess) return e;
  void* args[] = {const_cast<EngineArgs*>(&ea)};
  return cudaLaunchCooperativeKernel((const void*)k_engine, dim3(grid), dim3(kEngThreads), args, smem, st);
}

}  // namespace inp
