// The persistent engine kernel: one cooperative launch runs the fill loops
// of every image of every team to completion (single image: one team of all
// CTAs; batch: many teams, each with a list of images).  The per-image body
// for the image's patch radius is selected at run time.
#include "inpaint_engine.h"
#include "ptx.cuh"

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
  // the barriers sit at the start of shared memory
  EngBars* bars = reinterpret_cast<EngBars*>(x.smem);
  if (threadIdx.x == 0) {
    mbar_init(&bars->full[0], 1);
    mbar_init(&bars->full[1], 1);
    if (ea.tc_cols > 0) {
      for (int i = 0; i < kTcRing; ++i) {
        mbar_init(&bars->tc_full[i], 1);
        mbar_init(&bars->tc_empty[i], 2);  // one commit from each issuer
      }
      mbar_init(&bars->tc_done, 2);
    }
  }
  fence_mbar_init();
  // tensor memory of the tensor-core search: held for the whole launch (one
  // CTA per SM, so the allocation never waits on another engine CTA)
  if (ea.tc_cols > 0 && threadIdx.x < 32) tc_alloc(&bars->tmem, (uint32_t)ea.tc_cols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  x.tmem = ea.tc_cols > 0 ? bars->tmem : 0u;
  x.tc_rows = 0;
  x.tc_tiles = 0;
  x.tc_nb = 0;
  x.tc_pref = 0;
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
  // every tile's MMAs were waited for before its accumulators were read
  if (ea.tc_cols > 0) {
    tc_fence_before();
    __syncthreads();
    if (threadIdx.x < 32) {
      tc_fence_after();
      tc_dealloc(x.tmem, (uint32_t)ea.tc_cols);
    }
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
