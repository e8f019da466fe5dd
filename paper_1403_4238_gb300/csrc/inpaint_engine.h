// Host/device interface of the persistent fill-loop engine (engine.cu).
#pragma once
#include <cuda.h>
#include <cudaTypedefs.h>

#include "inpaint_internal.cuh"

namespace inp {

constexpr int kEngThreads = 512;
constexpr int kEngWarps = kEngThreads / 32;

// Per-team synchronisation words (global memory).
struct TeamCtl {
  unsigned epoch;   // iterations completed by the team (release-published)
  unsigned arrive;  // members arrived in the current iteration
  unsigned pad[30]; // keep teams on separate 128-byte lines
};

struct EngineArgs {
  const ImgState* imgs;        // [n_imgs]
  const CUtensorMap* tmaps;    // [n_imgs], 64-byte aligned
  const int* cta_team;         // [grid]
  const int* team_first;       // [n_teams + 1] first CTA of each team
  const int* team_img_off;     // [n_teams + 1] offsets into team_img
  const int* team_img;         // images of each team, in processing order
  TeamCtl* teams;              // [n_teams]
  unsigned long long* partials;// [grid]
  int* err;                    // INPAINT_ERR_TIMEOUT if a bounded wait gave up
  unsigned long long wait_limit_ns;
};

// Kernels of one patch radius (engine_r<R>.cu).
struct EngineFns {
  cudaError_t (*launch)(int srw, const EngineArgs& ea, int grid, cudaStream_t st);
  cudaError_t (*occupancy)(int srw, int* blocks_per_sm);
  cudaError_t (*update_fast)(const ImgState& s, unsigned long long cond, int use_cond,
                             cudaStream_t st);
  cudaError_t (*prio_init)(const ImgState& s, cudaStream_t st);
};
const EngineFns* engine_fns_r1();
const EngineFns* engine_fns_r2();
const EngineFns* engine_fns_r3();
const EngineFns* engine_fns_r4();
const EngineFns* engine_fns_r5();
const EngineFns* engine_fns_r6();
const EngineFns* engine_fns_r7();
const EngineFns* engine_fns_r8();

cudaError_t engine_occupancy(int r, int sr, int* blocks_per_sm);
cudaError_t engine_launch(int r, int sr, const EngineArgs& ea, int grid, cudaStream_t st);
int make_image_tmap(const ImgState& s, int srw, CUtensorMap* out);
cudaError_t launch_update_fast(const ImgState& s, unsigned long long cond, int use_cond,
                               cudaStream_t st);

}  // namespace inp
