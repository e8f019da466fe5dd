// Host/device interface of the persistent fill-loop engine (engine.cu).
#pragma once
#include <cuda.h>
#include <cudaTypedefs.h>

#include "inpaint_internal.cuh"

namespace inp {

constexpr int kEngThreads = 512;
constexpr int kEngWarps = kEngThreads / 32;
constexpr int kEngBatchRows = 32;  // candidate rows of a search batch (one per lane)

// Smallest staged width >= n words that is a multiple of 4 with an odd
// number of 16-byte chunks: rows of a tile then start in different bank
// quadruples, so 8 lanes reading 16 bytes each from 8 consecutive rows (one
// phase of a 128-bit shared load) touch 32 distinct banks.
__host__ __device__ constexpr int width_odd16(int n) {
  return ((((n + 3) & ~3) / 4) % 2) ? ((n + 3) & ~3) : ((n + 3) & ~3) + 4;
}
// Candidate columns of a search batch: 16 warps side by side, 4 * srw
// candidates per lane.
__host__ __device__ constexpr int eng_batch_cols(int srw) { return kEngWarps * 4 * srw; }
// TMA boxes of a batch: the source window (words) and the validity counts.
__host__ __device__ constexpr int eng_tile_width(int r, int srw) { return width_odd16(eng_batch_cols(srw) + 2 * r); }
__host__ __device__ constexpr int eng_count_width(int srw) { return eng_batch_cols(srw) + 4; }

// Per-team synchronisation words (global memory).
struct TeamCtl {
  unsigned long long pub;  // epoch | next px | next py | stop (release-published)
  unsigned expired;        // the launch's time budget ended this team's work
  unsigned pad[29];        // keep teams on separate 128-byte lines
};

struct EngineArgs {
  const ImgState* imgs;        // [n_imgs]
  const CUtensorMap* tmaps;    // [2 * n_imgs]: pixels, counts per image; 64-byte aligned
  const int* cta_team;         // [grid]
  const int* team_first;       // [n_teams + 1] first CTA of each team
  const int* team_img_off;     // [n_teams + 1] offsets into team_img
  const int* team_img;         // images of each team, in processing order
  TeamCtl* teams;              // [n_teams]
  unsigned long long* partials;// [grid] each CTA's best key of the round, tagged with the round
  int* err;                    // INPAINT_ERR_TIMEOUT if a bounded wait gave up
  unsigned long long wait_limit_ns;
  unsigned long long tick_ns;  // > 0: teams stop between iterations once the launch
                               // has run this long (serving ticks); 0: run to the end
  int withhold;                // failure injection: > 0 makes searcher rank withhold - 1
                               // of every team skip its arrival; 0 normally
};

// Per-CTA engine state carried from one image of a team's list to the next.
struct EngCtx {
  uint8_t* smem;                // dynamic shared memory, 128-byte aligned
  uint8_t* smem_end;            // end of the dynamic shared memory
  int rank, tsize;              // this CTA's rank in its team, team size
  TeamCtl* tc;
  unsigned long long* tpart;    // partial keys of the team's CTAs
  uint32_t ph0, ph1;            // phase parities of the two TMA barriers
  unsigned epoch;               // team publications seen
  unsigned long long t_start;   // global timer at the CTA's start (tick budget)
};

// Per-image engine body for radius R and SRW rows per warp (engine_r<R>.cu),
// called from the one engine kernel (engine_multi.cu) by the image's radius.
#define INP_DECL_RUN_IMAGE(R)                                            \
  __device__ void run_image_r##R##_s1(const EngineArgs& ea, int j, EngCtx& x); \
  __device__ void run_image_r##R##_s2(const EngineArgs& ea, int j, EngCtx& x);
INP_DECL_RUN_IMAGE(1)
INP_DECL_RUN_IMAGE(2)
INP_DECL_RUN_IMAGE(3)
INP_DECL_RUN_IMAGE(4)
INP_DECL_RUN_IMAGE(5)
INP_DECL_RUN_IMAGE(6)
INP_DECL_RUN_IMAGE(7)
INP_DECL_RUN_IMAGE(8)
#undef INP_DECL_RUN_IMAGE

// Host-side entry points of one patch radius (engine_r<R>.cu).
struct EngineFns {
  size_t (*smem_bytes)(int srw);  // least dynamic shared memory the engine needs for this radius
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

const EngineFns* engine_fns(int r);
// The engine kernel (engine_multi.cu); every launch takes engine_launch_smem()
// bytes, at least the largest engine_fns(r)->smem_bytes(srw) of its images.
cudaError_t engine_occupancy(size_t smem, int* blocks_per_sm);
// Dynamic shared memory of every engine launch: all an SM offers one CTA.
size_t engine_launch_smem();
cudaError_t engine_launch(size_t smem, const EngineArgs& ea, int grid, cudaStream_t st);
int make_image_tmap(const ImgState& s, int srw, CUtensorMap* out);  // writes out[0], out[1]
int make_image_tmap_box(const ImgState& s, int box_w, int box_h, CUtensorMap* out);
cudaError_t launch_update_fast(const ImgState& s, unsigned long long cond, int use_cond,
                               cudaStream_t st);

}  // namespace inp
