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

// Tensor-core search of the engine (Sec. 3, Eq. 3-4 as correlations; the
// exact BF16 form of the tensor-core search).  A tile is kTcRows candidate
// rows x 8N candidate columns (N = 64 or 128): the MMA's M = 128 rows are
// 16 candidate rows x 8 column shifts, its N columns blocks of 8 candidate
// columns.  Tiles are numbered row-major; searching CTA k of a team takes
// tiles k, k + ns, ...
constexpr int kTcRows = 16;
constexpr int kTcRing = 8;  // most slots of the shared-memory ring
constexpr int kTcRps = 2;   // source rows per ring slot (one bulk copy)
struct TcTiles {
  int N;         // MMA N: 8-column candidate blocks per tile (64 or 128)
  int ntx, nty;  // tiles per row / per column of the candidate rectangle
  int xs0;       // first source column of tile column 0 (a multiple of 8)
};
__host__ __device__ inline int tc_chunks(int r) { return (2 * r + 1 + 14) / 8; }  // 8-tap chunks of a row
__host__ __device__ inline TcTiles tc_tiles(const ImgState& s) {
  TcTiles t{0, 0, 0, 0};
  if (s.cx1 < s.cx0 || s.cy1 < s.cy0) return t;
  t.xs0 = (s.cx0 - s.r) & ~7;
  const int wneed = s.cx1 - s.r - t.xs0 + 1;  // candidate columns from the first tile's column 0
  t.ntx = (wneed + 1023) / 1024;
  t.N = (wneed + 8 * t.ntx - 1) / (8 * t.ntx) <= 64 ? 64 : 128;
  t.nty = (s.cy1 - s.cy0 + kTcRows) / kTcRows;
  return t;
}
// Plane geometry of an image (fills the tc_* fields and prows of s): the
// segment of tile column tx is columns [xs0 + 8N tx, + 8 (N + chunks - 1)),
// the rows every tile reads (y0 - r .. y0 + 15 + r) all exist.  Returns the
// plane elements to allocate (0: no tile).
__host__ __device__ inline size_t tc_plane_layout(ImgState& s) {
  const TcTiles t = tc_tiles(s);
  if (t.ntx == 0) return 0;
  s.tc_xs0 = t.xs0;
  s.tc_w = 8 * t.N;
  s.tc_len = 8 * (t.N + tc_chunks(s.r) - 1);
  s.tc_ntx = t.ntx;
  const int hr = s.cy0 + kTcRows * t.nty + s.r;
  s.prows = hr > s.H ? hr : s.H;
  return (size_t)t.ntx * s.prows * 5 * s.tc_len;
}
// The five planes of the image's current pixels (run before every engine
// launch of an image in the tensor-core form).
cudaError_t launch_planes(const ImgState& s, cudaStream_t st);

// Per-team synchronisation words (global memory).
struct TeamCtl {
  unsigned long long pub;  // epoch | next px | next py | stop (release-published)
  unsigned expired;        // the launch's time budget ended this team's work
  unsigned copied;         // e + 1 once round e's fill is in the image and its planes
                           // (release-published; the tensor-core searchers then
                           // prefetch the next round's source rows)
  unsigned pad[28];        // keep teams on separate 128-byte lines
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
  int tc_cols;                 // tensor-memory columns every CTA holds for the
                               // tensor-core search (0: no image uses it)
};

// The mbarriers of an engine CTA, at the start of its shared memory (the
// kernel initialises them once per launch).
struct EngBars {
  uint64_t full[2];               // TMA completion of the two streaming stages
  uint64_t tc_full[kTcRing];      // tensor-core search: source rows landed in ring slot
  uint64_t tc_empty[kTcRing];     // their MMAs (both issuers) completed: the slot is free
  uint64_t tc_done;               // a tile's MMAs (both issuers) completed
  uint32_t tmem;                  // tensor-memory base written by tcgen05.alloc
  uint32_t pad;
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
  uint32_t tmem;                // tensor-memory base address (tensor-core search)
  uint32_t tc_rows;             // ring slots filled so far (their phases)
  int tc_pref;                  // slots of the next round's first tile already requested
  uint32_t tc_tiles;            // tiles whose MMAs completed so far (done barrier phases)
  int tc_nb;                    // ring slots tc_rows was counted with (0: none yet)
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
