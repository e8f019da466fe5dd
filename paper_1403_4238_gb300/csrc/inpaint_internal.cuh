// Device-side state and helpers shared by the kernels of libinpaint.
//
// Data layout in HBM for one image of W x H pixels (patch radius r):
//   img    uint32[H*pitch]  RGBA8 (R in the low byte, A = 0): one pixel per
//                        word, so a pixel is one 32-bit load and byte-SIMD
//                        works on it; pitch = W rounded up to 4 words so rows
//                        start on 16-byte boundaries (TMA tiles need that)
//   omega  uint8[W*H]    1 = pixel of the target region Omega (still unknown)
//   gray   uint8[W*H]    integer luma of known pixels (0 under Omega)
//   conf   double[W*H]   confidence C (Eq. 2), 0 under Omega
//   count  int32[H*pitch] for a candidate centre q: unknown pixels in Psi_q
//                        (valid source patch iff 0); borders and the row
//                        padding hold a large value; same pitch as img so a
//                        TMA tile of counts can ride with the pixel tile
//   prio   uint64[W*H]   priority key of a front pixel: bits(P(p)) + 1; 0 off
//                        the front (P >= 0, so the bits order like the values)
//   pconf  double[W*H]   C(p) of the last priority evaluation at p
//   tiles0 PrioBest[]    best (key, idx) per 16x16-pixel tile of prio
//   tiles1 PrioBest[]    best per 16x16 block of tiles0 (256x256 pixels): the
//                        argmax over the front reads only these few entries
//   ctrl   Ctrl          loop control block (selected p^, counters, status)
//   trace  inpaint_step_info[trace_cap]   one record per iteration
//   planes uint16[5][prows*ppitch]  tensor-core form in the engine only: BF16
//                        R' G' B' (byte - 128) and the two halves of the
//                        square sum, the operands of its correlations
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include "inpaint.h"

namespace inp {

constexpr int kT0 = 16;         // edge of a level-0 priority tile (pixels)
constexpr int kT1 = 16;         // edge of a level-1 tile (level-0 tiles)
constexpr int kMaxRadius = 32;  // largest supported patch radius
constexpr int kCountInvalid = 1 << 28;  // count of a centre whose patch leaves the image

// Plain search tile: 8 candidate rows x 128 candidate columns per CTA, each
// thread computes 4 horizontally adjacent candidates.
constexpr int kSearchTW = 128;
constexpr int kSearchTH = 8;
constexpr int kSearchS = 4;
constexpr int kSearchThreads = (kSearchTW / kSearchS) * kSearchTH;  // 256
// Generic (large-radius) search tile.
constexpr int kGenTW = 64;
constexpr int kGenTH = 8;
constexpr int kGenS = 2;
constexpr int kGenThreads = (kGenTW / kGenS) * kGenTH;  // 256

constexpr int kUpdThreads = 512;

struct PrioBest {
  unsigned long long key;
  int idx;
  int pad;
};

struct Ctrl {
  int iter;        // iterations completed
  int remaining;   // |Omega|
  int status;      // 0 = running, else an inpaint_status error
  int px, py;      // target centre selected for the next iteration (-1: none)
  int n_valid;     // valid candidate centres inside the search rectangle
  int iter_limit;  // kernels do nothing once iter reaches this
  int n_adm;       // partial-overlap search: admissible candidates of the current search
  double prio;     // P(p^) of the selected target
  double conf;     // C(p^) of the selected target
  unsigned long long evals;  // sum over iterations of n_cand * n_known
  inpaint_step_info last;    // record of the most recent iteration
  // persistent-engine phase clocks (global timer, ns): search round (from the
  // previous publish to the last arrival) and update phase, summed
  unsigned long long t_search, t_update, t_last;
  int timed_iters;
  int tc_rounds;   // engine search rounds run in the tensor-core form
};

// Window codes of the speculative phase (update_fast.cuh): a pixel of the
// (4R+3)^2 priority window is outside the image, or in the image and not on
// the post-fill front; front pixels carry their packed normal instead.
constexpr int kSpecOutside = -2;   // window pixel outside the image
constexpr int kSpecNotFront = -1;  // in the image, not on the post-fill front

// Entry of a compact work list handled by thread t: consecutive entries go
// to warps 0..3 in turn (one warp per SM sub-partition), so a short list of
// long FP64 dependency chains uses all four sub-partitions with few active
// lanes each.
__device__ inline int list_entry(int t) { return ((t & 31) << 2) | ((t >> 5) & 3) | ((t >> 7) << 7); }

// The squared lengths nn = |n|^2 a Sobel normal of a binary mask can take
// (nx, ny in [-4, 4]) for the data term D = (dot / sqrt(nn)) / 510, dot in
// [0, 2040], and their codes.
constexpr int kDTabRows = 14;
__host__ __device__ inline int dtab_code(int nn) {
  switch (nn) {
    case 1: return 0;
    case 2: return 1;
    case 4: return 2;
    case 5: return 3;
    case 8: return 4;
    case 9: return 5;
    case 10: return 6;
    case 13: return 7;
    case 16: return 8;
    case 17: return 9;
    case 18: return 10;
    case 20: return 11;
    case 25: return 12;
    default: return 13;  // 32, the largest
  }
}
__host__ __device__ inline int dtab_nn(int code) {
  switch (code) {
    case 0: return 1;
    case 1: return 2;
    case 2: return 4;
    case 3: return 5;
    case 4: return 8;
    case 5: return 9;
    case 6: return 10;
    case 7: return 13;
    case 8: return 16;
    case 9: return 17;
    case 10: return 18;
    case 11: return 20;
    case 12: return 25;
    default: return 32;
  }
}

struct ImgState {
  int W, H, r;
  int pitch;               // words per image row (W rounded up to 4)
  int cx0, cx1, cy0, cy1;  // candidate-centre rectangle (inclusive)
  int t0x, t0y, t1x, t1y;  // level-0 / level-1 tile grid sizes
  int trace_cap;
  int srw;                 // engine search rows per warp (1 or 2)
  int n_partial;           // search CTAs writing partial[]
  int overlap;             // 1: partial-overlap search variant (Alg. 1, Sec. 5.4)
  uint32_t* img;
  uint8_t* omega;
  uint8_t* gray;
  double* conf;
  int32_t* count;          // unknown pixels of Psi_q per centre, row pitch `pitch`
  unsigned long long* prio;
  double* pconf;
  PrioBest* tiles0;
  PrioBest* tiles1;
  Ctrl* ctrl;
  inpaint_step_info* trace;
  unsigned long long* partial;  // per-CTA best search key of the iteration
  // tensor-core form in the persistent engine (null otherwise): five BF16
  // planes of the image, R' G' B' (byte - 128) and the square sum
  // sq = sum_c (byte_c - 128)^2 as 256 hi and lo (sq = 256 hi + lo), stored per tile column tx
  // of the search (columns [tc_xs0 + tx * tc_w, + tc_len)) as
  // [tx][row y < prows][plane][tc_len], zero outside W x H, so that two
  // source rows of a tile are one contiguous copy
  uint16_t* planes;
  int prows, tc_xs0, tc_w, tc_len, tc_ntx;
};

// BF16 bits of an integer with at most 8 significant bits (|v| <= 256, or
// 256 times such a value: exact, the low half of the float is zero).
__host__ __device__ inline uint32_t bf16_of_int(int v) {
  const float f = (float)v;
  uint32_t u;
  memcpy(&u, &f, 4);
  return u >> 16;
}

// The five plane values of pixel word w (R' G' B' hi lo) at offset o of
// tile column tx, row y.
__device__ inline void plane_store_at(const ImgState& s, int tx, int y, int o, uint32_t w) {
  const int d0 = (int)(w & 255u) - 128, d1 = (int)((w >> 8) & 255u) - 128, d2 = (int)((w >> 16) & 255u) - 128;
  const int sq = d0 * d0 + d1 * d1 + d2 * d2;
  uint16_t* row = s.planes + ((size_t)tx * s.prows + y) * 5 * s.tc_len + o;
  row[0] = (uint16_t)bf16_of_int(d0);
  row[s.tc_len] = (uint16_t)bf16_of_int(d1);
  row[2 * s.tc_len] = (uint16_t)bf16_of_int(d2);
  row[3 * s.tc_len] = (uint16_t)bf16_of_int(sq & ~255);  // 256 hi: hi < 256, exact in BF16
  row[4 * s.tc_len] = (uint16_t)bf16_of_int(sq & 255);
}

// Pixel (x, y) changed to w: its copies in the (at most two) tile columns
// whose segments hold column x.
__device__ inline void plane_store(const ImgState& s, int x, int y, uint32_t w) {
  const int xl = x - s.tc_xs0;
  if (xl < 0) return;  // left of every tile's source columns
  int tx = xl / s.tc_w;
  if (tx >= s.tc_ntx) tx = s.tc_ntx - 1;
  for (; tx >= 0 && xl - tx * s.tc_w < s.tc_len; --tx) plane_store_at(s, tx, y, xl - tx * s.tc_w, w);
}

__host__ __device__ inline uint32_t pack_rgb(uint32_t r, uint32_t g, uint32_t b) {
  return r | (g << 8) | (b << 16);
}

__host__ __device__ inline uint32_t luma_word(uint32_t w) {
  uint32_t r = w & 255u, g = (w >> 8) & 255u, b = (w >> 16) & 255u;
  return (299u * r + 587u * g + 114u * b + 500u) / 1000u;
}

// Loop is still running (uniform across a CTA: everyone reads the same word).
__device__ inline bool loop_active(const Ctrl* c) {
  return c->status == 0 && c->remaining > 0 && c->iter < c->iter_limit;
}

// Priority argmax order: larger key first, then lower index.
__device__ inline bool prio_better(unsigned long long ka, int ia, unsigned long long kb, int ib) {
  return ka > kb || (ka == kb && ia < ib);
}

// (k, i) = the better of (k, i) and (kk, ii), without a branch.
__device__ __forceinline__ void prio_take(unsigned long long& k, int& i, unsigned long long kk, int ii) {
  const bool b = prio_better(kk, ii, k, i);
  k = b ? kk : k;
  i = b ? ii : i;
}

__device__ inline unsigned long long warp_min_u64(unsigned long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    unsigned long long t = __shfl_xor_sync(0xffffffffu, v, o);
    v = t < v ? t : v;
  }
  return v;
}

__device__ inline void warp_best_prio(unsigned long long& k, int& i) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    unsigned long long tk = __shfl_xor_sync(0xffffffffu, k, o);
    int ti = __shfl_xor_sync(0xffffffffu, i, o);
    prio_take(k, i, tk, ti);
  }
}

// Block-wide best (key, idx); every thread gets the result.  scratch holds
// one entry per warp; blockDim.x must be a multiple of 32.
__device__ inline void block_best_prio(unsigned long long& k, int& i, PrioBest* scratch) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  warp_best_prio(k, i);
  __syncthreads();
  if (lane == 0) {
    scratch[wid].key = k;
    scratch[wid].idx = i;
  }
  __syncthreads();
  if (wid == 0) {
    unsigned long long kk = lane < nw ? scratch[lane].key : 0ull;
    int ii = lane < nw ? scratch[lane].idx : 0x7fffffff;
    warp_best_prio(kk, ii);
    if (lane == 0) {
      scratch[0].key = kk;
      scratch[0].idx = ii;
    }
  }
  __syncthreads();
  k = scratch[0].key;
  i = scratch[0].idx;
}

// Block reductions: one value per warp in scratch, then every warp reduces
// those itself (no lone warp between two barriers).  The leading barrier
// keeps the previous call's readers ahead of this call's writers.
__device__ inline unsigned long long block_min_u64(unsigned long long v, unsigned long long* scratch) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  v = warp_min_u64(v);
  __syncthreads();
  if (lane == 0) scratch[wid] = v;
  __syncthreads();
  return warp_min_u64(lane < nw ? scratch[lane] : ~0ull);
}

__device__ inline int block_sum_int(int v, int* scratch) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if (lane == 0) scratch[wid] = v;
  __syncthreads();
  int t = lane < nw ? scratch[lane] : 0;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  return t;
}

// ---- priority tiles: two-level argmax structure over the prio keys ----

// Rescans level-0 tile (tx, ty) from the pixel keys; one warp.  The eight
// loads of a lane are issued together (unrolled), then compared.
__device__ inline void warp_rescan_t0(const ImgState& s, int tx, int ty) {
  const int lane = threadIdx.x & 31;
  constexpr int N = kT0 * kT0 / 32;
  unsigned long long kk[N];
  int ii[N];
#pragma unroll
  for (int t = 0; t < N; ++t) {
    const int j = lane + 32 * t;
    const int x = tx * kT0 + (j & (kT0 - 1)), y = ty * kT0 + j / kT0;
    ii[t] = y * s.W + x;
    kk[t] = (x < s.W && y < s.H) ? __ldcg(&s.prio[ii[t]]) : 0ull;
  }
  unsigned long long k = 0ull;
  int idx = 0x7fffffff;
#pragma unroll
  for (int t = 0; t < N; ++t) prio_take(k, idx, kk[t], ii[t]);
  warp_best_prio(k, idx);
  if (lane == 0) {
    s.tiles0[ty * s.t0x + tx].key = k;
    s.tiles0[ty * s.t0x + tx].idx = idx;
  }
}

// Rescans level-1 tile (ux, uy) from the level-0 entries; one warp.
__device__ inline void warp_rescan_t1(const ImgState& s, int ux, int uy) {
  const int lane = threadIdx.x & 31;
  constexpr int N = kT1 * kT1 / 32;
  unsigned long long kk[N];
  int ii[N];
#pragma unroll
  for (int t = 0; t < N; ++t) {
    const int j = lane + 32 * t;
    const int tx = ux * kT1 + (j & (kT1 - 1)), ty = uy * kT1 + j / kT1;
    kk[t] = 0ull;
    ii[t] = 0x7fffffff;
    if (tx < s.t0x && ty < s.t0y) {
      kk[t] = __ldcg(&s.tiles0[ty * s.t0x + tx].key);
      ii[t] = __ldcg(&s.tiles0[ty * s.t0x + tx].idx);
    }
  }
  unsigned long long k = 0ull;
  int idx = 0x7fffffff;
#pragma unroll
  for (int t = 0; t < N; ++t) prio_take(k, idx, kk[t], ii[t]);
  warp_best_prio(k, idx);
  if (lane == 0) {
    s.tiles1[uy * s.t1x + ux].key = k;
    s.tiles1[uy * s.t1x + ux].idx = idx;
  }
}

// Best front pixel of the whole image from the level-1 entries; one warp,
// every lane gets the result.
__device__ inline void warp_global_best(const ImgState& s, unsigned long long& k, int& idx) {
  const int lane = threadIdx.x & 31;
  k = 0ull;
  idx = 0x7fffffff;
  const int n = s.t1x * s.t1y;
  for (int j = lane; j < n; j += 32) {
    const unsigned long long bk = __ldcg(&s.tiles1[j].key);
    const int bi = __ldcg(&s.tiles1[j].idx);
    prio_take(k, idx, bk, bi);
  }
  warp_best_prio(k, idx);
}

// After the prio keys of pixel rectangle [x0,x1] x [y0,y1] changed: refresh
// the tiles over it.  Whole block; ends with a __syncthreads.
__device__ inline void block_refresh_tiles(const ImgState& s, int x0, int x1, int y0, int y1) {
  const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int tx0 = x0 / kT0, tx1 = x1 / kT0, ty0 = y0 / kT0, ty1 = y1 / kT0;
  const int ntx = tx1 - tx0 + 1, nt = ntx * (ty1 - ty0 + 1);
  for (int t = w; t < nt; t += nw) warp_rescan_t0(s, tx0 + t % ntx, ty0 + t / ntx);
  __syncthreads();
  const int ux0 = tx0 / kT1, ux1 = tx1 / kT1, uy0 = ty0 / kT1, uy1 = ty1 / kT1;
  const int nux = ux1 - ux0 + 1, nu = nux * (uy1 - uy0 + 1);
  for (int t = w; t < nu; t += nw) warp_rescan_t1(s, ux0 + t % nux, uy0 + t / nux);
  __syncthreads();
}

// Selection of the next target p^ (highest priority, lowest index on ties)
// into the control block.  Called by warp 0 only.
__device__ inline void warp_select(const ImgState& s) {
  unsigned long long k;
  int idx;
  warp_global_best(s, k, idx);
  if ((threadIdx.x & 31) == 0) {
    Ctrl* c = s.ctrl;
    if (k == 0ull) {
      c->status = INPAINT_ERR_INTERNAL;  // Omega non-empty but no front
    } else {
      c->px = idx % s.W;
      c->py = idx / s.W;
      c->prio = __longlong_as_double((long long)(k - 1ull));
      c->conf = __ldcg(&s.pconf[idx]);
    }
  }
}

// ---- host-side launchers (defined in the .cu files) ----
void set_last_error(const char* msg);  // text returned by inpaint_last_error()
cudaError_t launch_init(const ImgState& s, const uint8_t* rgb, int rgb_stride, const uint8_t* mask,
                        int mask_stride, int32_t* sat, int* omega_count, cudaStream_t st);
cudaError_t launch_import(const ImgState& s, const uint8_t* rgb, const uint8_t* omega,
                          const double* conf, int32_t* sat, int* omega_count, cudaStream_t st);
int sat_chunks(int H);  // the integral image needs (W+1)(H+1) + sat_chunks(H)*W ints
cudaError_t prepare_search_plain(int r);
cudaError_t launch_prio_init_fast(const ImgState& s, cudaStream_t st);  // r <= 8
cudaError_t launch_search_plain(const ImgState& s, cudaStream_t st);
dim3 search_plain_grid(const ImgState& s);
// Tensor-core search (search_tc.cu), patch radius 1..8: a persistent grid over
// tiles of 8 candidate rows; one partial key per CTA (grid partials).
// Tensor-core search, one launch per iteration: one CTA per tile of the
// engine's tensor-core form (reads the image's BF16 planes).
struct TcPlan {
  int grid = 0, ntiles = 0, smem = 0, nb = 0, slot = 0;
};
// Geometry and launch shape (needs the search rectangle, not the buffers).
cudaError_t prepare_search_tc(const ImgState& s, TcPlan* plan);
cudaError_t launch_search_tc(const ImgState& s, const TcPlan& plan, cudaStream_t st);
cudaError_t launch_update(const ImgState& s, int do_fill, unsigned long long cond_handle,
                          int use_cond, cudaStream_t st);
cudaError_t launch_verify_count(const ImgState& s, cudaStream_t st);
cudaError_t launch_export(const ImgState& s, uint8_t* rgb_dense, cudaStream_t st);

}  // namespace inp
