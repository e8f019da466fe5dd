// Persistent fill-loop engine: the whole iterative stage of Sec. 4.2 in one
// cooperative kernel launch.
//
// CTAs form teams; a team runs the fill loop of one image at a time (a list
// of images per team gives the batched form).  One iteration of a team:
//   1. every member CTA searches its share of the candidate centres
//      (findBestPatch, Eq. 3-4): per warp, a unit of SR candidate rows x 128
//      candidate columns whose (SR+2R) x (128+2R) source window is brought
//      into shared memory by a TMA tile load, double-buffered, and reduced
//      to one (SSD << 32 | idx) key;
//   2. each member writes its key and arrives on the team counter; the last
//      to arrive runs the copy/update phase and the selection of the next
//      target (update_fast.cuh) and publishes the next epoch;
//   3. the others wait for that epoch (bounded wait, no trap) and go on.
// No host round trip and no kernel boundary per iteration.
#pragma once
#include <cuda.h>

#include "inpaint_engine.h"
#include "update_fast.cuh"

namespace inp {

// ---------------------------------------------------------------- PTX helpers

__device__ inline uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ inline unsigned long long globaltimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ inline void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
               : "memory");
}

__device__ inline void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}

__device__ inline bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait for a phase of an mbarrier; false after limit_ns.
__device__ inline bool mbar_wait(uint64_t* bar, uint32_t parity, unsigned long long limit_ns) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = globaltimer();
  while (!mbar_try_wait(bar, parity))
    if (globaltimer() - t0 > limit_ns) return false;
  return true;
}

__device__ inline void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_addr(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_addr(bar))
      : "memory");
}

__device__ inline unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ inline void st_release(unsigned* p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// ---------------------------------------------------------------- search batch

template <int R, int SRW>
struct EngGeom {
  static constexpr int P = 2 * R + 1;
  static constexpr int BW = (128 + 2 * R + 3) & ~3;  // staged width (words)
  static constexpr int B = kEngWarps * SRW;          // candidate rows per batch
  static constexpr int BH = B + 2 * R;               // staged rows
  static constexpr int STAGE_BYTES = ((BW * BH * 4 + 127) / 128) * 128;
  static constexpr int NROW = (4 + P - 1 + 3) & ~3;  // strip words per lane
  static constexpr unsigned FULL = (1u << P) - 1u;
};

// SSD of the SRW x 4 candidates of this lane (rows row0.. of the batch,
// columns lane*4..lane*4+3) against the staged target.  Fully-known target
// rows take a branch-free path; partly-known rows test a bit mask per column
// (warp-uniform).
template <int R, int SRW>
__device__ inline void compute_rows(const uint32_t* __restrict__ stage, int row0,
                                    const uint32_t* __restrict__ tgt,
                                    const uint32_t* __restrict__ rowmask, uint32_t (&acc)[SRW][4]) {
  using G = EngGeom<R, SRW>;
  constexpr int P = G::P, BW = G::BW, NROW = G::NROW;
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 0; o < SRW; ++o)
#pragma unroll
    for (int k = 0; k < 4; ++k) acc[o][k] = 0;
#pragma unroll 1
  for (int sr = 0; sr < SRW + 2 * R; ++sr) {
    uint32_t row[NROW];
    const uint4* sp = reinterpret_cast<const uint4*>(stage + (row0 + sr) * BW + lane * 4);
#pragma unroll
    for (int i = 0; i < NROW / 4; ++i) {
      const uint4 v = sp[i];
      row[4 * i] = v.x;
      row[4 * i + 1] = v.y;
      row[4 * i + 2] = v.z;
      row[4 * i + 3] = v.w;
    }
#pragma unroll
    for (int o = 0; o < SRW; ++o) {
      const int dy = sr - o;
      if (dy < 0 || dy >= P) continue;
      const uint32_t m = rowmask[dy];
      if (m == 0) continue;
      const uint32_t* trow = tgt + dy * P;
      if (m == G::FULL) {
#pragma unroll
        for (int dx = 0; dx < P; ++dx) {
          const uint32_t a = trow[dx];
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            const uint32_t d = __vabsdiffu4(a, row[k + dx]);
            acc[o][k] = __dp4a(d, d, acc[o][k]);
          }
        }
      } else {
#pragma unroll
        for (int dx = 0; dx < P; ++dx) {
          if (m & (1u << dx)) {
            const uint32_t a = trow[dx];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
              const uint32_t d = __vabsdiffu4(a, row[k + dx]);
              acc[o][k] = __dp4a(d, d, acc[o][k]);
            }
          }
        }
      }
    }
  }
}

// ---------------------------------------------------------------- kernel

struct EngSmemTail {
  uint64_t full[2];  // TMA completion barriers of the two stages
  unsigned long long red64[32];
  int red32[32];
  int flag;
  int stop;
};

constexpr int kTgtWords = 17 * 17 + 17 + 3;  // target words + row masks (R <= 8)
constexpr size_t kHeadBytes = ((sizeof(EngSmemTail) + kTgtWords * 4 + 127) / 128) * 128;

template <int R, int SRW>
__host__ __device__ constexpr size_t eng_smem_bytes() {
  using G = EngGeom<R, SRW>;
  const size_t srch = (size_t)2 * G::STAGE_BYTES;
  const size_t upd = sizeof(UpdSmem<R>);
  return kHeadBytes + (srch > upd ? srch : upd) + 128;
}

// Bounded wait until the team epoch moves past `epoch` (thread 0 only).
__device__ inline void wait_epoch(TeamCtl* tc, unsigned epoch, int* err, unsigned long long limit) {
  const unsigned long long t0 = globaltimer();
  while (ld_acquire(&tc->epoch) == epoch) {
    if (globaltimer() - t0 > limit) {
      atomicExch(err, INPAINT_ERR_TIMEOUT);
      return;
    }
    __nanosleep(64);
  }
}

template <int R, int SRW>
__global__ void __launch_bounds__(kEngThreads, 1) k_engine(EngineArgs ea) {
  using G = EngGeom<R, SRW>;
  constexpr int P = G::P, B = G::B;
  extern __shared__ __align__(128) uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
  EngSmemTail& tl = *reinterpret_cast<EngSmemTail*>(smem);
  uint32_t* tgt = reinterpret_cast<uint32_t*>(smem + sizeof(EngSmemTail));
  uint32_t* rowmask = tgt + P * P;
  uint8_t* big = smem + kHeadBytes;
  uint32_t* stage0 = reinterpret_cast<uint32_t*>(big);
  uint32_t* stage1 = reinterpret_cast<uint32_t*>(big + G::STAGE_BYTES);
  UpdSmem<R>& usm = *reinterpret_cast<UpdSmem<R>*>(big);

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int cta = blockIdx.x;
  const int team = ea.cta_team[cta];
  const int first = ea.team_first[team];
  const int rank = cta - first, tsize = ea.team_first[team + 1] - first;
  TeamCtl* tc = &ea.teams[team];
  unsigned long long* tpart = ea.partials + first;
  const unsigned long long limit = ea.wait_limit_ns;

  if (tid == 0) {
    mbar_init(&tl.full[0], 1);
    mbar_init(&tl.full[1], 1);
  }
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  __syncthreads();
  uint32_t ph0 = 0, ph1 = 0;
  unsigned epoch = ld_acquire(&tc->epoch);
  unsigned long long t_prev = globaltimer();

  for (int li = ea.team_img_off[team]; li < ea.team_img_off[team + 1]; ++li) {
    const int j = ea.team_img[li];
    const ImgState s = ea.imgs[j];
    const CUtensorMap* map = &ea.tmaps[j];
    Ctrl* c = s.ctrl;
    // candidate batches: B rows x 128 columns; the column grid is aligned so
    // that every TMA x coordinate is a multiple of 4 words
    const int xb = R + ((s.cx0 - R) & ~3);
    const int ncg = (s.cx1 - xb + 128) / 128;
    const int nrb = (s.cy1 - s.cy0 + B) / B;
    const int nbatch = ncg * nrb;
    // roles: searchers [0, ns), one speculative-phase CTA (the last rank),
    // the rest idle for this image; a team of one does everything itself
    const int ns = tsize >= 2 ? min(tsize - 1, nbatch) : 1;
    const bool spec_cta = tsize >= 2 ? rank == tsize - 1 : true;
    const bool searcher = rank < ns;
    const unsigned n_arrive = tsize >= 2 ? (unsigned)ns + 1u : 1u;
    const bool idle = !searcher && !spec_cta;
    while (true) {
      if (tid == 0) {
        tl.stop = !(__ldcg(&c->status) == 0 && __ldcg(&c->remaining) > 0 &&
                    __ldcg(&c->iter) < __ldcg(&c->iter_limit)) ||
                  __ldcg(ea.err) != 0;
      }
      __syncthreads();
      if (tl.stop) break;
      if (idle) {
        if (tid == 0) wait_epoch(tc, epoch, ea.err, limit);
        ++epoch;
        __syncthreads();
        continue;
      }
      unsigned long long best = ~0ull;
      if (spec_cta) {
        spec_phase<R>(s, usm);
        __threadfence();
        __syncthreads();
      }
      if (searcher) {
        const int px = __ldcg(&c->px), py = __ldcg(&c->py);
        if (tid < P) {  // target patch: known in-image pixels and per-row bit masks
          const int ty = py + tid - R;
          uint32_t m = 0;
          for (int dx = 0; dx < P; ++dx) {
            const int tx = px + dx - R;
            uint32_t w = 0;
            if (tx >= 0 && tx < s.W && ty >= 0 && ty < s.H &&
                __ldcg(&s.omega[(size_t)ty * s.W + tx]) == 0) {
              w = __ldcg(&s.img[(size_t)ty * s.pitch + tx]);
              m |= 1u << dx;
            }
            tgt[tid * P + dx] = w;
          }
          rowmask[tid] = m;
        }
        auto issue = [&](int b, uint32_t* st, uint64_t* bar) {
          const int gx = b % ncg, gy = b / ncg;
          asm volatile("fence.proxy.async;" ::: "memory");
          mbar_expect_tx(bar, (uint32_t)(G::BW * G::BH * 4));
          tma_load_2d(st, map, xb - R + 128 * gx, s.cy0 + B * gy - R, bar);
        };
        if (tid == 0 && rank < nbatch) issue(rank, stage0, &tl.full[0]);
        __syncthreads();  // target ready
        int cur = 0;
        bool ok = true;
        for (int b = rank; b < nbatch; b += ns) {
          const int nb = b + ns;
          if (tid == 0 && nb < nbatch) issue(nb, cur ? stage0 : stage1, &tl.full[cur ^ 1]);
          // validity of this lane's candidates, loaded while the tile arrives
          const int gx = b % ncg, gy = b / ncg;
          const int qx0 = xb + 128 * gx + lane * 4, qy0 = s.cy0 + B * gy + warp * SRW;
          int cnt[SRW][4];
#pragma unroll
          for (int o = 0; o < SRW; ++o)
#pragma unroll
            for (int k = 0; k < 4; ++k) {
              const int qx = qx0 + k, qy = qy0 + o;
              cnt[o][k] = (qx >= s.cx0 && qx <= s.cx1 && qy <= s.cy1)
                              ? __ldcg(&s.count[(size_t)qy * s.W + qx])
                              : 1;
            }
          const bool got = mbar_wait(&tl.full[cur], cur ? ph1 : ph0, limit);
          if (cur) ph1 ^= 1; else ph0 ^= 1;
          uint32_t acc[SRW][4];
          compute_rows<R, SRW>(cur ? stage1 : stage0, warp * SRW, tgt, rowmask, acc);
#pragma unroll
          for (int o = 0; o < SRW; ++o)
#pragma unroll
            for (int k = 0; k < 4; ++k)
              if (cnt[o][k] == 0) {
                const unsigned idx = (unsigned)((qy0 + o) * s.W + qx0 + k);
                const unsigned long long key = ((unsigned long long)acc[o][k] << 32) | idx;
                best = key < best ? key : best;
              }
          // every warp is done with this stage; a bounded wait that gave up
          // anywhere ends the search uniformly (after the prefetch landed)
          if (__syncthreads_or(!got)) {
            ok = false;
            if (nb < nbatch) {
              mbar_wait(&tl.full[cur ^ 1], cur ? ph0 : ph1, limit);
              if (cur) ph0 ^= 1; else ph1 ^= 1;
            }
            break;
          }
          cur ^= 1;
        }
        if (!ok && tid == 0) atomicExch(ea.err, INPAINT_ERR_TIMEOUT);
        best = block_min_u64(best, tl.red64);
      }

      // arrive; the last arrival applies the iteration
      if (tid == 0) {
        if (searcher) tpart[rank] = best;
        __threadfence();
        const unsigned old = atomicAdd(&tc->arrive, 1u);
        tl.flag = (old == n_arrive - 1u);
      }
      __syncthreads();
      if (tl.flag) {
        __threadfence();
        const unsigned long long t_a = globaltimer();
        update_phase<R>(s, tpart, ns, usm);
        __threadfence();
        __syncthreads();
        if (tid == 0) {
          const unsigned long long t_b = globaltimer();
          c->t_search += t_a - t_prev;
          c->t_update += t_b - t_a;
          c->t_last = t_b;
          c->timed_iters += 1;
          tc->arrive = 0u;
          __threadfence();
          st_release(&tc->epoch, epoch + 1u);
        }
      } else if (tid == 0) {
        wait_epoch(tc, epoch, ea.err, limit);
      }
      ++epoch;
      __syncthreads();
      t_prev = __ldcg(&c->t_last);
    }
  }
}

// ---------------------------------------------------------------- host side

template <int R, int SRW>
static cudaError_t launch_t(const EngineArgs& ea, int grid, cudaStream_t st) {
  const size_t smem = eng_smem_bytes<R, SRW>();
  cudaError_t e = cudaFuncSetAttribute(k_engine<R, SRW>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  void* args[] = {const_cast<EngineArgs*>(&ea)};
  return cudaLaunchCooperativeKernel((const void*)k_engine<R, SRW>, dim3(grid), dim3(kEngThreads),
                                     args, smem, st);
}

template <int R, int SRW>
static cudaError_t occupancy_t(int* blocks) {
  const size_t smem = eng_smem_bytes<R, SRW>();
  cudaError_t e = cudaFuncSetAttribute(k_engine<R, SRW>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, k_engine<R, SRW>, kEngThreads, smem);
}


}  // namespace inp


namespace inp {

// Single-CTA copy/update kernel of the graph-driven loop for R <= 8 (the same
// update phase the engine runs in its last-arriving CTA).
template <int R>
__global__ void __launch_bounds__(kEngThreads) k_update_fast(ImgState s, cudaGraphConditionalHandle cond,
                                                            int use_cond) {
  extern __shared__ __align__(16) uint8_t sm_raw[];
  UpdSmem<R>& usm = *reinterpret_cast<UpdSmem<R>*>(sm_raw);
  if (!loop_active(s.ctrl)) {
    if (use_cond && threadIdx.x == 0) cudaGraphSetConditional(cond, 0);
    return;
  }
  spec_phase<R>(s, usm);
  __syncthreads();
  const bool ok = update_phase<R>(s, s.partial, s.n_partial, usm);
  if (use_cond && threadIdx.x == 0) cudaGraphSetConditional(cond, ok && loop_active(s.ctrl) ? 1u : 0u);
}

template <int R>
static cudaError_t upd_fast_t(const ImgState& s, unsigned long long cond, int use_cond, cudaStream_t st) {
  const size_t smem = sizeof(UpdSmem<R>);
  cudaError_t e = cudaFuncSetAttribute(k_update_fast<R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  k_update_fast<R><<<1, kEngThreads, smem, st>>>(s, (cudaGraphConditionalHandle)cond, use_cond);
  return cudaGetLastError();
}





template <int R>
static cudaError_t prio_init_t(const ImgState& s, cudaStream_t st) {
  using G = UpdGeom<R>;
  const size_t smem = sizeof(UpdSmem<R>);
  cudaError_t e = cudaFuncSetAttribute(k_prio_init_fast<R>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const dim3 grid((s.W + G::NW - 1) / G::NW, (s.H + G::NW - 1) / G::NW);
  k_prio_init_fast<R><<<grid, 256, smem, st>>>(s);
  return cudaGetLastError();
}



}  // namespace inp

namespace inp {

// Entry points of one radius R, exported through EngineFns.
template <int R>
static cudaError_t eng_launch_r(int srw, const EngineArgs& ea, int grid, cudaStream_t st) {
  return srw == 2 ? launch_t<R, 2>(ea, grid, st) : launch_t<R, 1>(ea, grid, st);
}
template <int R>
static cudaError_t eng_occ_r(int srw, int* blocks) {
  return srw == 2 ? occupancy_t<R, 2>(blocks) : occupancy_t<R, 1>(blocks);
}
template <int R>
const EngineFns* engine_fns_for() {
  static const EngineFns f = {eng_launch_r<R>, eng_occ_r<R>, upd_fast_t<R>, prio_init_t<R>};
  return &f;
}

}  // namespace inp
