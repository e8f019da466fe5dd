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

// ---------------------------------------------------------------- search unit

template <int R, int SR>
struct EngGeom {
  static constexpr int P = 2 * R + 1;
  static constexpr int BW = (128 + 2 * R + 3) & ~3;  // box width (words)
  static constexpr int BH = SR + 2 * R;              // box height (rows)
  static constexpr int BUF_WORDS = BW * BH;
  static constexpr int BUF_BYTES = ((BUF_WORDS * 4 + 127) / 128) * 128;
  static constexpr int NROW = (4 + P - 1 + 3) & ~3;  // strip words per lane
  static constexpr unsigned FULL = (1u << P) - 1u;
};

// SSD of 4 adjacent candidates x SR rows against the staged target, from
// one staged (SR+2R) x BW window.  Fully-known target rows take a branch-free
// path; partly-known rows test the row bit mask per column (warp-uniform).
template <int R, int SR>
__device__ inline void compute_unit(const uint32_t* __restrict__ buf, const uint32_t* __restrict__ tgt,
                                    const uint32_t* __restrict__ rowmask, uint32_t (&acc)[SR][4]) {
  using G = EngGeom<R, SR>;
  constexpr int P = G::P, BW = G::BW, NROW = G::NROW;
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 0; o < SR; ++o)
#pragma unroll
    for (int k = 0; k < 4; ++k) acc[o][k] = 0;
  for (int sr = 0; sr < SR + 2 * R; ++sr) {
    uint32_t row[NROW];
    const uint4* sp = reinterpret_cast<const uint4*>(buf + sr * BW + lane * 4);
#pragma unroll
    for (int i = 0; i < NROW / 4; ++i) {
      const uint4 v = sp[i];
      row[4 * i] = v.x;
      row[4 * i + 1] = v.y;
      row[4 * i + 2] = v.z;
      row[4 * i + 3] = v.w;
    }
#pragma unroll
    for (int o = 0; o < SR; ++o) {
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
  uint64_t bars[2 * kEngWarps];
  unsigned long long wkey[kEngWarps];
  unsigned long long red64[32];
  int flag;
  int stop;
};

template <int R, int SR>
__host__ __device__ constexpr size_t eng_search_bytes() {
  return (size_t)2 * kEngWarps * EngGeom<R, SR>::BUF_BYTES;
}

template <int R, int SR>
__host__ __device__ constexpr size_t eng_smem_bytes() {
  using G = EngGeom<R, SR>;
  const size_t srch = eng_search_bytes<R, SR>();
  const size_t upd = sizeof(UpdSmem<R>);
  const size_t big = srch > upd ? srch : upd;
  const size_t tgt = (size_t)(G::P * G::P + G::P + 4) * 4;
  return big + ((tgt + 127) / 128) * 128 + sizeof(EngSmemTail) + 128;
}

template <int R, int SR>
__global__ void __launch_bounds__(kEngThreads, 1) k_engine(EngineArgs ea) {
  using G = EngGeom<R, SR>;
  constexpr int P = G::P;
  extern __shared__ __align__(128) uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
  constexpr size_t srch = eng_search_bytes<R, SR>();
  constexpr size_t upd = sizeof(UpdSmem<R>);
  constexpr size_t big = srch > upd ? srch : upd;
  uint32_t* bufs = reinterpret_cast<uint32_t*>(smem);
  UpdSmem<R>& usm = *reinterpret_cast<UpdSmem<R>*>(smem);
  uint32_t* tgt = reinterpret_cast<uint32_t*>(smem + big);
  uint32_t* rowmask = tgt + P * P;
  EngSmemTail& tl =
      *reinterpret_cast<EngSmemTail*>(smem + big + (((size_t)(P * P + P + 4) * 4 + 127) / 128) * 128);

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int cta = blockIdx.x;
  const int team = ea.cta_team[cta];
  const int first = ea.team_first[team];
  const int rank = cta - first, tsize = ea.team_first[team + 1] - first;
  TeamCtl* tc = &ea.teams[team];
  unsigned long long* tpart = ea.partials + first;
  const unsigned long long limit = ea.wait_limit_ns;

  if (lane == 0) {
    mbar_init(&tl.bars[2 * warp], 1);
    mbar_init(&tl.bars[2 * warp + 1], 1);
  }
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  __syncthreads();
  uint32_t ph0 = 0, ph1 = 0;  // phase parity of this warp's two buffers
  uint32_t* mybuf0 = bufs + (size_t)(2 * warp) * (G::BUF_BYTES / 4);
  uint32_t* mybuf1 = bufs + (size_t)(2 * warp + 1) * (G::BUF_BYTES / 4);
  unsigned epoch = ld_acquire(&tc->epoch);
  unsigned long long t_prev = globaltimer();  // start of this CTA's first search round

  for (int li = ea.team_img_off[team]; li < ea.team_img_off[team + 1]; ++li) {
    const int j = ea.team_img[li];
    const ImgState s = ea.imgs[j];
    const CUtensorMap* map = &ea.tmaps[j];
    Ctrl* c = s.ctrl;
    // column grid aligned so that every TMA x coordinate is a multiple of 4
    const int xb = R + ((s.cx0 - R) & ~3);
    const int ncg = (s.cx1 - xb + 128) / 128;
    const int nrg = (s.cy1 - s.cy0 + SR) / SR;
    const int nunits = ncg * nrg;
    while (true) {
      if (tid == 0) {
        tl.stop = !(__ldcg(&c->status) == 0 && __ldcg(&c->remaining) > 0 &&
                    __ldcg(&c->iter) < __ldcg(&c->iter_limit)) ||
                  __ldcg(ea.err) != 0;
      }
      __syncthreads();
      if (tl.stop) break;
      const int px = __ldcg(&c->px), py = __ldcg(&c->py);

      // target patch: known in-image pixels and per-row bit masks
      if (tid < P) {
        const int ty = py + tid - R;
        uint32_t m = 0;
        for (int dx = 0; dx < P; ++dx) {
          const int tx = px + dx - R;
          uint32_t w = 0;
          if (tx >= 0 && tx < s.W && ty >= 0 && ty < s.H && __ldcg(&s.omega[(size_t)ty * s.W + tx]) == 0) {
            w = __ldcg(&s.img[(size_t)ty * s.pitch + tx]);
            m |= 1u << dx;
          }
          tgt[tid * P + dx] = w;
        }
        rowmask[tid] = m;
      }
      __syncthreads();

      // search: unit u -> (row group u / ncg, column group u % ncg); units
      // are dealt to CTAs first, then to warps, so small images spread out.
      unsigned long long best = ~0ull;
      int u = rank + tsize * warp;
      const int ustride = tsize * kEngWarps;
      bool ok = true;
      auto issue = [&](int uu, uint32_t* b, uint64_t* bar) {
        if (lane == 0) {
          const int gx = uu % ncg, gy = uu / ncg;
          asm volatile("fence.proxy.async;" ::: "memory");
          mbar_expect_tx(bar, (uint32_t)(G::BW * G::BH * 4));
          tma_load_2d(b, map, xb - R + 128 * gx, s.cy0 + SR * gy - R, bar);
        }
      };
      int cur = 0;
      if (u < nunits) issue(u, mybuf0, &tl.bars[2 * warp]);
      for (; u < nunits; u += ustride) {
        const int nx = u + ustride;
        uint32_t* b = cur ? mybuf1 : mybuf0;
        if (nx < nunits) issue(nx, cur ? mybuf0 : mybuf1, &tl.bars[2 * warp + (cur ^ 1)]);
        const bool got = mbar_wait(&tl.bars[2 * warp + cur], cur ? ph1 : ph0, limit);
        if (cur) ph1 ^= 1; else ph0 ^= 1;
        if (!got) {
          ok = false;
          if (nx < nunits) {  // drain the prefetch before leaving
            mbar_wait(&tl.bars[2 * warp + (cur ^ 1)], cur ? ph0 : ph1, limit);
            if (cur) ph0 ^= 1; else ph1 ^= 1;
          }
          break;
        }
        uint32_t acc[SR][4];
        compute_unit<R, SR>(b, tgt, rowmask, acc);
        const int gx = u % ncg, gy = u / ncg;
        const int qx0 = xb + 128 * gx + lane * 4, qy0 = s.cy0 + SR * gy;
#pragma unroll
        for (int o = 0; o < SR; ++o) {
          const int qy = qy0 + o;
          if (qy > s.cy1) continue;
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            const int qx = qx0 + k;
            if (qx < s.cx0 || qx > s.cx1) continue;
            const int idx = qy * s.W + qx;
            if (__ldcg(&s.count[idx]) != 0) continue;
            const unsigned long long key = ((unsigned long long)acc[o][k] << 32) | (unsigned)idx;
            best = key < best ? key : best;
          }
        }
        __syncwarp();
        cur ^= 1;
      }
      if (!ok && lane == 0) atomicExch(ea.err, INPAINT_ERR_TIMEOUT);
      best = block_min_u64(best, tl.red64);

      // arrive; the last member of the team applies the iteration
      if (tid == 0) {
        tpart[rank] = best;
        __threadfence();
        const unsigned old = atomicAdd(&tc->arrive, 1u);
        tl.flag = (old == (unsigned)(tsize - 1));
      }
      __syncthreads();
      if (tl.flag) {
        __threadfence();
        const unsigned long long t_a = globaltimer();
        update_phase<R>(s, tpart, tsize, usm);
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
        const unsigned long long t0 = globaltimer();
        while (ld_acquire(&tc->epoch) == epoch) {
          if (globaltimer() - t0 > limit) {
            atomicExch(ea.err, INPAINT_ERR_TIMEOUT);
            break;
          }
          __nanosleep(64);
        }
      }
      ++epoch;
      __syncthreads();
      if (lane == 0) asm volatile("fence.proxy.async.global;" ::: "memory");
      t_prev = __ldcg(&c->t_last);
    }
  }
}

// ---------------------------------------------------------------- host side

template <int R, int SR>
static cudaError_t launch_t(const EngineArgs& ea, int grid, cudaStream_t st) {
  const size_t smem = eng_smem_bytes<R, SR>();
  cudaError_t e = cudaFuncSetAttribute(k_engine<R, SR>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  void* args[] = {const_cast<EngineArgs*>(&ea)};
  return cudaLaunchCooperativeKernel((const void*)k_engine<R, SR>, dim3(grid), dim3(kEngThreads),
                                     args, smem, st);
}

template <int R, int SR>
static cudaError_t occupancy_t(int* blocks) {
  const size_t smem = eng_smem_bytes<R, SR>();
  cudaError_t e = cudaFuncSetAttribute(k_engine<R, SR>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, k_engine<R, SR>, kEngThreads, smem);
}

#define ENG_DISPATCH(FN, R, SR, ...)                                         \
  switch (R * 10 + SR) {                                                     \
    case 11: return FN<1, 1>(__VA_ARGS__);                                   \
    case 12: return FN<1, 2>(__VA_ARGS__);                                   \
    case 14: return FN<1, 4>(__VA_ARGS__);                                   \
    case 21: return FN<2, 1>(__VA_ARGS__);                                   \
    case 22: return FN<2, 2>(__VA_ARGS__);                                   \
    case 24: return FN<2, 4>(__VA_ARGS__);                                   \
    case 31: return FN<3, 1>(__VA_ARGS__);                                   \
    case 32: return FN<3, 2>(__VA_ARGS__);                                   \
    case 34: return FN<3, 4>(__VA_ARGS__);                                   \
    case 41: return FN<4, 1>(__VA_ARGS__);                                   \
    case 42: return FN<4, 2>(__VA_ARGS__);                                   \
    case 44: return FN<4, 4>(__VA_ARGS__);                                   \
    case 51: return FN<5, 1>(__VA_ARGS__);                                   \
    case 52: return FN<5, 2>(__VA_ARGS__);                                   \
    case 54: return FN<5, 4>(__VA_ARGS__);                                   \
    case 61: return FN<6, 1>(__VA_ARGS__);                                   \
    case 62: return FN<6, 2>(__VA_ARGS__);                                   \
    case 64: return FN<6, 4>(__VA_ARGS__);                                   \
    case 71: return FN<7, 1>(__VA_ARGS__);                                   \
    case 72: return FN<7, 2>(__VA_ARGS__);                                   \
    case 74: return FN<7, 4>(__VA_ARGS__);                                   \
    case 81: return FN<8, 1>(__VA_ARGS__);                                   \
    case 82: return FN<8, 2>(__VA_ARGS__);                                   \
    case 84: return FN<8, 4>(__VA_ARGS__);                                   \
    default: return cudaErrorInvalidValue;                                   \
  }

cudaError_t engine_occupancy(int r, int sr, int* blocks_per_sm) {
  ENG_DISPATCH(occupancy_t, r, sr, blocks_per_sm)
}

cudaError_t engine_launch(int r, int sr, const EngineArgs& ea, int grid, cudaStream_t st) {
  ENG_DISPATCH(launch_t, r, sr, ea, grid, st)
}

size_t engine_smem_bytes(int r, int sr) {
  switch (r * 10 + sr) {
#define ENG_SM(R, SR) \
  case R * 10 + SR: return eng_smem_bytes<R, SR>();
    ENG_SM(1, 1) ENG_SM(1, 2) ENG_SM(1, 4) ENG_SM(2, 1) ENG_SM(2, 2) ENG_SM(2, 4)
    ENG_SM(3, 1) ENG_SM(3, 2) ENG_SM(3, 4) ENG_SM(4, 1) ENG_SM(4, 2) ENG_SM(4, 4)
    ENG_SM(5, 1) ENG_SM(5, 2) ENG_SM(5, 4) ENG_SM(6, 1) ENG_SM(6, 2) ENG_SM(6, 4)
    ENG_SM(7, 1) ENG_SM(7, 2) ENG_SM(7, 4) ENG_SM(8, 1) ENG_SM(8, 2) ENG_SM(8, 4)
#undef ENG_SM
    default: return 0;
  }
}

// TMA descriptor of an image's RGBA words: 2-D (W, H), row pitch in bytes,
// box (128 + 2r rounded up to 4) x (SR + 2r); out-of-image reads give 0.
int make_image_tmap(const ImgState& s, int sr, CUtensorMap* out) {
  static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  if (!encode) {
    cudaDriverEntryPointQueryResult q;
    void* fn = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault,
                                         &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn)
      return -1;
    encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }
  const cuuint64_t dims[2] = {(cuuint64_t)s.W, (cuuint64_t)s.H};
  const cuuint64_t strides[1] = {(cuuint64_t)s.pitch * 4};
  const cuuint32_t box[2] = {(cuuint32_t)((128 + 2 * s.r + 3) & ~3), (cuuint32_t)(sr + 2 * s.r)};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult r = encode(out, CU_TENSOR_MAP_DATA_TYPE_UINT32, 2, s.img, dims, strides, box, estr,
                            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? 0 : -1;
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

cudaError_t launch_update_fast(const ImgState& s, unsigned long long cond, int use_cond,
                               cudaStream_t st) {
  switch (s.r) {
    case 1: return upd_fast_t<1>(s, cond, use_cond, st);
    case 2: return upd_fast_t<2>(s, cond, use_cond, st);
    case 3: return upd_fast_t<3>(s, cond, use_cond, st);
    case 4: return upd_fast_t<4>(s, cond, use_cond, st);
    case 5: return upd_fast_t<5>(s, cond, use_cond, st);
    case 6: return upd_fast_t<6>(s, cond, use_cond, st);
    case 7: return upd_fast_t<7>(s, cond, use_cond, st);
    case 8: return upd_fast_t<8>(s, cond, use_cond, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace inp

namespace inp {

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

cudaError_t launch_prio_init_fast(const ImgState& s, cudaStream_t st) {
  switch (s.r) {
    case 1: return prio_init_t<1>(s, st);
    case 2: return prio_init_t<2>(s, st);
    case 3: return prio_init_t<3>(s, st);
    case 4: return prio_init_t<4>(s, st);
    case 5: return prio_init_t<5>(s, st);
    case 6: return prio_init_t<6>(s, st);
    case 7: return prio_init_t<7>(s, st);
    case 8: return prio_init_t<8>(s, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace inp
