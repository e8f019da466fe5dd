// findBestPatch, exact tensor-core form, one launch per iteration (the graph
// loop and the isolated search timing; Sec. 3, Eq. 3-4 written as
// correlations, the paper's own kernel being the CUDA-core Algorithm 1).
//
// The tile form of the persistent engine (search_tc_engine.cuh: the target
// as a Toeplitz A operand of 16 candidate rows x 8 column shifts, each
// source row as the B operand of N blocks of 8 candidate columns, BF16
// operands holding small integers, FP32 accumulators in tensor memory, the
// SSD exact), one CTA per tile: it stages the target and the validity bits
// of its tile, builds the A strips, streams the tile's source rows from the
// image's BF16 planes through a ring of shared-memory slots (one producer
// thread, two issuing warps) and reads the accumulators back into the best
// (SSD << 32 | idx) key of the tile, written to partial[tile].
#include "inpaint_engine.h"
#include "ptx.cuh"
#include "search_tc_engine.cuh"

namespace inp {
namespace {

constexpr unsigned long long kTcWaitNs = 2000000000ull;

// Head of the kernel's shared memory (the tile's state follows it).
struct TcHead {
  EngBars bars;
  int a2row[17];
  unsigned long long red64[32];
};
constexpr int kTcHeadBytes = (int)((sizeof(TcHead) + 127) / 128 * 128);

template <int R>
__host__ __device__ inline int tc_fixed_bytes(int N) {
  return kTcHeadBytes + TcEngGeom<R>::A_BYTES + TcEngGeom<R>::TPAD_BYTES + tc_bit_words(N) * 4;
}

template <int R>
__global__ void __launch_bounds__(kEngThreads, 1) k_search_tc(ImgState s, int nb, int slot) {
  using GT = TcEngGeom<R>;
  constexpr int P = GT::P, NSL = GT::NSL;
  extern __shared__ __align__(128) uint8_t tc_dyn[];
  uint8_t* sm = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(tc_dyn) + 127) & ~uintptr_t(127));
  TcHead& h = *reinterpret_cast<TcHead*>(sm);
  const Ctrl* c = s.ctrl;
  if (!loop_active(c)) return;
  const TcTiles tt = tc_tiles(s);
  const int t = blockIdx.x, ntiles = tt.ntx * tt.nty;
  const int tx = t % tt.ntx, y0 = s.cy0 + kTcRows * (t / tt.ntx), xs = tt.xs0 + 8 * tt.N * tx;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  TcArea ta;
  ta.a = sm + kTcHeadBytes;
  ta.tpad = reinterpret_cast<uint16_t*>(ta.a + GT::A_BYTES);
  ta.ring = ta.a + GT::A_BYTES + GT::TPAD_BYTES;
  ta.bits = reinterpret_cast<uint32_t*>(ta.ring + (size_t)nb * slot);
  ta.nb = nb;
  ta.ntl = 1;
  ta.slot = slot;
  if (tid == 0) {
    for (int i = 0; i < nb; ++i) {
      mbar_init(&h.bars.tc_full[i], 1);
      mbar_init(&h.bars.tc_empty[i], 2);  // one commit from each issuer
    }
    mbar_init(&h.bars.tc_done, 2);
  }
  fence_mbar_init();
  if (warp == 0) tc_alloc(&h.bars.tmem, 256);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = h.bars.tmem;
  const int px = __ldcg(&c->px), py = __ldcg(&c->py);
  const int npre = min(nb, NSL);
  int bad = 0;
  // the producer starts the tile's first rows at once
  if (warp == kEngWarps - 1 && lane == 0 && !tc_produce<R>(s, ta, h.bars, tx, y0, 0u, 0, npre, kTcWaitNs)) bad = 1;
  tc_bits_init<R>(s, tt, ta.bits, 1, t, ntiles);
  for (int e = tid; e < 4 * P * GT::TW; e += kEngThreads) ta.tpad[e] = 0;
  __syncthreads();
  // target patch: warp dy reads row dy (lane = dx) into the padded table
  for (int dy = warp; dy < P; dy += kEngWarps) {
    const int qx = px + lane - R, qy = py + dy - R;
    uint32_t w = 0;
    bool known = false;
    if (lane < P && qx >= 0 && qx < s.W && qy >= 0 && qy < s.H) {
      const uint8_t o = __ldcg(&s.omega[(size_t)qy * s.W + qx]);
      const uint32_t v = __ldcg(&s.img[(size_t)qy * s.pitch + qx]);
      known = o == 0;
      w = known ? v : 0u;
    }
    int sq = 0;
    if (lane < P) {
      const int d0 = known ? (int)(w & 255u) - 128 : 0, d1 = known ? (int)((w >> 8) & 255u) - 128 : 0,
                d2 = known ? (int)((w >> 16) & 255u) - 128 : 0;
      sq = d0 * d0 + d1 * d1 + d2 * d2;
      uint16_t* tp = ta.tpad + dy * GT::TW + 8 + lane;
      tp[0] = (uint16_t)bf16_of_int(d0);
      tp[P * GT::TW] = (uint16_t)bf16_of_int(d1);
      tp[2 * P * GT::TW] = (uint16_t)bf16_of_int(d2);
      tp[3 * P * GT::TW] = (uint16_t)bf16_of_int(known ? 1 : 0);
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, o);
    if (lane == 0) h.a2row[dy] = sq;
  }
  __syncthreads();
  // every warp but the producer's (its copies are in flight) writes A
  tc_build_a<R>(ta.a, ta.tpad, true, 32 * (kEngWarps - 1));
  __syncthreads();
  int a2 = 0;
#pragma unroll
  for (int dy = 0; dy < P; ++dy) a2 += h.a2row[dy];
  if (warp == kEngWarps - 1) {
    if (lane == 0 && !tc_produce<R>(s, ta, h.bars, tx, y0, 0u, npre, NSL, kTcWaitNs)) bad = 1;
    __syncwarp();
  } else if (warp == kEngWarps - 2) {
    if (!(tt.N == 128 ? tc_issue<R, 0, 128>(ta, h.bars, tmem, 0u, kTcWaitNs)
                      : tc_issue<R, 0, 64>(ta, h.bars, tmem, 0u, kTcWaitNs)))
      bad = 1;
    if (!mbar_wait(&h.bars.tc_done, 0u, kTcWaitNs)) bad = 1;  // the tile's MMAs
  } else if (warp == kEngWarps - 3) {
    if (!(tt.N == 128 ? tc_issue<R, 1, 128>(ta, h.bars, tmem, 0u, kTcWaitNs)
                      : tc_issue<R, 1, 64>(ta, h.bars, tmem, 0u, kTcWaitNs)))
      bad = 1;
  }
  tc_fence_before();
  const bool failed = __syncthreads_or(bad) != 0;
  tc_fence_after();
  unsigned long long best = ~0ull;
  if (!failed) best = tc_epilogue<R>(s, tmem, tt.N, a2, ta.bits, y0, xs, best);
  best = block_min_u64(best, h.red64);
  if (tid == 0) {
    s.partial[t] = best;
    if (failed) atomicCAS(const_cast<int*>(&c->status), 0, INPAINT_ERR_TIMEOUT);
  }
  if (failed && warp == kEngWarps - 1 && lane == 0) {
    // let the copies in flight land before the CTA exits (bounded)
    for (int g = 0; g < NSL && g < nb; ++g) mbar_wait(&h.bars.tc_full[g], 0u, kTcWaitNs);
  }
  // every tensor-memory read is complete before the columns are freed
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tc_dealloc(tmem, 256);
  }
}

template <int R>
cudaError_t prepare_r(const ImgState& s, TcPlan* plan) {
  const TcTiles tt = tc_tiles(s);
  plan->ntiles = tt.ntx * tt.nty;
  plan->grid = plan->ntiles;
  if (plan->ntiles == 0) return cudaSuccess;
  int dev = 0, optin = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e != cudaSuccess) return e;
  const int slot = tc_slot(tt.N, R), fixed = tc_fixed_bytes<R>(tt.N) + 128;  // + base alignment
  const int nb = (optin - fixed) / slot < kTcRing ? (optin - fixed) / slot : kTcRing;
  if (nb < 4) return cudaErrorInvalidConfiguration;
  plan->nb = nb;
  plan->slot = slot;
  plan->smem = fixed + nb * slot;
  return cudaFuncSetAttribute(k_search_tc<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, plan->smem);
}

template <int R>
cudaError_t launch_r(const ImgState& s, const TcPlan& p, cudaStream_t st) {
  k_search_tc<R><<<p.grid, kEngThreads, p.smem, st>>>(s, p.nb, p.slot);
  return cudaGetLastError();
}

}  // namespace

cudaError_t prepare_search_tc(const ImgState& s, TcPlan* plan) {
  switch (s.r) {
    case 1: return prepare_r<1>(s, plan);
    case 2: return prepare_r<2>(s, plan);
    case 3: return prepare_r<3>(s, plan);
    case 4: return prepare_r<4>(s, plan);
    case 5: return prepare_r<5>(s, plan);
    case 6: return prepare_r<6>(s, plan);
    case 7: return prepare_r<7>(s, plan);
    case 8: return prepare_r<8>(s, plan);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_search_tc(const ImgState& s, const TcPlan& p, cudaStream_t st) {
  if (p.grid <= 0) return cudaSuccess;
  if (!s.planes || p.nb < 4) return cudaErrorInvalidValue;
  switch (s.r) {
    case 1: return launch_r<1>(s, p, st);
    case 2: return launch_r<2>(s, p, st);
    case 3: return launch_r<3>(s, p, st);
    case 4: return launch_r<4>(s, p, st);
    case 5: return launch_r<5>(s, p, st);
    case 6: return launch_r<6>(s, p, st);
    case 7: return launch_r<7>(s, p, st);
    case 8: return launch_r<8>(s, p, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace inp
