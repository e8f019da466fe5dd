// findBestPatch, exact tensor-core form (Sec. 3, Eq. 3-4 written as
// correlations; the paper's own kernel is the CUDA-core Algorithm 1).
//
// With every byte shifted by 128 (b' = b - 128, |b'| <= 128, exact in BF16)
// and m the known-pixel indicator of the target patch Psi_p^:
//   SSD(q) = sum_d m(d) sum_c (t'_c(d) - s'_c(q+d))^2 = A2 - 2 X(q) + S(q)
//   A2   = sum_d m(d) sum_c t'_c(d)^2                       (one integer)
//   X(q) = sum_c sum_d [m(d) t'_c(d)] s'_c(q+d)             (3 correlations)
//   S(q) = sum_d m(d) sq(q+d),  sq = sum_c s'_c^2 <= 49152   (split as
//          sq = 256 hi + lo with hi, lo < 256, weights 256 m and m)
// Every product of two BF16 integers is exact and every partial sum is an
// integer of magnitude below 2^24 (|X| <= 17^2 * 3 * 128^2, S <= 17^2 * 49152),
// so the FP32 accumulators hold exact integers and the SSD equals the
// CUDA-core form's bit for bit.
//
// The correlations run as tcgen05 MMAs (kind::f16, BF16 operands in shared
// memory, FP32 accumulators in tensor memory) with no im2col copy:
//  * A (M = 128): row a is a block of 8 consecutive candidates (64 blocks of
//    one candidate row, then 64 of the next); it reads a plane row directly,
//    row a starting 16 bytes after row a - 1 (the canonical no-swizzle
//    K-major layout; consecutive rows overlap in memory).  The two 8-element
//    K halves of an MMA are two "items" (plane, 8-tap chunk): the leading
//    byte offset between the K core matrices is simply the distance between
//    the two items, so an MMA can pair chunks of different planes and only
//    ceil((P + 7) / 8) chunks per plane are needed.
//  * B (N = 8 RP for RP candidate row pairs): the Toeplitz matrix of target
//    rows, B[8k + b][j] = T[rho - 2k][j - b], for the plane row rho at which A
//    starts.  One MMA per (rho, item pair) updates all RP row pairs; B for
//    rho + 2 is B for rho shifted by one 8-row group, so one half-strip of
//    groups per (plane, chunk, parity of rho) serves every rho.
// A tile is RC candidate rows x TS candidate columns.  Per CTA the tiles
// run as a pipeline: one control warp issues the TMA load of tile i+1's RGBA
// rows into a staging buffer and the MMAs of tile i into one of two tensor-
// memory accumulator sets, while eight worker warps read the accumulators
// of tile i-1 back (tcgen05.ld), apply the validity test (count map) and
// keep the smallest (SSD << 32 | idx) key; the workers then convert the
// staged words of tile i+1 into the five BF16 planes (R', G', B', hi, lo).
#include "inpaint_engine.h"
#include "ptx.cuh"

namespace inp {
namespace {

constexpr int kTcWorkers = 16;                      // worker warps
constexpr int kTcThreads = 32 * (kTcWorkers + 1);   // + the control warp
constexpr int kTcPlaneW = 512;                      // plane row (BF16 elements)
constexpr int kTcMinSmem = 100 * 1024;  // at most two CTAs (2 x 256 TMEM columns) per SM
constexpr unsigned long long kTcWaitNs = 2000000000ull;

template <int R>
struct TcGeom {
  static constexpr int P = 2 * R + 1;
  static constexpr int RC = R == 8 ? 4 : 8;            // candidate rows per tile
  static constexpr int RP = RC / 2;                    // candidate row pairs
  static constexpr int N = 8 * RP;                     // MMA N
  static constexpr int NC8 = (P + 14) / 8;             // 8-tap chunks: taps j = b + dx < P + 7
  static constexpr int NX = 3 * NC8;                   // cross-term items (channel, chunk)
  static constexpr int NXP = (NX + 1) / 2;             // cross-term MMAs per plane row
  static constexpr int NHS = 5 * NC8 * 2 + 2;          // B half-strips (+ a zero pair)
  static constexpr int NR = RC + P - 1;                // plane rows of a tile
  static constexpr int NRHO = RC + P - 2;              // A start rows
  static constexpr int TMAX = (NRHO - 1) / 2;
  static constexpr int GB = TMAX + RP;                 // 8-row groups per B strip
  static constexpr int TS = (kTcPlaneW + 1 - P) & ~7;  // candidate columns per tile
  static constexpr int STG_BYTES = 2 * NR * 256 * 4;   // two 256-word TMA boxes
  static constexpr int PLANE_BYTES = NR * kTcPlaneW * 2 + 128;
  static constexpr int B_BYTES = NHS * GB * 128;
  static constexpr int OFF_PL = STG_BYTES;
  static constexpr int OFF_B = OFF_PL + 5 * PLANE_BYTES;
  static constexpr int OFF_T = OFF_B + B_BYTES;  // int16 T[4][P * P]
  static constexpr int OFF_MISC = (OFF_T + 4 * P * P * 2 + 15) & ~15;
  static constexpr int RAW = OFF_MISC + 384 + 128;  // + base alignment
  static constexpr int SMEM = RAW < kTcMinSmem ? kTcMinSmem : RAW;
  static constexpr uint32_t ACC = 2 * N;             // columns of one accumulator set (X, S)
  static constexpr uint32_t TMEM_COLS = 2 * ACC <= 64 ? 64 : 2 * ACC <= 128 ? 128 : 256;
  static_assert(RP <= 8, "at most two row pairs per worker warp");
  static_assert(N % 16 == 0 && N <= 256, "M = 128 needs N a multiple of 16");
  static_assert(NC8 * 8 >= P + 7, "chunks must cover every tap");
  static_assert(2 * ACC <= 256, "two accumulator sets in 256 columns");
  static_assert(SMEM <= 227 * 1024, "tile does not fit in shared memory");
};

// BF16 bits of a small integer (|v| <= 256 is exact).
__device__ inline uint32_t bf16_int(int v) { return __float_as_uint((float)v) >> 16; }

// Two byte values b0, b1 (0..255) shifted by `sub`, as a BF16 pair: the float
// 2^23 + b is exact, so subtracting (2^23 + sub) is exact and the high halves
// of the results are the BF16 encodings.
__device__ inline uint32_t bf16x2_bytes(uint32_t b0, uint32_t b1, float base) {
  const float f0 = __uint_as_float(0x4B000000u | b0) - base;
  const float f1 = __uint_as_float(0x4B000000u | b1) - base;
  return __byte_perm(__float_as_uint(f0), __float_as_uint(f1), 0x7632);
}

// Eight RGBA words -> the five BF16 plane words (R', G', B', hi, lo) x 4 pairs.
__device__ inline void convert8(const uint4& v0, const uint4& v1, uint4 (&o)[5]) {
  const uint32_t w[8] = {v0.x, v0.y, v0.z, v0.w, v1.x, v1.y, v1.z, v1.w};
  uint32_t out[5][4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    uint32_t hi2[2], lo2[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const uint32_t x = w[2 * i + h];
      const int d0 = (int)(x & 255u) - 128, d1 = (int)((x >> 8) & 255u) - 128,
                d2 = (int)((x >> 16) & 255u) - 128;
      const uint32_t sq = (uint32_t)(d0 * d0 + d1 * d1 + d2 * d2);
      hi2[h] = sq >> 8;
      lo2[h] = sq & 255u;
    }
    const uint32_t a = w[2 * i], b = w[2 * i + 1];
    out[0][i] = bf16x2_bytes(a & 255u, b & 255u, 8388736.0f);
    out[1][i] = bf16x2_bytes((a >> 8) & 255u, (b >> 8) & 255u, 8388736.0f);
    out[2][i] = bf16x2_bytes((a >> 16) & 255u, (b >> 16) & 255u, 8388736.0f);
    out[3][i] = bf16x2_bytes(hi2[0], hi2[1], 8388608.0f);
    out[4][i] = bf16x2_bytes(lo2[0], lo2[1], 8388608.0f);
  }
#pragma unroll
  for (int p = 0; p < 5; ++p) o[p] = make_uint4(out[p][0], out[p][1], out[p][2], out[p][3]);
}

template <int R>
struct TcTile {
  int x0, y0;
  __device__ TcTile(const ImgState& s, int tile, int nx) {
    x0 = ((s.cx0 - R) & ~7) + (tile % nx) * TcGeom<R>::TS;
    y0 = s.cy0 - R + (tile / nx) * TcGeom<R>::RC;
  }
};

template <int R>
__global__ void __launch_bounds__(kTcThreads, 1) k_search_tc(ImgState s, int nx, int ntiles,
                                                          const __grid_constant__ CUtensorMap tmap) {
  using G = TcGeom<R>;
  constexpr int P = G::P;
  extern __shared__ __align__(16) uint8_t tc_dyn[];
  const Ctrl* c = s.ctrl;
  if (!loop_active(c)) return;
  uint8_t* sm = tc_dyn + ((128u - (smem_addr(tc_dyn) & 127u)) & 127u);
  const uint32_t* stg = reinterpret_cast<const uint32_t*>(sm);
  int16_t* tv = reinterpret_cast<int16_t*>(sm + G::OFF_T);
  uint64_t* stg_bar = reinterpret_cast<uint64_t*>(sm + G::OFF_MISC);
  uint64_t* mma_bar = stg_bar + 1;  // [2]
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(sm + G::OFF_MISC + 24);
  int* a2_slot = reinterpret_cast<int*>(sm + G::OFF_MISC + 28);
  unsigned long long* red = reinterpret_cast<unsigned long long*>(sm + G::OFF_MISC + 32);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const bool ctl = warp == kTcWorkers, ctl0 = ctl && lane == 0;
  const int px = c->px, py = c->py;
  int tma_n = 0, mma_n0 = 0, mma_n1 = 0;  // operations issued (control lane)

  auto issue_tma = [&](int tile) {
    const TcTile<R> t(s, tile, nx);
    const bool two = t.x0 + 256 < s.W;  // the right box lies (partly) inside the image
    mbar_expect_tx(stg_bar, (uint32_t)((two ? 2 : 1) * G::NR * 256 * 4));
    tma_load_2d(sm, &tmap, t.x0, t.y0, stg_bar);
    if (two) tma_load_2d(sm + G::NR * 256 * 4, &tmap, t.x0 + 256, t.y0, stg_bar);
    ++tma_n;
  };

  if (ctl0) {
    mbar_init(stg_bar, 1);
    mbar_init(mma_bar, 1);
    mbar_init(mma_bar + 1, 1);
    fence_mbar_init();
    if ((int)blockIdx.x < ntiles) issue_tma(blockIdx.x);
  }
  if (warp == 0) tc_alloc(tmem_slot, G::TMEM_COLS);
  // Target patch: shifted values and the known indicator, T[kappa][dy * P + dx].
  for (int i = tid; i < P * P; i += kTcThreads) {
    const int dy = i / P, dx = i - dy * P;
    const int tx = px + dx - R, ty = py + dy - R;
    int v0 = 0, v1 = 0, v2 = 0, m = 0;
    if (tx >= 0 && tx < s.W && ty >= 0 && ty < s.H && !s.omega[(size_t)ty * s.W + tx]) {
      const uint32_t w = s.img[(size_t)ty * s.pitch + tx];
      v0 = (int)(w & 255u) - 128;
      v1 = (int)((w >> 8) & 255u) - 128;
      v2 = (int)((w >> 16) & 255u) - 128;
      m = 1;
    }
    tv[i] = (int16_t)v0;
    tv[P * P + i] = (int16_t)v1;
    tv[2 * P * P + i] = (int16_t)v2;
    tv[3 * P * P + i] = (int16_t)m;
  }
  // Zero the tails behind the planes (read only by discarded candidates).
  for (int i = tid; i < 5 * 32; i += kTcThreads)
    reinterpret_cast<uint32_t*>(sm + G::OFF_PL + (i / 32) * G::PLANE_BYTES +
                                G::NR * kTcPlaneW * 2)[i % 32] = 0u;
  __syncthreads();

  // B half-strips, one 16-byte core-matrix row per step: row rr of
  // half-strip hs = (kappa * NC8 + c) * 2 + par (the last two all zeros),
  // group gi, row b; kappa 0-2 channels (T'), 3 the weights 256 m, 4 m.
  constexpr int NBR = G::NHS * G::GB * 8;
  for (int rr = tid; rr < NBR; rr += kTcThreads) {
    const int b = rr & 7;
    int rest = rr >> 3;
    const int gi = rest % G::GB;
    const int hs = rest / G::GB;
    uint32_t wv[4] = {0u, 0u, 0u, 0u};
    if (hs < 5 * G::NC8 * 2) {
      const int par = hs & 1, c = (hs >> 1) % G::NC8, kap = (hs >> 1) / G::NC8;
      const int dy = par - 2 * (gi - G::TMAX);
      if (dy >= 0 && dy < P) {
        const int dx0 = 8 * c - b;
        const int16_t* trow = tv + (kap < 3 ? kap : 3) * P * P + dy * P;
        const int scale = kap == 3 ? 256 : 1;
#pragma unroll
        for (int jj = 0; jj < 8; jj += 2) {
          const int d0 = dx0 + jj, d1 = d0 + 1;
          const int v0 = (d0 >= 0 && d0 < P) ? scale * trow[d0] : 0;
          const int v1 = (d1 >= 0 && d1 < P) ? scale * trow[d1] : 0;
          wv[jj >> 1] = bf16_int(v0) | (bf16_int(v1) << 16);
        }
      }
    }
    *reinterpret_cast<uint4*>(sm + G::OFF_B + rr * 16) = make_uint4(wv[0], wv[1], wv[2], wv[3]);
  }
  if (warp == 0) {
    int a2 = 0;
    for (int i = lane; i < P * P; i += 32) {
      const int v0 = tv[i], v1 = tv[P * P + i], v2 = tv[2 * P * P + i];
      a2 += v0 * v0 + v1 * v1 + v2 * v2;  // zero where unknown
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) a2 += __shfl_xor_sync(0xffffffffu, a2, o);
    if (lane == 0) *a2_slot = a2;
  }
  fence_proxy_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const int a2 = *a2_slot;
  const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(G::N >> 3) << 17) |
                         ((uint32_t)(128 >> 4) << 24);
  // base descriptors (leading byte offsets are added per item pair)
  const uint64_t adesc0 = tc_desc(smem_addr(sm + G::OFF_PL), 0, 128);
  const uint64_t bdesc0 = tc_desc(smem_addr(sm + G::OFF_B), 0, 128);
  const int wq = warp & 3, kh = warp >> 2;  // TMEM lane quarter; row pairs kh, kh + 4, ...
  const int a = 32 * wq + lane, a_row = a >> 6, a_blk = a & 63;
  constexpr int KPW = (G::RP + 3) / 4;  // row pairs per worker warp
  unsigned long long best = ~0ull;
  int bad = 0;

  for (int i = 0;; ++i) {
    const int tile = blockIdx.x + i * gridDim.x;
    const bool has = tile < ntiles;
    // validity counts of the previous tile's candidates, loaded before the
    // conversion so that their latency is hidden behind it
    int cnt[KPW][8];
    if (!ctl && i > 0) {
      const TcTile<R> t(s, tile - gridDim.x, nx);
#pragma unroll
      for (int kk = 0; kk < KPW; ++kk) {
        const int k = kh + 4 * kk;
        const int qy = t.y0 + 2 * k + a_row + R;
#pragma unroll
        for (int b = 0; b < 8; ++b) {
          const int u = 8 * a_blk + b, qx = t.x0 + u + R;
          cnt[kk][b] = (k < G::RP && qy <= s.cy1 && u < G::TS && qx >= s.cx0 && qx <= s.cx1)
                           ? __ldcg(&s.count[(size_t)qy * s.pitch + qx])
                           : 1;
        }
      }
    }
    if (has && !ctl) {
      // staged words of this tile -> planes
      if (!mbar_wait(stg_bar, (uint32_t)(i & 1), kTcWaitNs)) {
        bad = 1;
      } else {
#pragma unroll 2
        for (int g = tid; g < G::NR * 64; g += 32 * kTcWorkers) {
          const int row = g >> 6, cg = g & 63;
          const uint4* src = reinterpret_cast<const uint4*>(
              stg + ((cg >> 5) * G::NR + row) * 256 + (cg & 31) * 8);
          uint4 o[5];
          convert8(src[0], src[1], o);
#pragma unroll
          for (int p = 0; p < 5; ++p)
            *reinterpret_cast<uint4*>(sm + G::OFF_PL + p * G::PLANE_BYTES + row * (kTcPlaneW * 2) +
                                      16 * cg) = o[p];
        }
      }
      fence_proxy_async_smem();
    }
    tc_fence_before();
    if (__syncthreads_or(bad)) break;
    if (ctl) {
      if (lane == 0 && has) {
        tc_fence_after();
        if (tile + (int)gridDim.x < ntiles) issue_tma(tile + gridDim.x);
        const uint32_t dcol = tmem + (uint32_t)((i & 1) * G::ACC);
        const uint32_t a_lo = (uint32_t)adesc0, a_hi = (uint32_t)(adesc0 >> 32);
        const uint32_t b_lo = (uint32_t)bdesc0, b_hi = (uint32_t)(bdesc0 >> 32);
        // item (kappa, c): A at plane kappa, column 8c; B half-strip
        // (kappa * NC8 + c) * 2 + parity.  Descriptor units are 16 bytes; the
        // leading byte offset sits at bit 16.  Every offset is a constant.
        constexpr uint32_t PLU = G::PLANE_BYTES / 16, HSU = G::GB * 8;  // plane, half-strip
        auto a_item = [&](int kap, int c) { return (uint32_t)(kap * PLU + c); };
        auto b_item = [&](int kap, int c) { return (uint32_t)((kap * G::NC8 + c) * 2 * HSU); };
#pragma unroll
        for (int rho = 0; rho < G::NRHO; ++rho) {
          const uint32_t arow = (uint32_t)(rho * (kTcPlaneW * 2 / 16));
          const uint32_t bsh = (uint32_t)(((rho & 1) * G::GB + G::TMAX - (rho >> 1)) * 8);
#pragma unroll
          for (int pi = 0; pi < G::NXP; ++pi) {  // cross-term item pairs into X
            const int i1 = 2 * pi, i2 = 2 * pi + 1;
            const int k1 = i1 / G::NC8, c1 = i1 % G::NC8;
            const uint32_t a1 = a_item(k1, c1), b1 = b_item(k1, c1);
            uint32_t a2, b2;
            if (i2 < G::NX) {
              a2 = a_item(i2 / G::NC8, i2 % G::NC8);
              b2 = b_item(i2 / G::NC8, i2 % G::NC8);
            } else {  // odd count: the second half meets the zero half-strips
              a2 = a1 + 1;
              b2 = b_item(5, 0);
            }
            const uint32_t alo = a_lo + arow + a1 + ((a2 - a1) << 16);
            const uint32_t blo = b_lo + b1 + bsh + ((b2 - b1) << 16);
            if (rho == 0 && pi == 0)
              tc_mma_lo<0>(dcol, alo, a_hi, blo, b_hi, idesc);
            else
              tc_mma_lo<1>(dcol, alo, a_hi, blo, b_hi, idesc);
          }
#pragma unroll
          for (int c = 0; c < G::NC8; ++c) {  // square items (hi, lo) into S
            const uint32_t a1 = a_item(3, c), a2 = a_item(4, c);
            const uint32_t b1 = b_item(3, c), b2 = b_item(4, c);
            const uint32_t alo = a_lo + arow + a1 + ((a2 - a1) << 16);
            const uint32_t blo = b_lo + b1 + bsh + ((b2 - b1) << 16);
            if (rho == 0 && c == 0)
              tc_mma_lo<0>(dcol + G::N, alo, a_hi, blo, b_hi, idesc);
            else
              tc_mma_lo<1>(dcol + G::N, alo, a_hi, blo, b_hi, idesc);
          }
        }
        tc_commit(mma_bar + (i & 1));
        if (i & 1) ++mma_n1; else ++mma_n0;
      }
      __syncwarp();
    } else if (i > 0) {
      // accumulators of the previous tile (its MMAs completed: waited below)
      const TcTile<R> t(s, tile - gridDim.x, nx);
      const uint32_t buf = (uint32_t)(((i - 1) & 1) * G::ACC);
#pragma unroll
      for (int kk = 0; kk < KPW; ++kk) {
        const int k = kh + 4 * kk;
        if (k >= G::RP) break;  // warp-uniform
        uint32_t X[8], Sv[8];
        const uint32_t ta = tmem + ((uint32_t)(32 * wq) << 16) + buf + (uint32_t)(8 * k);
        tc_ld8(ta, X);
        tc_ld8(ta + G::N, Sv);
        tc_wait_ld();
        const int qy = t.y0 + 2 * k + a_row + R;
#pragma unroll
        for (int b = 0; b < 8; ++b) {
          const int qx = t.x0 + 8 * a_blk + b + R;
          const int xv = __float2int_rn(__uint_as_float(X[b]));
          const int sv = __float2int_rn(__uint_as_float(Sv[b]));
          const uint32_t ssd = (uint32_t)(a2 - 2 * xv + sv);
          const unsigned long long key = ((unsigned long long)ssd << 32) | (unsigned)(qy * s.W + qx);
          if (cnt[kk][b] == 0 && key < best) best = key;
        }
      }
    }
    if (!has) break;
    // this tile's MMAs must finish before its planes are overwritten
    if (!mbar_wait(mma_bar + (i & 1), (uint32_t)((i >> 1) & 1), kTcWaitNs)) bad = 1;
    tc_fence_after();
  }

  if (bad) {
    if (tid == 0) atomicCAS(const_cast<int*>(&c->status), 0, INPAINT_ERR_TIMEOUT);
    if (ctl0) {  // let the copies and MMAs in flight finish (bounded) before freeing
      if (tma_n) mbar_wait(stg_bar, (uint32_t)((tma_n - 1) & 1), kTcWaitNs);
      if (mma_n0) mbar_wait(mma_bar, (uint32_t)((mma_n0 - 1) & 1), kTcWaitNs);
      if (mma_n1) mbar_wait(mma_bar + 1, (uint32_t)((mma_n1 - 1) & 1), kTcWaitNs);
    }
  }
  best = block_min_u64(best, red);
  if (tid == 0) s.partial[blockIdx.x] = best;
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tc_dealloc(tmem, G::TMEM_COLS);
  }
}

template <int R>
cudaError_t prepare_r(const ImgState& s, TcPlan* plan) {
  using G = TcGeom<R>;
  cudaError_t e = cudaFuncSetAttribute(k_search_tc<R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       G::SMEM);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0, bps = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k_search_tc<R>, kTcThreads, G::SMEM)) !=
      cudaSuccess)
    return e;
  if (bps < 1) return cudaErrorInvalidConfiguration;
  if (bps > 2) bps = 2;
  const int xb = (s.cx0 - R) & ~7;
  plan->nx = s.cx1 < s.cx0 ? 0 : (s.cx1 - R - xb) / G::TS + 1;
  const int ny = s.cy1 < s.cy0 ? 0 : (s.cy1 - s.cy0) / G::RC + 1;
  plan->ntiles = plan->nx * ny;
  plan->grid = plan->ntiles < sms * bps ? plan->ntiles : sms * bps;
  plan->smem = G::SMEM;
  plan->tmap_rows = G::NR;
  plan->tmap_ready = false;
  return cudaSuccess;
}

template <int R>
cudaError_t launch_r(const ImgState& s, const TcPlan& p, cudaStream_t st) {
  k_search_tc<R><<<p.grid, kTcThreads, p.smem, st>>>(s, p.nx, p.ntiles, p.tmap);
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

cudaError_t encode_search_tc(const ImgState& s, TcPlan* plan) {
  if (!s.img || plan->tmap_rows <= 0) return cudaErrorInvalidValue;
  if (make_image_tmap_box(s, 256, plan->tmap_rows, &plan->tmap) != 0) return cudaErrorInvalidValue;
  plan->tmap_ready = true;
  return cudaSuccess;
}

cudaError_t launch_search_tc(const ImgState& s, const TcPlan& p, cudaStream_t st) {
  if (p.grid <= 0) return cudaSuccess;
  if (!p.tmap_ready) return cudaErrorInvalidValue;
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
