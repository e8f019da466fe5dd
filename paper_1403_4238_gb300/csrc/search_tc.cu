// findBestPatch, exact tensor-core form (Sec. 3, Eq. 3-4 written as
// correlations; the paper's own kernel is the CUDA-core Algorithm 1).
//
// With every byte shifted by 128 (b' = b - 128, |b'| <= 128, exact in BF16)
// and m the known-pixel indicator of the target patch Psi_p^:
//   SSD(q) = sum_d m(d) sum_c (t'_c(d) - s'_c(q+d))^2 = A2 - 2 X(q) + S(q)
//   A2   = sum_d m(d) sum_c t'_c(d)^2                       (one integer)
//   X(q) = sum_c sum_d [m(d) t'_c(d)] s'_c(q+d)             (3 correlations)
//   S(q) = sum_d m(d) sq(q+d),  sq = sum_c s'_c^2 <= 49152   (split as
//          sq = 256 hi + lo with hi, lo < 256: two correlations)
// Every product of two BF16 integers is exact and every partial sum is an
// integer of magnitude below 2^24 (|X| <= 17^2 * 3 * 128^2, S parts below
// 17^2 * 255), so the FP32 accumulators hold exact integers and the SSD equals
// the CUDA-core form's bit for bit.
//
// The correlations run as tcgen05 MMAs (kind::f16, BF16 operands in shared
// memory, FP32 accumulators in tensor memory) with no im2col copy:
//  * A (M = 128): row a is a block of 8 consecutive candidates (64 blocks of
//    one candidate row, then 64 of the next); it reads the plane row directly,
//    row a starting 16 bytes after row a - 1.  That is the canonical
//    no-swizzle K-major layout with a 16-byte stride between the two K core
//    matrices of an MMA (consecutive rows overlap in memory).
//  * B (N = 8 RP for RP candidate row pairs): the Toeplitz matrix of target
//    rows, B[8k + b][j] = T[rho - 2k][j - b], for the plane row rho at which A
//    starts.  One MMA per (rho, K chunk, plane) updates all RP row pairs; B
//    for rho + 2 is B for rho shifted by one 8-row group, so one strip of
//    groups per (plane, K chunk, parity of rho) serves every rho.
// A tile is kTcRows candidate rows x TS candidate columns; its planes
// (R', G', B', hi, lo as BF16, 512 columns each) are converted from the RGBA
// image into shared memory, one elected thread issues the MMAs, and the
// eight warps read the accumulators back (tcgen05.ld), add the validity test
// (count map) and reduce to one (SSD << 32 | idx) key per CTA.
#include "inpaint_internal.cuh"
#include "ptx.cuh"

namespace inp {
namespace {

constexpr int kTcThreads = 256;
constexpr int kTcRows = 8;      // candidate rows per tile
constexpr int kTcPlaneW = 512;  // plane row length (BF16 elements)
constexpr unsigned long long kTcWaitNs = 2000000000ull;

template <int R>
struct TcGeom {
  static constexpr int P = 2 * R + 1;
  static constexpr int RC = kTcRows;
  static constexpr int RP = RC / 2;                    // candidate row pairs
  static constexpr int N = 8 * RP;                     // MMA N
  static constexpr int KC = (P + 22) / 16;             // K chunks: taps j = b + dx < P + 7
  static constexpr int NR = RC + P - 1;                // plane rows of a tile
  static constexpr int NRHO = RC + P - 2;              // A start rows
  static constexpr int TMAX = (NRHO - 1) / 2;
  static constexpr int GB = TMAX + RP;                 // 8-row groups per B strip
  static constexpr int TS = (kTcPlaneW + 1 - P) & ~7;  // candidate columns per tile
  static constexpr int PLANE_BYTES = NR * kTcPlaneW * 2 + 128;
  static constexpr int B_BYTES = 4 * KC * 2 * GB * 256;
  static constexpr int OFF_B = 5 * PLANE_BYTES;
  static constexpr int OFF_T = OFF_B + B_BYTES;  // int16 T[4][P * P]
  static constexpr int OFF_MISC = (OFF_T + 4 * P * P * 2 + 15) & ~15;
  static constexpr int SMEM = OFF_MISC + 16 + 32 * 8 + 128;  // + base alignment
  static constexpr uint32_t TMEM_COLS = 3 * N <= 32 ? 32 : 3 * N <= 64 ? 64 : 3 * N <= 128 ? 128 : 256;
  static_assert(RP % 2 == 0 && N % 16 == 0 && N <= 256, "M = 128 needs N a multiple of 16");
  static_assert(KC * 16 >= P + 7, "K chunks must cover every tap");
  static_assert(SMEM <= 227 * 1024, "tile does not fit in shared memory");
};

// ------------------------------------------------------------- tcgen05 PTX

__device__ inline uint64_t tc_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  // shared-memory matrix descriptor: start, leading (K) and stride (M/N) byte
  // offsets >> 4, descriptor version 1, no swizzle
  return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)(lbo >> 4) << 16) |
         ((uint64_t)(sbo >> 4) << 32) | (1ull << 46);
}

__device__ inline void tc_mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}

__device__ inline void tc_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   smem_addr(bar))
               : "memory");
}

__device__ inline void tc_alloc(uint32_t* slot, uint32_t cols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                   smem_addr(slot)),
               "r"(cols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ inline void tc_dealloc(uint32_t taddr, uint32_t cols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(cols)
               : "memory");
}

__device__ inline void tc_ld8(uint32_t taddr, uint32_t (&v)[8]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
        "=r"(v[7])
      : "r"(taddr)
      : "memory");
}

__device__ inline void tc_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
__device__ inline void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ inline void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ inline void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ inline void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

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
__global__ void __launch_bounds__(kTcThreads) k_search_tc(ImgState s, int nx, int ntiles) {
  using G = TcGeom<R>;
  constexpr int P = G::P;
  extern __shared__ __align__(16) uint8_t tc_dyn[];
  const Ctrl* c = s.ctrl;
  if (!loop_active(c)) return;
  uint8_t* sm = tc_dyn + ((128u - (smem_addr(tc_dyn) & 127u)) & 127u);
  int16_t* tv = reinterpret_cast<int16_t*>(sm + G::OFF_T);
  uint16_t* bsm = reinterpret_cast<uint16_t*>(sm + G::OFF_B);
  uint64_t* mbar = reinterpret_cast<uint64_t*>(sm + G::OFF_MISC);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(sm + G::OFF_MISC + 8);
  int* a2_slot = reinterpret_cast<int*>(sm + G::OFF_MISC + 12);
  unsigned long long* red = reinterpret_cast<unsigned long long*>(sm + G::OFF_MISC + 16);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int px = c->px, py = c->py;

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
    reinterpret_cast<uint32_t*>(sm + (i / 32) * G::PLANE_BYTES + G::NR * kTcPlaneW * 2)[i % 32] = 0u;
  if (tid == 0) {
    mbar_init(mbar, 1);
    fence_mbar_init();
  }
  if (warp == 0) tc_alloc(tmem_slot, G::TMEM_COLS);
  __syncthreads();

  // B strips: element e = (((kappa * KC + kc) * 2 + par) * GB + gi) * 128 + w;
  // w = core matrix cm (K half), row b, column jj.
  constexpr int NB = 4 * G::KC * 2 * G::GB * 128;
  for (int e = tid; e < NB; e += kTcThreads) {
    int rem = e;
    const int w = rem & 127;
    rem >>= 7;
    const int gi = rem % G::GB;
    rem /= G::GB;
    const int par = rem & 1;
    rem >>= 1;
    const int kc = rem % G::KC, kap = rem / G::KC;
    const int cm = w >> 6, b = (w >> 3) & 7, jj = w & 7;
    const int dy = par - 2 * (gi - G::TMAX);
    const int dx = 16 * kc + 8 * cm + jj - b;
    int v = 0;
    if (dy >= 0 && dy < P && dx >= 0 && dx < P) v = tv[kap * P * P + dy * P + dx];
    bsm[e] = (uint16_t)bf16_int(v);
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
  __syncthreads();
  const uint32_t tmem = *tmem_slot;
  const int a2 = *a2_slot;
  const uint32_t plane0 = smem_addr(sm), b0 = smem_addr(sm + G::OFF_B);
  const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(G::N >> 3) << 17) |
                         ((uint32_t)(128 >> 4) << 24);
  const int xb = (s.cx0 - R) & ~7, ys = s.cy0 - R;
  const int wq = warp & 3, kh = warp >> 2;
  const int a = 32 * wq + lane, a_row = a >> 6, a_blk = a & 63;
  unsigned long long best = ~0ull;
  uint32_t phase = 0;
  bool failed = false;

  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int x0 = xb + (tile % nx) * G::TS, y0 = ys + (tile / nx) * G::RC;
    // planes of rows y0 .. y0 + NR - 1, columns x0 .. x0 + 511
    for (int g = tid; g < G::NR * 64; g += kTcThreads) {
      const int row = g >> 6, cg = g & 63;
      const int y = y0 + row, x = x0 + 8 * cg;
      uint4 v0 = make_uint4(0, 0, 0, 0), v1 = v0;
      if (y < s.H) {
        const uint4* src = reinterpret_cast<const uint4*>(s.img + (size_t)y * s.pitch + x);
        if (x < s.pitch) v0 = __ldg(src);
        if (x + 4 < s.pitch) v1 = __ldg(src + 1);
      }
      uint4 o[5];
      convert8(v0, v1, o);
#pragma unroll
      for (int p = 0; p < 5; ++p)
        *reinterpret_cast<uint4*>(sm + p * G::PLANE_BYTES + row * (kTcPlaneW * 2) + 16 * cg) = o[p];
    }
    fence_proxy_async_smem();
    tc_fence_before();
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
      for (int rho = 0; rho < G::NRHO; ++rho) {
        const int par = rho & 1, t = rho >> 1;
        for (int kc = 0; kc < G::KC; ++kc) {
          const uint32_t aoff = (uint32_t)(rho * kTcPlaneW * 2 + 32 * kc);
          const uint32_t boff = (uint32_t)((G::TMAX - t) * 256);
          const uint32_t first = (rho == 0 && kc == 0) ? 1u : 0u;
#pragma unroll
          for (int ch = 0; ch < 3; ++ch) {
            const uint64_t ad = tc_desc(plane0 + ch * G::PLANE_BYTES + aoff, 16, 128);
            const uint64_t bd =
                tc_desc(b0 + ((ch * G::KC + kc) * 2 + par) * G::GB * 256 + boff, 128, 256);
            tc_mma(tmem, ad, bd, idesc, (first && ch == 0) ? 0u : 1u);
          }
          const uint64_t bm = tc_desc(b0 + ((3 * G::KC + kc) * 2 + par) * G::GB * 256 + boff, 128, 256);
          tc_mma(tmem + G::N, tc_desc(plane0 + 3 * G::PLANE_BYTES + aoff, 16, 128), bm, idesc,
                 first ? 0u : 1u);
          tc_mma(tmem + 2 * G::N, tc_desc(plane0 + 4 * G::PLANE_BYTES + aoff, 16, 128), bm, idesc,
                 first ? 0u : 1u);
        }
      }
      tc_commit(mbar);
    }
    const bool got = mbar_wait(mbar, phase, kTcWaitNs);
    phase ^= 1u;
    if (__syncthreads_or(!got)) {
      failed = true;
      break;
    }
    tc_fence_after();
#pragma unroll
    for (int kk = 0; kk < G::RP / 2; ++kk) {
      const int k = kh * (G::RP / 2) + kk;
      uint32_t X[8], Hv[8], Lv[8];
      const uint32_t ta = tmem + ((uint32_t)(32 * wq) << 16) + (uint32_t)(8 * k);
      tc_ld8(ta, X);
      tc_ld8(ta + G::N, Hv);
      tc_ld8(ta + 2 * G::N, Lv);
      tc_wait_ld();
      const int qy = y0 + 2 * k + a_row + R;
      if (qy > s.cy1) continue;
#pragma unroll
      for (int b = 0; b < 8; ++b) {
        const int u = 8 * a_blk + b, qx = x0 + u + R;
        if (u >= G::TS || qx < s.cx0 || qx > s.cx1) continue;
        const int xv = __float2int_rn(__uint_as_float(X[b]));
        const int hv = __float2int_rn(__uint_as_float(Hv[b]));
        const int lv = __float2int_rn(__uint_as_float(Lv[b]));
        const uint32_t ssd = (uint32_t)(a2 - 2 * xv + 256 * hv + lv);
        const int idx = qy * s.W + qx;
        const unsigned long long key = ((unsigned long long)ssd << 32) | (unsigned)idx;
        if (key < best && s.count[idx] == 0) best = key;
      }
    }
    tc_fence_before();
  }

  if (failed) {
    if (tid == 0) atomicCAS(const_cast<int*>(&c->status), 0, INPAINT_ERR_TIMEOUT);
    // let the MMAs in flight finish (bounded) before the accumulators are freed
    mbar_wait(mbar, phase ^ 1u, kTcWaitNs);
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
  if (bps > 2) bps = 2;  // at most 2 x 256 tensor-memory columns per SM
  const int xb = (s.cx0 - R) & ~7;
  plan->nx = s.cx1 < s.cx0 ? 0 : (s.cx1 - R - xb) / G::TS + 1;
  const int ny = s.cy1 < s.cy0 ? 0 : (s.cy1 - s.cy0) / G::RC + 1;
  plan->ntiles = plan->nx * ny;
  plan->grid = plan->ntiles < sms * bps ? plan->ntiles : sms * bps;
  plan->smem = G::SMEM;
  return cudaSuccess;
}

template <int R>
cudaError_t launch_r(const ImgState& s, const TcPlan& p, cudaStream_t st) {
  k_search_tc<R><<<p.grid, kTcThreads, p.smem, st>>>(s, p.nx, p.ntiles);
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
