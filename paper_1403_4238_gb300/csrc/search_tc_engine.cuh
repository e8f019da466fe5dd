// Tensor-core search of the persistent engine: the exact BF16 correlation
// form of the masked SSD (Sec. 3, Eq. 3-4) over the tiles of a searching
// CTA.
//
// With b' = byte - 128 (|b'| <= 128, exact in BF16) and m the known flags of
// the target patch Psi_p^ (zero outside the image):
//   SSD(q) = A2 - 2 X(q) + S(q),   A2 = sum_d m(d) sum_c t'_c(d)^2,
//   X(q) = sum_c sum_d m(d) t'_c(d) s'_c(q + d),
//   S(q) = sum_d m(d) sq(q + d),   sq = sum_c s'_c^2 = 256 hi + lo (hi, lo < 256).
// Every product is exact and every partial sum an integer below 2^24
// (|X| <= 17^2 * 3 * 128^2, S <= 17^2 * 49152), so the FP32 accumulation is
// exact and the SSD equals the CUDA-core form's bit for bit.
//
// One MMA (M = 128, N = 64 or 128, K = 16, BF16 operands in shared memory,
// FP32 accumulators in tensor memory) takes one source row y of a tile
// whose candidate rows are y0 .. y0 + 15 and whose candidate columns start
// at xs + R:
//  * A, the target as a Toeplitz matrix: row m = 8 i + b (candidate row
//    y0 + i, column shift b), K column kk of item (plane p, 8-tap chunk c)
//    holds w_p(k, 8c + kk - b) for target row k = y - y0 - i, where w is
//    m t'_p (p < 3) or m (p = 3, for both square planes), zero outside the
//    patch.  A strip (p, c) stores its 8x8 core matrices for target rows
//    P-1 .. 0 in that order between runs of 15 zero matrices, so the A
//    operand of row y is the 16 consecutive matrices that start at target
//    row y - y0, and an MMA's two K halves are two items of their own (the
//    leading byte offset is the distance between their strips).
//  * B, the source row itself: five plane-row segments side by side (R', G',
//    B', 256 hi -- exact in BF16, as hi < 256 -- and lo); row n of B
//    (candidate columns 8n .. 8n + 7) starts 16 bytes after row n - 1 (rows
//    overlap), chunk c 16 bytes further.
//  * D: accumulator X (the three channel planes, items paired across
//    planes) or S (256 hi and lo of one chunk against the same mask strip:
//    a leading byte offset of 0 in A); lane m, column n is candidate
//    (y0 + m / 8, xs + 8 n + m % 8 + R).
// Per tile one producer thread copies the tile's source rows into a ring of
// shared-memory slots (one bulk copy of two rows, five plane segments each,
// from the planes' tiled layout), two issuer threads issue the X and the S
// MMAs of a slot's rows once they have landed and free the slot with
// tcgen05.commit, and then all 16 warps read the accumulators back
// (tcgen05.ld), test validity against bits kept in shared memory and keep
// the smallest (SSD << 32 | idx) key.  The read-back works in FP32:
// fl(fl(S - 2X) + A2) is exact whenever the SSD is below 2^24 (then |S - 2X|
// < 2^24 too, as A2 < 2^24) and at least 2^24 otherwise (rounding is
// monotone), so a best value below 2^24 is the exact minimum; a thread
// whose best is not repeats its candidates in integers.
#pragma once
#include "inpaint_engine.h"
#include "ptx.cuh"

namespace inp {

template <int R>
struct TcEngGeom {
  static constexpr int P = 2 * R + 1;
  static constexpr int NC = (P + 14) / 8;              // 8-tap chunks: taps b + dx < P + 7
  static constexpr int NRS = kTcRows + P - 1;          // source rows of a tile
  static constexpr int NSL = NRS / kTcRps;             // ring slots a tile fills
  static constexpr int NSTRIP = 4 * NC;                // (plane, chunk) strips of A: 3 channels, mask
  static constexpr int ZG = 15;                        // zero matrices between strips
  static constexpr int ZERO = ZG + NSTRIP * (P + ZG);  // 16 zero matrices: the empty K half
  static constexpr int NGA = ZERO + 16;                // 8x8 core matrices of the A area
  static constexpr int A_BYTES = NGA * 128;
  static constexpr int NX = 3 * NC;                    // cross-term items of a source row
  static constexpr int NXP = (NX + 1) / 2;             // X MMAs of a source row
  static constexpr int TW = 32;                        // padded target row: taps -8 .. 23
  static constexpr int TPAD_BYTES = (4 * P * TW * 2 + 127) / 128 * 128;
  __host__ __device__ static constexpr int sg(int st) { return ZG + st * (P + ZG); }
  static_assert(NC == (R <= 4 ? 2 : 3), "chunks cover every tap");
  static_assert(NRS % kTcRps == 0, "whole slots per tile");
  static_assert(8 * NC <= TW - 8, "padded target row covers every chunk");
};
// Bytes of one plane-row segment of a tile and of a ring slot (kTcRps rows
// of five segments).
__host__ __device__ inline int tc_lrow(int N, int r) { return 16 * (N + tc_chunks(r) - 1); }
__host__ __device__ inline int tc_slot(int N, int r) { return (kTcRps * 5 * tc_lrow(N, r) + 16 + 127) & ~127; }
// Validity-bit words of one tile: kTcRows rows of 8N bits.
__host__ __device__ inline int tc_bit_words(int N) { return kTcRows * N / 4; }

// Where a tensor-core search keeps its state: A | padded target | ring | bits.
// The padded target table (written by the searcher's target staging):
// tpad[(p * P + k) * TW + 8 + jj] = w_p(k, jj) for p < 4 (R' G' B', the
// known flag) and jj in [-8, 24), zero outside the patch or where unknown.
struct TcArea {
  uint8_t* a;
  uint16_t* tpad;
  uint8_t* ring;
  uint32_t* bits;
  int nb;    // ring slots
  int ntl;   // tiles of this CTA
  int slot;  // bytes per slot
};

// Validity bits of this CTA's tiles from the counts (whole block).
template <int R>
__device__ __forceinline__ void tc_bits_init(const ImgState& s, const TcTiles& tt, uint32_t* bits, int ntl, int rank,
                                          int ns) {
  const int bw = tt.N / 4, ntiles = tt.ntx * tt.nty;
  for (int e = threadIdx.x; e < ntl * kTcRows * bw; e += blockDim.x) {
    const int kt = e / (kTcRows * bw), i = (e / bw) % kTcRows, w = e % bw;
    const int t = rank + kt * ns;
    uint32_t v = 0;
    if (t < ntiles) {
      const int qy = s.cy0 + kTcRows * (t / tt.ntx) + i;
      const int qx0 = tt.xs0 + 8 * tt.N * (t % tt.ntx) + 32 * w + R;
      if (qy <= s.cy1) {
        // all 32 loads in flight together (one L2 round trip)
        const int32_t* row = s.count + (size_t)qy * s.pitch;
        int cnt[32];
#pragma unroll
        for (int k = 0; k < 32; ++k) {
          const int qx = qx0 + k;
          cnt[k] = (qx >= s.cx0 && qx <= s.cx1) ? __ldcg(&row[qx]) : 1;
        }
#pragma unroll
        for (int k = 0; k < 32; ++k) v |= (cnt[k] == 0 ? 1u : 0u) << k;
      }
    }
    bits[e] = v;
  }
}

// Candidates within 2R of the previous target may have become valid (the
// fill only makes pixels known): set their bits (threads [0, nthr)).
template <int R>
__device__ __forceinline__ void tc_bits_refresh(const ImgState& s, const TcTiles& tt, uint32_t* bits, int rank, int ns,
                                             int ppx, int ppy, int nthr) {
  constexpr int NCW = 4 * R + 1;
  const int bw = tt.N / 4;
  for (int e = threadIdx.x; e < NCW * NCW; e += nthr) {
    const int qx = ppx + e % NCW - 2 * R, qy = ppy + e / NCW - 2 * R;
    if (qx < s.cx0 || qx > s.cx1 || qy < s.cy0 || qy > s.cy1) continue;
    const int xl = qx - R - tt.xs0;
    const int t = ((qy - s.cy0) / kTcRows) * tt.ntx + xl / (8 * tt.N);
    if (t % ns != rank) continue;
    if (__ldcg(&s.count[(size_t)qy * s.pitch + qx]) != 0) continue;
    const int kt = t / ns, i = (qy - s.cy0) % kTcRows, x = xl % (8 * tt.N);
    atomicOr(&bits[(kt * kTcRows + i) * bw + (x >> 5)], 1u << (x & 31));
  }
}

// The A strips from the padded target (threads [0, nthr)); the zero
// matrices are written only when `pads` (the first round of an image).  The
// writing threads order their stores before the MMAs' reads (proxy fence).
template <int R>
__device__ __forceinline__ void tc_build_a(uint8_t* A, const uint16_t* tpad, bool pads, int nthr) {
  using G = TcEngGeom<R>;
  constexpr int P = G::P, TW = G::TW;
  const int tid = threadIdx.x;
  if (tid >= nthr) return;
  if (pads) {
    for (int e = tid; e < G::NGA * 8; e += nthr) {
      const int rel = (e >> 3) - G::ZG;
      const bool strip = rel >= 0 && rel / (P + G::ZG) < G::NSTRIP && rel % (P + G::ZG) < P;
      if (!strip) reinterpret_cast<uint4*>(A)[e] = make_uint4(0u, 0u, 0u, 0u);
    }
  }
  for (int e = tid; e < G::NSTRIP * P * 8; e += nthr) {
    const int b = e & 7, j = (e >> 3) % P, st = (e >> 3) / P;
    const int p = st / G::NC, c = st - p * G::NC, k = P - 1 - j;
    // taps 8c - b .. 8c - b + 7 of target row k, plane p
    const uint16_t* src = tpad + (p * P + k) * TW + 8 + 8 * c - b;
    uint32_t w[4];
#pragma unroll
    for (int h = 0; h < 4; ++h) w[h] = (uint32_t)src[2 * h] | ((uint32_t)src[2 * h + 1] << 16);
    *reinterpret_cast<uint4*>(A + (G::sg(st) + j) * 128 + b * 16) = make_uint4(w[0], w[1], w[2], w[3]);
  }
  fence_proxy_async_smem();
}

// Producer: ring slots [h0, h1) of the tile in tile column tx whose source
// rows start at y0 - R (ring sequence numbers g0 + h; slot h holds rows
// 2h, 2h + 1, five plane segments of tc_len elements each).  One thread.
// Returns false if a bounded wait gave up.
template <int R>
__device__ __forceinline__ bool tc_produce(const ImgState& s, const TcArea& ta, EngBars& bars, int tx, int y0,
                                           uint32_t g0, int h0, int h1, unsigned long long limit) {
  const uint32_t bytes = (uint32_t)(kTcRps * 5 * 2 * s.tc_len);
  for (int h = h0; h < h1; ++h) {
    const uint32_t g = g0 + (uint32_t)h;
    const int slot = (int)(g % (uint32_t)ta.nb);
    if (g >= (uint32_t)ta.nb && !mbar_wait(&bars.tc_empty[slot], ((g / ta.nb) - 1u) & 1u, limit)) return false;
    mbar_expect_tx(&bars.tc_full[slot], bytes);
    const uint16_t* src = s.planes + ((size_t)tx * s.prows + (y0 - R + kTcRps * h)) * 5 * s.tc_len;
    bulk_load(ta.ring + (size_t)slot * ta.slot, src, bytes, &bars.tc_full[slot]);
  }
  return true;
}

// Issuer of the X MMAs (KIND 0) or the S MMAs (KIND 1) of a tile's NRS source
// rows, then a commit to the tile's done barrier.  One whole warp (the
// descriptor arithmetic is warp-uniform; one elected lane issues).  N is a
// template parameter so that every descriptor is a base plus an immediate.
template <int R, int KIND, int N>
__device__ __forceinline__ bool tc_issue(const TcArea& ta, EngBars& bars, uint32_t tmem, uint32_t g0,
                                      unsigned long long limit) {
  using G = TcEngGeom<R>;
  constexpr int P = G::P, NC = G::NC, NM = KIND == 0 ? G::NXP : NC;
  constexpr int LROW = 16 * (N + NC - 1);  // bytes of a plane-row segment
  constexpr uint32_t IDESC =
      (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
  const uint32_t hi = (128u >> 4) | (1u << 14);  // stride byte offset 128, descriptor version 1
  const uint32_t d = tmem + (KIND == 0 ? 0u : (uint32_t)N);
  const uint32_t a_lo0 = smem_addr(ta.a) >> 4, r_lo0 = smem_addr(ta.ring) >> 4;
  const int nb = ta.nb;
  const uint32_t slot_units = (uint32_t)ta.slot >> 4;
  int slot = (int)(g0 % (uint32_t)nb);
  uint32_t par = (g0 / (uint32_t)nb) & 1u;
  bool ok = true;
#pragma unroll 1
  for (int h = 0; h < G::NSL; ++h) {
    if (!__all_sync(0xffffffffu, mbar_wait(&bars.tc_full[slot], par, limit))) {
      ok = false;
      break;
    }
    tc_fence_after();
    const uint32_t b_slot = r_lo0 + (uint32_t)slot * slot_units;
#pragma unroll
    for (int rr = 0; rr < kTcRps; ++rr) {
      const int j = kTcRps * h + rr;
      const uint32_t a_row = a_lo0 + (uint32_t)(P - 1 - j) * 8u;
#pragma unroll
      for (int q = 0; q < NM; ++q) {
        // A: first item's core matrix for row j, leading byte offset to the second
        // (offsets relative to row j's A base a_lo0 + (P - 1 - j) * 8)
        int a1, a2, o1, o2;
        uint32_t zl = 0u;  // row-dependent part of a leading byte offset
        if (KIND == 0) {
          const int i1 = 2 * q, i2 = 2 * q + 1;
          a1 = G::sg(i1);
          if (i2 < G::NX) {
            a2 = G::sg(i2);
          } else {  // the second K half reads the zero matrices
            a2 = G::ZERO - (P - 1);
            zl = (uint32_t)(j * 8) << 16;
          }
          o1 = (i1 / NC) * LROW + 16 * (i1 % NC);
          o2 = i2 < G::NX ? (i2 / NC) * LROW + 16 * (i2 % NC) : o1 + 16;  // zero weights: any finite data
        } else {
          a1 = a2 = G::sg(3 * NC + q);  // both K halves: the mask strip
          o1 = 3 * LROW + 16 * q;
          o2 = o1 + LROW;
        }
        o1 += rr * 5 * LROW;
        o2 += rr * 5 * LROW;
        const uint32_t alo = a_row + (uint32_t)(a1 * 8 + ((a2 - a1) * 8 << 16)) + zl;
        const uint32_t blo = b_slot + (uint32_t)((o1 >> 4) + (((o2 - o1) >> 4) << 16));
        if (j == 0 && q == 0)
          tc_mma_lo_elect<0>(d, alo, hi, blo, hi, IDESC);
        else
          tc_mma_lo_elect<1>(d, alo, hi, blo, hi, IDESC);
      }
    }
    tc_commit_elect(&bars.tc_empty[slot]);
    if (++slot == nb) {
      slot = 0;
      par ^= 1u;
    }
  }
  tc_commit_elect(&bars.tc_done);  // also when a wait gave up: the MMAs issued so far
  return ok;
}

// Accumulators of tile (y0, xs) -> this thread's best key over its 16 or 32
// candidates (whole block, after the tile's done barrier): warp w reads the
// tensor-memory lanes of its quarter w % 4 and columns [w / 4 * N / 4, + N / 4),
// 16 at a time.
template <int R>
__device__ __forceinline__ unsigned long long tc_epilogue(const ImgState& s, uint32_t tmem, int N, int a2,
                                                       const uint32_t* tbits, int y0, int xs,
                                                       unsigned long long best) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int q = warp & 3, cg = warp >> 2;
  const int m = 32 * q + lane, i = m >> 3, b = m & 7;
  const int cols = N / 4;
  const int c0 = cg * cols;
  const uint32_t* brow = tbits + i * (N / 4) + c0 / 4;
  const int idx0 = (y0 + i) * s.W + xs + b + R + 8 * c0;  // candidate of this warp's first column
  const uint32_t ta = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)c0;
  const float a2f = (float)a2;  // exact: a2 < 2^24
  float bv = __int_as_float(0x7f800000);  // +inf
  int bi = 0;
  bool any = false;
  for (int h = 0; h < cols; h += 16) {
    uint32_t X[16], S[16];
    tc_ld16(ta + (uint32_t)h, X);
    tc_ld16(ta + (uint32_t)(N + h), S);
    const uint4 w = *reinterpret_cast<const uint4*>(brow + h / 4);
    tc_wait_ld();
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      // candidates in increasing index order: the strict test keeps the first of equals
      const float v = __fadd_rn(__fmaf_rn(-2.0f, __uint_as_float(X[k]), __uint_as_float(S[k])), a2f);
      const uint32_t word = k < 4 ? w.x : k < 8 ? w.y : k < 12 ? w.z : w.w;
      const bool valid = (word >> (8 * (k & 3) + b)) & 1u;
      any |= valid;
      if (valid && v < bv) {
        bv = v;
        bi = idx0 + 8 * (h + k);
      }
    }
  }
  if (!any) return best;
  if (bv < 16777216.0f) {  // exact
    const unsigned long long key = ((unsigned long long)(uint32_t)bv << 32) | (unsigned)bi;
    return key < best ? key : best;
  }
  // no candidate below 2^24: the exact integer pass over the same accumulators
  for (int h = 0; h < cols; h += 16) {
    uint32_t X[16], S[16];
    tc_ld16(ta + (uint32_t)h, X);
    tc_ld16(ta + (uint32_t)(N + h), S);
    const uint4 w = *reinterpret_cast<const uint4*>(brow + h / 4);
    tc_wait_ld();
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      const uint32_t word = k < 4 ? w.x : k < 8 ? w.y : k < 12 ? w.z : w.w;
      if ((word >> (8 * (k & 3) + b)) & 1u) {
        const int xv = __float2int_rz(__uint_as_float(X[k]));
        const int sv = __float2int_rz(__uint_as_float(S[k]));
        const uint32_t ssd = (uint32_t)(a2 - 2 * xv + sv);
        const unsigned long long key = ((unsigned long long)ssd << 32) | (unsigned)(idx0 + 8 * (h + k));
        best = key < best ? key : best;
      }
    }
  }
  return best;
}

}  // namespace inp
