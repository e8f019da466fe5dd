// Persistent fill-loop engine: the whole iterative stage of Sec. 4.2 in one
// cooperative kernel launch.
//
// CTAs form teams; a team runs the fill loop of one image at a time (a list
// of images per team gives the batched form).  One iteration of a team:
//   1. every member CTA searches its share of the candidate centres
//      (findBestPatch, Eq. 3-4).  Resident mode (large images): the CTA
//      owns a contiguous range of units of 32 candidate rows x 16 columns,
//      keeps their source window in shared memory for the whole removal and
//      only patches the pixels the previous iteration filled; streaming
//      mode (small images, small teams): batches of 32 rows x 64 or 128
//      columns whose source window and validity counts arrive by TMA,
//      double-buffered.  Each lane owns the candidates of one row; the
//      CTA reduces them to one (SSD << 32 | idx) key;
//   2. each member writes its key, tagged with the round, to its slot; the
//      leader polls the slots, runs the copy/update phase and the selection
//      of the next target (update_fast.cuh) and publishes the next epoch;
//   3. the others wait for that epoch (bounded wait, no trap) and go on.
// No host round trip and no kernel boundary per iteration.
#pragma once
#include <cstddef>
#include <type_traits>
#include <cuda.h>

#include "inpaint_engine.h"
#include "ptx.cuh"
#include "search_tc_engine.cuh"
#include "ssd_rows.cuh"
#include "update_fast.cuh"

namespace inp {

// ---------------------------------------------------------------- search batch

// A search batch is 32 candidate rows x BWC candidate columns.  Lane l of
// warp w owns the NCL adjacent candidates (row l, columns w*NCL ...): every
// lane of a warp uses the same target row at the same time (the row-mask
// branch stays warp-uniform), and the lanes' 128-bit loads of their source
// row strips fall on 32 consecutive tile rows, conflict-free.
template <int R, int SRW>
struct EngGeom {
  static constexpr int P = 2 * R + 1;
  static constexpr int NCL = 4 * SRW;              // candidates per lane (4 or 8)
  static constexpr int BWC = eng_batch_cols(SRW);  // candidate columns per batch (64 or 128)
  static constexpr int B = kEngBatchRows;          // candidate rows per batch (one per lane)
  static constexpr int BW = eng_tile_width(R, SRW);  // staged width (words)
  static constexpr int BH = B + 2 * R;             // staged rows
  static constexpr int PIX_BYTES = ((BW * BH * 4 + 127) / 128) * 128;
  static constexpr int CW = eng_count_width(SRW);  // count tile width (words), CW / 4 odd
  static constexpr int CNT_BYTES = ((CW * B * 4 + 127) / 128) * 128;
  static constexpr int VB_BYTES = kEngWarps * 32;  // validity bits: one byte per (warp, lane)
  static constexpr int SLOT_BYTES = PIX_BYTES + VB_BYTES;
  static constexpr int COFF = R & 3;  // first candidate column within the count tile
  static constexpr int NS = (NCL + P - 1 + 3) & ~3;  // strip words per lane
  static constexpr int TP = (P + 3) & ~3;            // padded target row (words)
  static constexpr unsigned FULL = (1u << P) - 1u;
  static_assert((kEngWarps - 1) * NCL + NS <= BW, "row strip must stay inside the tile");
  static_assert(kEngWarps * NCL + 4 <= CW, "count chunk must stay inside the tile row");
  static_assert(((CW / 4) & 1) == 1, "count rows must start in different bank quadruples");
};

template <int N>
__device__ __forceinline__ void lds_words(uint32_t (&d)[N], const uint32_t* p) {
  const uint4* q = reinterpret_cast<const uint4*>(p);
#pragma unroll
  for (int i = 0; i < N / 4; ++i) {
    const uint4 v = q[i];
    d[4 * i] = v.x;
    d[4 * i + 1] = v.y;
    d[4 * i + 2] = v.z;
    d[4 * i + 3] = v.w;
  }
}

// Row descriptor of a target row (computed once per target): which of its
// P pixels are known.  A row next to the fill front is usually known on one
// contiguous run that touches one end of the row, so the common shapes take
// one jump into a straight run of code instead of a test per column:
//   kRowSkip   nothing known;
//   kRowFrom   known on [s, P) (s = 0: the whole row), s in the low bits;
//   kRowUpTo   known on [0, e), e in the low bits;
//   kRowMask   anything else, the bit mask of known columns in the low bits.
constexpr uint32_t kRowSkip = 0u, kRowFrom = 1u << 30, kRowUpTo = 2u << 30, kRowMask = 3u << 30;

__device__ __forceinline__ uint32_t row_desc(uint32_t m, int P) {
  const uint32_t full = (1u << P) - 1u;
  if (m == 0) return kRowSkip;
  const int s = __ffs(m) - 1;           // lowest known column
  const int e = 32 - __clz(m);          // one past the highest known column
  if (m == ((full >> s) << s)) return kRowFrom | (uint32_t)s;
  if (s == 0 && m == (1u << e) - 1u) return kRowUpTo | (uint32_t)e;
  return kRowMask | m;
}

// SSD terms of target column DX for the lane's NCL candidates.
#define INP_SSD_COL(DX)                                                   \
  if constexpr ((DX) < P) {                                               \
    _Pragma("unroll") for (int k = 0; k < NCL; ++k) {                     \
      const uint32_t d_ = __vabsdiffu4(t[(DX)], r[k + (DX)]);             \
      acc[k] = __dp4a(d_, d_, acc[k]);                                    \
    }                                                                     \
  }

// SSD of this lane's NCL candidates against the staged target (Eq. 4): for
// every known target pixel one byte-SIMD absolute difference and one 4-way
// byte dot product per candidate (|a-b| per channel, squares summed; alpha
// is 0 on both sides).  `strip` points at the lane's row strip in the tile
// (row = lane, column = warp * NCL); `rowd` holds one row descriptor per
// target row.  A run of known columns [s, P) enters an ascending sequence of
// columns at s, a run [0, e) a descending one at e - 1 (one warp-uniform
// indirect jump per row); other rows test a bit per column.
template <int R, int SRW>
__device__ __forceinline__ void unit_ssd(const uint32_t* __restrict__ strip,
                                         const uint32_t* __restrict__ tgt,
                                         const uint32_t* __restrict__ rowd,
                                         uint32_t (&acc)[4 * SRW]) {
  using G = EngGeom<R, SRW>;
  constexpr int P = G::P, NS = G::NS, NCL = G::NCL, BW = G::BW, TP = G::TP;
  static_assert(P <= 17, "column sequences are written out for P <= 17");
#pragma unroll
  for (int k = 0; k < NCL; ++k) acc[k] = 0;
#pragma unroll 1
  for (int dy = 0; dy < P; ++dy) {
    const uint32_t desc = rowd[dy];
    if (desc == kRowSkip) continue;
    uint32_t r[NS], t[TP];
    lds_words(r, strip + dy * BW);
    lds_words(t, tgt + dy * TP);
    const uint32_t kind = desc & (3u << 30), arg = desc & 0xffffu;
    if (kind == kRowFrom) {
      switch (arg) {
        case 0: INP_SSD_COL(0) [[fallthrough]];
        case 1: INP_SSD_COL(1) [[fallthrough]];
        case 2: INP_SSD_COL(2) [[fallthrough]];
        case 3: INP_SSD_COL(3) [[fallthrough]];
        case 4: INP_SSD_COL(4) [[fallthrough]];
        case 5: INP_SSD_COL(5) [[fallthrough]];
        case 6: INP_SSD_COL(6) [[fallthrough]];
        case 7: INP_SSD_COL(7) [[fallthrough]];
        case 8: INP_SSD_COL(8) [[fallthrough]];
        case 9: INP_SSD_COL(9) [[fallthrough]];
        case 10: INP_SSD_COL(10) [[fallthrough]];
        case 11: INP_SSD_COL(11) [[fallthrough]];
        case 12: INP_SSD_COL(12) [[fallthrough]];
        case 13: INP_SSD_COL(13) [[fallthrough]];
        case 14: INP_SSD_COL(14) [[fallthrough]];
        case 15: INP_SSD_COL(15) [[fallthrough]];
        case 16: INP_SSD_COL(16) [[fallthrough]];
        default: break;
      }
    } else if (kind == kRowUpTo) {
      switch (arg) {
        case 17: INP_SSD_COL(16) [[fallthrough]];
        case 16: INP_SSD_COL(15) [[fallthrough]];
        case 15: INP_SSD_COL(14) [[fallthrough]];
        case 14: INP_SSD_COL(13) [[fallthrough]];
        case 13: INP_SSD_COL(12) [[fallthrough]];
        case 12: INP_SSD_COL(11) [[fallthrough]];
        case 11: INP_SSD_COL(10) [[fallthrough]];
        case 10: INP_SSD_COL(9) [[fallthrough]];
        case 9: INP_SSD_COL(8) [[fallthrough]];
        case 8: INP_SSD_COL(7) [[fallthrough]];
        case 7: INP_SSD_COL(6) [[fallthrough]];
        case 6: INP_SSD_COL(5) [[fallthrough]];
        case 5: INP_SSD_COL(4) [[fallthrough]];
        case 4: INP_SSD_COL(3) [[fallthrough]];
        case 3: INP_SSD_COL(2) [[fallthrough]];
        case 2: INP_SSD_COL(1) [[fallthrough]];
        case 1: INP_SSD_COL(0) [[fallthrough]];
        default: break;
      }
    } else {
      const uint32_t m = desc;  // kRowMask: bits of the known columns (P <= 17 < 30)
#pragma unroll
      for (int dx = 0; dx < P; ++dx) {
        if (m & (1u << dx)) {
#pragma unroll
          for (int k = 0; k < NCL; ++k) {
            const uint32_t d = __vabsdiffu4(t[dx], r[k + dx]);
            acc[k] = __dp4a(d, d, acc[k]);
          }
        }
      }
    }
  }
}
#undef INP_SSD_COL

// The compute of a search round, outside the engine body so that its
// registers hold only the row strips, the target row and the accumulators
// (the engine body keeps the leader's state live across the search).

// Smallest key (SSD << 32 | idx) of this lane's candidates in one unit:
// `bits` marks the valid ones, idx0 is the linear index of the first.
template <int R, int SRW>
__device__ __noinline__ unsigned long long unit_best(const uint32_t* strip, const uint32_t* tgt,
                                                     const uint32_t* rowd, uint32_t bits, unsigned idx0) {
  uint32_t acc[4 * SRW];
  unit_ssd<R, SRW>(strip, tgt, rowd, acc);
  unsigned long long best = ~0ull;
#pragma unroll
  for (int k = 0; k < 4 * SRW; ++k) {
    const unsigned long long key = ((unsigned long long)acc[k] << 32) | (idx0 + (unsigned)k);
    if ((bits & (1u << k)) && key < best) best = key;
  }
  return best;
}

// ---------------------------------------------------------------- resident search

// Resident mode: the candidate rectangle is cut into units of 32 candidate
// rows (one per lane) x 16 candidate columns (one lane's candidates); the
// units, in band-major order, are split into contiguous ranges of equal
// size, one per searching CTA.  A CTA keeps the source window of its units
// in shared memory for the whole removal (one tile per 32-row band its range
// touches) and after each publication only patches the pixels the previous
// iteration filled and the validity of the candidates near them.
constexpr int kResCols = 16;   // candidates per lane
constexpr int kResRows = 32;   // candidate rows per unit (one per lane)
constexpr int kResMaxSeg = 4;  // bands one CTA's tiles may span

struct ResSeg {
  int band;      // 32-row band of the search rectangle
  int c_lo;      // first unit column of the band in this CTA's range
  int pitch;     // tile row pitch (words), pitch / 4 odd
  int off;       // byte offset of the tile in the CTA's tile area
};

struct ResPlan {
  int u0, u1;        // this CTA's units [u0, u1), band-major
  int ncu;           // unit columns per band
  int nseg;
  int bits_off;      // byte offset of the validity bits (uint16 per unit and lane)
  ResSeg seg[kResMaxSeg];
};

template <int R>
struct ResGeom {
  static constexpr int P = 2 * R + 1;
  static constexpr int NS = (kResCols + P - 1 + 3) & ~3;  // strip words per lane
  static constexpr int TP = (P + 3) & ~3;
  static constexpr int TH = kResRows + 2 * R;             // tile rows
};

// SSD of this lane's 16 candidates (Eq. 4) for one unit: per target row one
// indexed jump into the row sequences of ssd_rows.cuh (known run [s, P) or
// [0, e)); other row shapes test a bit per column.
template <int R>
__device__ __forceinline__ void unit16_ssd(const uint32_t* __restrict__ strip, int pitch,
                                           const uint32_t* __restrict__ tgt,
                                           const uint32_t* __restrict__ rowd, uint32_t (&acc)[kResCols]) {
  using G = ResGeom<R>;
  constexpr int P = G::P, NS = G::NS, TP = G::TP;
#pragma unroll
  for (int k = 0; k < kResCols; ++k) acc[k] = 0;
#pragma unroll 1
  for (int dy = 0; dy < P; ++dy) {
    const uint32_t desc = rowd[dy];
    if (desc == kRowSkip) continue;
    uint32_t r[NS], t[TP];
    lds_words(r, strip + dy * pitch);
    lds_words(t, tgt + dy * G::TP);
    const uint32_t kind = desc & (3u << 30);
    if (kind != kRowMask) {
      const uint32_t arg = desc & 0xffffu;
      // entry of the jump table: [0, P) ascending from column s, [P, 2P)
      // descending from column e - 1; clamped so that it stays in the table
      const uint32_t idx = min(kind == kRowFrom ? arg : (uint32_t)P + arg - 1u, (uint32_t)(2 * P - 1));
      if constexpr (P == 3) INP_SSD_ROW16_P3(acc, r, t, idx);
      if constexpr (P == 5) INP_SSD_ROW16_P5(acc, r, t, idx);
      if constexpr (P == 7) INP_SSD_ROW16_P7(acc, r, t, idx);
      if constexpr (P == 9) INP_SSD_ROW16_P9(acc, r, t, idx);
      if constexpr (P == 11) INP_SSD_ROW16_P11(acc, r, t, idx);
      if constexpr (P == 13) INP_SSD_ROW16_P13(acc, r, t, idx);
      if constexpr (P == 15) INP_SSD_ROW16_P15(acc, r, t, idx);
      if constexpr (P == 17) INP_SSD_ROW16_P17(acc, r, t, idx);
    } else {
#pragma unroll
      for (int dx = 0; dx < P; ++dx) {
        if (desc & (1u << dx)) {
#pragma unroll
          for (int k = 0; k < kResCols; ++k) {
            const uint32_t d = __vabsdiffu4(t[dx], r[k + dx]);
            acc[k] = __dp4a(d, d, acc[k]);
          }
        }
      }
    }
  }
}

// Smallest key (SSD << 32 | idx) of this lane's 16 candidates of one unit:
// `vb` marks the valid ones, idx0 is the linear index of the first.
template <int R>
__device__ __noinline__ unsigned long long unit16_best(const uint32_t* strip, int pitch, const uint32_t* tgt,
                                                       const uint32_t* rowd, uint32_t vb, unsigned idx0) {
  uint32_t acc[kResCols];
  unit16_ssd<R>(strip, pitch, tgt, rowd, acc);
  unsigned long long best = ~0ull;
#pragma unroll
  for (int k = 0; k < kResCols; ++k) {
    const unsigned long long key = ((unsigned long long)acc[k] << 32) | (idx0 + (unsigned)k);
    if ((vb & (1u << k)) && key < best) best = key;
  }
  return best;
}

// All units of this CTA for the current target, warp w taking its local
// units w, w + 16, ...; returns the lane's smallest key.
template <int R>
__device__ __noinline__ unsigned long long resident_units16(const ResPlan* pl, const uint8_t* tiles, int xb,
                                                            int cy0, int W, const uint32_t* tgt,
                                                            const uint32_t* rowd) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int u0 = pl->u0, n = pl->u1 - pl->u0, ncu = pl->ncu, b0 = pl->seg[0].band;
  const uint16_t* bits = reinterpret_cast<const uint16_t*>(tiles + pl->bits_off);
  unsigned long long best = ~0ull;
#pragma unroll 1
  for (int j = warp; j < n; j += kEngWarps) {
    const int u = u0 + j, band = u / ncu, col = u - band * ncu;
    const ResSeg& sg = pl->seg[band - b0];
    const uint32_t* strip = reinterpret_cast<const uint32_t*>(tiles + sg.off) + lane * sg.pitch +
                            (col - sg.c_lo) * kResCols;
    const unsigned idx0 = (unsigned)((cy0 + band * kResRows + lane) * W + xb + col * kResCols);
    const unsigned long long k = unit16_best<R>(strip, sg.pitch, tgt, rowd, bits[j * 32 + lane], idx0);
    best = k < best ? k : best;
  }
  return best;
}

// Plan of rank `rank`'s units: the tile of each band its range touches.
// Returns the bytes of shared memory the plan needs (tiles + validity
// bits), or -1 when the range spans more bands than kResMaxSeg.
template <int R>
__host__ __device__ inline long long res_plan(ResPlan& pl, int ncu, int nbands, int rank, int ns) {
  using G = ResGeom<R>;
  const long long U = (long long)ncu * nbands;
  pl.u0 = (int)(U * rank / ns);
  pl.u1 = (int)(U * (rank + 1) / ns);
  pl.ncu = ncu;
  pl.nseg = 0;
  if (pl.u1 <= pl.u0) {
    pl.bits_off = 0;
    return 0;
  }
  const int b_lo = pl.u0 / ncu, b_hi = (pl.u1 - 1) / ncu;
  if (b_hi - b_lo + 1 > kResMaxSeg) return -1;
  long long off = 0;
  for (int b = b_lo; b <= b_hi; ++b) {
    const int c_lo = b == b_lo ? pl.u0 % ncu : 0;
    const int c_hi = b == b_hi ? (pl.u1 - 1) % ncu + 1 : ncu;
    ResSeg& sg = pl.seg[pl.nseg++];
    sg.band = b;
    sg.c_lo = c_lo;
    sg.pitch = width_odd16((c_hi - c_lo) * kResCols + 2 * R);
    sg.off = (int)off;
    off += (((long long)sg.pitch * G::TH * 4) + 127) / 128 * 128;
  }
  pl.bits_off = (int)off;
  off += (long long)(pl.u1 - pl.u0) * 32 * 2;
  return off;
}

// ---------------------------------------------------------------- kernel

struct EngSmemTail {
  EngBars bars;      // mbarriers (streaming stages, tensor-core ring), tensor-memory base
  ImgState img;      // the image's state block (a leader that does not search reads it here)
  unsigned long long red64[32];
  int red32[32];
  unsigned long long key;  // best key of the round (leader)
  int flag;
  int allow;  // leader: no iteration limit, status or error stops the loop after this iteration
  int stop;
  int px, py;
  int a2row[17];  // tensor-core search: per target row, sum of the known pixels' squared shifted values
  int tc_pref;  // tensor-core search: slots the producer prefetched for the next round
  CtrlSnap snap;  // leader: the control fields its update reads (kept by the leader itself)
  int lim, status, err;  // leader: iteration limit, status and error word (the stop decision)
  EarlySel es;           // leader: the early selection's inputs and outcome
  uint8_t known[2][17 * 17];  // known flags of the last two targets (by round parity)
  ResPlan plan;               // resident mode: this CTA's units and tiles
};

static_assert(offsetof(EngSmemTail, bars) == 0, "the kernel initialises the barriers at the start of shared memory");

constexpr int kTgtWords = 17 * 20 + 17 + 3;  // padded target rows + row masks (R <= 8)
constexpr size_t kHeadBytes = ((((sizeof(EngSmemTail) + 15) & ~size_t(15)) + kTgtWords * 4 + 127) / 128) * 128;

// Shared memory of an engine CTA: head | (the leader only) update state and
// update cache | two count tiles | tile slots.  The slots hold the source
// tiles of the CTA's search batches: all of them, resident across the
// iterations of a removal, when they fit, else two used as a double buffer.
// A searching CTA that does not lead starts its count tiles right after the
// head.  The kernel is launched with all the shared memory an SM offers and
// takes as many slots as fit.
template <int R>
__host__ __device__ constexpr size_t upd_smem_bytes() {
  return ((sizeof(UpdSmem<R>) + 127) / 128) * 128 + sizeof(UpdCache<R>);
}

// The least shared memory an engine CTA needs: a searching leader with two
// slots (the streaming double buffer).
template <int R, int SRW>
__host__ __device__ constexpr size_t eng_smem_bytes() {
  using G = EngGeom<R, SRW>;
  return kHeadBytes + ((upd_smem_bytes<R>() + 127) / 128) * 128 + (size_t)2 * G::CNT_BYTES +
         (size_t)2 * G::SLOT_BYTES + 128;
}

static_assert(eng_smem_bytes<8, 2>() <= 227 * 1024, "engine CTA must fit in shared memory");
static_assert(eng_smem_bytes<7, 2>() <= 227 * 1024, "engine CTA must fit in shared memory");

template <int R>
__device__ inline UpdCache<R>& upd_cache_of(uint8_t* upd_base) {
  return *reinterpret_cast<UpdCache<R>*>(upd_base + ((sizeof(UpdSmem<R>) + 127) / 128) * 128);
}

// Team publication word: epoch (bits 0-31), next target px (32-46), py
// (47-61), stop flag (62).  One acquire load gives a waiting CTA everything
// it needs to start the next search round.
__device__ inline unsigned long long pub_pack(unsigned epoch, int px, int py, bool stop) {
  return (unsigned long long)epoch | ((unsigned long long)(px & 0x7fff) << 32) |
         ((unsigned long long)(py & 0x7fff) << 47) | ((unsigned long long)(stop ? 1 : 0) << 62);
}

__device__ inline unsigned long long ld_acquire64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

__device__ inline void st_release64(unsigned long long* p, unsigned long long v) {
  asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ inline void st_relaxed64(unsigned long long* p, unsigned long long v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ inline unsigned long long ld_relaxed64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

// The leader's publishing thread: the last one.  It is the update phase's
// fence thread: its warp has no isophote or row-maximum work there, so the
// fence it issues after the copy waits off the path, and the same fence
// makes its later publication of the next round a release.
constexpr int kPubThread = kEngThreads - 1;


// Bounded wait (thread 0) for a publication with an epoch other than `epoch`;
// returns it, or a stop word after setting *err on timeout.
__device__ inline unsigned long long wait_pub(TeamCtl* tc, unsigned epoch, int* err,
                                              unsigned long long limit) {
  unsigned long long v = ld_acquire64(&tc->pub);
  if ((unsigned)v != epoch) return v;
  const unsigned long long t0 = globaltimer();
  while (true) {
    v = ld_acquire64(&tc->pub);
    if ((unsigned)v != epoch) return v;
    if (globaltimer() - t0 > limit) {
      atomicExch(err, INPAINT_ERR_TIMEOUT);
      return pub_pack(epoch + 1u, 0, 0, true);
    }
  }
}

// A searcher's best key of a round travels to the leader tagged with the
// round: (SSD << 38) | (idx << 8) | tag, tag = epoch mod 128 (SSD < 2^26 for
// radius <= 8, idx < 2^30), so the leader polls the keys themselves and no
// separate arrival counter is needed.  Keys of one round carry the same tag,
// so the tagged values order like (SSD, idx).  Slots are set to all ones
// (tag 0xff, never a round's) before every launch.
__device__ inline unsigned long long key_tag(unsigned long long key, unsigned epoch) {
  if (key == ~0ull) return ~0ull & ~0xffull | (epoch & 0x7fu);
  return ((key >> 32) << 38) | ((key & 0x3fffffffull) << 8) | (epoch & 0x7fu);
}

__device__ inline unsigned long long key_untag(unsigned long long t) {
  const unsigned long long ssd = t >> 38, idx = (t >> 8) & 0x3fffffffull;
  if (ssd == 0x3ffffffull && idx == 0x3fffffffull) return ~0ull;
  return (ssd << 32) | idx;
}

// Leader: the best key of the round over the tagged slots [0, n), each
// polled (bounded) by one thread until it carries the round's tag; the
// untagged minimum lands in *out.  Returns false (every thread) when a
// slot did not arrive in time.  Whole block; ends with a __syncthreads.
__device__ inline bool gather_keys(const unsigned long long* slots, int n, unsigned epoch, int* err,
                                   unsigned long long limit, unsigned long long* red,
                                   unsigned long long* out) {
  // a key is a message of its own (the leader reads nothing else the
  // searchers write), so relaxed loads suffice; warp 0 polls up to eight
  // slots per lane at a time and reduces them, the other warps wait at the
  // one barrier
  if (threadIdx.x < 32) {
    constexpr int U = 8;
    const int lane = threadIdx.x;
    const unsigned tag = epoch & 0x7fu;
    unsigned long long best = ~0ull;
    bool late = false;
    const unsigned long long t0 = globaltimer();
    for (int b = 0; b < n && !late; b += 32 * U) {
      unsigned pending = 0u;
#pragma unroll
      for (int u = 0; u < U; ++u)
        if (b + lane + 32 * u < n) pending |= 1u << u;
      while (pending) {
        unsigned long long v[U];
#pragma unroll
        for (int u = 0; u < U; ++u) v[u] = (pending >> u) & 1u ? ld_relaxed64(&slots[b + lane + 32 * u]) : 0ull;
#pragma unroll
        for (int u = 0; u < U; ++u)
          if (((pending >> u) & 1u) && (v[u] & 0xffu) == tag) {
            const unsigned long long k = key_untag(v[u]);
            best = k < best ? k : best;
            pending &= ~(1u << u);
          }
        if (pending && globaltimer() - t0 > limit) {
          late = true;
          break;
        }
      }
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
      const unsigned long long ob = __shfl_xor_sync(0xffffffffu, best, o);
      best = ob < best ? ob : best;
    }
    late = __any_sync(0xffffffffu, late);
    if (lane == 0) {
      red[0] = late ? 1ull : 0ull;
      *out = best;
    }
  }
  __syncthreads();
  if (red[0] != 0ull) {
    if (threadIdx.x == 0) atomicExch(err, INPAINT_ERR_TIMEOUT);
    return false;
  }
  return true;
}

__device__ inline bool ctrl_active(const Ctrl* c) {
  return __ldcg(&c->status) == 0 && __ldcg(&c->remaining) > 0 &&
         __ldcg(&c->iter) < __ldcg(&c->iter_limit);
}

// Roles of a team on one image: CTAs [0, ns) search; the last CTA (the
// leader) runs the speculative phase of each iteration while they search,
// waits for them, applies the update and publishes the next round; any other
// CTA idles until the image is done.  A team of one CTA does all of it in
// sequence.
// Per-image part of the engine: the fill loop of image j for this CTA's
// team (roles below).  Called by k_engine (engine_multi.cu) through
// run_image_r<R>_s<SRW>, once per image of the team's list.
template <int R, int SRW, bool kLeadOnly = false>
__device__ __forceinline__ void run_image(const EngineArgs& ea, int j, EngCtx& x);

// The loop of a searching CTA in the tensor-core form (the image's state
// block, the stop flag and the first target are in shared memory), compiled
// as a function of its own with every phase inlined: a call would save and
// restore the caller's registers through local memory, which misses L1
// while shared memory takes nearly all of it.
template <int R>
__device__ __noinline__ void run_tc_search(const EngineArgs& ea, EngCtx& x, const TcTiles tt, TcArea tca, int ns) {
  using GT = TcEngGeom<R>;
  constexpr int P = GT::P, NSL = GT::NSL;
  // the context lives in the kernel's local memory, which misses L1 (shared
  // memory takes nearly all of it) and is re-read after every barrier or
  // fence: keep working copies in registers, write them back at the end
  uint8_t* const smem = x.smem;
  const uint32_t tmem = x.tmem;
  uint32_t tc_rows = x.tc_rows, tc_tiles = x.tc_tiles;
  int tc_pref = x.tc_pref, tc_nb = x.tc_nb;
  unsigned long long* const tpart = x.tpart;
  EngSmemTail& tl = *reinterpret_cast<EngSmemTail*>(smem);
  const ImgState& s = tl.img;
  Ctrl* c = s.ctrl;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int rank = x.rank;
  TeamCtl* tc = x.tc;
  const unsigned long long limit = ea.wait_limit_ns;
  unsigned epoch = x.epoch;
  // A | padded target | ring | validity bits
  uint8_t* area = smem + kHeadBytes;
  tca.a = area;
  tca.tpad = reinterpret_cast<uint16_t*>(area + GT::A_BYTES);
  tca.ring = area + GT::A_BYTES + GT::TPAD_BYTES;
  tca.bits = reinterpret_cast<uint32_t*>(tca.ring + (size_t)tca.nb * tca.slot);
  if (tc_nb != tca.nb) {
    // the ring's phases are counted from the slot sequence number modulo the
    // slot count: a new slot count restarts them (every slot of an earlier
    // image was consumed, so no barrier has a pending phase)
    if (tc_nb != 0 && tid == 0) {
      for (int i = 0; i < kTcRing; ++i) {
        mbar_inval(&tl.bars.tc_full[i]);
        mbar_inval(&tl.bars.tc_empty[i]);
        mbar_init(&tl.bars.tc_full[i], 1);
        mbar_init(&tl.bars.tc_empty[i], 2);
      }
    }
    fence_mbar_init();
    __syncthreads();
    tc_nb = tca.nb;
    tc_rows = 0;
  }
  const int ntiles = tt.ntx * tt.nty;
  const int first_y = s.cy0 + kTcRows * (rank / tt.ntx), first_tx = rank % tt.ntx;  // this CTA's first tile
  const int npre = min(tca.nb, NSL);
  int prev_px = -1000000, prev_py = -1000000;
  int round = 0;
  while (!tl.stop) {
    const int px = tl.px, py = tl.py;
    const bool first = round == 0;
    int bad = 0;
    // the producer starts the first tile's rows at once, unless it
    // prefetched them while the leader was updating
    if (tc_pref == 0 && warp == kEngWarps - 1 && lane == 0 &&
        !tc_produce<R>(s, tca, tl.bars, first_tx, first_y, tc_rows, 0, npre, limit))
      bad = 1;
    if (first) {
      tc_bits_init<R>(s, tt, tca.bits, tca.ntl, rank, ns);
      // the padded target table's columns outside the patch stay zero
      for (int e = tid; e < 4 * P * GT::TW; e += kEngThreads) tca.tpad[e] = 0;
      __syncthreads();
    }
    // target patch: warp dy reads row dy (lane = dx) and writes its
    // entries of the padded target table (R' G' B' and the known flag, zero
    // where unknown) and the row's share of A2
    for (int dy = warp; dy < P; dy += kEngWarps) {
      const int tx = px + lane - R, ty = py + dy - R;
      uint32_t w = 0;
      bool known = false;
      if (lane < P && tx >= 0 && tx < s.W && ty >= 0 && ty < s.H) {
        const uint8_t o = __ldcg(&s.omega[(size_t)ty * s.W + tx]);
        const uint32_t v = __ldcg(&s.img[(size_t)ty * s.pitch + tx]);
        known = o == 0;
        w = known ? v : 0u;
      }
      int sq = 0;
      if (lane < P) {
        const int d0 = known ? (int)(w & 255u) - 128 : 0, d1 = known ? (int)((w >> 8) & 255u) - 128 : 0,
                  d2 = known ? (int)((w >> 16) & 255u) - 128 : 0;
        sq = d0 * d0 + d1 * d1 + d2 * d2;
        uint16_t* tp = tca.tpad + dy * GT::TW + 8 + lane;
        tp[0] = (uint16_t)bf16_of_int(d0);
        tp[P * GT::TW] = (uint16_t)bf16_of_int(d1);
        tp[2 * P * GT::TW] = (uint16_t)bf16_of_int(d2);
        tp[3 * P * GT::TW] = (uint16_t)bf16_of_int(known ? 1 : 0);
      }
#pragma unroll
      for (int o = 16; o; o >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, o);
      if (lane == 0) tl.a2row[dy] = sq;
    }
    __syncthreads();
    // every warp but the producer's (its copies are in flight) writes A
    tc_build_a<R>(tca.a, tca.tpad, first, 32 * (kEngWarps - 1));
    __syncthreads();
    int a2 = 0;
#pragma unroll
    for (int dy = 0; dy < P; ++dy) a2 += tl.a2row[dy];
    unsigned long long best = ~0ull;
    for (int kt = 0; kt < tca.ntl; ++kt) {
      const int t = rank + kt * ns;
      if (t >= ntiles) break;  // uniform
      const int y0 = s.cy0 + kTcRows * (t / tt.ntx), xs = tt.xs0 + 8 * tt.N * (t % tt.ntx);
      const uint32_t g0 = tc_rows;
      if (warp == kEngWarps - 1) {
        if (lane == 0 && !tc_produce<R>(s, tca, tl.bars, t % tt.ntx, y0, g0, kt == 0 ? npre : 0, NSL, limit))
          bad = 1;
        __syncwarp();
      } else if (warp == kEngWarps - 2) {
        if (!(tt.N == 128 ? tc_issue<R, 0, 128>(tca, tl.bars, tmem, g0, limit)
                          : tc_issue<R, 0, 64>(tca, tl.bars, tmem, g0, limit)))
          bad = 1;
        // the one warp that waits for the tile's MMAs (the others sleep at
        // the block barrier: spinning warps would take issue slots from the
        // issuers)
        if (!mbar_wait(&tl.bars.tc_done, tc_tiles & 1u, limit)) bad = 1;
      } else if (warp == kEngWarps - 3) {
        if (!(tt.N == 128 ? tc_issue<R, 1, 128>(tca, tl.bars, tmem, g0, limit)
                          : tc_issue<R, 1, 64>(tca, tl.bars, tmem, g0, limit)))
          bad = 1;
      } else if (kt == 0 && !first) {
        // validity bits near the previous fill: needed only by the read-back
        tc_bits_refresh<R>(s, tt, tca.bits, rank, ns, prev_px, prev_py, 32 * (kEngWarps - 3));
      }
      tc_fence_before();
      if (__syncthreads_or(bad)) break;
      tc_fence_after();
      best = tc_epilogue<R>(s, tmem, tt.N, a2, tca.bits + kt * tc_bit_words(tt.N), y0, xs, best);
      tc_fence_before();
      ++tc_tiles;
      tc_rows += NSL;
      __syncthreads();  // the accumulators are read before the next tile's MMAs
    }
    tc_pref = 0;
    best = block_min_u64(best, tl.red64);
    ++round;
    if (bad && tid == 0) atomicExch(ea.err, INPAINT_ERR_TIMEOUT);
    if (tid == 0 && rank + 1 != ea.withhold) st_relaxed64(&tpart[rank], key_tag(best, epoch));
    if (rank == 0 && tid == 0) atomicAdd(&c->tc_rounds, 1);
    if (warp == kEngWarps - 1 && lane == 0) {
      // once the leader has written this round's fill, the next round's
      // first source rows are final: request them now, while the leader
      // updates (no prefetch if the next publication comes first)
      int n = 0;
      const unsigned long long t0 = globaltimer();
      while (true) {
        if ((int)(ld_acquire(&tc->copied) - (epoch + 1u)) >= 0) {
          asm volatile("fence.proxy.async.global;" ::: "memory");
          n = npre;
          if (!tc_produce<R>(s, tca, tl.bars, first_tx, first_y, tc_rows, 0, n, limit))
            atomicExch(ea.err, INPAINT_ERR_TIMEOUT);
          break;
        }
        if ((unsigned)ld_acquire64(&tc->pub) != epoch || globaltimer() - t0 > limit) break;
      }
      tl.tc_pref = n;
    }
    // wait for the next round
    if (tid == 0) {
      const unsigned long long v = wait_pub(tc, epoch, ea.err, limit);
      tl.stop = ((v >> 62) & 1ull) != 0;
      tl.px = (int)((v >> 32) & 0x7fff);
      tl.py = (int)((v >> 47) & 0x7fff);
    }
    ++epoch;
    prev_px = px;
    prev_py = py;
    __syncthreads();
    tc_pref = tl.tc_pref;
    if (lane == 0) asm volatile("fence.proxy.async.global;" ::: "memory");
  }
  if (tc_pref > 0) {
    // the loop stopped with a prefetch in flight: let it land and release
    // its slots (two arrivals stand for the two issuers' commits)
    if (warp == kEngWarps - 1 && lane == 0) {
      for (int h = 0; h < tc_pref; ++h) {
        const uint32_t g = tc_rows + (uint32_t)h;
        const int slot = (int)(g % (uint32_t)tca.nb);
        if (!mbar_wait(&tl.bars.tc_full[slot], (g / tca.nb) & 1u, limit)) atomicExch(ea.err, INPAINT_ERR_TIMEOUT);
        mbar_arrive(&tl.bars.tc_empty[slot]);
        mbar_arrive(&tl.bars.tc_empty[slot]);
      }
    }
    tc_rows += (uint32_t)tc_pref;
    tc_pref = 0;
    __syncthreads();
  }
  x.epoch = epoch;
  x.tc_rows = tc_rows;
  x.tc_tiles = tc_tiles;
  x.tc_pref = tc_pref;
  x.tc_nb = tc_nb;
}

// The loop of a leader that does not search, compiled as a function of its
// own: none of the search state is live through its phases, so its
// registers hold the update's working set.
template <int R, int SRW>
__device__ __noinline__ void run_lead_only(const EngineArgs& ea, int j, EngCtx& x) {
  run_image<R, SRW, true>(ea, j, x);
}

template <int R, int SRW, bool kLeadOnly>
__device__ __forceinline__ void run_image(const EngineArgs& ea, int j, EngCtx& x) {
  using G = EngGeom<R, SRW>;
  using RG = ResGeom<R>;
  constexpr int P = G::P, B = G::B;
  uint8_t* smem = x.smem;
  EngSmemTail& tl = *reinterpret_cast<EngSmemTail*>(smem);
  uint32_t* tgt = reinterpret_cast<uint32_t*>(smem + ((sizeof(EngSmemTail) + 15) & ~size_t(15)));
  uint32_t* rowd = tgt + P * G::TP;  // row descriptors of the target
  uint8_t* upd_base = smem + kHeadBytes;
  UpdSmem<R>& usm = *reinterpret_cast<UpdSmem<R>*>(upd_base);
  UpdCache<R>& uca = upd_cache_of<R>(upd_base);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int rank = x.rank, tsize = x.tsize;
  TeamCtl* tc = x.tc;
  unsigned long long* tpart = x.tpart;
  const unsigned long long t_start = x.t_start;  // (the context is in local memory)
  const unsigned long long limit = ea.wait_limit_ns;
  uint32_t ph0 = x.ph0, ph1 = x.ph1;
  unsigned epoch = x.epoch;

  // every role reads the image's fields from shared memory, which keeps
  // about forty registers free for its phases
  if constexpr (!kLeadOnly) {
    if (tid == 0) tl.img = ea.imgs[j];
    __syncthreads();
  }
  const ImgState& s = tl.img;
  const CUtensorMap* map = &ea.tmaps[2 * j];
  const CUtensorMap* cmap = &ea.tmaps[2 * j + 1];
  Ctrl* c = s.ctrl;
  const int xb = R + ((s.cx0 - R) & ~3);
  const int ncg = s.cx1 >= s.cx0 ? (s.cx1 - xb + G::BWC) / G::BWC : 0;
  const int nrb = s.cy1 >= s.cy0 ? (s.cy1 - s.cy0 + B) / B : 0;
  const int nbatch = ncg * nrb;
  // Roles: CTAs [0, ns) search, batch b going to CTA b mod ns (batches cost
  // alike).  The last CTA of the team is the leader: it runs the speculative
  // phase of each iteration while the others search, waits for their keys,
  // applies the update and publishes the next round.  When the image has
  // many batches per CTA (small teams in the batched form) the leader also
  // searches its share after the speculative phase, which is short next to
  // a CTA's share of such a search.  A CTA that neither searches nor leads
  // idles until the image is done.
  // Tensor-core form (an image given planes, a team of two or more): every
  // CTA but the leader searches whole tiles, when its A strips, a ring of
  // at least four source-row slots and the validity bits of its tiles fit.
  const TcTiles tt = s.planes ? tc_tiles(s) : TcTiles{0, 0, 0, 0};
  const int tc_ntiles = tt.ntx * tt.nty;
  TcArea tca{nullptr, nullptr, nullptr, nullptr, 0, 0, 0};
  bool tcmode = false;
  if (s.planes && ea.tc_cols >= 2 * tt.N && tsize >= 2 && tc_ntiles > 0) {
    const int nsq = min(tsize - 1, tc_ntiles);
    const int ntl = (tc_ntiles + nsq - 1) / nsq;
    const long long avail = (long long)(x.smem_end - (smem + kHeadBytes));
    const int slot = tc_slot(tt.N, R);
    const long long fixed =
        TcEngGeom<R>::A_BYTES + TcEngGeom<R>::TPAD_BYTES + (long long)ntl * tc_bit_words(tt.N) * 4;
    const long long nbl = (avail - fixed) / slot;
    if (ntl <= 8 && nbl >= 4) {
      tcmode = true;
      tca.nb = nbl < kTcRing ? (int)nbl : kTcRing;
      tca.ntl = ntl;
      tca.slot = slot;
    }
  }
  const bool lead_searches = !tcmode && (tsize == 1 || nbatch >= 8 * tsize);
  const int ns = tcmode ? min(tsize - 1, tc_ntiles) : lead_searches ? tsize : min(tsize - 1, nbatch);
  const bool leader = rank == tsize - 1;
  const bool searcher = rank < ns;
  if constexpr (!kLeadOnly) {
    if (leader && !searcher) {
      run_lead_only<R, SRW>(ea, j, x);
      return;
    }
    if (tcmode && searcher) {
      if (tid == 0) {
        tl.stop = !ctrl_active(c) || __ldcg(ea.err) != 0;
        tl.px = __ldcg(&c->px);
        tl.py = __ldcg(&c->py);
      }
      __syncthreads();
      run_tc_search<R>(ea, x, tt, tca, ns);
      return;
    }
  }
  // the CTA's work area (a searching leader keeps its update state below it)
  uint8_t* area = smem + kHeadBytes + (leader ? ((upd_smem_bytes<R>() + 127) / 128) * 128 : 0);
  // streaming mode: two count tiles and two tile slots (double buffer)
  uint32_t* cnt_t[2] = {reinterpret_cast<uint32_t*>(area),
                        reinterpret_cast<uint32_t*>(area + G::CNT_BYTES)};
  uint8_t* slots = area + 2 * G::CNT_BYTES;
  auto slot_pix = [&](int i) { return reinterpret_cast<uint32_t*>(slots + (size_t)i * G::SLOT_BYTES); };
  // resident mode when every searching CTA's tiles fit (the same decision
  // in every CTA of the team: the bound below depends only on the image,
  // the team and the smallest work area, a searching leader's)
  const int ncu = s.cx1 >= s.cx0 ? (s.cx1 - xb + kResCols) / kResCols : 0;
  const int nbands = s.cy1 >= s.cy0 ? (s.cy1 - s.cy0 + kResRows) / kResRows : 0;
  bool resident = false;
  {
    const long long U = (long long)ncu * nbands;
    const long long m = ns > 0 ? (U + ns - 1) / ns : 0;  // most units of one CTA
    const long long avail =
        (long long)(x.smem_end - (smem + kHeadBytes)) -
        (lead_searches ? ((long long)(upd_smem_bytes<R>() + 127) / 128) * 128 : 0);
    // two tiles (a range may straddle a band boundary) plus the bits; more
    // than one band of units per CTA streams instead
    const long long need = (long long)(kResRows + 2 * R) * 4 *
                               (m * kResCols + 2 * (2 * R + 8)) + 256 + m * 64;
    // at least half a unit per warp, else the batches of the streaming
    // mode spread the search over more warps
    resident = !tcmode && m >= kEngWarps / 2 && m <= ncu && need <= avail;
  }
  // large images: the leader publishes the next target as soon as the
  // window's priorities are known and updates its tile maxima afterwards
  const bool early_sel = (resident || tcmode) && !lead_searches;
  ResPlan& pl = tl.plan;
  if (resident && searcher) {
    if (tid == 0) res_plan<R>(pl, ncu, nbands, rank, ns);
    __syncthreads();
  }
  if (tid == 0) {
    tl.stop = !ctrl_active(c) || __ldcg(ea.err) != 0;
    tl.px = __ldcg(&c->px);
    tl.py = __ldcg(&c->py);
  }
  __syncthreads();
  int prev_px = -1000000, prev_py = -1000000;
  int round = 0;        // search rounds of this image in this launch
  bool staged = false;  // leader: neighbourhood of the next p^ already in shared memory

  // One search round for target (px, py): this CTA's batches; returns its
  // best key.  Whole block.
  auto search_round = [&](int px, int py) -> unsigned long long {
    const int b0 = rank < ns ? rank : nbatch;
    const int par = round & 1;
    // a batch's stage in streaming mode: its RGBA window and the validity
    // counts of its candidates, on one mbarrier
    auto issue = [&](int b, uint32_t* st, uint32_t* ct, uint64_t* bar) {
      const int gx = b % ncg, gy = b / ncg;
      // (the stage's previous generic reads are ordered before this by the
      // block barrier that ends every batch)
      mbar_expect_tx(bar, (uint32_t)(G::BW * G::BH * 4 + G::CW * B * 4));
      tma_load_2d(st, map, xb - R + G::BWC * gx, s.cy0 + B * gy - R, bar);
      tma_load_2d(ct, cmap, xb - G::COFF + G::BWC * gx, s.cy0 + B * gy, bar);
    };
    const bool first = round == 0;
    if (!resident && tid == 0 && b0 < nbatch) issue(b0, slot_pix(0), cnt_t[0], &tl.bars.full[0]);
    const uint8_t* tiles = area;
    if (resident && first) {
      // the source windows of every band segment (plain 16-byte loads;
      // outside the image: zero), then the validity bits of every unit
      for (int g = 0; g < pl.nseg; ++g) {
        const ResSeg sg = pl.seg[g];
        const int x0 = xb - R + sg.c_lo * kResCols, y0 = s.cy0 + sg.band * kResRows - R;
        const int nq = sg.pitch / 4;
        uint4* dst = reinterpret_cast<uint4*>(area + sg.off);
        for (int i = tid; i < RG::TH * nq; i += kEngThreads) {
          const int row = i / nq, q = i - row * nq, y = y0 + row, xw = x0 + 4 * q;
          uint4 v = make_uint4(0u, 0u, 0u, 0u);
          if (y >= 0 && y < s.H && xw + 3 < s.pitch)
            v = __ldcg(reinterpret_cast<const uint4*>(s.img + (size_t)y * s.pitch + xw));
          dst[i] = v;
        }
      }
      uint16_t* bits = reinterpret_cast<uint16_t*>(area + pl.bits_off);
      for (int jj = warp; jj < pl.u1 - pl.u0; jj += kEngWarps) {
        const int u = pl.u0 + jj, band = u / ncu, col = u - band * ncu;
        const int qy = s.cy0 + band * kResRows + lane, qx0 = xb + col * kResCols;
        uint32_t v = 0;
        if (qy <= s.cy1) {
#pragma unroll
          for (int k = 0; k < kResCols; ++k) {
            const int qx = qx0 + k;
            if (qx >= s.cx0 && qx <= s.cx1 && __ldcg(&s.count[(size_t)qy * s.pitch + qx]) == 0) v |= 1u << k;
          }
        }
        bits[jj * 32 + lane] = (uint16_t)v;
      }
    } else if (resident && pl.u1 > pl.u0) {
      // the previous target's filled pixels (its unknown in-image pixels),
      // copied by the leader before the publication, into every tile that
      // holds them
      const uint8_t* kprev = tl.known[par ^ 1];
      if (tid < P * P) {
        const int tx = prev_px + tid % P - R, ty = prev_py + tid / P - R;
        if (tx >= 0 && tx < s.W && ty >= 0 && ty < s.H && !kprev[tid]) {
          const uint32_t w = __ldcg(&s.img[(size_t)ty * s.pitch + tx]);
          for (int g = 0; g < pl.nseg; ++g) {
            const ResSeg& sg = pl.seg[g];
            const int lx = tx - (xb - R + sg.c_lo * kResCols), ly = ty - (s.cy0 + sg.band * kResRows - R);
            if (lx >= 0 && lx < sg.pitch && ly >= 0 && ly < RG::TH)
              reinterpret_cast<uint32_t*>(area + sg.off)[ly * sg.pitch + lx] = w;
          }
        }
      }
      // candidates within 2R of the previous target may have become valid
      constexpr int NCW = 4 * R + 1;
      for (int jj = tid; jj < NCW * NCW; jj += kEngThreads) {
        const int qx = prev_px + jj % NCW - 2 * R, qy = prev_py + jj / NCW - 2 * R;
        if (qx < s.cx0 || qx > s.cx1 || qy < s.cy0 || qy > s.cy1) continue;
        const int band = (qy - s.cy0) / kResRows, col = (qx - xb) / kResCols;
        const int u = band * ncu + col;
        if (u < pl.u0 || u >= pl.u1) continue;
        if (__ldcg(&s.count[(size_t)qy * s.pitch + qx]) != 0) continue;
        const int e = (u - pl.u0) * 32 + (qy - s.cy0) % kResRows;
        atomicOr(reinterpret_cast<unsigned*>(area + pl.bits_off) + (e >> 1),
                 (1u << ((qx - xb) % kResCols)) << (16 * (e & 1)));
      }
    }
    // target patch: warp dy reads row dy (lane = dx); the ballot of the
    // known flags gives the row descriptor
    {
      uint8_t* kn = tl.known[par];
      for (int dy = warp; dy < P; dy += kEngWarps) {
        const int tx = px + lane - R, ty = py + dy - R;
        uint32_t w = 0;
        bool known = false;
        if (lane < P && tx >= 0 && tx < s.W && ty >= 0 && ty < s.H) {
          // both reads in flight together; the pixel is kept only if known
          const uint8_t o = __ldcg(&s.omega[(size_t)ty * s.W + tx]);
          const uint32_t v = __ldcg(&s.img[(size_t)ty * s.pitch + tx]);
          known = o == 0;
          w = known ? v : 0u;
        }
        const unsigned bal = __ballot_sync(0xffffffffu, known);
        if (lane < P) {
          tgt[dy * G::TP + lane] = w;
          kn[dy * P + lane] = (uint8_t)known;
        }
        if (lane == 0) rowd[dy] = row_desc(bal & G::FULL, P);
      }
    }
    __syncthreads();
    unsigned long long best = ~0ull;
    bool ok = true;
    if (resident) {
      if (pl.u1 > pl.u0) best = resident_units16<R>(&pl, tiles, xb, s.cy0, s.W, tgt, rowd);
    } else {
      int cur = 0;
      for (int b = b0; b < nbatch; b += ns) {
        const int nb = b + ns;
        if (tid == 0 && nb < nbatch) issue(nb, slot_pix(cur ^ 1), cnt_t[cur ^ 1], &tl.bars.full[cur ^ 1]);
        const int gx = b % ncg, gy = b / ncg;
        const bool got = mbar_wait(&tl.bars.full[cur], cur ? ph1 : ph0, limit);
        if (cur) ph1 ^= 1; else ph0 ^= 1;
        // validity of this lane's candidates from the count tile (16-byte
        // aligned chunk) and the search rectangle
        uint32_t cw[G::NCL + 4];
        lds_words(cw, cnt_t[cur] + lane * G::CW + G::NCL * warp);
        const int qy = s.cy0 + B * gy + lane, qx0 = xb + G::BWC * gx + G::NCL * warp;
        uint32_t bits = 0;
#pragma unroll
        for (int k = 0; k < G::NCL; ++k) {
          const int qx = qx0 + k;
          if (qx >= s.cx0 && qx <= s.cx1 && qy <= s.cy1 && cw[G::COFF + k] == 0) bits |= 1u << k;
        }
        const unsigned long long kb = unit_best<R, SRW>(slot_pix(cur) + lane * G::BW + G::NCL * warp, tgt, rowd,
                                                        bits, (unsigned)(qy * s.W + qx0));
        best = kb < best ? kb : best;
        if (__syncthreads_or(!got)) {  // a bounded wait gave up: stop uniformly
          ok = false;
          if (nb < nbatch) {
            mbar_wait(&tl.bars.full[cur ^ 1], cur ? ph0 : ph1, limit);
            if (cur) ph0 ^= 1; else ph1 ^= 1;
          }
          break;
        }
        cur ^= 1;
      }
    }
    ++round;
    if (!ok && tid == 0) atomicExch(ea.err, INPAINT_ERR_TIMEOUT);
    return block_min_u64(best, tl.red64);
  };

  // One iteration of the leader for target (px, py): speculative phase (and
  // its own search share when it searches), the searchers' keys, update,
  // publication of the next round, bookkeeping.  Whole block.
  auto lead_round = [&](int px, int py, bool searches) {
    const unsigned long long t_a = globaltimer();
    spec_phase<R>(s, usm, uca, staged, early_sel);
    if (tid == 32) {
      // the stop decision's inputs that other CTAs may change, read by a
      // thread outside the warp that gathers the keys; everything the update
      // reads stays in shared memory (no local-memory state: it would miss
      // L1, which the shared memory leaves nearly empty)
      tl.status = __ldcg(&c->status);
      tl.err = __ldcg(ea.err);
      tl.allow = usm.spec_iter + 1 < tl.lim && tl.status == 0 && tl.err == 0;
      tl.es.pub = early_sel ? &tc->pub : nullptr;
      tl.es.epoch = epoch;
      tl.es.allow = tl.allow != 0;
      tl.es.tick_ns = ea.tick_ns;
      tl.es.t_start = t_start;
      tl.es.expired = &tc->expired;
      tl.es.pub_thread = kPubThread;
      tl.es.published = false;
    }
    if constexpr (!kLeadOnly) {
      if (searches) {
        const unsigned long long best = search_round(px, py);
        if (tid == 0) st_relaxed64(&tpart[rank], key_tag(best, epoch));
      }
    }
    tl.flag = gather_keys(tpart, ns, epoch, ea.err, limit, tl.red64, &tl.key);
    bool stop = true, ok = false;
    int npx = 0, npy = 0;
    unsigned long long t_b = 0ull;
    if (tl.flag) {
      t_b = globaltimer();
      ok = update_phase<R>(s, nullptr, 0, usm, uca, kPubThread, false, &tl.key, &tl.es,
                           tcmode ? &tc->copied : nullptr, epoch + 1u, &tl.snap);  // ends with a __syncthreads
      if (ok && tl.es.published) {
        // the next round (or the stop) went out inside the update phase
        if (tid == 0) tl.stop = usm.early_stop;
        npx = usm.next_idx % s.W;
        npy = usm.next_idx / s.W;
      } else if (ok) {
        // the next target is known: publish it before the bookkeeping.
        // Thread 0 decides (the inputs are global and may change under
        // other threads' feet) and the barrier below shares the decision.
        if (tid == 0) {
          bool st = usm.remaining <= 0 || usm.next_key == 0ull || usm.it + 1 >= tl.lim || tl.status != 0 ||
                    tl.err != 0;
          if (!st && ea.tick_ns && globaltimer() - t_start > ea.tick_ns) {
            st = true;  // the launch's time budget is spent: resume in the next launch
            tc->expired = 1u;
          }
          tl.stop = st;
        }
        npx = usm.next_idx % s.W;
        npy = usm.next_idx / s.W;
      }
    }
    __syncthreads();
    stop = ok ? tl.stop != 0 : true;
    // publication: the update phase's fence (same thread) already ordered
    // every write the searchers read before this store; without an update
    // (timeout or error) the store carries its own release
    if (tid == kPubThread && !(ok && tl.es.published)) {
      if (ok)
        st_relaxed64(&tc->pub, pub_pack(epoch + 1u, npx, npy, stop));
      else
        st_release64(&tc->pub, pub_pack(epoch + 1u, npx, npy, stop));
    }
    if (tid == 0) {
      tl.stop = stop;
      tl.px = npx;
      tl.py = npy;
    }
    staged = ok && !stop;
    if (staged) stage_next<R>(s, npx, npy, usm, &tl.snap.conf);  // next speculative phase's input
    if (ok) {
      update_finish<R>(s, usm, staged, false, &tl.snap);  // and the next round's snapshot
      if (tid == 0) {
        atomicAdd(&c->t_search, t_b - t_a);
        atomicAdd(&c->t_update, globaltimer() - t_b);
        atomicAdd(&c->timed_iters, 1);
      }
    }
    ++epoch;
    prev_px = px;
    prev_py = py;
    __syncthreads();
    if (lane == 0) asm volatile("fence.proxy.async.global;" ::: "memory");
  };

  if (leader) stage_dterm<R>(usm);  // (the first speculative phase's barriers publish it)
  if (leader && tid == 0) {
    // the leader's snapshot of the control block; update_finish keeps it
    // current from here on
    tl.snap.px = __ldcg(&c->px);
    tl.snap.py = __ldcg(&c->py);
    tl.snap.conf = __ldcg(&c->conf);
    tl.snap.prio = __ldcg(&c->prio);
    tl.snap.n_cand = __ldcg(&c->n_valid);
    tl.snap.it = __ldcg(&c->iter);
    tl.snap.remaining = __ldcg(&c->remaining);
    tl.lim = __ldcg(&c->iter_limit);
  }
  if constexpr (kLeadOnly) {
    if (tid == 0) usm.tiles_pending = 0;
    __syncthreads();
    while (!tl.stop) lead_round(tl.px, tl.py, false);
    // the last update's tile maxima, deferred by the early selection
    if (usm.tiles_pending) update_tiles<R>(s, usm, uca, 0);
    x.epoch = epoch;
    return;
  }
  while (!tl.stop) {
    const int px = tl.px, py = tl.py;
    if (leader) {
      lead_round(px, py, true);
      continue;
    }
    if (searcher) {
      const unsigned long long best = search_round(px, py);
      if (tid == 0 && rank + 1 != ea.withhold) st_relaxed64(&tpart[rank], key_tag(best, epoch));
    }
    // searchers and idle CTAs: wait for the next round
    if (tid == 0) {
      const unsigned long long v = wait_pub(tc, epoch, ea.err, limit);
      tl.stop = ((v >> 62) & 1ull) != 0;
      tl.px = (int)((v >> 32) & 0x7fff);
      tl.py = (int)((v >> 47) & 0x7fff);
    }
    ++epoch;
    prev_px = px;
    prev_py = py;
    __syncthreads();
    if (lane == 0) asm volatile("fence.proxy.async.global;" ::: "memory");
  }
  x.ph0 = ph0;
  x.ph1 = ph1;
  x.epoch = epoch;
}

// Shared-memory bytes the engine needs for radius R and SRW rows per warp.
template <int R, int SRW>
constexpr size_t engine_smem_for() {
  return eng_smem_bytes<R, SRW>();
}

}  // namespace inp


namespace inp {

// Single-CTA copy/update kernel of the graph-driven loop for R <= 8 (the same
// update phase the engine runs in its last-arriving CTA).
template <int R>
__global__ void __launch_bounds__(kEngThreads) k_update_fast(ImgState s, cudaGraphConditionalHandle cond,
                                                            int use_cond) {
  extern __shared__ __align__(128) uint8_t sm_raw[];
  UpdSmem<R>& usm = *reinterpret_cast<UpdSmem<R>*>(sm_raw);
  UpdCache<R>& uca = upd_cache_of<R>(sm_raw);
  if (!loop_active(s.ctrl)) {
    if (use_cond && threadIdx.x == 0) cudaGraphSetConditional(cond, 0);
    return;
  }
  stage_dterm<R>(usm);  // (spec_phase's barriers publish it)
  spec_phase<R>(s, usm, uca, false);
  const bool ok = update_phase<R>(s, s.partial, s.n_partial, usm, uca, -1, s.overlap != 0);
  if (ok) update_finish<R>(s, usm, false, s.overlap != 0);
  if (use_cond && threadIdx.x == 0) cudaGraphSetConditional(cond, ok && loop_active(s.ctrl) ? 1u : 0u);
}

template <int R>
static cudaError_t upd_fast_t(const ImgState& s, unsigned long long cond, int use_cond, cudaStream_t st) {
  const size_t smem = upd_smem_bytes<R>();
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

// Host entry points of one radius R, exported through EngineFns.
template <int R>
static size_t eng_smem_r(int srw) {
  return srw == 2 ? engine_smem_for<R, 2>() : engine_smem_for<R, 1>();
}
template <int R>
const EngineFns* engine_fns_for() {
  static const EngineFns f = {eng_smem_r<R>, upd_fast_t<R>, prio_init_t<R>};
  return &f;
}

}  // namespace inp
