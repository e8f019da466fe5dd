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
#include <type_traits>
#include <cuda.h>

#include "inpaint_engine.h"
#include "ptx.cuh"
#include "update_fast.cuh"

namespace inp {

// ---------------------------------------------------------------- search batch

template <int R, int SRW>
struct EngGeom {
  static constexpr int P = 2 * R + 1;
  static constexpr int BW = (128 + 2 * R + 3) & ~3;  // staged width (words)
  static constexpr int B = kEngWarps * SRW;          // candidate rows per batch
  static constexpr int BH = B + 2 * R;               // staged rows
  static constexpr int PIX_BYTES = ((BW * BH * 4 + 127) / 128) * 128;
  static constexpr int CNT_BYTES = ((kEngCountW * B * 4 + 127) / 128) * 128;
  static constexpr int STAGE_BYTES = PIX_BYTES + CNT_BYTES;  // pixel tile | count tile
  static constexpr int COFF = R & 3;  // first candidate column within the count tile
  static constexpr int NROW = (4 + P - 1 + 3) & ~3;  // strip words per lane
  static constexpr int TP = (P + 3) & ~3;            // padded target row (words)
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
#pragma unroll
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
      uint32_t t[G::TP];
      const uint4* tp = reinterpret_cast<const uint4*>(tgt + dy * G::TP);
#pragma unroll
      for (int i = 0; i < G::TP / 4; ++i) {
        const uint4 v = tp[i];
        t[4 * i] = v.x;
        t[4 * i + 1] = v.y;
        t[4 * i + 2] = v.z;
        t[4 * i + 3] = v.w;
      }
      if (m == G::FULL) {
#pragma unroll
        for (int dx = 0; dx < P; ++dx) {
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            const uint32_t d = __vabsdiffu4(t[dx], row[k + dx]);
            acc[o][k] = __dp4a(d, d, acc[o][k]);
          }
        }
      } else {
#pragma unroll
        for (int dx = 0; dx < P; ++dx) {
          if (m & (1u << dx)) {
#pragma unroll
            for (int k = 0; k < 4; ++k) {
              const uint32_t d = __vabsdiffu4(t[dx], row[k + dx]);
              acc[o][k] = __dp4a(d, d, acc[o][k]);
            }
          }
        }
      }
    }
  }
}

// Two-row batches (SRW = 2): half-warps take two adjacent candidate rows and
// each lane eight adjacent candidates (columns (lane & 15) * 8 ...), so both
// half-warps use the same target row at a time: the row-mask branch stays
// warp-uniform and costs half as much per evaluation as with four candidates.
// SSD terms of target columns dx in [D0, D0 + L) for eight candidates, no
// per-column test (a contiguous run of known target pixels).
template <int R, int D0, int L, int TP, int N8>
__device__ __forceinline__ void ssd_run8(const uint32_t (&t)[TP], const uint32_t (&r)[N8],
                                         uint32_t (&acc)[16]) {
  // even and odd columns go to separate accumulators: twice the independent
  // dot-product chains per lane
#pragma unroll
  for (int dx = D0; dx < D0 + L; ++dx)
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const uint32_t d = __vabsdiffu4(t[dx], r[k + dx]);
      acc[(dx & 1) * 8 + k] = __dp4a(d, d, acc[(dx & 1) * 8 + k]);
    }
}

template <int R>
__device__ inline void compute_rows8(const uint32_t* __restrict__ stage, int row, int col,
                                     const uint32_t* __restrict__ tgt,
                                     const uint32_t* __restrict__ rowmask, uint32_t (&acc)[8]) {
  using G = EngGeom<R, 2>;
  constexpr int P = G::P, BW = G::BW, N8 = (8 + P - 1 + 3) & ~3;
  static_assert(15 * 8 + N8 <= BW, "row strip must stay inside the tile");
  uint32_t acc2[16];
#pragma unroll
  for (int k = 0; k < 16; ++k) acc2[k] = 0;
#pragma unroll 1
  for (int dy = 0; dy < P; ++dy) {
    const uint32_t m = rowmask[dy];
    if (m == 0) continue;
    uint32_t r[N8];
    const uint4* sp = reinterpret_cast<const uint4*>(stage + (row + dy) * BW + col);
#pragma unroll
    for (int i = 0; i < N8 / 4; ++i) {
      const uint4 v = sp[i];
      r[4 * i] = v.x;
      r[4 * i + 1] = v.y;
      r[4 * i + 2] = v.z;
      r[4 * i + 3] = v.w;
    }
    uint32_t t[G::TP];
    const uint4* tp = reinterpret_cast<const uint4*>(tgt + dy * G::TP);
#pragma unroll
    for (int i = 0; i < G::TP / 4; ++i) {
      const uint4 v = tp[i];
      t[4 * i] = v.x;
      t[4 * i + 1] = v.y;
      t[4 * i + 2] = v.z;
      t[4 * i + 3] = v.w;
    }
    const uint32_t um = ~m & G::FULL;  // unknown columns of the row
    if (m == G::FULL) {
      ssd_run8<R, 0, P>(t, r, acc2);
    } else if ((m & (m + 1)) == 0 || (um & (um + 1)) == 0) {
      // the known columns are one run at the start or at the end of the row
      // (the usual shape next to the fill front): straight-line code
      const bool at_end = (m & 1u) == 0;
      switch (__popc(m)) {
#define INP_RUN8(n)                                             \
  case n:                                                       \
    if constexpr (n < P) {                                      \
      if (at_end) ssd_run8<R, P - n, n>(t, r, acc2);            \
      else ssd_run8<R, 0, n>(t, r, acc2);                       \
    }                                                           \
    break;
        INP_RUN8(1) INP_RUN8(2) INP_RUN8(3) INP_RUN8(4) INP_RUN8(5) INP_RUN8(6) INP_RUN8(7)
        INP_RUN8(8) INP_RUN8(9) INP_RUN8(10) INP_RUN8(11) INP_RUN8(12) INP_RUN8(13) INP_RUN8(14)
        INP_RUN8(15) INP_RUN8(16)
#undef INP_RUN8
        default:
          break;
      }
    } else {
#pragma unroll
      for (int dx = 0; dx < P; ++dx) {
        if (m & (1u << dx)) {
#pragma unroll
          for (int k = 0; k < 8; ++k) {
            const uint32_t d = __vabsdiffu4(t[dx], r[k + dx]);
            acc2[(dx & 1) * 8 + k] = __dp4a(d, d, acc2[(dx & 1) * 8 + k]);
          }
        }
      }
    }
  }
#pragma unroll
  for (int k = 0; k < 8; ++k) acc[k] = acc2[k] + acc2[8 + k];
}

// ---------------------------------------------------------------- kernel

struct EngSmemTail {
  uint64_t full[2];  // TMA completion barriers of the two stages
  ImgState img;      // the image's state block (a leader that does not search reads it here)
  unsigned long long red64[32];
  int red32[32];
  int flag;
  int stop;
  int px, py;
  uint8_t known[17 * 17];
};

constexpr int kTgtWords = 17 * 20 + 17 + 3;  // padded target rows + row masks (R <= 8)
constexpr size_t kHeadBytes = ((((sizeof(EngSmemTail) + 15) & ~size_t(15)) + kTgtWords * 4 + 127) / 128) * 128;

// Shared memory of an engine CTA: head | two search stages | update state |
// update cache (the leader keeps its speculative state while it searches).
template <int R>
__host__ __device__ constexpr size_t upd_smem_bytes() {
  return ((sizeof(UpdSmem<R>) + 127) / 128) * 128 + sizeof(UpdCache<R>);
}

template <int R, int SRW>
__host__ __device__ constexpr size_t eng_smem_bytes() {
  using G = EngGeom<R, SRW>;
  return kHeadBytes + (size_t)2 * G::STAGE_BYTES + upd_smem_bytes<R>() + 128;
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

// The leader's publishing thread: the last one, in a warp with no level-0
// tile to scan in most iterations, so that its fence waits off the path.
constexpr int kPubThread = kEngThreads - 1;

__device__ inline void red_release_add(unsigned* p, unsigned v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Bounded wait (thread 0) for a publication with an epoch other than `epoch`;
// returns it, or a stop word after setting *err on timeout.
__device__ inline unsigned long long wait_pub(TeamCtl* tc, unsigned epoch, int* err,
                                              unsigned long long limit) {
  unsigned long long v = ld_acquire64(&tc->pub);
  if ((unsigned)v != epoch) return v;
  const unsigned long long t0 = globaltimer();
  while (true) {
    __nanosleep(20);
    v = ld_acquire64(&tc->pub);
    if ((unsigned)v != epoch) return v;
    if (globaltimer() - t0 > limit) {
      atomicExch(err, INPAINT_ERR_TIMEOUT);
      return pub_pack(epoch + 1u, 0, 0, true);
    }
  }
}

// Bounded wait (thread 0) until `n` searchers arrived; false on timeout.
__device__ inline bool wait_arrivals(TeamCtl* tc, unsigned n, int* err, unsigned long long limit) {
  if (ld_acquire(&tc->arrive) >= n) return true;
  const unsigned long long t0 = globaltimer();
  while (ld_acquire(&tc->arrive) < n) {
    if (globaltimer() - t0 > limit) {
      atomicExch(err, INPAINT_ERR_TIMEOUT);
      return false;
    }
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
  constexpr int P = G::P, B = G::B;
  uint8_t* smem = x.smem;
  EngSmemTail& tl = *reinterpret_cast<EngSmemTail*>(smem);
  uint32_t* tgt = reinterpret_cast<uint32_t*>(smem + ((sizeof(EngSmemTail) + 15) & ~size_t(15)));
  uint32_t* rowmask = tgt + P * G::TP;
  uint8_t* big = smem + kHeadBytes;
  uint32_t* stage0 = reinterpret_cast<uint32_t*>(big);
  uint32_t* stage1 = reinterpret_cast<uint32_t*>(big + G::STAGE_BYTES);
  UpdSmem<R>& usm = *reinterpret_cast<UpdSmem<R>*>(big + 2 * G::STAGE_BYTES);
  UpdCache<R>& uca = upd_cache_of<R>(big + 2 * G::STAGE_BYTES);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int rank = x.rank, tsize = x.tsize;
  TeamCtl* tc = x.tc;
  unsigned long long* tpart = x.tpart;
  const unsigned long long limit = ea.wait_limit_ns;
  uint32_t ph0 = x.ph0, ph1 = x.ph1;
  unsigned epoch = x.epoch;

  // a leader that does not search reads the image's fields from shared
  // memory, which keeps about forty registers free for its phases
  if constexpr (kLeadOnly) {
    if (tid == 0) tl.img = ea.imgs[j];
    __syncthreads();
  }
  std::conditional_t<kLeadOnly, const ImgState&, const ImgState> s = kLeadOnly ? tl.img : ea.imgs[j];
  const CUtensorMap* map = &ea.tmaps[2 * j];
  const CUtensorMap* cmap = &ea.tmaps[2 * j + 1];
  Ctrl* c = s.ctrl;
  const int xb = R + ((s.cx0 - R) & ~3);
  const int ncg = s.cx1 >= s.cx0 ? (s.cx1 - xb + 128) / 128 : 0;
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
  const bool lead_searches = tsize == 1 || nbatch >= 8 * tsize;
  const int ns = lead_searches ? tsize : min(tsize - 1, nbatch);
  const bool leader = rank == tsize - 1;
  const bool searcher = rank < ns;
  const unsigned n_wait = (unsigned)(lead_searches ? ns - 1 : ns);
  if constexpr (!kLeadOnly) {
    if (leader && !searcher) {
      run_lead_only<R, SRW>(ea, j, x);
      return;
    }
  }
  bool resident = false;  // stage0 holds this CTA's only batch of the image
  if (tid == 0) {
    tl.stop = !ctrl_active(c) || __ldcg(ea.err) != 0;
    tl.px = __ldcg(&c->px);
    tl.py = __ldcg(&c->py);
  }
  __syncthreads();
  int prev_px = -1000000, prev_py = -1000000;
  bool staged = false;  // leader: neighbourhood of the next p^ already in shared memory

  // One search round for target (px, py): this CTA's batches; returns its
  // best key.  Whole block.
  auto search_round = [&](int px, int py) -> unsigned long long {
    const int b0 = rank < ns ? rank : nbatch;
    const bool need0 = !resident ||
                       (abs(prev_px - (xb + 128 * (b0 % max(ncg, 1)) + 64)) <= 64 + 2 * R + 4 &&
                        abs(prev_py - (s.cy0 + B * (b0 / max(ncg, 1)) + B / 2)) <= B / 2 + 2 * R + 1);
    // a batch's stage: its RGBA window (unless still resident) and the
    // validity counts of its candidates, on one mbarrier
    auto issue = [&](int b, uint32_t* st, uint64_t* bar, bool pixels) {
      const int gx = b % ncg, gy = b / ncg;
      // (the stage's previous generic reads are ordered before this by the
      // block barrier that ends every batch)
      mbar_expect_tx(bar, (uint32_t)((pixels ? G::BW * G::BH * 4 : 0) + kEngCountW * B * 4));
      if (pixels) tma_load_2d(st, map, xb - R + 128 * gx, s.cy0 + B * gy - R, bar);
      tma_load_2d(reinterpret_cast<uint8_t*>(st) + G::PIX_BYTES, cmap, xb - G::COFF + 128 * gx,
                  s.cy0 + B * gy, bar);
    };
    if (tid == 0 && b0 < nbatch) issue(b0, stage0, &tl.full[0], need0);
    // target patch: one thread per pixel, then the row masks
    if (tid < P * P) {
      const int tx = px + tid % P - R, ty = py + tid / P - R;
      uint32_t w = 0;
      int known = 0;
      if (tx >= 0 && tx < s.W && ty >= 0 && ty < s.H) {
        // both reads in flight together; the pixel is kept only if known
        const uint8_t o = __ldcg(&s.omega[(size_t)ty * s.W + tx]);
        const uint32_t v = __ldcg(&s.img[(size_t)ty * s.pitch + tx]);
        known = o == 0;
        w = known ? v : 0u;
      }
      tgt[(tid / P) * G::TP + tid % P] = w;
      tl.known[tid] = (uint8_t)known;
    }
    __syncthreads();
    if (tid < P) {
      uint32_t m = 0;
      for (int dx = 0; dx < P; ++dx) m |= (uint32_t)tl.known[tid * P + dx] << dx;
      rowmask[tid] = m;
    }
    __syncthreads();
    unsigned long long best = ~0ull;
    int cur = 0;
    bool ok = true;
    int nproc = 0;
    for (int b = b0; b < nbatch; b += ns) {
      const int nb = b + ns;
      if (tid == 0 && nb < nbatch) issue(nb, cur ? stage0 : stage1, &tl.full[cur ^ 1], true);
      const int gx = b % ncg, gy = b / ncg;
      const int qx0 = xb + 128 * gx + lane * 4, qy0 = s.cy0 + B * gy + warp * SRW;
      const bool got = mbar_wait(&tl.full[cur], cur ? ph1 : ph0, limit);
      if (cur) ph1 ^= 1; else ph0 ^= 1;
      const uint32_t* stg = cur ? stage1 : stage0;
      const int* cst = reinterpret_cast<const int*>(reinterpret_cast<const uint8_t*>(stg) + G::PIX_BYTES);
      if constexpr (SRW == 2) {
        // lane: candidate row warp*2 + lane/16, columns (lane & 15)*8 + [0, 8)
        const int lrow = warp * 2 + (lane >> 4), lcol = (lane & 15) * 8;
        uint32_t acc[8];
        compute_rows8<R>(stg, lrow, lcol, tgt, rowmask, acc);
        const int qy = s.cy0 + B * gy + lrow;
        int cw[12];  // counts of this lane's candidates (vector loads, 16-byte aligned)
        const int4* cp4 = reinterpret_cast<const int4*>(cst + lrow * kEngCountW + lcol);
#pragma unroll
        for (int i = 0; i < 3; ++i) {
          const int4 v = cp4[i];
          cw[4 * i] = v.x;
          cw[4 * i + 1] = v.y;
          cw[4 * i + 2] = v.z;
          cw[4 * i + 3] = v.w;
        }
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          const int qx = xb + 128 * gx + lcol + k;
          const bool in = qx >= s.cx0 && qx <= s.cx1 && qy <= s.cy1;
          if (in && cw[G::COFF + k] == 0) {
            const unsigned idx = (unsigned)(qy * s.W + qx);
            const unsigned long long key = ((unsigned long long)acc[k] << 32) | idx;
            best = key < best ? key : best;
          }
        }
      } else {
        uint32_t acc[SRW][4];
        compute_rows<R, SRW>(stg, warp * SRW, tgt, rowmask, acc);
#pragma unroll
        for (int o = 0; o < SRW; ++o) {
          int cw[8];  // counts of this lane's candidates (vector loads, 16-byte aligned)
          const int4* cp4 = reinterpret_cast<const int4*>(cst + (warp * SRW + o) * kEngCountW + lane * 4);
          const int4 v0 = cp4[0], v1 = cp4[1];
          cw[0] = v0.x; cw[1] = v0.y; cw[2] = v0.z; cw[3] = v0.w;
          cw[4] = v1.x; cw[5] = v1.y; cw[6] = v1.z; cw[7] = v1.w;
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            const int qx = qx0 + k, qy = qy0 + o;
            const bool in = qx >= s.cx0 && qx <= s.cx1 && qy <= s.cy1;
            if (in && cw[G::COFF + k] == 0) {
              const unsigned idx = (unsigned)(qy * s.W + qx);
              const unsigned long long key = ((unsigned long long)acc[o][k] << 32) | idx;
              best = key < best ? key : best;
            }
          }
        }
      }
      ++nproc;
      if (__syncthreads_or(!got)) {  // a bounded wait gave up: stop uniformly
        ok = false;
        if (nb < nbatch) {
          mbar_wait(&tl.full[cur ^ 1], cur ? ph0 : ph1, limit);
          if (cur) ph0 ^= 1; else ph1 ^= 1;
        }
        break;
      }
      cur ^= 1;
    }
    // the tile stays resident when it was this CTA's only batch (the leader's
    // shared memory is reused by its update phase)
    resident = ok && !leader && b0 < nbatch && nproc == 1;
    if (!ok && tid == 0) atomicExch(ea.err, INPAINT_ERR_TIMEOUT);
    return block_min_u64(best, tl.red64);
  };

  // One iteration of the leader for target (px, py): speculative phase (and
  // its own search share when it searches), the searchers' keys, update,
  // publication of the next round, bookkeeping.  Whole block.
  auto lead_round = [&](int px, int py, bool searches) {
    const unsigned long long t_a = globaltimer();
    // the stop decision's global inputs, read now so that their latency
    // hides behind the phases (a stop seen here ends the loop one iteration
    // later at most)
    int lim = 0, status = 0, err = 0;
    if (tid == 0) {
      lim = __ldcg(&c->iter_limit);
      status = __ldcg(&c->status);
      err = __ldcg(ea.err);
    }
    spec_phase<R>(s, usm, uca, staged);
    if (searches) {
      const unsigned long long best = search_round(px, py);
      if (tid == 0) tpart[rank] = best;
    }
    if (tid == 0) {
      tl.flag = wait_arrivals(tc, n_wait, ea.err, limit);
      tc->arrive = 0u;  // all keys are in; ordered before the next publication by its fence
    }
    __syncthreads();
    bool stop = true, ok = false;
    int npx = 0, npy = 0;
    unsigned long long t_b = 0ull;
    if (tl.flag) {
      t_b = globaltimer();
      ok = update_phase<R>(s, tpart, ns, usm, uca, kPubThread);  // ends with a __syncthreads
      if (ok) {
        // the next target is known: publish it before the bookkeeping.
        // Thread 0 decides (the inputs are global and may change under
        // other threads' feet) and the barrier below shares the decision.
        if (tid == 0) {
          bool st = usm.remaining <= 0 || usm.next_key == 0ull || usm.it + 1 >= lim || status != 0 ||
                    err != 0;
          if (!st && ea.tick_ns && globaltimer() - x.t_start > ea.tick_ns) {
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
    if (tid == kPubThread) {
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
    if (staged) stage_next<R>(s, npx, npy, usm);  // next speculative phase's input
    if (ok) {
      update_finish<R>(s, usm, staged);
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

  if constexpr (kLeadOnly) {
    while (!tl.stop) lead_round(tl.px, tl.py, false);
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
      if (tid == 0) {
        tpart[rank] = best;
        if (rank + 1 != ea.withhold) red_release_add(&tc->arrive, 1u);
      }
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
