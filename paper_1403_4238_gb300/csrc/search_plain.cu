// findBestPatch, plain CUDA-core form (Sec. 3 Eq. 3-4; Algorithm 1 and the
// local-memory staging of Algorithm 2 / Sec. 5.5 as prior art).
//
// For the selected target centre p^ and every valid candidate centre q (patch
// inside the image and fully known: unknown count 0), the SSD over the known
// in-image pixels d of Psi_p^ is
//     SSD(q) = sum_d sum_{c in RGB} (I[p^+d]_c - I[q+d]_c)^2,
// an exact 32-bit integer (at most 65^2 * 3 * 255^2 < 2^31).  Each CTA
// reduces its candidates to one key (SSD << 32 | idx(q)); the smallest key
// over all CTAs is the best patch, ties going to the lowest index.
//
// GB300 design: a CTA stages an (8 + 2r) x (128 + 2r) tile of RGBA words in
// shared memory (every pixel is reused by up to P^2 candidates), each thread
// keeps 4 adjacent candidates in registers, reads one row strip of the tile
// per patch row with 128-bit loads, and per known target pixel issues one
// byte-SIMD absolute difference and one 4-way byte dot product per candidate
// (|a-b| per channel, then sum of squares; alpha is 0 on both sides).
// Unknown target pixels are skipped by a warp-uniform branch on a per-row
// bit mask, so the work is |K| evaluations per candidate, not P^2.
#include "inpaint_internal.cuh"

namespace inp {

__device__ inline unsigned long long cand_key(const ImgState& s, uint32_t ssd, int qx, int qy) {
  if (qx > s.cx1 || qy > s.cy1) return ~0ull;
  const int idx = qy * s.W + qx;
  if (s.count[(size_t)qy * s.pitch + qx] != 0) return ~0ull;
  return ((unsigned long long)ssd << 32) | (unsigned)idx;
}

// Stage a rows x pitch window of image words whose top-left is (x0, y0);
// out-of-image words read as 0 (never used by a valid candidate).
__device__ inline void stage_tile(const ImgState& s, uint32_t* dst, int x0, int y0, int rows,
                                  int pitch) {
  const int n = rows * pitch;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const int yy = y0 + i / pitch, xx = x0 + i % pitch;
    uint32_t w = 0;
    if (xx >= 0 && xx < s.W && yy >= 0 && yy < s.H) w = s.img[(size_t)yy * s.pitch + xx];
    dst[i] = w;
  }
}

__device__ inline void write_partial(const ImgState& s, unsigned long long best,
                                     unsigned long long* scratch) {
  best = block_min_u64(best, scratch);
  if (threadIdx.x == 0) s.partial[blockIdx.y * gridDim.x + blockIdx.x] = best;
}

template <int R>
__global__ void __launch_bounds__(kSearchThreads) k_search_plain(ImgState s) {
  constexpr int P = 2 * R + 1;
  constexpr int TW = kSearchTW, TH = kSearchTH, S = kSearchS;
  constexpr int SW = (TW + 2 * R + 3) & ~3;       // tile pitch (words), multiple of 4
  constexpr int SH = TH + 2 * R;
  constexpr int NROW = (S + P - 1 + 3) & ~3;      // words of one row strip
  static_assert(31 * S + NROW <= SW, "row strip must stay inside the tile");
  __shared__ __align__(16) uint32_t src[SH * SW];
  __shared__ uint32_t tgt[P * P];
  __shared__ uint32_t rowmask[P];
  __shared__ unsigned long long red[32];

  const Ctrl* c = s.ctrl;
  if (!loop_active(c)) return;
  const int px = c->px, py = c->py;
  const int ox = s.cx0 + blockIdx.x * TW, oy = s.cy0 + blockIdx.y * TH;
  const int tid = threadIdx.x;

  // Target patch: known in-image pixels with their RGBA words, one bit mask per row.
  if (tid < P) {
    const int ty = py + tid - R;
    uint32_t m = 0;
    for (int dx = 0; dx < P; ++dx) {
      const int tx = px + dx - R;
      uint32_t w = 0;
      if (tx >= 0 && tx < s.W && ty >= 0 && ty < s.H) {
        const size_t t = (size_t)ty * s.W + tx;
        if (!s.omega[t]) {
          w = s.img[(size_t)ty * s.pitch + tx];
          m |= 1u << dx;
        }
      }
      tgt[tid * P + dx] = w;
    }
    rowmask[tid] = m;
  }
  stage_tile(s, src, ox - R, oy - R, SH, SW);
  __syncthreads();

  const int lane = tid & 31, wr = tid >> 5;  // warp = one candidate row of the tile
  uint32_t acc[S];
#pragma unroll
  for (int k = 0; k < S; ++k) acc[k] = 0;

  for (int dy = 0; dy < P; ++dy) {
    const uint32_t m = rowmask[dy];
    if (m == 0) continue;
    uint32_t row[NROW];
    const uint4* sp = reinterpret_cast<const uint4*>(&src[(wr + dy) * SW + lane * S]);
#pragma unroll
    for (int i = 0; i < NROW / 4; ++i) {
      const uint4 v = sp[i];
      row[4 * i] = v.x;
      row[4 * i + 1] = v.y;
      row[4 * i + 2] = v.z;
      row[4 * i + 3] = v.w;
    }
    const uint32_t* trow = &tgt[dy * P];
#pragma unroll
    for (int dx = 0; dx < P; ++dx) {
      if (m & (1u << dx)) {
        const uint32_t a = trow[dx];
#pragma unroll
        for (int k = 0; k < S; ++k) {
          const uint32_t d = __vabsdiffu4(a, row[k + dx]);
          acc[k] = __dp4a(d, d, acc[k]);
        }
      }
    }
  }

  unsigned long long best = ~0ull;
  const int qy = oy + wr;
#pragma unroll
  for (int k = 0; k < S; ++k) {
    const unsigned long long key = cand_key(s, acc[k], ox + lane * S + k, qy);
    best = key < best ? key : best;
  }
  write_partial(s, best, red);
}

// Stage a rows x pitch window of image words for the partial-overlap search:
// the alpha byte says whether the pixel may be used as a source (0: known and
// in the image; 0xFF: unknown or outside the image, RGB bytes 0).
__device__ inline void stage_tile_avail(const ImgState& s, uint32_t* dst, int x0, int y0, int rows,
                                        int pitch) {
  const int n = rows * pitch;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const int yy = y0 + i / pitch, xx = x0 + i % pitch;
    uint32_t w = 0xff000000u;
    if (xx >= 0 && xx < s.W && yy >= 0 && yy < s.H) {
      const uint8_t o = s.omega[(size_t)yy * s.W + xx];
      const uint32_t v = s.img[(size_t)yy * s.pitch + xx];
      w = o ? 0xff000000u : v;
    }
    dst[i] = w;
  }
}

// findBestPatch, partial-overlap variant (Algorithm 1 and Sec. 5.4): every
// centre q of the search rectangle is a candidate, also when Psi_q overlaps
// Omega or crosses the image border.  SSD(q) runs over the offsets whose
// target pixel and source pixel are both known and in the image; q is
// admissible only if a known in-image source pixel lies under every unknown
// in-image target pixel (the copy of Sec. 3 reads those).  Same tiles and
// byte-SIMD arithmetic as k_search_plain, with the source's availability in
// the alpha byte of its staged word: the absolute difference's alpha byte is
// then 0xFF exactly when the source pixel is unavailable, and shifting the
// RGB mask 0x00ffffff right by (difference >> 27) = 31 drops that term.  The
// number of admissible candidates goes to ctrl->n_adm (the update phase's
// work count reads and clears it).
template <int R>
__global__ void __launch_bounds__(kSearchThreads) k_search_overlap(ImgState s) {
  constexpr int P = 2 * R + 1;
  constexpr int TW = kSearchTW, TH = kSearchTH, S = kSearchS;
  constexpr int SW = (TW + 2 * R + 3) & ~3;
  constexpr int SH = TH + 2 * R;
  constexpr int NROW = (S + P - 1 + 3) & ~3;
  static_assert(31 * S + NROW <= SW, "row strip must stay inside the tile");
  __shared__ __align__(16) uint32_t src[SH * SW];
  __shared__ uint32_t tgt[P * P];
  __shared__ uint32_t rowmask[P], unkmask[P];
  __shared__ unsigned long long red[32];
  __shared__ int red32[32];

  Ctrl* c = s.ctrl;
  if (!loop_active(c)) return;
  const int px = c->px, py = c->py;
  const int ox = s.cx0 + blockIdx.x * TW, oy = s.cy0 + blockIdx.y * TH;
  const int tid = threadIdx.x;

  // target patch: known pixels (words, bit masks per row) and unknown in-image pixels
  if (tid < P) {
    const int ty = py + tid - R;
    uint32_t m = 0, u = 0;
    for (int dx = 0; dx < P; ++dx) {
      const int tx = px + dx - R;
      uint32_t w = 0;
      if (tx >= 0 && tx < s.W && ty >= 0 && ty < s.H) {
        if (!s.omega[(size_t)ty * s.W + tx]) {
          w = s.img[(size_t)ty * s.pitch + tx];
          m |= 1u << dx;
        } else {
          u |= 1u << dx;
        }
      }
      tgt[tid * P + dx] = w;
    }
    rowmask[tid] = m;
    unkmask[tid] = u;
  }
  stage_tile_avail(s, src, ox - R, oy - R, SH, SW);
  __syncthreads();

  const int lane = tid & 31, wr = tid >> 5;
  uint32_t acc[S], bad[S];
#pragma unroll
  for (int k = 0; k < S; ++k) {
    acc[k] = 0;
    bad[k] = 0;
  }

  for (int dy = 0; dy < P; ++dy) {
    const uint32_t m = rowmask[dy], u = unkmask[dy];
    if ((m | u) == 0) continue;
    uint32_t row[NROW];
    const uint4* sp = reinterpret_cast<const uint4*>(&src[(wr + dy) * SW + lane * S]);
#pragma unroll
    for (int i = 0; i < NROW / 4; ++i) {
      const uint4 v = sp[i];
      row[4 * i] = v.x;
      row[4 * i + 1] = v.y;
      row[4 * i + 2] = v.z;
      row[4 * i + 3] = v.w;
    }
    const uint32_t* trow = &tgt[dy * P];
#pragma unroll
    for (int dx = 0; dx < P; ++dx) {
      if (m & (1u << dx)) {
        const uint32_t a = trow[dx];
#pragma unroll
        for (int k = 0; k < S; ++k) {
          const uint32_t d = __vabsdiffu4(a, row[k + dx]);
          const uint32_t e = d & (0x00ffffffu >> (d >> 27));
          acc[k] = __dp4a(e, e, acc[k]);
        }
      } else if (u & (1u << dx)) {
#pragma unroll
        for (int k = 0; k < S; ++k) bad[k] |= row[k + dx] >> 24;
      }
    }
  }

  unsigned long long best = ~0ull;
  int n_adm = 0;
  const int qy = oy + wr;
#pragma unroll
  for (int k = 0; k < S; ++k) {
    const int qx = ox + lane * S + k;
    if (qx <= s.cx1 && qy <= s.cy1 && bad[k] == 0) {
      const unsigned long long key = ((unsigned long long)acc[k] << 32) | (unsigned)(qy * s.W + qx);
      best = key < best ? key : best;
      ++n_adm;
    }
  }
  n_adm = block_sum_int(n_adm, red32);
  if (tid == 0 && n_adm) atomicAdd(&c->n_adm, n_adm);
  write_partial(s, best, red);
}

// Any radius up to kMaxRadius: the known target pixels are compacted into a
// list in shared memory and each evaluation reads its source word from there.
__global__ void __launch_bounds__(kGenThreads) k_search_generic(ImgState s) {
  extern __shared__ __align__(16) uint32_t dyn[];
  __shared__ unsigned long long red[32];
  __shared__ int nk_s;
  const Ctrl* c = s.ctrl;
  if (!loop_active(c)) return;
  const int R = s.r, P = 2 * R + 1;
  const int TW = kGenTW, TH = kGenTH, S = kGenS;
  const int SW = TW + 2 * R, SH = TH + 2 * R;
  uint32_t* src = dyn;                          // SH * SW
  uint32_t* koff = dyn + SH * SW;               // P * P offsets into the tile
  uint32_t* kval = koff + P * P;                // P * P target words
  const int px = c->px, py = c->py;
  const int ox = s.cx0 + blockIdx.x * TW, oy = s.cy0 + blockIdx.y * TH;
  const int tid = threadIdx.x;
  if (tid == 0) {
    int n = 0;
    for (int dy = 0; dy < P; ++dy)
      for (int dx = 0; dx < P; ++dx) {
        const int tx = px + dx - R, ty = py + dy - R;
        if (tx >= 0 && tx < s.W && ty >= 0 && ty < s.H) {
          const size_t t = (size_t)ty * s.W + tx;
          if (!s.omega[t]) {
            koff[n] = dy * SW + dx;
            kval[n] = s.img[(size_t)ty * s.pitch + tx];
            ++n;
          }
        }
      }
    nk_s = n;
  }
  stage_tile(s, src, ox - R, oy - R, SH, SW);
  __syncthreads();
  const int nk = nk_s;
  const int lane = tid & 31, wr = tid >> 5;
  uint32_t acc[kGenS] = {0, 0};
  const uint32_t* base = src + wr * SW + lane * S;
  for (int k = 0; k < nk; ++k) {
    const uint32_t a = kval[k];
    const uint32_t* b = base + koff[k];
#pragma unroll
    for (int j = 0; j < S; ++j) {
      const uint32_t d = __vabsdiffu4(a, b[j]);
      acc[j] = __dp4a(d, d, acc[j]);
    }
  }
  unsigned long long best = ~0ull;
  const int qy = oy + wr;
#pragma unroll
  for (int j = 0; j < S; ++j) {
    const unsigned long long key = cand_key(s, acc[j], ox + lane * S + j, qy);
    best = key < best ? key : best;
  }
  write_partial(s, best, red);
}

static size_t generic_smem(int R) {
  const int P = 2 * R + 1;
  return (size_t)((kGenTH + 2 * R) * (kGenTW + 2 * R) + 2 * P * P) * sizeof(uint32_t);
}

cudaError_t prepare_search_plain(int r) {
  if (r <= 8) return cudaSuccess;
  return cudaFuncSetAttribute(k_search_generic, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)generic_smem(r));
}

dim3 search_plain_grid(const ImgState& s) {
  const int cw = s.cx1 - s.cx0 + 1, ch = s.cy1 - s.cy0 + 1;
  if (cw <= 0 || ch <= 0) return dim3(0, 0, 1);
  if (s.r <= 8) return dim3((cw + kSearchTW - 1) / kSearchTW, (ch + kSearchTH - 1) / kSearchTH, 1);
  return dim3((cw + kGenTW - 1) / kGenTW, (ch + kGenTH - 1) / kGenTH, 1);
}

cudaError_t launch_search_plain(const ImgState& s, cudaStream_t st) {
  const dim3 g = search_plain_grid(s);
  if (g.x == 0) return cudaSuccess;
  if (s.overlap) {
    switch (s.r) {
      case 1: k_search_overlap<1><<<g, kSearchThreads, 0, st>>>(s); break;
      case 2: k_search_overlap<2><<<g, kSearchThreads, 0, st>>>(s); break;
      case 3: k_search_overlap<3><<<g, kSearchThreads, 0, st>>>(s); break;
      case 4: k_search_overlap<4><<<g, kSearchThreads, 0, st>>>(s); break;
      case 5: k_search_overlap<5><<<g, kSearchThreads, 0, st>>>(s); break;
      case 6: k_search_overlap<6><<<g, kSearchThreads, 0, st>>>(s); break;
      case 7: k_search_overlap<7><<<g, kSearchThreads, 0, st>>>(s); break;
      case 8: k_search_overlap<8><<<g, kSearchThreads, 0, st>>>(s); break;
      default: return cudaErrorInvalidValue;  // the variant is built for r <= 8
    }
    return cudaGetLastError();
  }
  switch (s.r) {
    case 1: k_search_plain<1><<<g, kSearchThreads, 0, st>>>(s); break;
    case 2: k_search_plain<2><<<g, kSearchThreads, 0, st>>>(s); break;
    case 3: k_search_plain<3><<<g, kSearchThreads, 0, st>>>(s); break;
    case 4: k_search_plain<4><<<g, kSearchThreads, 0, st>>>(s); break;
    case 5: k_search_plain<5><<<g, kSearchThreads, 0, st>>>(s); break;
    case 6: k_search_plain<6><<<g, kSearchThreads, 0, st>>>(s); break;
    case 7: k_search_plain<7><<<g, kSearchThreads, 0, st>>>(s); break;
    case 8: k_search_plain<8><<<g, kSearchThreads, 0, st>>>(s); break;
    default:
      k_search_generic<<<g, kGenThreads, generic_smem(s.r), st>>>(s);
  }
  return cudaGetLastError();
}

}  // namespace inp
