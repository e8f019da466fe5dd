// Copy/update phase of one fill iteration for patch radius R <= 8, executed
// by a single CTA (the update kernel of the graph loop, or the last CTA of a
// search round inside the persistent engine).
//
// Sec. 3: after findBestPatch the pixels of Psi_q~ are copied into the
// unknown part of Psi_p^, those pixels take the confidence C(p^), and the
// priorities P(p) = C(p) D(p) (Eq. 1-2) that depend on them are recomputed
// before the next target is selected.  Everything this touches lies within
// 3R+2 pixels of p^, so that neighbourhood (mask, grey level, confidence) is
// staged in shared memory once; the priorities of the front pixels within
// 2R+1 of p^ are then evaluated from shared memory, each in one thread with
// the confidence sum in row-major patch order (bit-identical to the CPU).
#pragma once
#include "inpaint_internal.cuh"

namespace inp {

template <int R>
struct UpdGeom {
  static constexpr int P = 2 * R + 1;
  static constexpr int RB = 3 * R + 2;  // staged neighbourhood radius
  static constexpr int NS = 2 * RB + 1;
  static constexpr int R2 = 2 * R + 1;  // priorities that can change
  static constexpr int NW = 2 * R2 + 1;
  static constexpr int NC = 4 * R + 1;  // validity counts that can change
};

template <int R>
struct __align__(16) UpdSmem {
  using G = UpdGeom<R>;
  double cf[G::NS * G::NS];
  int mag[G::NS * G::NS];  // isophote |grad|^2 at a local pixel, -1 if not eligible
  int gxy[G::NS * G::NS];  // (gx + 512) << 16 | (gy + 512)
  int fsat[(G::P + 1) * (G::P + 1)];
  uint16_t flist[G::NW * G::NW];
  uint8_t om[G::NS * G::NS];  // 0 known, 1 Omega, 2 outside the image
  uint8_t gr[G::NS * G::NS];
  uint8_t filled[G::P * G::P];
  int nfront;
  unsigned long long red64[32];
  PrioBest redpb[32];
  int red32[32];
};

__device__ inline int ldcg_i(const int* p) { return __ldcg(p); }

// P(p) of Eq. 1-2 from the staged neighbourhood; (lx, ly) are p's local
// coordinates, (x, y) its image coordinates.
template <int R>
__device__ inline double prio_local(const UpdSmem<R>& sm, const ImgState& s, int lx, int ly, int x,
                                    int y, double* c_out) {
  using G = UpdGeom<R>;
  constexpr int NS = G::NS;
  double sum = 0.0;
  int n_in = 0;
#pragma unroll 1
  for (int dy = -R; dy <= R; ++dy) {
#pragma unroll
    for (int dx = -R; dx <= R; ++dx) {
      const int l = (ly + dy) * NS + lx + dx;
      const int o = sm.om[l];
      if (o != 2) {
        ++n_in;
        if (o == 0) sum = __dadd_rn(sum, sm.cf[l]);
      }
    }
  }
  const double c = __ddiv_rn(sum, (double)n_in);

  // Sobel of the Omega indicator with replicated image borders.
  const int xl = x > 0 ? -1 : 0, xr = x < s.W - 1 ? 1 : 0;
  const int yu = y > 0 ? -1 : 0, yd = y < s.H - 1 ? 1 : 0;
  auto M = [&](int ox, int oy) { return sm.om[(ly + oy) * NS + lx + ox] == 1 ? 1 : 0; };
  const int m_lu = M(xl, yu), m_cu = M(0, yu), m_ru = M(xr, yu);
  const int m_lc = M(xl, 0), m_rc = M(xr, 0);
  const int m_ld = M(xl, yd), m_cd = M(0, yd), m_rd = M(xr, yd);
  const int nx = (m_ru + 2 * m_rc + m_rd) - (m_lu + 2 * m_lc + m_ld);
  const int ny = (m_ld + 2 * m_cd + m_rd) - (m_lu + 2 * m_cu + m_ru);

  // Isophote: strongest precomputed gradient in Psi_p, first in row-major order.
  int best = -1, bl = 0;
#pragma unroll 1
  for (int dy = -R; dy <= R; ++dy) {
#pragma unroll
    for (int dx = -R; dx <= R; ++dx) {
      const int l = (ly + dy) * NS + lx + dx;
      const int m = sm.mag[l];
      if (m > best) {
        best = m;
        bl = l;
      }
    }
  }
  int gx = 0, gy = 0;
  if (best >= 0) {
    const int g = sm.gxy[bl];
    gx = (g >> 16) - 512;
    gy = (g & 0xffff) - 512;
  }
  int dot = (-gy) * nx + gx * ny;
  dot = dot < 0 ? -dot : dot;
  const int nn = nx * nx + ny * ny;
  double d = 0.0;
  if (nn != 0) d = __ddiv_rn(__ddiv_rn((double)dot, __dsqrt_rn((double)nn)), 510.0);
  *c_out = c;
  return __dmul_rn(c, d);
}


// Stages mask / grey / confidence of the NS x NS neighbourhood of (cx, cy).
template <int R>
__device__ inline void stage_nbhd(const ImgState& s, int cx, int cy, UpdSmem<R>& sm) {
  using G = UpdGeom<R>;
  constexpr int RB = G::RB, NS = G::NS;
  for (int i = threadIdx.x; i < NS * NS; i += blockDim.x) {
    const int x = cx - RB + i % NS, y = cy - RB + i / NS;
    uint8_t o = 2, g = 0;
    double cf = 0.0;
    if (x >= 0 && x < s.W && y >= 0 && y < s.H) {
      const size_t q = (size_t)y * s.W + x;
      o = __ldcg(&s.omega[q]);
      g = __ldcg(&s.gray[q]);
      cf = __ldcg(&s.conf[q]);
    }
    sm.om[i] = o;
    sm.gr[i] = g;
    sm.cf[i] = cf;
  }
}

// Isophote candidates of the staged neighbourhood: pixels whose four
// neighbours are known, with their central-difference grey gradient.
template <int R>
__device__ inline void stage_isophotes(UpdSmem<R>& sm) {
  constexpr int NS = UpdGeom<R>::NS;
  for (int i = threadIdx.x; i < NS * NS; i += blockDim.x) {
    const int lx = i % NS, ly = i / NS;
    int m = -1, g = 0;
    if (lx >= 1 && lx < NS - 1 && ly >= 1 && ly < NS - 1 && sm.om[i] == 0 && sm.om[i - 1] == 0 &&
        sm.om[i + 1] == 0 && sm.om[i - NS] == 0 && sm.om[i + NS] == 0) {
      const int gx = (int)sm.gr[i + 1] - (int)sm.gr[i - 1];
      const int gy = (int)sm.gr[i + NS] - (int)sm.gr[i - NS];
      m = gx * gx + gy * gy;
      g = ((gx + 512) << 16) | (gy + 512);
    }
    sm.mag[i] = m;
    sm.gxy[i] = g;
  }
}

// Front pixels of the NW x NW window around (cx, cy) go to sm.flist; the
// other in-image window pixels get priority key 0.  sm.nfront must be 0.
template <int R>
__device__ inline void window_front(const ImgState& s, int cx, int cy, UpdSmem<R>& sm) {
  using G = UpdGeom<R>;
  constexpr int RB = G::RB, NS = G::NS, R2 = G::R2, NW = G::NW;
  for (int i = threadIdx.x; i < NW * NW; i += blockDim.x) {
    const int wx = i % NW - R2, wy = i / NW - R2;
    const int l = (RB + wy) * NS + RB + wx;
    if (sm.om[l] == 2) continue;
    const bool front = sm.om[l] == 1 && (sm.om[l - 1] == 0 || sm.om[l + 1] == 0 ||
                                         sm.om[l - NS] == 0 || sm.om[l + NS] == 0);
    if (front) {
      sm.flist[atomicAdd(&sm.nfront, 1)] = (uint16_t)i;
    } else {
      const size_t p = (size_t)(cy + wy) * s.W + cx + wx;
      s.prio[p] = 0ull;
      s.pconf[p] = 0.0;
    }
  }
}

// Priority key of front-list entry i of the window around (cx, cy).
template <int R>
__device__ inline void window_prio(const ImgState& s, int cx, int cy, const UpdSmem<R>& sm, int i) {
  using G = UpdGeom<R>;
  constexpr int RB = G::RB, R2 = G::R2, NW = G::NW;
  const int wi = sm.flist[i];
  const int wx = wi % NW - R2, wy = wi / NW - R2;
  double cc;
  const double pr = prio_local<R>(sm, s, RB + wx, RB + wy, cx + wx, cy + wy, &cc);
  const size_t p = (size_t)(cy + wy) * s.W + cx + wx;
  s.prio[p] = (unsigned long long)__double_as_longlong(pr) + 1ull;
  s.pconf[p] = cc;
}

// Initial priorities, one CTA per NW x NW window of the image.
template <int R>
__global__ void __launch_bounds__(256) k_prio_init_fast(ImgState s) {
  using G = UpdGeom<R>;
  extern __shared__ __align__(16) uint8_t sm_raw[];
  UpdSmem<R>& sm = *reinterpret_cast<UpdSmem<R>*>(sm_raw);
  const int cx = G::R2 + blockIdx.x * G::NW, cy = G::R2 + blockIdx.y * G::NW;
  if (threadIdx.x == 0) sm.nfront = 0;
  stage_nbhd<R>(s, cx, cy, sm);
  __syncthreads();
  stage_isophotes<R>(sm);
  window_front<R>(s, cx, cy, sm);
  __syncthreads();
  for (int i = threadIdx.x; i < sm.nfront; i += blockDim.x) window_prio<R>(s, cx, cy, sm, i);
}

// Returns false (status already written) when no source patch exists or the
// state is inconsistent; true when the iteration was applied.  Whole block.
template <int R>
__device__ bool update_phase(const ImgState& s, const unsigned long long* partial, int n_partial,
                             UpdSmem<R>& sm) {
  using G = UpdGeom<R>;
  constexpr int P = G::P, RB = G::RB, NS = G::NS, R2 = G::R2, NW = G::NW, NC = G::NC;
  Ctrl* c = s.ctrl;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int W = s.W, H = s.H;
  const int px = __ldcg(&c->px), py = __ldcg(&c->py);
  const double cp = __ldcg(&c->conf), pp = __ldcg(&c->prio);
  const int n_cand = __ldcg(&c->n_valid), it = __ldcg(&c->iter);
  int remaining = __ldcg(&c->remaining);

  // U0 + U1: best source key over the search CTAs; stage the neighbourhood.
  unsigned long long best = ~0ull;
  for (int i = tid; i < n_partial; i += nt) {
    const unsigned long long v = __ldcg(&partial[i]);
    best = v < best ? v : best;
  }
  stage_nbhd<R>(s, px, py, sm);
  if (tid == 0) sm.nfront = 0;
  best = block_min_u64(best, sm.red64);
  if (best == ~0ull) {
    if (tid == 0) c->status = INPAINT_ERR_NO_SOURCE;
    return false;
  }
  const uint32_t ssd = (uint32_t)(best >> 32);
  const int q = (int)(best & 0xffffffffull);
  const int qx = q % W, qy = q / W;

  // U2: copy the unknown in-image part of Psi_p^ from Psi_q~.
  int my_filled = 0;
  for (int i = tid; i < P * P; i += nt) {
    const int dy = i / P - R, dx = i % P - R;
    const int l = (RB + dy) * NS + RB + dx;
    uint8_t f = 0;
    if (sm.om[l] == 1) {
      const int tx = px + dx, ty = py + dy;
      const uint32_t w = __ldcg(&s.img[(size_t)(qy + dy) * s.pitch + qx + dx]);
      const uint8_t g = (uint8_t)luma_word(w);
      const size_t t = (size_t)ty * W + tx;
      s.img[(size_t)ty * s.pitch + tx] = w;
      s.gray[t] = g;
      s.conf[t] = cp;
      s.omega[t] = 0;
      sm.om[l] = 0;
      sm.gr[l] = g;
      sm.cf[l] = cp;
      f = 1;
      ++my_filled;
    }
    sm.filled[i] = f;
  }
  const int filled = block_sum_int(my_filled, sm.red32);
  if (filled == 0) {  // p^ must lie in Omega
    if (tid == 0) c->status = INPAINT_ERR_INTERNAL;
    return false;
  }
  const int nx_in = min(px + R, W - 1) - max(px - R, 0) + 1;
  const int ny_in = min(py + R, H - 1) - max(py - R, 0) + 1;
  const int n_known = nx_in * ny_in - filled;

  // U3: isophote candidates, integral image of the filled flags, front list.
  stage_isophotes<R>(sm);
  if (tid < 32) {
    constexpr int P1 = P + 1;
    for (int v = tid; v <= P; v += 32) {
      sm.fsat[v] = 0;
      sm.fsat[v * P1] = 0;
    }
    __syncwarp();
    for (int v = tid; v < P; v += 32) {
      int run = 0;
      for (int u = 0; u < P; ++u) {
        run += sm.filled[v * P + u];
        sm.fsat[(v + 1) * P1 + u + 1] = run;
      }
    }
    __syncwarp();
    for (int u = tid + 1; u <= P; u += 32)
      for (int v = 2; v <= P; ++v) sm.fsat[v * P1 + u] += sm.fsat[(v - 1) * P1 + u];
  }
  window_front<R>(s, px, py, sm);
  __syncthreads();

  // U4: validity counts around p^ and the priorities of the front pixels.
  int newly = 0;
  const int nfront = sm.nfront;
  for (int i = tid; i < NC * NC + nfront; i += nt) {
    if (i < nfront) {
      window_prio<R>(s, px, py, sm, i);
    } else {
      const int j = i - nfront;
      const int wy = j / NC - 2 * R, wx = j % NC - 2 * R;
      const int x = px + wx, y = py + wy;
      if (x < 0 || x >= W || y < 0 || y >= H) continue;
      const int u0 = max(0, wx), u1 = min(P - 1, wx + 2 * R);
      const int v0 = max(0, wy), v1 = min(P - 1, wy + 2 * R);
      constexpr int P1 = P + 1;
      const int dec = sm.fsat[(v1 + 1) * P1 + u1 + 1] - sm.fsat[v0 * P1 + u1 + 1] -
                      sm.fsat[(v1 + 1) * P1 + u0] + sm.fsat[v0 * P1 + u0];
      if (dec) {
        const size_t qi = (size_t)y * W + x;
        const int nv = __ldcg(&s.count[qi]) - dec;
        s.count[qi] = nv;
        if (nv == 0 && x >= s.cx0 && x <= s.cx1 && y >= s.cy0 && y <= s.cy1) ++newly;
      }
    }
  }
  newly = block_sum_int(newly, sm.red32);

  // U5: tiles over the window, then the next target.
  block_refresh_tiles(s, max(0, px - R2), min(W - 1, px + R2), max(0, py - R2), min(H - 1, py + R2));
  remaining -= filled;
  if (tid == 0) {
    inpaint_step_info* e = &c->last;
    e->iter = it;
    e->px = px;
    e->py = py;
    e->qx = qx;
    e->qy = qy;
    e->ssd = ssd;
    e->priority = pp;
    e->confidence = cp;
    e->filled = filled;
    e->remaining = remaining;
    e->n_known = n_known;
    e->n_cand = n_cand;
    if (it < s.trace_cap) s.trace[it] = *e;
    c->remaining = remaining;
    c->iter = it + 1;
    c->n_valid = n_cand + newly;
    c->evals += (unsigned long long)n_cand * (unsigned long long)n_known;
    c->px = -1;
    c->py = -1;
  }
  __syncthreads();
  if (remaining > 0 && tid < 32) warp_select(s);
  __syncthreads();
  return true;
}

}  // namespace inp
