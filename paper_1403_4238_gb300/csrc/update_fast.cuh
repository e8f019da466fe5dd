// Copy/update phase of one fill iteration for patch radius R <= 8.
//
// Sec. 3: after findBestPatch the pixels of Psi_q~ are copied into the
// unknown part of Psi_p^, those pixels take the confidence C(p^), and the
// priorities P(p) = C(p) D(p) (Eq. 1-2) that depend on them are recomputed
// before the next target is selected.  Everything involved lies within 3R+2
// pixels of p^, so that neighbourhood is staged in shared memory.
//
// The work is split in two phases.  Which pixels are filled (Psi_p^ ∩ Omega)
// and the confidence they receive (C(p^)) are known as soon as p^ is
// selected; only their colours depend on the search result q~.  So the
// *speculative phase* (spec_phase) runs while the search is still going: it
// builds the post-fill mask and confidences, finds the post-fill front pixels
// within 2R+1 of p^, and evaluates their confidence terms C(p) -- the
// sequential FP64 sums, in row-major patch order (the part with the longest
// dependency chain) -- and their front normals.  The *update phase*
// (update_phase) then only copies the pixels, recomputes the isophotes from
// the new grey levels, and combines them into the data terms D(p) and the
// priorities.  The data term D = (|dot| / sqrt(nn)) / 510 takes one of a
// finite set of values (nn = |n|^2 <= 32, |dot| <= 2040); the library
// evaluates that set once with the same IEEE operations and reads it back
// here, which gives the same bits as evaluating the expression.
#pragma once
#include "inpaint_internal.cuh"
#include "ptx.cuh"

namespace inp {

template <int R>
struct UpdGeom {
  static constexpr int P = 2 * R + 1;
  static constexpr int RB = 3 * R + 2;  // staged neighbourhood radius
  static constexpr int NS = 2 * RB + 1;
  static constexpr int R2 = 2 * R + 1;  // priorities that can change
  static constexpr int NW = 2 * R2 + 1;
  static constexpr int NC = 4 * R + 1;  // validity counts that can change
  // level-0 / level-1 priority tiles an NW x NW window can touch (per axis)
  static constexpr int KT0 = (NW + kT0 - 2) / kT0 + 1;
  static constexpr int KT1 = 2;
};

constexpr int kT1Cache = 512;  // level-1 entries kept in shared memory (images up to 2^25 px)

// State the update phase reads that the search does not change, loaded
// while the search runs (update_prefetch): validity counts of the count
// window, the priority keys of the level-0 tiles the priority window
// touches, the level-0 entries of the level-1 tiles over them, and the
// level-1 entries of the whole image.
template <int R>
struct __align__(16) UpdCache {
  using G = UpdGeom<R>;
  unsigned long long tp[G::KT0 * G::KT0 * kT0 * kT0];
  PrioBest t0c[G::KT1 * G::KT1 * kT1 * kT1];
  PrioBest t1c[kT1Cache];
  int cnt[G::NC * G::NC];
  int tx0, ty0, ntx, nty;  // level-0 tiles [tx0, tx0 + ntx) x [ty0, ty0 + nty)
  int ux0, uy0, nux, nuy;  // level-1 tiles
  int t1n;                 // level-1 entries cached (0: read them from global memory)
};

template <int R>
struct __align__(16) UpdSmem {
  using G = UpdGeom<R>;
  double cf[G::NS * G::NS];
  double sC[G::NW * G::NW];  // post-fill C(p) of the window (from the speculative phase)
  int snrm[G::NW * G::NW];   // packed normal, or kSpecNotFront / kSpecOutside
  int mag[G::NS * G::NS];    // isophote |grad|^2 at a local pixel, -1 if not eligible
  int gxy[G::NS * G::NS];    // (gx + 512) << 16 | (gy + 512)
  int fsat[(G::P + 1) * (G::P + 1)];
  uint8_t om[G::NS * G::NS];  // 0 known, 1 Omega, 2 outside the image
  uint8_t gr[G::NS * G::NS];
  uint8_t filled[G::P * G::P];
  uint16_t list[G::NW * G::NW];
  int nlist;
  unsigned long long red64[32];
  int red32[32];
  int spec_iter, spec_filled, nfront;  // speculative phase outcome
  // the next target as staged by stage_next: centre, iteration, C(p^)
  int nx_px, nx_py, nx_it;
  double nx_cp;
  // outcome of update_phase, consumed by update_finish
  unsigned long long next_key;  // priority key of the next target (0: none)
  int next_idx;
  int it, remaining, n_filled, n_known, n_cand, newly, qx, qy;
  uint32_t ssd;
  int px, py;
  double pp, cp;
  // the best front pixel whose priority this iteration's fill cannot change
  // (outside the NW x NW window), found by spec_phase when asked
  unsigned long long out_key;
  int out_idx;
  int early_stop;  // early selection: the loop stops after this iteration
  int upd_ok;      // update_phase: the speculation matches the iteration
  int iso_next;    // spec_phase: next chunk of the isophotes the fill cannot change
  // the data term's divisors: s = sqrt(nn) for the 14 normal lengths, their
  // reciprocals and that of 510 (stage_dterm, once per launch)
  double dsq[kDTabRows], dinv[kDTabRows], dinv510;
  // early selection: the tile maxima of the last update and the check of
  // its selection are pending (run by the next speculative phase's spare
  // warps, or by the leader before it leaves the image)
  int tiles_pending;
  unsigned long long pend_key;  // the published next target's key, index
  int pend_idx;
  int pend_rem;  // |Omega| after that update
  PrioBest red_pb[32];
};

// a / b rounded to nearest for a divisor known in advance, from y = RN(1/b):
// q0 = RN(a y), the remainder a - q0 b exact by one FMA, then the corrected
// quotient RN(q0 + r y) (Markstein's division, IBM J. Res. Dev. 34(1), 1990).
// Used only where it is checked to equal RN(a / b) for every input: the data
// term below, for all 14 normal lengths and all 2041 dot products.
__device__ inline double div_known(double a, double b, double y) {
  const double q0 = __dmul_rn(a, y);
  const double r = __fma_rn(-q0, b, a);
  return __fma_rn(r, y, q0);
}

// The data term's divisors into shared memory (threads 0-14; a barrier must
// follow before data_term_known reads them): correctly rounded square roots
// and reciprocals, the same values the host computes.
template <int R>
__device__ inline void stage_dterm(UpdSmem<R>& sm) {
  const int t = threadIdx.x;
  if (t < kDTabRows) {
    const double s = __dsqrt_rn((double)dtab_nn(t));
    sm.dsq[t] = s;
    sm.dinv[t] = __ddiv_rn(1.0, s);
  } else if (t == kDTabRows) {
    sm.dinv510 = __ddiv_rn(1.0, 510.0);
  }
}

// D of Eq. 2, the same bits as data_term_direct: fl(fl(dot / s) / 510), both
// quotients by div_known with the staged divisors (no global load on the
// update's path).
template <int R>
__device__ inline double data_term_known(const UpdSmem<R>& sm, int dot, int nn) {
  if (nn == 0) return 0.0;
  const int c = dtab_code(nn);
  return div_known(div_known((double)dot, sm.dsq[c], sm.dinv[c]), 510.0, sm.dinv510);
}

// Sobel normal of the Omega indicator at local (lx, ly) = image (x, y),
// replicated image borders, packed as (nx + 8) << 8 | (ny + 8).
template <int R>
__device__ inline int normal_local(const UpdSmem<R>& sm, const ImgState& s, int lx, int ly, int x,
                                   int y) {
  constexpr int NS = UpdGeom<R>::NS;
  const int xl = x > 0 ? -1 : 0, xr = x < s.W - 1 ? 1 : 0;
  const int yu = y > 0 ? -1 : 0, yd = y < s.H - 1 ? 1 : 0;
  auto M = [&](int ox, int oy) { return sm.om[(ly + oy) * NS + lx + ox] == 1 ? 1 : 0; };
  const int m_lu = M(xl, yu), m_cu = M(0, yu), m_ru = M(xr, yu);
  const int m_lc = M(xl, 0), m_rc = M(xr, 0);
  const int m_ld = M(xl, yd), m_cd = M(0, yd), m_rd = M(xr, yd);
  const int nx = (m_ru + 2 * m_rc + m_rd) - (m_lu + 2 * m_lc + m_ld);
  const int ny = (m_ld + 2 * m_cd + m_rd) - (m_lu + 2 * m_cu + m_ru);
  return ((nx + 8) << 8) | (ny + 8);
}

// C(p) of Eq. 2: the known part of Psi_p summed in row-major order (dy
// outer, dx inner, one addition at a time), over the in-image area.
// Unknown and out-of-image entries hold +0.0 in sm.cf, and adding +0.0 to a
// non-negative double leaves it unchanged, so summing every entry gives
// exactly the sum over the known pixels.
template <int R>
__device__ inline double conf_local(const UpdSmem<R>& sm, const ImgState& s, int lx, int ly, int x,
                                    int y) {
  constexpr int NS = UpdGeom<R>::NS;
  double sum = 0.0;
#pragma unroll 1
  for (int dy = -R; dy <= R; ++dy) {
#pragma unroll
    for (int dx = -R; dx <= R; ++dx) sum = __dadd_rn(sum, sm.cf[(ly + dy) * NS + lx + dx]);
  }
  const int n_in = (min(x + R, s.W - 1) - max(x - R, 0) + 1) * (min(y + R, s.H - 1) - max(y - R, 0) + 1);
  return __ddiv_rn(sum, (double)n_in);
}

// Strongest precomputed isophote in Psi_p, first in row-major order.
template <int R>
__device__ inline void isophote_local(const UpdSmem<R>& sm, int lx, int ly, int* gx, int* gy) {
  constexpr int NS = UpdGeom<R>::NS;
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
  *gx = 0;
  *gy = 0;
  if (best >= 0) {
    const int g = sm.gxy[bl];
    *gx = (g >> 16) - 512;
    *gy = (g & 0xffff) - 512;
  }
}

__device__ inline int dot_abs(int gx, int gy, int nrm) {
  const int nx = (nrm >> 8) - 8, ny = (nrm & 0xff) - 8;
  const int d = (-gy) * nx + gx * ny;
  return d < 0 ? -d : d;
}

__device__ inline int nn_of(int nrm) {
  const int nx = (nrm >> 8) - 8, ny = (nrm & 0xff) - 8;
  return nx * nx + ny * ny;
}

// D of Eq. 2 evaluated directly (initialisation).
__device__ inline double data_term_direct(int dot, int nn) {
  if (nn == 0) return 0.0;
  return __ddiv_rn(__ddiv_rn((double)dot, __dsqrt_rn((double)nn)), 510.0);
}


// Stages the NS x NS neighbourhood of (cx, cy): mask (2 outside the image),
// optionally grey levels and confidences (+0.0 under Omega and outside).
template <int R, bool GRAY, bool CONF>
__device__ inline void stage_nbhd(const ImgState& s, int cx, int cy, UpdSmem<R>& sm) {
  using G = UpdGeom<R>;
  constexpr int RB = G::RB, NS = G::NS;
  constexpr int U = 4;  // entries per thread with their loads in flight together
  const int step = blockDim.x;
  for (int i0 = threadIdx.x; i0 < NS * NS; i0 += U * step) {
    uint8_t o[U], g[U];
    double cf[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int i = i0 + u * step;
      const int x = cx - RB + i % NS, y = cy - RB + i / NS;
      o[u] = 2;
      g[u] = 0;
      cf[u] = 0.0;
      if (i < NS * NS && x >= 0 && x < s.W && y >= 0 && y < s.H) {
        const size_t q = (size_t)y * s.W + x;
        o[u] = __ldcg(&s.omega[q]);
        if (GRAY) g[u] = __ldcg(&s.gray[q]);
        if (CONF) cf[u] = __ldcg(&s.conf[q]);  // read unconditionally, kept for known pixels
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int i = i0 + u * step;
      if (i >= NS * NS) break;
      sm.om[i] = o[u];
      if (GRAY) sm.gr[i] = g[u];
      if (CONF) sm.cf[i] = o[u] ? 0.0 : cf[u];
    }
  }
}

// Isophote candidate at local pixel (lx, ly): eligible when it and its four
// neighbours are known, with its central-difference grey gradient.
template <int R>
__device__ inline void isophote_at(UpdSmem<R>& sm, int lx, int ly) {
  constexpr int NS = UpdGeom<R>::NS;
  const int i = ly * NS + lx;
  int m = -1, g = 0;
  if (lx >= 1 && lx < NS - 1 && ly >= 1 && ly < NS - 1) {
    // all nine reads issued together (no short-circuit chain of loads)
    const int o = sm.om[i] | sm.om[i - 1] | sm.om[i + 1] | sm.om[i - NS] | sm.om[i + NS];
    const int gx = (int)sm.gr[i + 1] - (int)sm.gr[i - 1];
    const int gy = (int)sm.gr[i + NS] - (int)sm.gr[i - NS];
    if (o == 0) {
      m = gx * gx + gy * gy;
      g = ((gx + 512) << 16) | (gy + 512);
    }
  }
  sm.mag[i] = m;
  sm.gxy[i] = g;
}

// Isophote candidates of the whole staged neighbourhood.
template <int R>
__device__ inline void stage_isophotes(UpdSmem<R>& sm) {
  constexpr int NS = UpdGeom<R>::NS;
  for (int i = threadIdx.x; i < NS * NS; i += blockDim.x) isophote_at<R>(sm, i % NS, i / NS);
}

// Isophote candidates of part of the neighbourhood of p^.  The fill of the
// iteration changes grey levels and the mask only inside Psi_p^, so a
// candidate can change only within one pixel of it: in the box of
// Chebyshev radius R + 1 around p^.  kRing false: every candidate outside
// that box (the speculative phase, before the search ends, threads
// [first, blockDim.x)); kRing true: the box itself, from the copied pixels.
template <int R, bool kRing>
__device__ inline void stage_isophotes_part(UpdSmem<R>& sm, int first, int last = -1) {
  constexpr int NS = UpdGeom<R>::NS, RB = UpdGeom<R>::RB, RR = R + 1, NB = 2 * RR + 1;
  constexpr int n = kRing ? NB * NB : NS * NS;
  if (last < 0) last = (int)blockDim.x;
  if ((int)threadIdx.x < first || (int)threadIdx.x >= last) return;
  for (int k = (int)threadIdx.x - first; k < n; k += last - first) {
    if (kRing) {
      isophote_at<R>(sm, RB - RR + k % NB, RB - RR + k / NB);
    } else {
      const int lx = k % NS, ly = k / NS;
      if (abs(lx - RB) > RR || abs(ly - RB) > RR) isophote_at<R>(sm, lx, ly);
    }
  }
}

// stage_isophotes_part<R, false> with the work handed out in chunks of 32
// positions from sm.iso_next (0 on entry): a warp that starts late takes
// fewer.  Whole warps.  No barrier.
template <int R>
__device__ inline void stage_isophotes_dyn(UpdSmem<R>& sm) {
  constexpr int NS = UpdGeom<R>::NS, RB = UpdGeom<R>::RB, RR = R + 1;
  const int lane = threadIdx.x & 31;
  while (true) {
    int base = 0;
    if (lane == 0) base = atomicAdd(&sm.iso_next, 32);
    base = __shfl_sync(0xffffffffu, base, 0);
    if (base >= NS * NS) break;
    const int k = base + lane;
    if (k < NS * NS) {
      const int lx = k % NS, ly = k / NS;
      if (abs(lx - RB) > RR || abs(ly - RB) > RR) isophote_at<R>(sm, lx, ly);
    }
  }
}

__device__ inline bool front_local(const uint8_t* om, int l, int NS) {
  // the five reads are independent (no short-circuit chain of loads)
  const int c = om[l], a = om[l - 1], b = om[l + 1], u = om[l - NS], d = om[l + NS];
  return c == 1 && (a == 0 || b == 0 || u == 0 || d == 0);
}

// Initial priorities, one CTA per NW x NW window of the image (direct
// evaluation of every term).
template <int R>
__global__ void __launch_bounds__(256, 2) k_prio_init_fast(ImgState s) {
  using G = UpdGeom<R>;
  constexpr int RB = G::RB, NS = G::NS, R2 = G::R2, NW = G::NW;
  extern __shared__ __align__(16) uint8_t sm_raw[];
  UpdSmem<R>& sm = *reinterpret_cast<UpdSmem<R>*>(sm_raw);
  const int cx = R2 + blockIdx.x * NW, cy = R2 + blockIdx.y * NW;
  stage_nbhd<R, true, true>(s, cx, cy, sm);
  __syncthreads();
  stage_isophotes<R>(sm);
  __syncthreads();
  for (int i = threadIdx.x; i < NW * NW; i += blockDim.x) {
    const int wx = i % NW - R2, wy = i / NW - R2;
    const int lx = RB + wx, ly = RB + wy, l = ly * NS + lx;
    if (sm.om[l] == 2) continue;
    const int x = cx + wx, y = cy + wy;
    unsigned long long key = 0ull;
    double c = 0.0;
    if (front_local(sm.om, l, NS)) {
      c = conf_local<R>(sm, s, lx, ly, x, y);
      const int nrm = normal_local<R>(sm, s, lx, ly, x, y);
      int gx, gy;
      isophote_local<R>(sm, lx, ly, &gx, &gy);
      const double d = data_term_direct(dot_abs(gx, gy, nrm), nn_of(nrm));
      key = (unsigned long long)__double_as_longlong(__dmul_rn(c, d)) + 1ull;
    }
    const size_t p = (size_t)y * s.W + x;
    s.prio[p] = key;
    s.pconf[p] = c;
  }
}

// Loads what the update phase of target (px, py) reads but the search does
// not change (see UpdCache), with threads [first, blockDim.x).  No barrier.
template <int R>
__device__ void update_prefetch(const ImgState& s, UpdCache<R>& ca, int first, int px, int py) {
  using G = UpdGeom<R>;
  constexpr int R2 = G::R2, NC = G::NC;
  const int W = s.W, H = s.H;
  const int tx0 = max(0, px - R2) / kT0, tx1 = min(W - 1, px + R2) / kT0;
  const int ty0 = max(0, py - R2) / kT0, ty1 = min(H - 1, py + R2) / kT0;
  const int ntx = tx1 - tx0 + 1, nty = ty1 - ty0 + 1;
  const int ux0 = tx0 / kT1, ux1 = tx1 / kT1, uy0 = ty0 / kT1, uy1 = ty1 / kT1;
  const int nux = ux1 - ux0 + 1, nuy = uy1 - uy0 + 1;
  const int n1 = s.t1x * s.t1y;
  if ((int)threadIdx.x < first) return;
  // every load is an asynchronous copy into the cache, all in flight at once
  const int step = (int)blockDim.x - first, t0 = (int)threadIdx.x - first;
  for (int j = t0; j < NC * NC; j += step) {
    const int x = px + j % NC - 2 * R, y = py + j / NC - 2 * R;
    const bool ok = x >= 0 && x < W && y >= 0 && y < H;
    cp_async4(&ca.cnt[j], ok ? &s.count[(size_t)y * s.pitch + x] : s.count, ok);
  }
  {
    const int n = ntx * nty * kT0 * kT0;
    for (int e = t0; e < n; e += step) {
      const int t = e / (kT0 * kT0), j = e % (kT0 * kT0);
      const int x = (tx0 + t % ntx) * kT0 + (j & (kT0 - 1)), y = (ty0 + t / ntx) * kT0 + j / kT0;
      const bool ok = x < W && y < H;
      cp_async8(&ca.tp[e], ok ? &s.prio[(size_t)y * W + x] : s.prio, ok);
    }
  }
  {
    const int n = nux * nuy * kT1 * kT1;
    for (int e = t0; e < n; e += step) {
      const int u = e / (kT1 * kT1), j = e % (kT1 * kT1);
      const int tx = (ux0 + u % nux) * kT1 + (j & (kT1 - 1)), ty = (uy0 + u / nux) * kT1 + j / kT1;
      if (tx < s.t0x && ty < s.t0y) {
        cp_async16(&ca.t0c[e], &s.tiles0[ty * s.t0x + tx]);
      } else {
        ca.t0c[e].key = 0ull;
        ca.t0c[e].idx = 0x7fffffff;
        ca.t0c[e].pad = 0;
      }
    }
  }
  if (n1 <= kT1Cache)
    for (int e = t0; e < n1; e += step) cp_async16(&ca.t1c[e], &s.tiles1[e]);
  cp_async_wait_all();
  if ((int)threadIdx.x == first) {
    ca.tx0 = tx0;
    ca.ty0 = ty0;
    ca.ntx = ntx;
    ca.nty = nty;
    ca.ux0 = ux0;
    ca.uy0 = uy0;
    ca.nux = nux;
    ca.nuy = nuy;
    ca.t1n = n1 <= kT1Cache ? n1 : 0;
  }
}

// Integral image of the filled flags of Psi_p^ (validity-count
// decrements); one warp.
template <int R>
__device__ inline void warp_fsat(UpdSmem<R>& sm) {
  constexpr int P = UpdGeom<R>::P, P1 = P + 1;
  const int lane = threadIdx.x & 31;
  for (int v = lane; v <= P; v += 32) {
    sm.fsat[v] = 0;
    sm.fsat[v * P1] = 0;
  }
  __syncwarp();
  for (int v = lane; v < P; v += 32) {
    int run = 0;
    for (int u = 0; u < P; ++u) {
      run += sm.filled[v * P + u];
      sm.fsat[(v + 1) * P1 + u + 1] = run;
    }
  }
  __syncwarp();
  for (int u = lane + 1; u <= P; u += 32)
    for (int v = 2; v <= P; ++v) sm.fsat[v * P1 + u] += sm.fsat[(v - 1) * P1 + u];
}

// The next iteration's input, once update_phase has selected the next
// target (npx, npy): its neighbourhood, and in sm.nx_* its centre,
// iteration number and confidence C(p^), so that spec_phase(staged = true)
// reads no global control state.  The thread that reads C(p^) also installs
// it in the control block.  Whole block; the caller's barrier makes it
// visible.
template <int R>
__device__ void stage_next(const ImgState& s, int npx, int npy, UpdSmem<R>& sm, double* conf_out = nullptr) {
  const int t_cp = (int)blockDim.x - 1;  // a thread with the fewest staging entries
  double ncp = 0.0;
  if ((int)threadIdx.x == t_cp) ncp = __ldcg(&s.pconf[sm.next_idx]);
  stage_nbhd<R, true, true>(s, npx, npy, sm);
  if ((int)threadIdx.x == t_cp) {
    sm.nx_px = npx;
    sm.nx_py = npy;
    sm.nx_it = sm.it + 1;
    sm.nx_cp = ncp;
    s.ctrl->conf = ncp;
    if (conf_out) *conf_out = ncp;
  }
}

// Speculative phase: post-fill mask, grey levels and confidences of the
// neighbourhood of p^, the filled set and its integral image, the post-fill
// front of the window with its normals and confidence terms.  Everything
// stays in shared memory for update_phase.  Whole block.
// `staged`: the neighbourhood of p^ is already in shared memory (the engine
// stages it while it records the previous iteration).
// Best (key, idx) of the priorities outside the NW x NW window around
// (px, py), from the caches update_prefetch filled: level-1 tiles the window
// does not touch, level-0 tiles it does not touch inside the level-1 tiles
// it does, and the pixels outside it inside the level-0 tiles it touches.
// Those priorities are the ones the fill of this iteration leaves alone.
// Whole block.
template <int R>
__device__ void best_outside_window(const ImgState& s, UpdSmem<R>& sm, const UpdCache<R>& ca, int px,
                                    int py) {
  constexpr int R2 = UpdGeom<R>::R2;
  const int W = s.W;
  unsigned long long k = 0ull;
  int idx = 0x7fffffff;
  const int n1 = s.t1x * s.t1y;
  for (int e = threadIdx.x; e < n1; e += blockDim.x) {
    const int ux = e % s.t1x, uy = e / s.t1x;
    if (ux >= ca.ux0 && ux < ca.ux0 + ca.nux && uy >= ca.uy0 && uy < ca.uy0 + ca.nuy) continue;
    if (ca.t1n) prio_take(k, idx, ca.t1c[e].key, ca.t1c[e].idx);
    else prio_take(k, idx, __ldcg(&s.tiles1[e].key), __ldcg(&s.tiles1[e].idx));
  }
  for (int e = threadIdx.x; e < ca.nux * ca.nuy * kT1 * kT1; e += blockDim.x) {
    const int u = e / (kT1 * kT1), j = e % (kT1 * kT1);
    const int tx = (ca.ux0 + u % ca.nux) * kT1 + (j & (kT1 - 1)), ty = (ca.uy0 + u / ca.nux) * kT1 + j / kT1;
    if (tx >= ca.tx0 && tx < ca.tx0 + ca.ntx && ty >= ca.ty0 && ty < ca.ty0 + ca.nty) continue;
    prio_take(k, idx, ca.t0c[e].key, ca.t0c[e].idx);
  }
  for (int e = threadIdx.x; e < ca.ntx * ca.nty * kT0 * kT0; e += blockDim.x) {
    const int t = e / (kT0 * kT0), j = e % (kT0 * kT0);
    const int x = (ca.tx0 + t % ca.ntx) * kT0 + (j & (kT0 - 1)), y = (ca.ty0 + t / ca.ntx) * kT0 + j / kT0;
    if (x >= W || y >= s.H || (abs(x - px) <= R2 && abs(y - py) <= R2)) continue;
    prio_take(k, idx, ca.tp[e], y * W + x);
  }
  block_best_prio(k, idx, sm.red_pb);  // ends with a __syncthreads
  if (threadIdx.x == 0) {
    sm.out_key = k;
    sm.out_idx = idx;
  }
}

// best_outside_window for the threads [g0, blockDim.x) only (g0 a multiple
// of 32, the group synchronised by named barrier 1): the speculative
// phase's spare warps run it while the other warps' FP64 chains go on.
// Writes sm.out_key / sm.out_idx; a block barrier must follow before they
// are read.
template <int R>
__device__ void best_outside_window_group(const ImgState& s, UpdSmem<R>& sm, const UpdCache<R>& ca, int px,
                                          int py, int g0) {
  constexpr int R2 = UpdGeom<R>::R2;
  const int W = s.W;
  const int nt = (int)blockDim.x - g0, t0 = (int)threadIdx.x - g0;
  // the group's cache loads (update_prefetch) are complete and visible
  asm volatile("bar.sync 1, %0;" ::"r"(nt) : "memory");
  unsigned long long k = 0ull;
  int idx = 0x7fffffff;
  const int n1 = s.t1x * s.t1y;
  for (int e = t0; e < n1; e += nt) {
    const int ux = e % s.t1x, uy = e / s.t1x;
    if (ux >= ca.ux0 && ux < ca.ux0 + ca.nux && uy >= ca.uy0 && uy < ca.uy0 + ca.nuy) continue;
    if (ca.t1n) prio_take(k, idx, ca.t1c[e].key, ca.t1c[e].idx);
    else prio_take(k, idx, __ldcg(&s.tiles1[e].key), __ldcg(&s.tiles1[e].idx));
  }
  for (int e = t0; e < ca.nux * ca.nuy * kT1 * kT1; e += nt) {
    const int u = e / (kT1 * kT1), j = e % (kT1 * kT1);
    const int tx = (ca.ux0 + u % ca.nux) * kT1 + (j & (kT1 - 1)), ty = (ca.uy0 + u / ca.nux) * kT1 + j / kT1;
    if (tx >= ca.tx0 && tx < ca.tx0 + ca.ntx && ty >= ca.ty0 && ty < ca.ty0 + ca.nty) continue;
    prio_take(k, idx, ca.t0c[e].key, ca.t0c[e].idx);
  }
  for (int e = t0; e < ca.ntx * ca.nty * kT0 * kT0; e += nt) {
    const int t = e / (kT0 * kT0), j = e % (kT0 * kT0);
    const int x = (ca.tx0 + t % ca.ntx) * kT0 + (j & (kT0 - 1)), y = (ca.ty0 + t / ca.ntx) * kT0 + j / kT0;
    if (x >= W || y >= s.H || (abs(x - px) <= R2 && abs(y - py) <= R2)) continue;
    prio_take(k, idx, ca.tp[e], y * W + x);
  }
  warp_best_prio(k, idx);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, w0 = g0 >> 5, nw = (int)(blockDim.x >> 5);
  if (lane == 0) {
    sm.red_pb[wid].key = k;
    sm.red_pb[wid].idx = idx;
  }
  asm volatile("bar.sync 1, %0;" ::"r"(nt) : "memory");
  if (wid == w0) {
    unsigned long long kk = w0 + lane < nw ? sm.red_pb[w0 + lane].key : 0ull;
    int ii = w0 + lane < nw ? sm.red_pb[w0 + lane].idx : 0x7fffffff;
    warp_best_prio(kk, ii);
    if (lane == 0) {
      sm.out_key = kk;
      sm.out_idx = ii;
    }
  }
}

// The control-block fields the update phase reads, taken early by a caller
// that knows nothing writes them before the update (the engine's leader
// reads them at the start of its round, so their latency is hidden).
struct CtrlSnap {
  int px, py, n_cand, it, remaining;
  double conf, prio;
};

// The tile maxima of the last update (level-0 tiles of its priority window
// from the cached keys, then their level-1 tiles, in global memory and the
// caches) and the check that the best of the tiles is the target the early
// selection published.  Threads [g0, blockDim.x) (g0 a multiple of 32; named
// barrier 2 when g0 > 0).  Runs before update_prefetch replaces the caches.
template <int R>
__device__ void update_tiles(const ImgState& s, UpdSmem<R>& sm, UpdCache<R>& ca, int g0) {
  const int W = s.W, nt = (int)blockDim.x - g0, t0 = (int)threadIdx.x - g0;
  auto gsync = [&]() {
    if (g0 == 0)
      __syncthreads();
    else
      asm volatile("bar.sync 2, %0;" ::"r"(nt) : "memory");
  };
  const int lane = t0 & 31, wid = t0 >> 5, nw = nt >> 5;
  for (int t = wid; t < ca.ntx * ca.nty; t += nw) {
    const int tx = ca.tx0 + t % ca.ntx, ty = ca.ty0 + t / ca.ntx;
    unsigned long long k = 0ull;
    int idx = 0x7fffffff;
#pragma unroll
    for (int r8 = 0; r8 < kT0 * kT0 / 32; ++r8) {
      const int j = lane + 32 * r8;
      const int x = tx * kT0 + (j & (kT0 - 1)), y = ty * kT0 + j / kT0;
      prio_take(k, idx, ca.tp[t * (kT0 * kT0) + j], y * W + x);
    }
    warp_best_prio(k, idx);
    if (lane == 0) {
      s.tiles0[ty * s.t0x + tx].key = k;
      s.tiles0[ty * s.t0x + tx].idx = idx;
      const int u = (ty / kT1 - ca.uy0) * ca.nux + (tx / kT1 - ca.ux0);
      PrioBest& e = ca.t0c[u * (kT1 * kT1) + (ty & (kT1 - 1)) * kT1 + (tx & (kT1 - 1))];
      e.key = k;
      e.idx = idx;
    }
  }
  gsync();
  for (int u = wid; u < ca.nux * ca.nuy; u += nw) {
    const int ux = ca.ux0 + u % ca.nux, uy = ca.uy0 + u / ca.nux;
    unsigned long long k = 0ull;
    int idx = 0x7fffffff;
#pragma unroll
    for (int r8 = 0; r8 < kT1 * kT1 / 32; ++r8) {
      const PrioBest& e = ca.t0c[u * (kT1 * kT1) + lane + 32 * r8];
      prio_take(k, idx, e.key, e.idx);
    }
    warp_best_prio(k, idx);
    if (lane == 0) {
      s.tiles1[uy * s.t1x + ux].key = k;
      s.tiles1[uy * s.t1x + ux].idx = idx;
      if (ca.t1n) {
        ca.t1c[uy * s.t1x + ux].key = k;
        ca.t1c[uy * s.t1x + ux].idx = idx;
      }
    }
  }
  gsync();
  if (wid == 0 && sm.pend_rem > 0) {
    unsigned long long k = 0ull;
    int idx = 0x7fffffff;
    if (ca.t1n) {
      for (int j = lane; j < ca.t1n; j += 32) prio_take(k, idx, ca.t1c[j].key, ca.t1c[j].idx);
      warp_best_prio(k, idx);
    } else {
      warp_global_best(s, k, idx);
    }
    if (lane == 0 && (k != sm.pend_key || (k != 0ull && idx != sm.pend_idx)))
      s.ctrl->status = INPAINT_ERR_INTERNAL;  // the tiles and the early selection disagree
  }
  gsync();  // every read of the caches is done before they are replaced
  if (t0 == 0) sm.tiles_pending = 0;
}

template <int R>
__device__ void spec_phase(const ImgState& s, UpdSmem<R>& sm, UpdCache<R>& ca, bool staged,
                           bool want_outside = false) {
  using G = UpdGeom<R>;
  constexpr int P = G::P, RB = G::RB, NS = G::NS, R2 = G::R2, NW = G::NW;
  const Ctrl* c = s.ctrl;
  int px, py, it;
  double cp;
  if (staged) {
    px = sm.nx_px;
    py = sm.nx_py;
    it = sm.nx_it;
    cp = sm.nx_cp;
  } else {
    px = __ldcg(&c->px);
    py = __ldcg(&c->py);
    it = __ldcg(&c->iter);
    cp = __ldcg(&c->conf);
    stage_nbhd<R, true, true>(s, px, py, sm);
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    sm.nlist = 0;
    sm.iso_next = 0;
  }
  int my = 0;
  for (int i = threadIdx.x; i < P * P; i += blockDim.x) {
    const int l = (RB + i / P - R) * NS + RB + i % P - R;
    uint8_t f = 0;
    if (sm.om[l] == 1) {
      sm.om[l] = 0;
      sm.cf[l] = cp;
      f = 1;
      ++my;
    }
    sm.filled[i] = f;
  }
  const int filled = block_sum_int(my, sm.red32);  // includes __syncthreads
  // post-fill front of the window, compacted
  for (int i = threadIdx.x; i < NW * NW; i += blockDim.x) {
    const int l = (RB + i / NW - R2) * NS + RB + i % NW - R2;
    int nrm = kSpecOutside;
    if (sm.om[l] != 2) {
      nrm = kSpecNotFront;
      if (front_local(sm.om, l, NS)) sm.list[atomicAdd(&sm.nlist, 1)] = (uint16_t)i;
    }
    sm.snrm[i] = nrm;  // front entries are overwritten below
  }
  __syncthreads();
  const int nfront = sm.nlist;
  // FP64 confidence sums (Eq. 2) by the first warps, warp 4 builds the
  // filled-flag integral image, and warps 0-4 share the isophotes the fill
  // cannot change; the other warps (the spare group) bring the tiles up to
  // date, load the update phase's cache and find the best priority outside
  // the fill's window
  const int nt = (int)blockDim.x;
  const bool spare = nt >= 256;
  if (spare) {
    constexpr int g0 = 160;
    // one dependent row-major chain per front pixel, packed into as few
    // warps as the front needs: up to three warps of chains still run at the
    // 64 cycles of one dependent add, four at 76 (the unit takes a warp
    // instruction about every 19 cycles whatever the active lanes)
    const int cw = nfront <= 96 ? (nfront + 31) >> 5 : 4;
    if ((int)threadIdx.x < 32 * cw) {
      for (int k = threadIdx.x; k < nfront; k += 32 * cw) {
        const int i = sm.list[k];
        const int wx = i % NW - R2, wy = i / NW - R2;
        const int lx = RB + wx, ly = RB + wy, x = px + wx, y = py + wy;
        sm.sC[i] = conf_local<R>(sm, s, lx, ly, x, y);
        sm.snrm[i] = normal_local<R>(sm, s, lx, ly, x, y);
      }
    } else if ((int)(threadIdx.x >> 5) == 4) {
      warp_fsat<R>(sm);
    }
    if ((int)threadIdx.x >= g0) {
      if (want_outside && sm.tiles_pending) update_tiles<R>(s, sm, ca, g0);
      update_prefetch<R>(s, ca, g0, px, py);
      if (want_outside) best_outside_window_group<R>(s, sm, ca, px, py, g0);
    } else {
      // the warps without chains at once, the chain warps when done
      stage_isophotes_dyn<R>(sm);
    }
  } else {
    for (int k = threadIdx.x; k < nfront; k += nt) {
      const int i = sm.list[k];
      const int wx = i % NW - R2, wy = i / NW - R2;
      const int lx = RB + wx, ly = RB + wy, x = px + wx, y = py + wy;
      sm.sC[i] = conf_local<R>(sm, s, lx, ly, x, y);
      sm.snrm[i] = normal_local<R>(sm, s, lx, ly, x, y);
    }
    if (threadIdx.x < 32) warp_fsat<R>(sm);
    if (want_outside && sm.tiles_pending) update_tiles<R>(s, sm, ca, 0);
    update_prefetch<R>(s, ca, 0, px, py);
    stage_isophotes_part<R, false>(sm, 0);
  }
  if (threadIdx.x == 0) {
    sm.nfront = nfront;
    sm.spec_iter = it;
    sm.spec_filled = filled;
  }
  __syncthreads();
  if (want_outside && !spare) {
    best_outside_window<R>(s, sm, ca, px, py);
    __syncthreads();
  }
}

// Early selection (persistent engine, resident mode): the next target is
// the better of the best new priority in the window and the best one
// outside it (found by spec_phase), so it is published as soon as the
// window's priorities are known; the tile maxima are brought up to date
// after the publication, off the searchers' path.
struct EarlySel {
  unsigned long long* pub;  // the team's publication word; nullptr: select through the tiles first
  unsigned epoch;           // epoch of the round being applied
  bool allow;               // no iteration limit, status or error stops the loop after this one
  unsigned long long tick_ns, t_start;  // the launch's time budget (0: none) and start
  unsigned* expired;        // set when the time budget stops the loop
  int pub_thread;
  bool published;           // out (every thread): the next round (or the stop) went out
};

__device__ inline unsigned long long pub_word(unsigned epoch, int px, int py, bool stop) {
  return (unsigned long long)epoch | ((unsigned long long)(px & 0x7fff) << 32) |
         ((unsigned long long)(py & 0x7fff) << 47) | ((unsigned long long)(stop ? 1 : 0) << 62);
}

// Update phase: applies the iteration whose best source key is *best_in, or
// the minimum of partial[0..n_partial), on the state prepared by spec_phase and
// update_prefetch.  Returns false (status written) when there is no source
// patch or the state is inconsistent.  Whole block; ends with a __syncthreads.
// Thread `fence_thread` (if any) issues a gpu-scope fence once the pixel,
// mask and count writes of the iteration are issued (see the engine's
// publication).  `overlap_counts`: the search was the partial-overlap variant,
// whose admissible candidates it counted in ctrl->n_adm.
template <int R>
__device__ bool update_phase(const ImgState& s, const unsigned long long* partial, int n_partial,
                             UpdSmem<R>& sm, UpdCache<R>& ca, int fence_thread = -1,
                             bool overlap_counts = false, const unsigned long long* best_in = nullptr,
                             EarlySel* es = nullptr, unsigned* copied = nullptr, unsigned copied_val = 0u,
                             const CtrlSnap* snap = nullptr) {
  using G = UpdGeom<R>;
  constexpr int P = G::P, RB = G::RB, NS = G::NS, R2 = G::R2, NW = G::NW, NC = G::NC;
  Ctrl* c = s.ctrl;
  const int tid = threadIdx.x, nt = blockDim.x;

  // best source key: given (already reduced, in shared memory), or the
  // minimum of the partial keys in global memory
  unsigned long long best = ~0ull;
  if (best_in) {
    best = *best_in;
  } else {
    for (int i = tid; i < n_partial; i += nt) {
      const unsigned long long v = __ldcg(&partial[i]);
      best = v < best ? v : best;
    }
    best = block_min_u64(best, sm.red64);
  }
  if (best == ~0ull) {
    if (tid == 0) c->status = INPAINT_ERR_NO_SOURCE;
    __syncthreads();
    return false;
  }
  // The iteration's scalars go to shared memory once (they are also the
  // record update_finish writes): each phase below reads the ones it needs,
  // so that none stays in a register across the phases.  A spilled one
  // would come back from L2, since local memory misses the L1 that the
  // shared memory leaves nearly empty.  Candidates of this iteration's
  // search: the validity-count total, or the admissible ones the
  // partial-overlap search counted.
  if (tid == 0) {
    const int px = snap ? snap->px : __ldcg(&c->px), py = snap ? snap->py : __ldcg(&c->py);
    const int it = snap ? snap->it : __ldcg(&c->iter);
    const int filled = sm.spec_filled, q = (int)(best & 0xffffffffull), W = s.W, H = s.H;
    sm.px = px;
    sm.py = py;
    sm.cp = snap ? snap->conf : __ldcg(&c->conf);
    sm.pp = snap ? snap->prio : __ldcg(&c->prio);
    sm.n_cand = snap ? snap->n_cand : overlap_counts ? __ldcg(&c->n_adm) : __ldcg(&c->n_valid);
    sm.it = it;
    sm.n_filled = filled;
    sm.remaining = (snap ? snap->remaining : __ldcg(&c->remaining)) - filled;
    sm.qx = q % W;
    sm.qy = q / W;
    sm.ssd = (uint32_t)(best >> 32);
    sm.n_known = (min(px + R, W - 1) - max(px - R, 0) + 1) * (min(py + R, H - 1) - max(py - R, 0) + 1) - filled;
    sm.newly = 0;
    sm.upd_ok = filled != 0 && sm.spec_iter == it;
  }
  __syncthreads();
  if (!sm.upd_ok) {
    if (tid == 0) c->status = INPAINT_ERR_INTERNAL;  // p^ not in Omega, or stale speculation
    __syncthreads();
    return false;
  }
  // the window's keys before this update (every key of the cached level-0
  // tiles, from update_prefetch); a front pixel's key is never 0
  auto cache_key = [&](int x, int y) -> unsigned long long& {
    const int t = (y / kT0 - ca.ty0) * ca.ntx + (x / kT0 - ca.tx0);
    return ca.tp[t * (kT0 * kT0) + (y & (kT0 - 1)) * kT0 + (x & (kT0 - 1))];
  };

  // one pass over: the copy of the unknown in-image part of Psi_p^ from
  // Psi_q~ (first, so that its loads go out at once), the validity counts of
  // the candidates the fill touches (they depend on the filled pixels only),
  // and key 0 for the window's pixels off the new front; everything the next
  // search reads is written here, before the fence below
  {
    const int px = sm.px, py = sm.py, qx = sm.qx, qy = sm.qy, W = s.W, H = s.H;
    const double cp = sm.cp;
    int newly = 0;
    for (int t = tid; t < P * P + NC * NC + NW * NW; t += nt) {
      if (t < P * P) {
        const int i = t;
        if (!sm.filled[i]) continue;
        const int dy = i / P - R, dx = i % P - R;
        const int l = (RB + dy) * NS + RB + dx;
        const int tx = px + dx, ty = py + dy;
        const uint32_t w = __ldcg(&s.img[(size_t)(qy + dy) * s.pitch + qx + dx]);
        const uint8_t g = (uint8_t)luma_word(w);
        const size_t q = (size_t)ty * W + tx;
        s.img[(size_t)ty * s.pitch + tx] = w;
        if (s.planes) plane_store(s, tx, ty, w);  // the tensor-core search's operands
        s.gray[q] = g;
        s.conf[q] = cp;
        s.omega[q] = 0;
        sm.gr[l] = g;
      } else if (t < P * P + NC * NC) {
        const int j = t - P * P;
        const int wy = j / NC - 2 * R, wx = j % NC - 2 * R;
        const int x = px + wx, y = py + wy;
        if (x < 0 || x >= W || y < 0 || y >= H) continue;
        const int u0 = max(0, wx), u1 = min(P - 1, wx + 2 * R);
        const int v0 = max(0, wy), v1 = min(P - 1, wy + 2 * R);
        constexpr int P1 = P + 1;
        const int dec = sm.fsat[(v1 + 1) * P1 + u1 + 1] - sm.fsat[v0 * P1 + u1 + 1] -
                        sm.fsat[(v1 + 1) * P1 + u0] + sm.fsat[v0 * P1 + u0];
        if (dec) {
          const int nv = ca.cnt[j] - dec;
          s.count[(size_t)y * s.pitch + x] = nv;
          if (nv == 0 && x >= s.cx0 && x <= s.cx1 && y >= s.cy0 && y <= s.cy1) ++newly;
        }
      } else {
        const int i = t - P * P - NC * NC;
        if (sm.snrm[i] != kSpecNotFront) continue;  // outside, or a front pixel
        const int x = px + i % NW - R2, y = py + i / NW - R2;
        unsigned long long& ck = cache_key(x, y);
        if (ck == 0ull) continue;  // not on the old front: key and C are 0 already
        const size_t p = (size_t)y * W + x;
        s.prio[p] = 0ull;
        s.pconf[p] = 0.0;
        ck = 0ull;
      }
    }
    if (newly) atomicAdd(&sm.newly, newly);
  }
  __syncthreads();
  const int fthread = fence_thread >= 0 ? fence_thread : copied ? 0 : -1;
  if (tid == fthread) {
    // every write the next search reads (pixels, planes, mask, counts) is
    // issued; the barrier above orders the other threads' ones before this
    // fence, which also serves the thread's later publication of the next
    // round.  The fence thread has no isophote or row-maximum work below, so
    // its wait overlaps them.  Then the searchers may prefetch the next
    // round's first source rows.
    asm volatile("fence.acq_rel.gpu;" ::: "memory");
    if (copied) asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(copied), "r"(copied_val) : "memory");
  }

  // isophotes of the new grey levels (the ones the fill cannot change were
  // computed by the speculative phase), then for every front pixel the
  // strongest one of its patch (first in row-major order on ties) as a
  // separable windowed maximum of keys (|grad|^2 + 1) << 12 | (4095 - l) over
  // local indices l: rows here, columns in the priority loop below; the
  // confidence array is free here and holds the row maxima
  stage_isophotes_part<R, true>(sm, 0);
  __syncthreads();
  constexpr int HR = NW + 2 * R;  // rows of the horizontal pass
  uint32_t* hkey = reinterpret_cast<uint32_t*>(sm.cf);
  static_assert(sizeof(sm.cf) >= sizeof(uint32_t) * HR * NW, "key scratch");
  static_assert(NS * NS <= 4096, "local index fits in 12 bits");
  const int nhk = nt >= 512 ? nt - 32 : nt;  // the last warp (the fence thread's) sits out
  for (int i = tid; i < HR * NW && tid < nhk; i += nhk) {
    const int ly = RB - R2 - R + i / NW, lx = RB - R2 + i % NW;
    uint32_t best = 0u;
#pragma unroll
    for (int dx = -R; dx <= R; ++dx) {
      const int l = ly * NS + lx + dx;
      const int m = sm.mag[l];
      const uint32_t key = m >= 0 ? ((uint32_t)(m + 1) << 12) | (uint32_t)(4095 - l) : 0u;
      best = key > best ? key : best;
    }
    hkey[i] = best;
  }
  __syncthreads();

  // priorities of the new front (from the compact list, spread over the
  // sub-partitions); the new keys also go to the cached level-0 tiles
  unsigned long long wk = 0ull;  // best new key of the window (early selection)
  int wi = 0x7fffffff;
  {
    const int px = sm.px, py = sm.py, W = s.W, nfront = sm.nfront;
    const int nlist = (nfront + 127) & ~127;
    for (int t = tid; t < nlist; t += nt) {
      const int k = list_entry(t);
      if (k >= nfront) continue;
      const int i = sm.list[k];
      const int wx = i % NW - R2, wy = i / NW - R2;
      int gx, gy;
      uint32_t ik = 0u;  // column maximum of the row maxima
  #pragma unroll
      for (int dy = 0; dy <= 2 * R; ++dy) {
        const uint32_t key = hkey[(i / NW + dy) * NW + i % NW];
        ik = key > ik ? key : ik;
      }
      gx = 0;
      gy = 0;
      if (ik) {
        const int g = sm.gxy[4095 - (int)(ik & 4095u)];
        gx = (g >> 16) - 512;
        gy = (g & 0xffff) - 512;
      }
      const double cc = sm.sC[i];
      const int nrm = sm.snrm[i];
      const double d = data_term_known(sm, dot_abs(gx, gy, nrm), nn_of(nrm));
      const int x = px + wx, y = py + wy;
      const size_t p = (size_t)y * W + x;
      const unsigned long long key = (unsigned long long)__double_as_longlong(__dmul_rn(cc, d)) + 1ull;
      s.prio[p] = key;
      s.pconf[p] = cc;
      cache_key(x, y) = key;
      prio_take(wk, wi, key, (int)p);
    }
  }
  const bool early = es && es->pub;
  if (early) {
    // the next target: the better of the window's best and the best outside
    // it; published now unless the loop stops, in which case the stop goes
    // out (the publishing thread is the fence thread: its fence after the
    // copy makes this store a release of everything the search reads)
    block_best_prio(wk, wi, sm.red_pb);  // every thread gets the window's best
    prio_take(wk, wi, sm.out_key, sm.out_idx);
    if ((int)threadIdx.x == es->pub_thread) {
      bool st = sm.remaining <= 0 || wk == 0ull || !es->allow;
      if (!st && es->tick_ns && globaltimer() - es->t_start > es->tick_ns) {
        st = true;  // the launch's time budget is spent: resume in the next launch
        *es->expired = 1u;
      }
      const int W = s.W;
      asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(es->pub),
                   "l"(pub_word(es->epoch + 1u, st ? 0 : wi % W, st ? 0 : wi / W, st))
                   : "memory");
      sm.early_stop = st;
    }
    es->published = true;
    // the outcome is known: the tile maxima and the check of this selection
    // are left to the next speculative phase's spare warps
    if (tid == 0) {
      const int rem = sm.remaining;
      sm.next_key = rem > 0 ? wk : 0ull;
      sm.next_idx = wi;
      sm.pend_key = wk;
      sm.pend_idx = wi;
      sm.pend_rem = rem;
      sm.tiles_pending = 1;
    }
    __syncthreads();
    return true;
  }
  __syncthreads();  // the priority loop's cache writes before the tiles read them

  // level-0 tiles from the cached keys, then level-1, then the best
  const int lane = tid & 31, wid = tid >> 5, nw = nt >> 5;
  for (int t = wid; t < ca.ntx * ca.nty; t += nw) {
    const int tx = ca.tx0 + t % ca.ntx, ty = ca.ty0 + t / ca.ntx;
    unsigned long long k = 0ull;
    int idx = 0x7fffffff;
#pragma unroll
    for (int r8 = 0; r8 < kT0 * kT0 / 32; ++r8) {
      const int j = lane + 32 * r8;
      const int x = tx * kT0 + (j & (kT0 - 1)), y = ty * kT0 + j / kT0;
      const unsigned long long kk = ca.tp[t * (kT0 * kT0) + j];
      const int ii = y * s.W + x;
      prio_take(k, idx, kk, ii);
    }
    warp_best_prio(k, idx);
    if (lane == 0) {
      s.tiles0[ty * s.t0x + tx].key = k;
      s.tiles0[ty * s.t0x + tx].idx = idx;
      const int u = (ty / kT1 - ca.uy0) * ca.nux + (tx / kT1 - ca.ux0);
      PrioBest& e = ca.t0c[u * (kT1 * kT1) + (ty & (kT1 - 1)) * kT1 + (tx & (kT1 - 1))];
      e.key = k;
      e.idx = idx;
    }
  }
  __syncthreads();
  for (int u = wid; u < ca.nux * ca.nuy; u += nw) {
    const int ux = ca.ux0 + u % ca.nux, uy = ca.uy0 + u / ca.nux;
    unsigned long long k = 0ull;
    int idx = 0x7fffffff;
#pragma unroll
    for (int r8 = 0; r8 < kT1 * kT1 / 32; ++r8) {
      const PrioBest& e = ca.t0c[u * (kT1 * kT1) + lane + 32 * r8];
      prio_take(k, idx, e.key, e.idx);
    }
    warp_best_prio(k, idx);
    if (lane == 0) {
      s.tiles1[uy * s.t1x + ux].key = k;
      s.tiles1[uy * s.t1x + ux].idx = idx;
      if (ca.t1n) {
        ca.t1c[uy * s.t1x + ux].key = k;
        ca.t1c[uy * s.t1x + ux].idx = idx;
      }
    }
  }
  __syncthreads();
  {
    // every warp takes the same decision: a lone warp running while the
    // others wait at the barrier was several times slower here
    unsigned long long k = 0ull;
    int idx = 0x7fffffff;
    if (sm.remaining > 0) {
      if (ca.t1n) {
        for (int j = lane; j < ca.t1n; j += 32) prio_take(k, idx, ca.t1c[j].key, ca.t1c[j].idx);
        warp_best_prio(k, idx);
      } else {
        warp_global_best(s, k, idx);
      }
    }
    if (tid == 0) {
      sm.next_key = k;
      sm.next_idx = idx;
    }
  }
  __syncthreads();
  return true;
}

// Records the iteration applied by update_phase (trace, counters) and
// installs the next target p^ with its priority and confidence in the
// control block (stage_next has installed the confidence when
// `cp_staged`).  Neither the image state nor the tiles change here, so the
// persistent engine publishes the next target to its searchers first.
// Whole block; ends with a __syncthreads.
template <int R>
__device__ void update_finish(const ImgState& s, const UpdSmem<R>& sm, bool cp_staged,
                              bool overlap_counts = false, CtrlSnap* next_snap = nullptr) {
  Ctrl* c = s.ctrl;
  const bool next = sm.remaining > 0 && sm.next_key != 0ull;
  if (threadIdx.x == 0) {
    // the record is built in registers: no global read-backs on the
    // leader's critical path
    inpaint_step_info e;
    e.iter = sm.it;
    e.px = sm.px;
    e.py = sm.py;
    e.qx = sm.qx;
    e.qy = sm.qy;
    e.ssd = sm.ssd;
    e.priority = sm.pp;
    e.confidence = sm.cp;
    e.filled = sm.n_filled;
    e.remaining = sm.remaining;
    e.n_known = sm.n_known;
    e.n_cand = sm.n_cand;
    c->last = e;
    if (sm.it < s.trace_cap) s.trace[sm.it] = e;
    c->remaining = sm.remaining;
    c->iter = sm.it + 1;
    c->n_valid = sm.n_cand + sm.newly;
    if (next_snap) {
      next_snap->remaining = sm.remaining;
      next_snap->it = sm.it + 1;
      next_snap->n_cand = sm.n_cand + sm.newly;
    }
    if (overlap_counts) c->n_adm = 0;  // the next search counts afresh
    atomicAdd(&c->evals, (unsigned long long)sm.n_cand * (unsigned long long)sm.n_known);
    if (!next) {
      c->px = -1;
      c->py = -1;
      if (sm.remaining > 0) c->status = INPAINT_ERR_INTERNAL;  // Omega non-empty but no front
    }
  }
  if (next && (int)threadIdx.x == (blockDim.x > 32 ? 32 : 0)) {
    // the next target, from another warp (its confidence is a global read)
    const double prio = __longlong_as_double((long long)(sm.next_key - 1ull));
    c->px = sm.next_idx % s.W;
    c->py = sm.next_idx / s.W;
    c->prio = prio;
    if (!cp_staged) {
      const double conf = __ldcg(&s.pconf[sm.next_idx]);
      c->conf = conf;
      if (next_snap) next_snap->conf = conf;  // (staged: stage_next wrote it)
    }
    if (next_snap) {
      next_snap->px = sm.next_idx % s.W;
      next_snap->py = sm.next_idx / s.W;
      next_snap->prio = prio;
    }
  }
  __syncthreads();
}

}  // namespace inp
