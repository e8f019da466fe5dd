// Initialisation, priority and copy/update kernels of the fill loop.
//
// Sec. 3 of the paper: the fill front dOmega, the priority P(p) = C(p) D(p)
// (Eq. 1-2), the copy of the best source patch into the unknown part of the
// target patch, and the confidence update.  Table 2 lists these as the grey
// conversion, border update, source marking, priority and confidence updates
// and the RGB/grey update; here they are: one init pass per image, then one
// single-CTA update kernel per iteration that touches only the neighbourhood
// of the filled patch.
//
// Bit-exactness of the FP64 priority: the library is compiled with
// --fmad=false, the confidence sum runs in row-major patch order (dy outer,
// dx inner) in one thread, and division/sqrt use the IEEE round-to-nearest
// intrinsics, so each value equals the single-threaded CPU evaluation of the
// same expression.
#include "inpaint_internal.cuh"

namespace inp {

// ---------------------------------------------------------------- priority

__device__ inline bool known_px(const ImgState& s, int x, int y) {
  return x >= 0 && x < s.W && y >= 0 && y < s.H && s.omega[(size_t)y * s.W + x] == 0;
}

__device__ inline int omega_clamped(const ImgState& s, int x, int y) {
  x = x < 0 ? 0 : (x >= s.W ? s.W - 1 : x);
  y = y < 0 ? 0 : (y >= s.H ? s.H - 1 : y);
  return s.omega[(size_t)y * s.W + x] ? 1 : 0;
}

// Fill front membership: p in Omega with an in-image 4-neighbour in Phi.
__device__ inline bool on_front(const ImgState& s, int x, int y) {
  if (s.omega[(size_t)y * s.W + x] == 0) return false;
  return known_px(s, x - 1, y) || known_px(s, x + 1, y) || known_px(s, x, y - 1) ||
         known_px(s, x, y + 1);
}

// P(p) of Eq. 1 with C(p), D(p) of Eq. 2; writes C(p) to *c_out.
__device__ double priority_at(const ImgState& s, int x, int y, double* c_out) {
  const int W = s.W, H = s.H, r = s.r;
  // Confidence term: known part of Psi_p over its in-image area, summed in
  // row-major order.
  double sum = 0.0;
  int n_in = 0;
  for (int dy = -r; dy <= r; ++dy) {
    const int qy = y + dy;
    if (qy < 0 || qy >= H) continue;
    for (int dx = -r; dx <= r; ++dx) {
      const int qx = x + dx;
      if (qx < 0 || qx >= W) continue;
      ++n_in;
      const size_t q = (size_t)qy * W + qx;
      if (s.omega[q] == 0) sum = __dadd_rn(sum, s.conf[q]);
    }
  }
  const double c = __ddiv_rn(sum, (double)n_in);

  // Normal to the front: Sobel of the Omega indicator (replicated borders).
  const int m_lu = omega_clamped(s, x - 1, y - 1), m_cu = omega_clamped(s, x, y - 1);
  const int m_ru = omega_clamped(s, x + 1, y - 1), m_lc = omega_clamped(s, x - 1, y);
  const int m_rc = omega_clamped(s, x + 1, y), m_ld = omega_clamped(s, x - 1, y + 1);
  const int m_cd = omega_clamped(s, x, y + 1), m_rd = omega_clamped(s, x + 1, y + 1);
  const int nx = (m_ru + 2 * m_rc + m_rd) - (m_lu + 2 * m_lc + m_ld);
  const int ny = (m_ld + 2 * m_cd + m_rd) - (m_lu + 2 * m_cu + m_ru);

  // Isophote: strongest central-difference grey gradient among pixels of
  // Psi_p whose four neighbours are known (first in row-major order on ties).
  int best = -1, gx = 0, gy = 0;
  for (int dy = -r; dy <= r; ++dy) {
    const int qy = y + dy;
    if (qy < 1 || qy >= H - 1) continue;
    for (int dx = -r; dx <= r; ++dx) {
      const int qx = x + dx;
      if (qx < 1 || qx >= W - 1) continue;
      const size_t q = (size_t)qy * W + qx;
      if (s.omega[q] | s.omega[q - 1] | s.omega[q + 1] | s.omega[q - W] | s.omega[q + W]) continue;
      const int tx = (int)s.gray[q + 1] - (int)s.gray[q - 1];
      const int ty = (int)s.gray[q + W] - (int)s.gray[q - W];
      const int mag = tx * tx + ty * ty;
      if (mag > best) {
        best = mag;
        gx = tx;
        gy = ty;
      }
    }
  }
  int dot = (-gy) * nx + gx * ny;
  dot = dot < 0 ? -dot : dot;
  const int nn = nx * nx + ny * ny;
  double d = 0.0;
  if (nn != 0) d = __ddiv_rn(__ddiv_rn((double)dot, __dsqrt_rn((double)nn)), 510.0);
  *c_out = c;
  return __dmul_rn(c, d);
}

__device__ inline void eval_pixel(const ImgState& s, int x, int y) {
  const size_t i = (size_t)y * s.W + x;
  unsigned long long key = 0ull;
  double c = 0.0;
  if (on_front(s, x, y)) {
    const double p = priority_at(s, x, y, &c);
    key = (unsigned long long)__double_as_longlong(p) + 1ull;
  }
  s.prio[i] = key;
  s.pconf[i] = c;
}

// ---------------------------------------------------------------- init

__global__ void k_ctrl_init(Ctrl* c) {
  c->iter = 0;
  c->remaining = 0;
  c->status = 0;
  c->px = -1;
  c->py = -1;
  c->n_valid = 0;
  c->iter_limit = 0x7fffffff;
  c->n_adm = 0;
  c->prio = 0.0;
  c->conf = 0.0;
  c->evals = 0ull;
  c->t_search = 0ull;
  c->t_update = 0ull;
  c->t_last = 0ull;
  c->timed_iters = 0;
  c->tc_rounds = 0;
}

// RGB (or RGBA words) + mask -> packed state; counts |Omega|.
__global__ void k_unpack(ImgState s, const uint8_t* rgb, int rgb_stride, const uint8_t* mask,
                         int mask_stride, const double* conf_in) {
  __shared__ int scratch[32];
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y;
  int om = 0;
  if (x < s.W) {
    const uint8_t* p = rgb + (size_t)y * rgb_stride + 3 * (size_t)x;
    const uint32_t w = pack_rgb(p[0], p[1], p[2]);
    const size_t i = (size_t)y * s.W + x;
    om = mask[(size_t)y * mask_stride + x] != 0;
    s.img[(size_t)y * s.pitch + x] = w;
    s.omega[i] = (uint8_t)om;
    s.gray[i] = om ? 0 : (uint8_t)luma_word(w);
    s.conf[i] = om ? 0.0 : (conf_in ? conf_in[i] : 1.0);
  }
  const int tot = block_sum_int(om, scratch);
  if (threadIdx.x == 0 && tot) atomicAdd(&s.ctrl->remaining, tot);
}

// Integral image of Omega: sat[y][x] = #Omega in [0,x) x [0,y), (W+1) x (H+1).
// Pass 1: prefix along each row (one warp per row).  Pass 2: prefix down each
// column within chunks of kSatChunk rows.  Pass 3: exclusive prefix of the
// chunk totals per column.  Pass 4: add each chunk's offset.
constexpr int kSatChunk = 64;

__global__ void k_sat_rows(ImgState s, int32_t* sat) {
  const int lane = threadIdx.x & 31;
  const int y = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (y > s.H) return;
  const int W1 = s.W + 1;
  int32_t* row = sat + (size_t)y * W1;
  if (y == 0) {
    for (int x = lane; x < W1; x += 32) row[x] = 0;
    return;
  }
  const uint8_t* om = s.omega + (size_t)(y - 1) * s.W;
  if (lane == 0) row[0] = 0;
  int carry = 0;
  for (int base = 0; base < s.W; base += 32) {
    const int x = base + lane;
    int v = x < s.W ? (int)om[x] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, v, o);
      if (lane >= o) v += t;
    }
    v += carry;
    if (x < s.W) row[x + 1] = v;
    carry = __shfl_sync(0xffffffffu, v, 31);
  }
}

__global__ void k_sat_cols_chunk(ImgState s, int32_t* sat, int32_t* tot) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int ch = blockIdx.y;
  if (x >= s.W) return;
  const int W1 = s.W + 1;
  const int y0 = 1 + ch * kSatChunk, y1 = min(s.H, ch * kSatChunk + kSatChunk);
  int run = 0;
  for (int y = y0; y <= y1; ++y) {
    int32_t* p = sat + (size_t)y * W1 + x + 1;
    run += *p;
    *p = run;
  }
  tot[(size_t)ch * s.W + x] = run;
}

__global__ void k_sat_chunk_prefix(ImgState s, int32_t* tot, int nchunks) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= s.W) return;
  int run = 0;
  for (int ch = 0; ch < nchunks; ++ch) {
    int32_t* p = tot + (size_t)ch * s.W + x;
    const int v = *p;
    *p = run;
    run += v;
  }
}

__global__ void k_sat_cols_apply(ImgState s, int32_t* sat, const int32_t* tot) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y + 1 + kSatChunk;  // the first chunk needs no offset
  if (x >= s.W || y > s.H) return;
  const int ch = (y - 1) / kSatChunk;
  sat[(size_t)y * (s.W + 1) + x + 1] += tot[(size_t)ch * s.W + x];
}

__device__ inline bool in_rect(const ImgState& s, int x, int y) {
  return x >= s.cx0 && x <= s.cx1 && y >= s.cy0 && y <= s.cy1;
}

// Unknown count per candidate centre from the integral image; counts the
// valid centres inside the search rectangle.
__global__ void k_count(ImgState s, const int32_t* sat) {
  __shared__ int scratch[32];
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y;
  const int r = s.r, W1 = s.W + 1;
  int valid = 0;
  if (x < s.W) {
    int cnt = kCountInvalid;
    if (x - r >= 0 && x + r < s.W && y - r >= 0 && y + r < s.H) {
      const size_t a = (size_t)(y - r) * W1, b = (size_t)(y + r + 1) * W1;
      cnt = sat[b + x + r + 1] - sat[a + x + r + 1] - sat[b + x - r] + sat[a + x - r];
    }
    s.count[(size_t)y * s.pitch + x] = cnt;
    valid = (cnt == 0 && in_rect(s, x, y)) ? 1 : 0;
  } else if (x < s.pitch) {
    s.count[(size_t)y * s.pitch + x] = kCountInvalid;  // row padding
  }
  const int tot = block_sum_int(valid, scratch);
  if (threadIdx.x == 0 && tot) atomicAdd(&s.ctrl->n_valid, tot);
}

__global__ void k_prio_all(ImgState s) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y;
  if (x < s.W) eval_pixel(s, x, y);
}

// Level-0 tiles from the pixel keys, then level-1 tiles: one warp per tile.
__global__ void k_tiles0_all(ImgState s) {
  const int t = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (t < s.t0x * s.t0y) warp_rescan_t0(s, t % s.t0x, t / s.t0x);
}

__global__ void k_tiles1_all(ImgState s) {
  const int t = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (t < s.t1x * s.t1y) warp_rescan_t1(s, t % s.t1x, t / s.t1x);
}

// ---------------------------------------------------------------- update

struct UpdSmem {
  uint8_t filled[(2 * kMaxRadius + 1) * (2 * kMaxRadius + 1)];
  int32_t fsat[(2 * kMaxRadius + 2) * (2 * kMaxRadius + 2)];
  PrioBest pb[32];
  unsigned long long u64s[32];
  int ints[32];
};

// One iteration's copy/update and the selection of the next target patch.
// Single CTA.  With do_fill == 0 only the selection runs (initialisation).
__global__ void __launch_bounds__(kUpdThreads) k_update(ImgState s, int do_fill,
                                                       cudaGraphConditionalHandle cond,
                                                       int use_cond) {
  __shared__ UpdSmem sm;
  Ctrl* c = s.ctrl;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int W = s.W, H = s.H, r = s.r, P = 2 * r + 1;
  if (!loop_active(c)) {
    if (use_cond && tid == 0) cudaGraphSetConditional(cond, 0);
    return;
  }
  int remaining = c->remaining;
  if (do_fill) {
    // findBestPatch result: lowest (SSD << 32 | idx) over all search CTAs.
    unsigned long long best = ~0ull;
    for (int i = tid; i < s.n_partial; i += nt) {
      const unsigned long long v = s.partial[i];
      best = v < best ? v : best;
    }
    best = block_min_u64(best, sm.u64s);
    if (best == ~0ull) {  // no fully-known source patch: leave the state as is
      if (tid == 0) {
        c->status = INPAINT_ERR_NO_SOURCE;
        if (use_cond) cudaGraphSetConditional(cond, 0);
      }
      return;
    }
    const uint32_t ssd = (uint32_t)(best >> 32);
    const int q = (int)(best & 0xffffffffull);
    const int qx = q % W, qy = q / W;
    const int px = c->px, py = c->py;
    const double cp = c->conf, pp = c->prio;
    const int n_cand = c->n_valid;

    // Copy Psi_q~ into the unknown in-image part of Psi_p^; those pixels
    // take confidence C(p^) and leave Omega.  Sources are known pixels, so
    // they are never written here.
    int my_filled = 0;
    for (int i = tid; i < P * P; i += nt) {
      const int dy = i / P - r, dx = i % P - r;
      const int tx = px + dx, ty = py + dy;
      uint8_t f = 0;
      if (tx >= 0 && tx < W && ty >= 0 && ty < H) {
        const size_t t = (size_t)ty * W + tx;
        if (s.omega[t]) {
          const uint32_t w = s.img[(size_t)(qy + dy) * s.pitch + qx + dx];
          s.img[(size_t)ty * s.pitch + tx] = w;
          if (s.planes) plane_store(s, tx, ty, w);
          s.gray[t] = (uint8_t)luma_word(w);
          s.conf[t] = cp;
          s.omega[t] = 0;
          f = 1;
          ++my_filled;
        }
      }
      sm.filled[i] = f;
    }
    const int filled = block_sum_int(my_filled, sm.ints);  // has __syncthreads
    const int nx_in = min(px + r, W - 1) - max(px - r, 0) + 1;
    const int ny_in = min(py + r, H - 1) - max(py - r, 0) + 1;
    const int n_known = nx_in * ny_in - filled;

    // Integral image of the filled flags over the patch, in shared memory.
    const int P1 = P + 1;
    for (int v = tid; v <= P; v += nt) {
      sm.fsat[v] = 0;           // row 0
      sm.fsat[v * P1] = 0;      // column 0
    }
    __syncthreads();
    for (int v = tid; v < P; v += nt) {
      int run = 0;
      for (int u = 0; u < P; ++u) {
        run += sm.filled[v * P + u];
        sm.fsat[(v + 1) * P1 + u + 1] = run;
      }
    }
    __syncthreads();
    for (int u = tid + 1; u <= P; u += nt)
      for (int v = 2; v <= P; ++v) sm.fsat[v * P1 + u] += sm.fsat[(v - 1) * P1 + u];
    __syncthreads();

    // Validity map: every centre within 2r of p^ loses the filled pixels of
    // its patch from its unknown count.
    const int side = 4 * r + 1;
    int newly = 0;
    for (int j = tid; j < side * side; j += nt) {
      const int wy = j / side - 2 * r, wx = j % side - 2 * r;
      const int x = px + wx, y = py + wy;
      if (x < 0 || x >= W || y < 0 || y >= H) continue;
      const int u0 = max(0, wx), u1 = min(P - 1, wx + 2 * r);
      const int v0 = max(0, wy), v1 = min(P - 1, wy + 2 * r);
      if (u0 > u1 || v0 > v1) continue;
      const int dec = sm.fsat[(v1 + 1) * P1 + u1 + 1] - sm.fsat[v0 * P1 + u1 + 1] -
                      sm.fsat[(v1 + 1) * P1 + u0] + sm.fsat[v0 * P1 + u0];
      if (dec) {
        const size_t qi = (size_t)y * s.pitch + x;
        const int nv = s.count[qi] - dec;
        s.count[qi] = nv;
        if (nv == 0 && in_rect(s, x, y)) ++newly;
      }
    }
    newly = block_sum_int(newly, sm.ints);  // also orders the global writes above

    // Priorities that can change: front pixels within 2r+1 of p^.
    const int R2 = 2 * r + 1, side2 = 2 * R2 + 1;
    for (int j = tid; j < side2 * side2; j += nt) {
      const int x = px - R2 + j % side2, y = py - R2 + j / side2;
      if (x >= 0 && x < W && y >= 0 && y < H) eval_pixel(s, x, y);
    }
    __syncthreads();
    block_refresh_tiles(s, max(0, px - R2), min(W - 1, px + R2), max(0, py - R2),
                        min(H - 1, py + R2));

    remaining -= filled;
    if (filled == 0) {  // p^ must lie in Omega; stop rather than loop without progress
      if (tid == 0) {
        c->status = INPAINT_ERR_INTERNAL;
        if (use_cond) cudaGraphSetConditional(cond, 0);
      }
      return;
    }
    if (tid == 0) {
      const int it = c->iter;
      {
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
      }
      c->remaining = remaining;
      c->iter = it + 1;
      c->n_valid = n_cand + newly;
      c->evals += (unsigned long long)n_cand * (unsigned long long)n_known;
      c->px = -1;
      c->py = -1;
    }
    __syncthreads();
  }

  // Selection of the next target: highest priority on the front, lowest
  // index on ties, from the level-1 tile maxima.
  if (remaining > 0 && tid < 32) warp_select(s);
  __syncthreads();
  if (use_cond && tid == 0) cudaGraphSetConditional(cond, loop_active(c) ? 1u : 0u);
}

// Debug self-check: recount every candidate's unknown pixels and re-evaluate
// every priority key from scratch; any difference sets INPAINT_ERR_INTERNAL.
__global__ void k_verify(ImgState s) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y;
  if (x >= s.W || s.ctrl->status != 0) return;
  const int r = s.r;
  const size_t i = (size_t)y * s.W + x, ic = (size_t)y * s.pitch + x;
  bool bad = false;
  if (x - r >= 0 && x + r < s.W && y - r >= 0 && y + r < s.H) {
    int cnt = 0;
    for (int dy = -r; dy <= r; ++dy)
      for (int dx = -r; dx <= r; ++dx) cnt += s.omega[(size_t)(y + dy) * s.W + x + dx];
    bad |= cnt != s.count[ic];
  } else {
    bad |= s.count[ic] < kCountInvalid - (2 * r + 1) * (2 * r + 1);
  }
  unsigned long long key = 0ull;
  if (on_front(s, x, y)) {
    double c;
    key = (unsigned long long)__double_as_longlong(priority_at(s, x, y, &c)) + 1ull;
  }
  bad |= key != s.prio[i];
  if (bad) atomicCAS(&s.ctrl->status, 0, (int)INPAINT_ERR_INTERNAL);
}

__global__ void k_export(ImgState s, uint8_t* rgb) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (size_t)s.W * s.H) return;
  const uint32_t w = s.img[(i / s.W) * s.pitch + i % s.W];
  rgb[3 * i] = (uint8_t)(w & 255u);
  rgb[3 * i + 1] = (uint8_t)((w >> 8) & 255u);
  rgb[3 * i + 2] = (uint8_t)((w >> 16) & 255u);
}

// ---------------------------------------------------------------- launchers

int sat_chunks(int H) { return (H + kSatChunk - 1) / kSatChunk; }

static cudaError_t init_tail(const ImgState& s, int32_t* sat, cudaStream_t st) {
  const int W = s.W, H = s.H;
  int32_t* tot = sat + (size_t)(W + 1) * (H + 1);
  const int nch = sat_chunks(H);
  k_sat_rows<<<(H + 1 + 7) / 8, 256, 0, st>>>(s, sat);
  k_sat_cols_chunk<<<dim3((W + 127) / 128, nch), 128, 0, st>>>(s, sat, tot);
  k_sat_chunk_prefix<<<(W + 127) / 128, 128, 0, st>>>(s, tot, nch);
  if (H > kSatChunk) k_sat_cols_apply<<<dim3((W + 127) / 128, H - kSatChunk), 128, 0, st>>>(s, sat, tot);
  const dim3 rows((W + 255) / 256, H);
  k_count<<<dim3((s.pitch + 255) / 256, H), 256, 0, st>>>(s, sat);
  if (s.r <= 8) {
    const cudaError_t e = launch_prio_init_fast(s, st);
    if (e != cudaSuccess) return e;
  } else {
    k_prio_all<<<rows, 256, 0, st>>>(s);
  }
  k_tiles0_all<<<(s.t0x * s.t0y + 7) / 8, 256, 0, st>>>(s);
  k_tiles1_all<<<(s.t1x * s.t1y + 7) / 8, 256, 0, st>>>(s);
  k_update<<<1, kUpdThreads, 0, st>>>(s, 0, 0ull, 0);
  return cudaGetLastError();
}

cudaError_t launch_init(const ImgState& s, const uint8_t* rgb, int rgb_stride, const uint8_t* mask,
                        int mask_stride, int32_t* sat, int* /*omega_count*/, cudaStream_t st) {
  k_ctrl_init<<<1, 1, 0, st>>>(s.ctrl);
  k_unpack<<<dim3((s.W + 255) / 256, s.H), 256, 0, st>>>(s, rgb, rgb_stride, mask, mask_stride,
                                                          nullptr);
  return init_tail(s, sat, st);
}

cudaError_t launch_import(const ImgState& s, const uint8_t* rgb, const uint8_t* omega,
                          const double* conf, int32_t* sat, int* /*omega_count*/, cudaStream_t st) {
  k_ctrl_init<<<1, 1, 0, st>>>(s.ctrl);
  k_unpack<<<dim3((s.W + 255) / 256, s.H), 256, 0, st>>>(s, rgb, 3 * s.W, omega, s.W, conf);
  return init_tail(s, sat, st);
}

cudaError_t launch_update(const ImgState& s, int do_fill, unsigned long long cond_handle,
                          int use_cond, cudaStream_t st) {
  k_update<<<1, kUpdThreads, 0, st>>>(s, do_fill, (cudaGraphConditionalHandle)cond_handle,
                                      use_cond);
  return cudaGetLastError();
}

cudaError_t launch_verify_count(const ImgState& s, cudaStream_t st) {
  k_verify<<<dim3((s.W + 127) / 128, s.H), 128, 0, st>>>(s);
  return cudaGetLastError();
}

cudaError_t launch_export(const ImgState& s, uint8_t* rgb_dense, cudaStream_t st) {
  const size_t n = (size_t)s.W * s.H;
  k_export<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(s, rgb_dense);
  return cudaGetLastError();
}

}  // namespace inp
