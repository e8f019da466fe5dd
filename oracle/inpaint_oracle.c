/*
 * Plain single-threaded CPU oracle of exemplar-based object removal.
 *
 * TEST INFRASTRUCTURE ONLY (see inpaint_oracle.h): loaded by the tests, the
 * smoke entry point and the benchmark's CPU-baseline leg, never by the
 * library.  Built with -O2 -ffp-contract=off so that no floating-point
 * expression is contracted into a fused multiply-add on any host.
 *
 * The steps follow Sec. 3 of the paper in its order: fill front dOmega,
 * priorities P(p) = C(p) D(p) (Eq. 1-2), best patch by masked SSD (Eq. 3-4,
 * the findBestPatch kernel of Table 2 / Algorithm 1), copy of the best patch
 * into the unknown part of the target patch, confidence update, repeat until
 * Omega is empty.  Where the paper is silent the readings are:
 *   - confidence sum over Psi_p intersected with Phi (Eq. 2 prints Omega,
 *     which would make every priority 0), divided by the number of in-image
 *     pixels of Psi_p, summed in row-major order (dy outer, dx inner);
 *   - C = 1 on Phi and 0 on Omega at the start; a filled pixel takes C(p^);
 *   - grey level: integer BT.601 luma (299 R + 587 G + 114 B + 500) / 1000;
 *   - front normal n_p: integer Sobel of the Omega indicator with replicated
 *     borders; isophote: the largest central-difference gradient of the grey
 *     level among known pixels of Psi_p whose four neighbours are known and
 *     in the image (first in row-major order on ties);
 *   - data term D = |grad_perp . n| / |n| / (2 * 255), 0 when n = 0
 *     (alpha = 255 of Eq. 2, times 2 for the central difference);
 *   - priority ties and SSD ties go to the lowest linear index;
 *   - a candidate patch must lie inside the image and inside the current
 *     known region (filled pixels count as known); the SSD sums RGB squared
 *     differences over the known in-image pixels of the target patch, at the
 *     same offset in the candidate patch (Eq. 4);
 *   - the copy writes only pixels that are in Omega and in the image.
 */
#include "inpaint_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

uint8_t oracle_gray(uint8_t r, uint8_t g, uint8_t b) {
  return (uint8_t)((299u * r + 587u * g + 114u * b + 500u) / 1000u);
}

static int in_image(int x, int y, int W, int H) {
  return x >= 0 && x < W && y >= 0 && y < H;
}

/* A pixel of Phi: inside the image and not in Omega. */
static int known(const uint8_t* omega, int x, int y, int W, int H) {
  return in_image(x, y, W, H) && omega[(size_t)y * W + x] == 0;
}

void oracle_front(const uint8_t* omega, int W, int H, uint8_t* front) {
  for (int y = 0; y < H; ++y)
    for (int x = 0; x < W; ++x) {
      size_t i = (size_t)y * W + x;
      front[i] = 0;
      if (!omega[i]) continue;
      if (known(omega, x - 1, y, W, H) || known(omega, x + 1, y, W, H) ||
          known(omega, x, y - 1, W, H) || known(omega, x, y + 1, W, H))
        front[i] = 1;
    }
}

/* Omega indicator with replicated borders, for the Sobel normal. */
static int omega_clamped(const uint8_t* omega, int x, int y, int W, int H) {
  if (x < 0) x = 0;
  if (x >= W) x = W - 1;
  if (y < 0) y = 0;
  if (y >= H) y = H - 1;
  return omega[(size_t)y * W + x] ? 1 : 0;
}

double oracle_priority(const uint8_t* gray, const double* conf,
                       const uint8_t* omega, int W, int H, int r, int x, int y,
                       double* c_out, double* d_out) {
  /* Confidence term C(p), Eq. 2 first line. */
  double sum = 0.0;
  int n_in = 0;
  for (int dy = -r; dy <= r; ++dy)
    for (int dx = -r; dx <= r; ++dx) {
      int qx = x + dx, qy = y + dy;
      if (!in_image(qx, qy, W, H)) continue;
      ++n_in;
      if (omega[(size_t)qy * W + qx] == 0) sum += conf[(size_t)qy * W + qx];
    }
  double c = sum / (double)n_in;

  /* Normal n_p to the front: Sobel of the Omega indicator. */
  int m_l_u = omega_clamped(omega, x - 1, y - 1, W, H);
  int m_c_u = omega_clamped(omega, x, y - 1, W, H);
  int m_r_u = omega_clamped(omega, x + 1, y - 1, W, H);
  int m_l_c = omega_clamped(omega, x - 1, y, W, H);
  int m_r_c = omega_clamped(omega, x + 1, y, W, H);
  int m_l_d = omega_clamped(omega, x - 1, y + 1, W, H);
  int m_c_d = omega_clamped(omega, x, y + 1, W, H);
  int m_r_d = omega_clamped(omega, x + 1, y + 1, W, H);
  int nx = (m_r_u + 2 * m_r_c + m_r_d) - (m_l_u + 2 * m_l_c + m_l_d);
  int ny = (m_l_d + 2 * m_c_d + m_r_d) - (m_l_u + 2 * m_c_u + m_r_u);

  /* Isophote: strongest grey gradient among fully-known pixels of Psi_p. */
  int best_mag = -1, gx = 0, gy = 0;
  for (int dy = -r; dy <= r; ++dy)
    for (int dx = -r; dx <= r; ++dx) {
      int qx = x + dx, qy = y + dy;
      if (!known(omega, qx, qy, W, H)) continue;
      if (!known(omega, qx - 1, qy, W, H) || !known(omega, qx + 1, qy, W, H) ||
          !known(omega, qx, qy - 1, W, H) || !known(omega, qx, qy + 1, W, H))
        continue;
      int tx = (int)gray[(size_t)qy * W + qx + 1] - (int)gray[(size_t)qy * W + qx - 1];
      int ty = (int)gray[(size_t)(qy + 1) * W + qx] - (int)gray[(size_t)(qy - 1) * W + qx];
      int mag = tx * tx + ty * ty;
      if (mag > best_mag) {
        best_mag = mag;
        gx = tx;
        gy = ty;
      }
    }

  /* Data term D(p), Eq. 2 second line: isophote (-gy, gx) against n_p. */
  int dot = (-gy) * nx + gx * ny;
  if (dot < 0) dot = -dot;
  int nn = nx * nx + ny * ny;
  double d = 0.0;
  if (nn != 0) d = ((double)dot / sqrt((double)nn)) / 510.0;

  if (c_out) *c_out = c;
  if (d_out) *d_out = d;
  /* Eq. 1. */
  return c * d;
}

void oracle_search_rect(const uint8_t* mask, int W, int H, int r, double alpha,
                        int* cx0, int* cx1, int* cy0, int* cy1) {
  oracle_search_rect2(mask, W, H, r, alpha, 0, cx0, cx1, cy0, cy1);
}

void oracle_search_rect2(const uint8_t* mask, int W, int H, int r, double alpha,
                         int overlap, int* cx0, int* cx1, int* cy0, int* cy1) {
  /* Candidates whose patch crosses the image border exist only in the
   * partial-overlap variant: there the rectangle is clamped to the image. */
  int lo_x = r, hi_x = W - 1 - r, lo_y = r, hi_y = H - 1 - r;
  if (overlap) {
    lo_x = 0;
    hi_x = W - 1;
    lo_y = 0;
    hi_y = H - 1;
  }
  if (alpha >= 0.0) {
    /* Bounding box of the object (Sec. 5.3): w x h. */
    int x0 = W, x1 = -1, y0 = H, y1 = -1;
    for (int y = 0; y < H; ++y)
      for (int x = 0; x < W; ++x)
        if (mask[(size_t)y * W + x]) {
          if (x < x0) x0 = x;
          if (x > x1) x1 = x;
          if (y < y0) y0 = y;
          if (y > y1) y1 = y;
        }
    if (x1 >= 0) {
      int w = x1 - x0 + 1, h = y1 - y0 + 1;
      /* Eq. 6: expand by alpha*w left/right and alpha*h up/down. */
      int ex = (int)floor(alpha * (double)w);
      int ey = (int)floor(alpha * (double)h);
      if (x0 - ex > lo_x) lo_x = x0 - ex;
      if (x1 + ex < hi_x) hi_x = x1 + ex;
      if (y0 - ey > lo_y) lo_y = y0 - ey;
      if (y1 + ey < hi_y) hi_y = y1 + ey;
    }
  }
  *cx0 = lo_x;
  *cx1 = hi_x;
  *cy0 = lo_y;
  *cy1 = hi_y;
}

int oracle_ssd_map(const uint8_t* rgb, const uint8_t* omega, int W, int H,
                   int r, int px, int py, int cx0, int cx1, int cy0, int cy1,
                   uint32_t* ssd_out, int* n_known) {
  /* K: known in-image pixels of the target patch. */
  int nk = 0;
  for (int dy = -r; dy <= r; ++dy)
    for (int dx = -r; dx <= r; ++dx)
      if (known(omega, px + dx, py + dy, W, H)) ++nk;
  if (n_known) *n_known = nk;

  int n_cand = 0;
  for (int qy = 0; qy < H; ++qy)
    for (int qx = 0; qx < W; ++qx) {
      size_t qi = (size_t)qy * W + qx;
      ssd_out[qi] = UINT32_MAX;
      if (qx < cx0 || qx > cx1 || qy < cy0 || qy > cy1) continue;
      if (qx - r < 0 || qx + r >= W || qy - r < 0 || qy + r >= H) continue;
      int ok = 1;
      for (int dy = -r; dy <= r && ok; ++dy)
        for (int dx = -r; dx <= r; ++dx)
          if (omega[(size_t)(qy + dy) * W + qx + dx]) {
            ok = 0;
            break;
          }
      if (!ok) continue;
      ++n_cand;
      /* Eq. 4: squared RGB differences over the known target pixels. */
      uint64_t s = 0;
      for (int dy = -r; dy <= r; ++dy)
        for (int dx = -r; dx <= r; ++dx) {
          if (!known(omega, px + dx, py + dy, W, H)) continue;
          const uint8_t* a = rgb + 3 * ((size_t)(py + dy) * W + px + dx);
          const uint8_t* b = rgb + 3 * ((size_t)(qy + dy) * W + qx + dx);
          for (int c = 0; c < 3; ++c) {
            int64_t e = (int64_t)a[c] - (int64_t)b[c];
            s += (uint64_t)(e * e);
          }
        }
      /* r <= 32 keeps every SSD below 2^32 - 1: 65^2 * 3 * 255^2 < 2^30. */
      ssd_out[qi] = (uint32_t)s;
    }
  return n_cand;
}

int oracle_ssd_map_overlap(const uint8_t* rgb, const uint8_t* omega, int W,
                           int H, int r, int px, int py, int cx0, int cx1,
                           int cy0, int cy1, uint32_t* ssd_out, int* n_known) {
  int nk = 0;
  for (int dy = -r; dy <= r; ++dy)
    for (int dx = -r; dx <= r; ++dx)
      if (known(omega, px + dx, py + dy, W, H)) ++nk;
  if (n_known) *n_known = nk;

  int n_cand = 0;
  for (int qy = 0; qy < H; ++qy)
    for (int qx = 0; qx < W; ++qx) {
      size_t qi = (size_t)qy * W + qx;
      ssd_out[qi] = UINT32_MAX;
      if (qx < cx0 || qx > cx1 || qy < cy0 || qy > cy1) continue;
      /* The copy needs a known source pixel under every unknown in-image
       * pixel of the target patch. */
      int ok = 1;
      for (int dy = -r; dy <= r && ok; ++dy)
        for (int dx = -r; dx <= r; ++dx) {
          int tx = px + dx, ty = py + dy;
          if (!in_image(tx, ty, W, H) || !omega[(size_t)ty * W + tx]) continue;
          if (!known(omega, qx + dx, qy + dy, W, H)) {
            ok = 0;
            break;
          }
        }
      if (!ok) continue;
      ++n_cand;
      /* Alg. 1 / Sec. 5.4: squared RGB differences over the pixel pairs
       * with both the target pixel and the source pixel known and in the
       * image (an empty sum is 0). */
      uint64_t s = 0;
      for (int dy = -r; dy <= r; ++dy)
        for (int dx = -r; dx <= r; ++dx) {
          if (!known(omega, px + dx, py + dy, W, H)) continue;
          if (!known(omega, qx + dx, qy + dy, W, H)) continue;
          const uint8_t* a = rgb + 3 * ((size_t)(py + dy) * W + px + dx);
          const uint8_t* b = rgb + 3 * ((size_t)(qy + dy) * W + qx + dx);
          for (int c = 0; c < 3; ++c) {
            int64_t e = (int64_t)a[c] - (int64_t)b[c];
            s += (uint64_t)(e * e);
          }
        }
      ssd_out[qi] = (uint32_t)s;
    }
  return n_cand;
}

int oracle_run_from_state(uint8_t* rgb, uint8_t* omega, double* conf, int W,
                          int H, int r, int cx0, int cx1, int cy0, int cy1,
                          int max_iters, oracle_trace* trace, int trace_cap,
                          int* iters_done, uint64_t* evals) {
  return oracle_run_from_state2(rgb, omega, conf, W, H, r, cx0, cx1, cy0, cy1,
                                0, max_iters, trace, trace_cap, iters_done,
                                evals);
}

int oracle_run_from_state2(uint8_t* rgb, uint8_t* omega, double* conf, int W,
                           int H, int r, int cx0, int cx1, int cy0, int cy1,
                           int overlap, int max_iters, oracle_trace* trace,
                           int trace_cap, int* iters_done, uint64_t* evals) {
  size_t n = (size_t)W * H;
  int it = 0;
  uint64_t ev = 0;
  int status = ORACLE_OK;
  uint8_t* gray = (uint8_t*)calloc(n, 1);
  uint8_t* front = (uint8_t*)calloc(n, 1);
  uint32_t* ssd = (uint32_t*)malloc(n * sizeof(uint32_t));
  if (!gray || !front || !ssd) {
    free(gray);
    free(front);
    free(ssd);
    return ORACLE_ERR_ARG;
  }
  int remaining = 0;
  for (size_t i = 0; i < n; ++i) {
    if (omega[i])
      ++remaining;
    else
      gray[i] = oracle_gray(rgb[3 * i], rgb[3 * i + 1], rgb[3 * i + 2]);
  }

  while (remaining > 0 && (max_iters <= 0 || it < max_iters)) {
    /* 1. Fill front. */
    oracle_front(omega, W, H, front);

    /* 2. Priorities on the front; p^ = argmax, ties to the lowest index. */
    long best = -1;
    double best_p = 0.0, best_c = 0.0;
    for (size_t i = 0; i < n; ++i) {
      if (!front[i]) continue;
      double c;
      double p = oracle_priority(gray, conf, omega, W, H, r, (int)(i % W),
                                 (int)(i / W), &c, NULL);
      if (best < 0 || p > best_p) {
        best = (long)i;
        best_p = p;
        best_c = c;
      }
    }
    if (best < 0) { /* cannot happen while Phi is non-empty */
      status = ORACLE_ERR_ARG;
      break;
    }
    int px = (int)(best % W), py = (int)(best / W);

    /* 3. findBestPatch: q~ = argmin SSD, ties to the lowest index (Eq. 3). */
    int nk = 0;
    int n_cand = overlap ? oracle_ssd_map_overlap(rgb, omega, W, H, r, px, py,
                                                  cx0, cx1, cy0, cy1, ssd, &nk)
                         : oracle_ssd_map(rgb, omega, W, H, r, px, py, cx0,
                                          cx1, cy0, cy1, ssd, &nk);
    long bq = -1;
    for (size_t i = 0; i < n; ++i)
      if (ssd[i] != UINT32_MAX && (bq < 0 || ssd[i] < ssd[bq])) bq = (long)i;
    if (bq < 0) {
      status = ORACLE_ERR_NO_SOURCE;
      break;
    }
    int qx = (int)(bq % W), qy = (int)(bq / W);

    /* 4. Copy Psi_q~ into the unknown part of Psi_p^, update C and Omega. */
    int filled = 0;
    for (int dy = -r; dy <= r; ++dy)
      for (int dx = -r; dx <= r; ++dx) {
        int tx = px + dx, ty = py + dy;
        if (!in_image(tx, ty, W, H)) continue;
        size_t t = (size_t)ty * W + tx;
        if (!omega[t]) continue;
        size_t s = (size_t)(qy + dy) * W + qx + dx;
        rgb[3 * t] = rgb[3 * s];
        rgb[3 * t + 1] = rgb[3 * s + 1];
        rgb[3 * t + 2] = rgb[3 * s + 2];
        gray[t] = oracle_gray(rgb[3 * t], rgb[3 * t + 1], rgb[3 * t + 2]);
        conf[t] = best_c;
        omega[t] = 0;
        ++filled;
      }
    remaining -= filled;
    ev += (uint64_t)n_cand * (uint64_t)nk;

    if (trace && it < trace_cap) {
      oracle_trace* e = &trace[it];
      e->iter = it;
      e->px = px;
      e->py = py;
      e->qx = qx;
      e->qy = qy;
      e->ssd = ssd[bq];
      e->priority = best_p;
      e->confidence = best_c;
      e->filled = filled;
      e->remaining = remaining;
      e->n_known = nk;
      e->n_cand = n_cand;
    }
    ++it;
  }
  free(gray);
  free(front);
  free(ssd);
  if (iters_done) *iters_done = it;
  if (evals) *evals = ev;
  return status;
}

int oracle_run(const uint8_t* rgb, const uint8_t* mask, int W, int H, int r,
               double alpha, int max_iters, uint8_t* rgb_out,
               uint8_t* mask_out, double* conf_out, oracle_trace* trace,
               int trace_cap, int* iters_done, uint64_t* evals) {
  return oracle_run2(rgb, mask, W, H, r, alpha, 0, max_iters, rgb_out,
                     mask_out, conf_out, trace, trace_cap, iters_done, evals);
}

int oracle_run2(const uint8_t* rgb, const uint8_t* mask, int W, int H, int r,
                double alpha, int overlap, int max_iters, uint8_t* rgb_out,
                uint8_t* mask_out, double* conf_out, oracle_trace* trace,
                int trace_cap, int* iters_done, uint64_t* evals) {
  if (iters_done) *iters_done = 0;
  if (evals) *evals = 0;
  if (!rgb || !mask || r < 1 || r > 32 || W < 2 * r + 1 || H < 2 * r + 1)
    return ORACLE_ERR_ARG;
  size_t n = (size_t)W * H;
  size_t n_omega = 0;
  for (size_t i = 0; i < n; ++i)
    if (mask[i]) ++n_omega;
  if (n_omega == n) return ORACLE_ERR_ARG; /* no known pixel at all */

  uint8_t* img = (uint8_t*)malloc(3 * n);
  uint8_t* omega = (uint8_t*)malloc(n);
  double* conf = (double*)malloc(n * sizeof(double));
  if (!img || !omega || !conf) {
    free(img);
    free(omega);
    free(conf);
    return ORACLE_ERR_ARG;
  }
  memcpy(img, rgb, 3 * n);
  for (size_t i = 0; i < n; ++i) {
    omega[i] = mask[i] ? 1 : 0;
    conf[i] = mask[i] ? 0.0 : 1.0;
  }
  int cx0, cx1, cy0, cy1;
  oracle_search_rect2(mask, W, H, r, alpha, overlap, &cx0, &cx1, &cy0, &cy1);

  int status = ORACLE_DONE;
  if (n_omega > 0)
    status = oracle_run_from_state2(img, omega, conf, W, H, r, cx0, cx1, cy0,
                                    cy1, overlap, max_iters, trace, trace_cap,
                                    iters_done, evals);
  if (rgb_out) memcpy(rgb_out, img, 3 * n);
  if (mask_out) memcpy(mask_out, omega, n);
  if (conf_out) memcpy(conf_out, conf, n * sizeof(double));
  free(img);
  free(omega);
  free(conf);
  return status;
}
