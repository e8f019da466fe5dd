/*
 * Oracle for exemplar-based object removal (Criminisi-style inpainting as
 * described in Sec. 3 of Wang, Xiong, Yun, Cavallaro, "Computer Vision
 * Accelerators for Mobile Systems based on OpenCL GPGPU Co-Processing",
 * J. Sign. Process. Syst. 2014).
 *
 * TEST INFRASTRUCTURE ONLY.  This is a plain, slow, single-threaded CPU
 * restatement of the algorithm, used to check the CUDA library.  Only the
 * test suite, the smoke entry point and the benchmark's CPU-baseline leg may
 * load it.  It shares no code, header or constant with the CUDA path.
 *
 * Conventions: images are W x H, row-major, linear index idx(x,y) = y*W + x.
 * RGB input is 3 interleaved bytes per pixel; mask nonzero = pixel to remove
 * (the target region Omega); everything else is the source region Phi.
 * Patch radius r, patch side P = 2r+1.
 *
 * Every function is "parity pinned" by the tests in tests/test_oracle_*.py
 * (brute force in an independent numpy implementation, hand-computed
 * priorities, planted copies, invariants).  The fill loop as a whole is
 * pinned only through those pieces and invariants: the paper prints no
 * per-iteration values and no result images.
 */
#ifndef INPAINT_ORACLE_H
#define INPAINT_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes (own copy; the CUDA library has its own). */
#define ORACLE_OK 0
#define ORACLE_DONE 1
#define ORACLE_ERR_ARG (-1)
#define ORACLE_ERR_NO_SOURCE (-4)

/* One entry per fill iteration. */
typedef struct {
  int32_t iter;        /* 0-based iteration number */
  int32_t px, py;      /* selected target centre p^ (max priority) */
  int32_t qx, qy;      /* chosen source centre q~ (min SSD) */
  uint32_t ssd;        /* SSD of q~ against the known part of Psi_p^ */
  double priority;     /* P(p^) = C(p^) * D(p^) */
  double confidence;   /* C(p^) */
  int32_t filled;      /* pixels copied this iteration */
  int32_t remaining;   /* |Omega| after this iteration */
  int32_t n_known;     /* |K|: known in-image pixels of Psi_p^ */
  int32_t n_cand;      /* number of valid candidate centres searched */
} oracle_trace;

/* Integer BT.601 luma of one pixel. */
uint8_t oracle_gray(uint8_t r, uint8_t g, uint8_t b);

/* Fill front dOmega: front[i] = 1 iff omega[i] and an in-image 4-neighbour is
 * in Phi. */
void oracle_front(const uint8_t* omega, int W, int H, uint8_t* front);

/* Priority P(p) = C(p) * D(p) of pixel (x,y) (Eq. 1-2).  gray is valid on
 * Phi; conf holds C (0 on Omega).  Writes C(p) and D(p) when non-NULL. */
double oracle_priority(const uint8_t* gray, const double* conf,
                       const uint8_t* omega, int W, int H, int r, int x, int y,
                       double* c_out, double* d_out);

/* SSD of every candidate centre against target p (Eq. 4).  ssd_out[idx] is
 * the SSD for a valid candidate and UINT32_MAX otherwise.  A candidate is
 * valid iff its patch lies inside the image and inside Phi, and its centre is
 * inside the rectangle [cx0,cx1] x [cy0,cy1] (inclusive).  Returns the number
 * of valid candidates; *n_known receives |K|. */
int oracle_ssd_map(const uint8_t* rgb, const uint8_t* omega, int W, int H,
                   int r, int px, int py, int cx0, int cx1, int cy0, int cy1,
                   uint32_t* ssd_out, int* n_known);

/* Candidate-centre rectangle for search factor alpha (Sec. 5.3, Eq. 6):
 * alpha < 0 selects the exhaustive search (every interior centre). */
void oracle_search_rect(const uint8_t* mask, int W, int H, int r, double alpha,
                        int* cx0, int* cx1, int* cy0, int* cy1);

/* Partial-overlap variant of the search (Alg. 1 and Sec. 5.4): every centre
 * of the rectangle is a candidate, also when its patch overlaps Omega or
 * crosses the image border, provided a known in-image source pixel lies
 * under every unknown in-image pixel of the target patch (so that the copy
 * is defined).  SSD(q) sums the squared RGB differences over the offsets
 * whose target pixel and source pixel are both known and in the image (0
 * when there is none).  Same outputs as oracle_ssd_map. */
int oracle_ssd_map_overlap(const uint8_t* rgb, const uint8_t* omega, int W,
                           int H, int r, int px, int py, int cx0, int cx1,
                           int cy0, int cy1, uint32_t* ssd_out, int* n_known);

/* oracle_search_rect; with overlap != 0 the rectangle is clamped to the
 * image instead of the interior centres (the partial-overlap variant). */
void oracle_search_rect2(const uint8_t* mask, int W, int H, int r, double alpha,
                         int overlap, int* cx0, int* cx1, int* cy0, int* cy1);

/* The whole removal loop.  rgb_out (3*W*H), mask_out (W*H) and conf_out
 * (W*H) receive the final state when non-NULL; trace receives up to
 * trace_cap entries; *iters_done and *evals (sum over iterations of
 * n_cand * n_known) are always written.  max_iters <= 0 runs to completion.
 * Returns ORACLE_OK, ORACLE_DONE (nothing to fill), ORACLE_ERR_ARG or
 * ORACLE_ERR_NO_SOURCE (the state is left as before that iteration). */
int oracle_run(const uint8_t* rgb, const uint8_t* mask, int W, int H, int r,
               double alpha, int max_iters, uint8_t* rgb_out,
               uint8_t* mask_out, double* conf_out, oracle_trace* trace,
               int trace_cap, int* iters_done, uint64_t* evals);

/* Same loop, but starting from an explicit state (rgb, omega, conf) rather
 * than from an image + mask; the search rectangle is given directly.  Used
 * to check single iterations taken from the middle of a long run. */
int oracle_run_from_state(uint8_t* rgb, uint8_t* omega, double* conf, int W,
                          int H, int r, int cx0, int cx1, int cy0, int cy1,
                          int max_iters, oracle_trace* trace, int trace_cap,
                          int* iters_done, uint64_t* evals);

/* oracle_run / oracle_run_from_state with the search variant chosen by
 * `overlap` (0: candidates fully known and inside the image; 1: the
 * partial-overlap variant of oracle_ssd_map_overlap).  The work count adds
 * n_cand * n_known per iteration in both. */
int oracle_run2(const uint8_t* rgb, const uint8_t* mask, int W, int H, int r,
                double alpha, int overlap, int max_iters, uint8_t* rgb_out,
                uint8_t* mask_out, double* conf_out, oracle_trace* trace,
                int trace_cap, int* iters_done, uint64_t* evals);
int oracle_run_from_state2(uint8_t* rgb, uint8_t* omega, double* conf, int W,
                           int H, int r, int cx0, int cx1, int cy0, int cy1,
                           int overlap, int max_iters, oracle_trace* trace,
                           int trace_cap, int* iters_done, uint64_t* evals);

#ifdef __cplusplus
}
#endif
#endif
