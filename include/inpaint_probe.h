/*
 * Measurement and failure-injection aids of libinpaint.  The paper has no
 * counterpart to any of them: a hardware rate probe (the instruction rates
 * that bound the search kernels, so that their roofline fractions use
 * measured denominators), an isolated timing of one findBestPatch search,
 * and a run of the persistent engine in which one searcher never reports,
 * which exercises its bounded waits.
 */
#ifndef INPAINT_PROBE_H
#define INPAINT_PROBE_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  double ssd_evals_per_s; /* byte-SIMD abs-diff + 4-way byte dot product pairs per second
                             (one candidate-pixel SSD evaluation each), all SMs */
  double imad_per_s;      /* 32-bit integer multiply-adds per second, all SMs */
  double iadd3_per_s;     /* 32-bit three-input integer adds per second, all SMs */
  double dadd_per_s;      /* FP64 add per second, all SMs */
  double sm_clock_mhz;    /* SM clock seen during the probe (clock64 vs global timer) */
  int sm_count;
} inpaint_peaks;

/* Runs the probe kernels on the current device (about a second; uses the
 * legacy default stream and synchronises it).  Returns 0 or a negative
 * inpaint_status. */
int inpaint_probe_peaks(inpaint_peaks* out);

/* Times one findBestPatch search (Sec. 3, Eq. 3-4) of the given form on a
 * context's current state, in isolation: the search kernel of that form is
 * launched `reps` times for the context's current target p^ (after one
 * untimed launch), between CUDA events on the context's stream, without the
 * copy/update step, so the state does not change.  Needs a pending target
 * (after create/reset or a step, before the removal finishes; otherwise
 * INPAINT_DONE).  Outputs: ms_per_search, the smallest packed key
 * (SSD << 32 | idx) found (equal for every form), and evals = valid
 * candidate centres x known target pixels of this search.  form: an
 * INPAINT_FORM_* value (the plain form is the stand-alone graph-loop
 * kernel).  Allocates and frees its own partial-key buffer; synchronises
 * the stream.  The paper has no counterpart; this is a measurement aid. */
struct inpaint_ctx;
int inpaint_time_search(struct inpaint_ctx* ctx, int form, int reps, double* ms_per_search,
                        unsigned long long* best_key, unsigned long long* evals);

/* Failure injection for the persistent engine's bounded waits.  Runs
 * inpaint_run(ctx, max_iters, iters_done, NULL, 0) once with the engine's
 * wait limit set to wait_limit_s seconds (0 < wait_limit_s <= 10; normally
 * 4 s) and with searcher CTA `rank` (>= 0) of the team never reporting its
 * key.  The team's leader then gives up waiting for the keys after
 * wait_limit_s, applies no update, and publishes a stop that every other CTA
 * of the team reads; the launch ends and the call returns
 * INPAINT_ERR_TIMEOUT with the removal state exactly as before the
 * interrupted iteration (the iterations before it stay applied), so the
 * context stays usable and a later inpaint_run continues the removal.  A
 * rank that does not search in this image (one at or beyond the number of
 * searching CTAs) has no effect and the run completes normally.  The wait
 * limit and the reporting are restored before the call returns.  Errors:
 * INPAINT_ERR_ARG (null ctx, rank < 0, wait_limit_s out of range),
 * INPAINT_ERR_UNSUPPORTED (the context does not run the persistent engine:
 * graph loop, tensor-core form, partial-overlap search or r > 8), and every
 * error of inpaint_run. */
int inpaint_run_withheld(struct inpaint_ctx* ctx, int rank, double wait_limit_s, int max_iters,
                         int* iters_done);

#ifdef __cplusplus
}
#endif
#endif
