/*
 * Hardware rate probe of libinpaint.  The paper has no counterpart: it
 * measures, on the GPU at hand, the instruction rates that bound the search
 * kernels, so that their roofline fractions use measured denominators.
 */
#ifndef INPAINT_PROBE_H
#define INPAINT_PROBE_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  double ssd_evals_per_s; /* byte-SIMD abs-diff + 4-way byte dot product pairs per second
                             (one candidate-pixel SSD evaluation each), all SMs */
  double imad_per_s;      /* 32-bit integer multiply-add per second, all SMs */
  double iadd3_per_s;     /* dependent 32-bit integer adds per second, all SMs */
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

#ifdef __cplusplus
}
#endif
#endif
