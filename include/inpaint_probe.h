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

#ifdef __cplusplus
}
#endif
#endif
