/*
 * teno_probe.h -- measurement helper shipped beside the TENO-AA library.
 *
 * The paper has no counterpart: this is the FP64 arithmetic-peak probe used
 * as the roofline denominator of the FP64-bound TENO-AA kernels (the GPU's
 * FP64 rate is not in the measured-peaks file).
 */
#ifndef TENO_PROBE_H
#define TENO_PROBE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Run a dependent-free DFMA stream on every SM: blocks x 256 threads, each
 * with 8 independent accumulators, iters iterations.  Writes the elapsed
 * device time in milliseconds (CUDA events on the given stream) and the
 * number of DFMA instructions executed per thread lane.  out_sink (device,
 * blocks*256 doubles) receives the accumulators so nothing is optimised out.
 * Returns 0 on success, 2 on a CUDA error. */
int teno_probe_dfma(int blocks, int iters, double *out_sink, double *ms, int64_t *dfma_total,
                    void *stream);

#ifdef __cplusplus
}
#endif

#endif
