/*
 * Integer issue-rate microbenchmark of the GPU the decoder runs on.
 *
 * Not part of the decoding method (the paper has no counterpart): it measures
 * the denominator of the decoder's roofline.  FWBF decoding (Sec. III) is
 * bound by plain integer instructions, not by memory or tensor cores, and the
 * GPU's integer issue rate is published nowhere, so it is measured here with
 * chains of independent 32-bit integer instructions.
 */
#ifndef FWBF_PEAK_H
#define FWBF_PEAK_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/*
 * Runs a kernel of independent integer instruction chains on the current
 * device, on `stream` (a cudaStream_t, NULL = legacy default stream), and
 * reports the lane-operations it issued per second.
 *   mix      0: 3-input logic operations only (the integer ALU pipe);
 *            1: logic operations and integer multiply-adds alternating
 *               (the ALU and the multiply-add pipes together).
 *   ms       target run time in milliseconds (1..10000); the kernel is sized
 *            from a short calibration launch.
 *   out_ops_per_s  result, lane-operations per second (one 32-bit integer
 *            instruction executed by one thread counts as one).
 *   out_ops  lane-operations the timed launch issued (may be NULL).
 * Blocks the calling thread until the timed launch ends.  Returns 0 or a
 * negative FWBF_* error code (fwbf.h): FWBF_EINVAL for a bad argument,
 * FWBF_ECUDA for a CUDA error.
 */
int fwbf_peak_int_issue(int mix, double ms, void *stream, double *out_ops_per_s, double *out_ops);

#ifdef __cplusplus
}
#endif

#endif
