/*
 * Diagnostics of the GPU the decoder runs on (not part of the decoding method).
 *
 * Integer issue-rate microbenchmark.
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

/*
 * Bounded-wait probe (for tests of the timeout path without a GPU fault): one
 * block of 32 threads runs the bounded mbarrier wait that every decoding
 * kernel uses while its code tables are staged into shared memory, on a
 * barrier that expects expect_bytes bytes.  No copy is issued, so with
 * expect_bytes > 0 nothing completes the barrier: the wait gives up after its
 * limit (one second of the GPU's global timer) and the kernel records
 * FWBF_ETIMEOUT -- what a decoding kernel reports through fwbf_last_status /
 * fwbf_batch_status when a table copy does not land -- and returns, leaving
 * the context usable.  With expect_bytes = 0 the barrier completes at once
 * (FWBF_OK).  Not part of the method.
 *   expect_bytes  0..65536
 *   out_status    host int: FWBF_OK or FWBF_ETIMEOUT
 * Blocks until the kernel has finished.  Returns 0, FWBF_EINVAL or FWBF_ECUDA.
 */
int fwbf_probe_bounded_wait(uint32_t expect_bytes, void *stream, int *out_status);

#ifdef __cplusplus
}
#endif

#endif
