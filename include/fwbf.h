/*
 * fwbf.h - C ABI of libfwbf.so: GB300 (sm_103a) decoding of LDPC codes with
 * the fast weighted bit-flipping (FWBF) algorithm of Ma, Li, Zhu, Zhang and Qi,
 * "An Improved WBF Algorithm for Higher-Speed Decoding of LDPC Codes".
 *
 * What is computed (paper Sec. II, Eq. 1 and Sec. III):
 *   Initialisation  z_0[n] = 1 iff y_n < 0;  w_{n,m} = min_{i in N(m)\n} |y_i|.
 *   Step 1          s_k = z_k H^T; stop if its weight is 0 or k = max_iter.
 *   Step 2          E_n = sum_{m in M(n)} (2 s_m - 1) w_{n,m} - alpha |y_n|   (Eq. 1);
 *                   split the bits into contiguous blocks of p (the last one may
 *                   be short); in every block take the first index of largest E
 *                   and flip it if E > 0.  All blocks read the same s_k.
 *                   k = k + 1, back to Step 1.
 * Conventions shared by every entry point:
 *   - Return value: FWBF_OK (0) or a negative FWBF_E* code; fwbf_strerror()
 *     names it and fwbf_last_error() gives this thread's detail message.
 *     Argument checks happen before any work is queued.  No C++ exception
 *     crosses the ABI.
 *   - Device pointers are plain CUDA device addresses owned by the caller;
 *     host pointers are only read during the call.  Work is queued on the given
 *     stream (a cudaStream_t passed as void*, NULL = legacy default stream) and
 *     is asynchronous: results are ready when the stream reaches that point.
 *   - Bit-packed decisions: frame f, bit n lives in word f*ceil(N/32) + n/32,
 *     bit position n%32.
 *   - Iteration counts: k >= 0 when the syndrome of z_k is zero (k flip passes
 *     were run), -max_iter when it is still non-zero after max_iter passes.
 *   - A code handle is immutable after creation; calls on different streams may
 *     share it.
 */
#ifndef FWBF_H
#define FWBF_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define FWBF_OK 0
#define FWBF_EINVAL -1        /* an argument is out of range or inconsistent */
#define FWBF_ENOMEM -2        /* host or device allocation failed */
#define FWBF_ECUDA -3         /* a CUDA runtime call failed */
#define FWBF_EUNSUPPORTED -4  /* valid input the library does not handle */
#define FWBF_ETIMEOUT -5      /* a kernel gave up a bounded wait (see fwbf_last_status) */

typedef struct fwbf_code_s *fwbf_code;

typedef struct {
    int32_t N;          /* bits (columns of H) */
    int32_t M;          /* checks (rows of H) */
    int64_t nnz;        /* ones in H */
    int32_t Z;          /* circulant size found in H (1 = no circulant structure) */
    int32_t dv_max;     /* largest column weight */
    int32_t dc_max;     /* largest row weight */
    int32_t seg_len;    /* p, block length of the bit-choose */
    int32_t n_blocks;   /* ceil(N / p) */
    int64_t table_bytes;/* device bytes of the index tables */
} fwbf_code_info;

/*
 * Builds a code handle from the ones of H (Sec. II: H = [h_mn], M x N).
 *   N, M       1 <= N, M <= 65535
 *   nnz        number of ones; row_idx[e], col_idx[e] (host arrays, copied) are
 *              the check m and bit n of the e-th one.  Order is free; duplicates
 *              are rejected.
 *   seg_len    p of Sec. III Step 2, 1 <= p <= N.
 *   out        receives the handle (release with fwbf_destroy).
 * Validation: indices in range, no duplicate, every check has at least two bits
 * (otherwise N(m)\n is empty in Eq. 1) and at most 255, every bit at most 255
 * checks.  When H is built from Z x Z circulant blocks (cyclic and
 * quasi-cyclic codes), the largest such Z is found and the index tables are
 * stored in that compressed form.  Errors: FWBF_EINVAL, FWBF_EUNSUPPORTED,
 * FWBF_ENOMEM, FWBF_ECUDA.  Uses the current CUDA device.
 */
int fwbf_code_create(int32_t N, int32_t M, int64_t nnz, const int32_t *row_idx,
                     const int32_t *col_idx, int32_t seg_len, fwbf_code *out);

/* Releases a handle (waits for the device to finish using it).  NULL is a no-op. */
int fwbf_destroy(fwbf_code c);

/* Copies the handle's parameters into *out. */
int fwbf_code_query(fwbf_code c, fwbf_code_info *out);

/*
 * int8 channel values for the integer decoder:
 *   q[i] = saturate_{[-127,127]}(round_half_to_even(16 * y[i])), NaN -> 0.
 *   y      device float[count]        q   device int8[count]
 * Any alignment; count >= 0.
 */
int fwbf_quantize(const float *y, int8_t *q, int64_t count, void *stream);

/*
 * FWBF on int8 channel values (Sec. III with Eq. 1 in fixed point).
 *   y          device int8 [n_frames][N], frames packed back to back (stride N
 *              bytes); the base address must be 16-byte aligned.
 *   n_frames   >= 0 (0 queues nothing)
 *   max_iter   K_max >= 1
 *   alpha      weighting factor of Eq. 1, 0 <= alpha <= 64; it is used as
 *              alpha_q = round_half_to_even(256 alpha) and the metric is
 *              E'_n = 256 sum (2 s_m - 1) w_{n,m} - alpha_q |q_n|, exact in int32.
 *   out_bits   device uint32 [n_frames][ceil(N/32)]
 *   out_iters  device int32 [n_frames]
 * Results are bit-identical to the definition above for every input.
 */
int fwbf_decode(fwbf_code c, const int8_t *y, int64_t n_frames, int32_t max_iter,
                float alpha, uint32_t *out_bits, int32_t *out_iters, void *stream);

/*
 * fwbf_decode without any device memory allocation.  The paper has no
 * counterpart: this entry point exists for callers that cannot allocate device
 * memory once they are running, such as real-time receivers that fix their
 * memory at start-up so the decode path has no allocation latency or
 * out-of-memory failure, and hosts where the stream-ordered allocator is not
 * available.  fwbf_decode takes its 8-byte frame work counter from a
 * stream-ordered allocation on every call; this variant takes it from a fixed
 * 256-byte array in the library's device memory, which every GPU that loads the
 * library holds until the process exits.  Arguments, results and errors are
 * those of fwbf_decode.
 *   - The first call on a device looks up the array's device address; make
 *     that first call before any stream capture.
 *   - The array is shared by every call and keeps the last call's contents; the
 *     counter is cleared on the stream before each launch.  Calls whose work
 *     overlaps on the GPU (other streams, other threads) race on it: order them
 *     on one stream or serialise them.
 *   - A decode whose scratch would not fit the fixed array is rejected with
 *     FWBF_EUNSUPPORTED (this decoder needs 8 of the 256 bytes).
 * No cudaMalloc, cudaFree or other allocating call is made.
 */
int fwbf_decode_noalloc(fwbf_code c, const int8_t *y, int64_t n_frames, int32_t max_iter,
                        float alpha, uint32_t *out_bits, int32_t *out_iters, void *stream);

/*
 * FWBF on real channel values, metric of Eq. 1 in float32.
 *   y          device float [n_frames][N] (finite values), any 4-byte alignment
 *   other arguments as fwbf_decode.
 * Decisions equal those of exact arithmetic except where two metrics, or a
 * metric and 0, lie within float32 rounding of each other.
 */
int fwbf_decode_f32(fwbf_code c, const float *y, int64_t n_frames, int32_t max_iter,
                    float alpha, uint32_t *out_bits, int32_t *out_iters, void *stream);

/*
 * The metric of Eq. 1 (float32) of the first pass, for every bit:
 *   out_E      device float [n_frames][N], E_n for z_0 and s_0.
 */
int fwbf_metric_f32(fwbf_code c, const float *y, int64_t n_frames, float alpha, float *out_E,
                    void *stream);

/*
 * Waits for the stream, then reports and clears the device status word that
 * kernels set when a bounded wait runs out: FWBF_OK or FWBF_ETIMEOUT.
 */
int fwbf_last_status(void *stream);

/* Static description of a status code. */
const char *fwbf_strerror(int status);

/* Detail message of this thread's last failing call ("" if none). */
const char *fwbf_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* FWBF_H */
