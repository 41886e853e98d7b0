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
    int32_t max_row_overlap; /* most bits any two checks share: the RC constraint
                                of Sec. II (no two rows with two common ones)
                                holds iff this is <= 1; the decoder works either way */
    int32_t decoder;    /* kernel fwbf_decode (and its _noalloc / _host forms)
                           runs for this code: FWBF_DECODER_LIST, _CYCLIC or _QC */
} fwbf_code_info;

/* fwbf_code_info.decoder.  All three compute the same results (bit-identical);
 * they differ in the layout they exploit. */
#define FWBF_DECODER_LIST 0   /* explicit index lists, any H */
#define FWBF_DECODER_CYCLIC 1 /* packed: H one circulant (N = M = Z, e.g. EG codes) */
#define FWBF_DECODER_QC 2     /* packed: H blocks of Z x Z circulants, Z % 64 == 0 */

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
 *              bytes); the base address must be 16-byte aligned.  The decoder
 *              works on the range fwbf_quantize writes, [-127, 127]: an input
 *              of -128 is read as -127.
 *   n_frames   >= 0 (0 queues nothing)
 *   max_iter   K_max >= 1
 *   alpha      weighting factor of Eq. 1, 0 <= alpha <= 64; it is used as
 *              alpha_q = round_half_to_even(256 alpha) and the metric is
 *              E'_n = 256 sum (2 s_m - 1) w_{n,m} - alpha_q |q_n|, exact in int32.
 *   out_bits   device uint32 [n_frames][ceil(N/32)]
 *   out_iters  device int32 [n_frames]
 * Results are bit-identical to the definition above for every input in that range.
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
 *     that first call before any stream capture.  The address is kept for the
 *     life of the process: after cudaDeviceReset on that device it is stale,
 *     so do not use this entry point on a device that has been reset.
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
 * End to end from host memory: the float channel values of n_frames frames are
 * copied to the device, quantised (fwbf_quantize) and decoded (fwbf_decode), and
 * the decisions and pass counts copied back, in chunks of chunk_frames frames
 * that alternate between two internal streams so that one chunk's copies
 * overlap another's decoding.  The work is ordered after the work already
 * queued on `stream`, and `stream` reaches the end of the call only when every
 * chunk has been copied back (so the caller synchronises on its own stream).
 *   y_host      host float [n_frames][N] (page-locked for asynchronous copies)
 *   bits_host   host uint32 [n_frames][ceil(N/32)]
 *   iters_host  host int32 [n_frames]
 *   chunk_frames  >= 1 (e.g. 32768: on GB300, where host-to-device copies run
 *               at about 210 GB/s, 2^15 EG(1023) frames per chunk keep the
 *               pipeline within 6 % of the copy time); device memory used: 2 chunks of float
 *               input, int8 frames and outputs, from the stream-ordered
 *               allocator, released on `stream`.
 * Host buffers must stay valid until `stream` has completed the call.
 */
int fwbf_decode_host(fwbf_code c, const float *y_host, int64_t n_frames, int32_t max_iter,
                     float alpha, uint32_t *bits_host, int32_t *iters_host,
                     int64_t chunk_frames, void *stream);

/*
 * Comparison rule: lambda-largest selection (MLP-WBF's bit-choose, Sec. III)
 * with the IMWBF metric of Eq. 1 in place of FWBF's p-blocks.  Every pass
 * computes E'_n for all bits from the same syndrome, takes the lambda bits with
 * the largest metrics one after another (largest remaining, lowest index first
 * among equals) and flips those with E' > 0.  lambda = 1 is single-bit flipping
 * (FWBF with p = N); lambda >= N flips every positive metric (FWBF with p = 1).
 * Arguments as fwbf_decode, plus lambda >= 1 (values above N act as N).
 */
int fwbf_decode_lambda(fwbf_code c, const int8_t *y, int64_t n_frames, int32_t max_iter,
                       float alpha, int32_t lambda, uint32_t *out_bits, int32_t *out_iters,
                       void *stream);

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

/* ------------------------------------------------------------------------ */
/* Batched decoding of several codes in one persistent launch               */
/* ------------------------------------------------------------------------ */

/*
 * The paper decodes one code at a time; this is a throughput form of the same
 * decoder (results are those of fwbf_decode for every job): codes of
 * different N, M and row / column weight, each with its own frames and
 * outputs, share one persistent kernel launch.
 */
typedef struct fwbf_batch_s *fwbf_batch;

typedef struct {
    fwbf_code code;        /* code handle (its seg_len p is used) */
    const int8_t *y;       /* device int8 [n_frames][N], 16-byte aligned */
    int64_t n_frames;      /* >= 0 */
    int32_t max_iter;      /* >= 1 */
    float alpha;           /* 0 <= alpha <= 64 */
    uint32_t *out_bits;    /* device uint32 [n_frames][ceil(N/32)] */
    int32_t *out_iters;    /* device int32 [n_frames] */
    const void *mlp;       /* NULL: plain FWBF; else the learned network (see
                              fwbf_decode_learned), cyclic codes with packed = 1 or 2 */
    int32_t k_learn;       /* learned passes before the plain fallback (mlp != NULL) */
    int32_t gate_dv;       /* network consulted on learned passes with W_k >= gate_dv d_v
                              (see fwbf_decode_learned) */
} fwbf_batch_job;

/*
 * Builds a batch of 1..16 jobs (the descriptors are copied; buffers must stay
 * valid while the batch is used).
 *   warps_per_cta   1..16: warps per CTA of the launch (packed = 0 or 1)
 *   packed          1: cyclic codes use the packed two-positions-per-register
 *                   decoder, and quasi-cyclic codes with Z a multiple of 256
 *                   (plain jobs, warps_per_cta >= 4) the packed quasi-cyclic
 *                   decoder with 4 or 8 warps per frame; 0: every code uses the
 *                   list decoder; 2: as 1, with every frame decoded by a group
 *                   of warps in two 512-thread CTAs per SM when every job
 *                   allows it (cyclic codes with H / 32 divisible by 4 and at
 *                   least 8: 2 or 4 warps; those quasi-cyclic codes: 4, 8 or
 *                   16; any code of the list decoder: 2, 4 or 8), else as 1
 *                   (warps_per_cta is then ignored when the grouped launch is
 *                   taken).  Results are the same for every choice.
 * Allocates one device frame counter per job (owned by the handle); the job
 * table travels with every launch as its parameter block.  Errors:
 * FWBF_EINVAL, FWBF_EUNSUPPORTED (a code too large for one warp's shared
 * memory), FWBF_ENOMEM, FWBF_ECUDA.
 */
int fwbf_batch_create(const fwbf_batch_job *jobs, int32_t n_jobs, int32_t warps_per_cta,
                      int32_t packed, fwbf_batch *out);

/*
 * Decodes every job of the batch: clears the job counters and queues one
 * persistent launch on the stream.  It allocates nothing and does not
 * synchronise, so the call can be captured into a CUDA graph and replayed
 * (the buffers are those given at create time).  Calls of the same batch must
 * not overlap on the GPU (they share the counters).
 */
int fwbf_decode_batch(fwbf_batch b, void *stream);

/* How a batch decodes job `job` (0 <= job < the batch's job count), as chosen
 * at create time. */
typedef struct {
    int32_t decoder;          /* FWBF_DECODER_LIST, _CYCLIC or _QC */
    int32_t warps_per_frame;  /* warps that decode one frame together */
    int32_t frames_per_cta;   /* frames a CTA decodes at once for this job */
    int32_t grouped;          /* 1: the launch is the grouped kernel (two 512-thread
                                 CTAs per SM, every frame by a warp group) */
} fwbf_batch_job_info;

int fwbf_batch_query(fwbf_batch b, int32_t job, fwbf_batch_job_info *out);

/* Waits for the stream; FWBF_ETIMEOUT if a batch kernel gave up a bounded wait. */
int fwbf_batch_status(void *stream);

/* Releases a batch (waits for the device). NULL is a no-op. */
int fwbf_batch_destroy(fwbf_batch b);

/* ------------------------------------------------------------------------ */
/* Per-pass schedules and the learned schedule                              */
/* ------------------------------------------------------------------------ */

/*
 * The weighting factor alpha of Eq. 1 and the flip threshold of Sec. III
 * Step 2 (0 in the paper: flip iff E_b > 0) are the method's only parameters;
 * these entry points vary them per pass.  Both need a cyclic code (a single
 * circulant H, e.g. the EG(2,2^s) codes); other codes give FWBF_EUNSUPPORTED.
 *
 * Per-pass features (float [8], also what the learned network reads), for the
 * state at the start of pass k of a frame:
 *   0 W_k / N    1 W_{k-1} / N (W_0 at k = 0)    2 W_0 / N    3 k / 16
 *   4 flips of pass k-1 / n_blocks (0 at k = 0)
 *   5 bits with sum_m (2 s_m - 1) w_{n,m} >= 1 at pass k-1, / N (0 at k = 0)
 *   6 mean |q_n| / 127                            7 fraction of |q_n| < 8
 * (W_k: syndrome weight, N = M for a cyclic code.)
 */
#define FWBF_MLP_IN 8
#define FWBF_MLP_HIDDEN 64
#define FWBF_MLP_OUT 2
#define FWBF_MLP_PARAMS 4866
#define FWBF_MLP_BLOB_BYTES 10000

/*
 * fwbf_decode with alpha_q / theta_q (x256 fixed point, as alpha_q of
 * fwbf_decode) of pass k of frame f read from device arrays at
 * [f * sched_stride + k], k < max_iter (sched_stride = 0: one schedule for all
 * frames).  Values are clamped to alpha_q in [0, 16384], theta_q >= 0.  The
 * no-flip shortcut is not used (a later pass may use other parameters).
 *   out_feat    device float [n_frames][feat_passes][8] or NULL: the features
 *               above at the start of every pass k < feat_passes (unwritten for
 *               passes a frame does not run).
 */
int fwbf_decode_sched(fwbf_code c, const int8_t *y, int64_t n_frames, int32_t max_iter,
                      const int32_t *alpha_q, const int32_t *theta_q, int64_t sched_stride,
                      uint32_t *out_bits, int32_t *out_iters, float *out_feat,
                      int32_t feat_passes, void *stream);

/*
 * FWBF whose pass parameters come from the learned network, with plain FWBF
 * as the fallback.  For pass k < k_learn the decoding warps evaluate the
 * network on the features above: outputs (o0, o1) give alpha = o0 and
 * theta = 16 o1 (in units of the int8 metric; theta_q = 256 theta),
 * then snapped to steps of 1/2 (alpha) and 4 (theta) and clamped to [0, 64]
 * and [0, 4096].  The network is consulted only on passes whose syndrome
 * weight W_k is at least gate_dv d_v (d_v the largest column weight: about
 * gate_dv bit errors' worth of unsatisfied checks, the passes whose labels
 * most often differ from plain FWBF's parameters); the other passes use
 * (alpha_fallback, 0).  gate_dv >= 0 (0: every pass).  A larger gate evaluates
 * the network less often (faster) and keeps less of its frame-error gain.
 * Fallback: a frame whose syndrome is not zero after k_learn learned passes
 * gets plain FWBF's own result for it (what fwbf_decode with alpha_fallback
 * and max_iter gives: decisions and pass count).  If every learned pass so far
 * used (alpha_fallback, 0), the frame's state already is plain FWBF's and
 * decoding continues from it; otherwise the frame is decoded again from its
 * channel values.  (A learned pass at the fallback parameters that flips
 * nothing is treated alike at once: every later learned pass would repeat it.)
 *   mlp          device weight blob, FWBF_MLP_BLOB_BYTES, 16-byte aligned
 *                (written by fwbf_mlp_pack / fwbf_mlp_adam):
 *                W1 bf16[64][8] | W2 bf16 | W3 bf16[2][64] |
 *                b1 f32[64] | b2 f32[64] | b3 f32[2]  (bytes 0, 1024, 9216,
 *                9472, 9728, 9984).  W2 (unit u, input c) is stored in 512
 *                groups of eight: group 64 (c / 8) + u, element c % 8, so that
 *                lanes taking consecutive units read contiguous bytes.
 *   out_sched    device int32 [n_frames][k_learn][2] or NULL: the (alpha_q,
 *                theta_q) used in every learned pass that ran (unwritten for
 *                the passes a frame skips)
 *   out_feat, feat_passes   as fwbf_decode_sched
 */
int fwbf_decode_learned(fwbf_code c, const int8_t *y, int64_t n_frames, int32_t max_iter,
                        int32_t k_learn, int32_t gate_dv, float alpha_fallback, const void *mlp,
                        uint32_t *out_bits, int32_t *out_iters, int32_t *out_sched,
                        float *out_feat, int32_t feat_passes, void *stream);

/*
 * Training kernels of the network (float32 master parameters in the blob's
 * order: W1, W2, W3, b1, b2, b3, FWBF_MLP_PARAMS floats, device).
 *   fwbf_mlp_pack     master -> blob (weights rounded to bf16)
 *   fwbf_mlp_forward  out[n][2] = network(x[n][8]) with the blob's weights
 *   fwbf_mlp_grad     adds to grad the gradient, with respect to the blob's
 *                     weights, of sum over the n samples of
 *                     ||network(x_s) - target_s||^2 / n_total, and that sum to
 *                     *loss (device float)
 *   fwbf_mlp_adam     one Adam step (step >= 1) on master with grad; rewrites
 *                     the blob and clears grad
 */
int fwbf_mlp_pack(const float *master, void *blob, void *stream);
int fwbf_mlp_forward(const void *blob, const float *x, int64_t n, float *out, void *stream);
int fwbf_mlp_grad(const void *blob, const float *x, const float *target, int64_t n, int64_t n_total,
                  float *grad, float *loss, void *stream);
int fwbf_mlp_adam(float *master, void *blob, float *grad, float *m, float *v, int64_t step,
                  float lr, float beta1, float beta2, float eps, void *stream);

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
