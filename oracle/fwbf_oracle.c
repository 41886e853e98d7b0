/*
 * CPU oracle for FWBF (fast weighted bit-flipping) LDPC decoding.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously correct
 * statement of what the decoder computes.  Only the tests, the smoke check and
 * the benchmark's CPU-baseline leg may load it; the decoding library never
 * does, and it shares no code, header or table with the CUDA path.
 *
 * What it follows (Ma, Li, Zhu, Zhang, Qi, "An Improved WBF Algorithm for
 * Higher-Speed Decoding of LDPC Codes"):
 *   Sec. II      notation: H (M x N), N(m) = bits of check m, M(n) = checks of
 *                bit n, syndrome s = z H^T and its weight w_k.
 *   Eq. 1        IMWBF metric E_n = sum_{m in M(n)} (2 s_m - 1) w_{n,m} - alpha |y_n|
 *                with w_{n,m} = min_{i in N(m)\n} |y_i|.
 *   Sec. III     FWBF: initialisation (z_0 = (1 - sgn y)/2, weights w_{n,m});
 *                Step 1 (syndrome weight, stop test); Step 2 (per p-length block:
 *                arg-max of E, flip it if its metric is positive); k = k + 1.
 *   footnote 1   a short last block is padded with "null" metrics that never win.
 *
 * Readings where the paper is silent or garbled (each one is listed with its
 * reason in the design notes):
 *   sgn(0)       z_0[n] = 1 iff y_n < 0 (q_n < 0); zero maps to bit 0.
 *   stop test    at most max_iter flip passes; the result after pass k is z_k.
 *                iters = k when the syndrome of z_k is zero, -max_iter when it
 *                is still non-zero after max_iter passes.
 *   ties         inside a block the lowest bit index wins.
 *   flip test    strict: flip iff E_b > theta (theta = 0 in the paper).
 *   blocks       contiguous [i p, min(N, (i+1) p)), B = ceil(N / p); all blocks
 *                read the same syndrome s_k and their flips are applied together.
 *   weights      w_{n,m} is computed once, from the channel values, at
 *                initialisation.
 *   int8 path    q_n = saturate_{+-127}(round_half_even(16 y_n)), NaN -> 0;
 *                the decoders read an int8 input of -128 (outside that range)
 *                as -127; a_n = |q_n|; the metric is scaled by 256 so that
 *                E'_n = 256 sum (2 s_m - 1) w_{n,m} - alpha_q a_n with
 *                alpha_q = round_half_even(256 alpha) is an exact integer.
 *
 * Build: gcc -O2 -shared -fPIC fwbf_oracle.c -o liboracle.so -lm
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* An int8 channel value as the decoders read it: the quantiser's range is the
 * symmetric [-127, 127], and -128 is read as -127. */
static int32_t channel_q(int8_t v) { return v < -127 ? -127 : (int32_t)v; }

#define ORACLE_OK 0
#define ORACLE_EINVAL -1
#define ORACLE_ENOMEM -2
#define ORACLE_EOVERFLOW -3

/* ------------------------------------------------------------------------ */
/* H as index lists (Sec. II: N(m) and M(n))                                 */
/* ------------------------------------------------------------------------ */

typedef struct {
    int N, M;
    int64_t nnz;
    int64_t *row_ptr;  /* [M+1]  N(m) = row_bit[row_ptr[m] .. row_ptr[m+1]) */
    int32_t *row_bit;  /* [nnz]  bits of each check, ascending */
    int64_t *col_ptr;  /* [N+1]  M(n) = col_chk[col_ptr[n] .. col_ptr[n+1]) */
    int32_t *col_chk;  /* [nnz]  checks of each bit, ascending */
} ocode;

static void ocode_free(ocode *c) {
    free(c->row_ptr);
    free(c->row_bit);
    free(c->col_ptr);
    free(c->col_chk);
    memset(c, 0, sizeof(*c));
}

static int cmp_i32(const void *a, const void *b) {
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

static int ocode_build(int N, int M, int64_t nnz, const int32_t *rows,
                       const int32_t *cols, ocode *c) {
    memset(c, 0, sizeof(*c));
    if (N <= 0 || M <= 0 || nnz <= 0) return ORACLE_EINVAL;
    c->N = N;
    c->M = M;
    c->nnz = nnz;
    c->row_ptr = calloc((size_t)M + 1, sizeof(int64_t));
    c->col_ptr = calloc((size_t)N + 1, sizeof(int64_t));
    c->row_bit = malloc((size_t)nnz * sizeof(int32_t));
    c->col_chk = malloc((size_t)nnz * sizeof(int32_t));
    if (!c->row_ptr || !c->col_ptr || !c->row_bit || !c->col_chk) {
        ocode_free(c);
        return ORACLE_ENOMEM;
    }
    for (int64_t e = 0; e < nnz; ++e) {
        if (rows[e] < 0 || rows[e] >= M || cols[e] < 0 || cols[e] >= N) {
            ocode_free(c);
            return ORACLE_EINVAL;
        }
        c->row_ptr[rows[e] + 1]++;
        c->col_ptr[cols[e] + 1]++;
    }
    for (int m = 0; m < M; ++m) c->row_ptr[m + 1] += c->row_ptr[m];
    for (int n = 0; n < N; ++n) c->col_ptr[n + 1] += c->col_ptr[n];
    int64_t *rfill = calloc((size_t)M, sizeof(int64_t));
    int64_t *cfill = calloc((size_t)N, sizeof(int64_t));
    if (!rfill || !cfill) {
        free(rfill);
        free(cfill);
        ocode_free(c);
        return ORACLE_ENOMEM;
    }
    for (int64_t e = 0; e < nnz; ++e) {
        c->row_bit[c->row_ptr[rows[e]] + rfill[rows[e]]++] = cols[e];
        c->col_chk[c->col_ptr[cols[e]] + cfill[cols[e]]++] = rows[e];
    }
    free(rfill);
    free(cfill);
    for (int m = 0; m < M; ++m)
        qsort(c->row_bit + c->row_ptr[m], (size_t)(c->row_ptr[m + 1] - c->row_ptr[m]),
              sizeof(int32_t), cmp_i32);
    for (int n = 0; n < N; ++n)
        qsort(c->col_chk + c->col_ptr[n], (size_t)(c->col_ptr[n + 1] - c->col_ptr[n]),
              sizeof(int32_t), cmp_i32);
    /* a check needs at least two bits for N(m)\n to be non-empty (Eq. 1) */
    for (int m = 0; m < M; ++m)
        if (c->row_ptr[m + 1] - c->row_ptr[m] < 2) {
            ocode_free(c);
            return ORACLE_EINVAL;
        }
    return ORACLE_OK;
}

/* ------------------------------------------------------------------------ */
/* Quantiser (int8 channel values)                                           */
/* ------------------------------------------------------------------------ */

/* q = saturate to [-127, 127] of round-half-to-even(16 y); NaN -> 0.
 * 16 y is exact in double, and nearbyint rounds half to even in the default
 * rounding mode. */
int oracle_quantize(const float *y, int8_t *q, int64_t count) {
    for (int64_t i = 0; i < count; ++i) {
        double v = (double)y[i] * 16.0;
        double r;
        if (isnan(v))
            r = 0.0;
        else {
            r = nearbyint(v);
            if (r > 127.0) r = 127.0;
            if (r < -127.0) r = -127.0;
        }
        q[i] = (int8_t)r;
    }
    return ORACLE_OK;
}

/* round-half-to-even of 256 * alpha (fixed-point weighting factor) */
int32_t oracle_alpha_q(double alpha) { return (int32_t)nearbyint(alpha * 256.0); }

/* ------------------------------------------------------------------------ */
/* FWBF on int8 channel values (Sec. III with Eq. 1)                         */
/* ------------------------------------------------------------------------ */

/*
 * Decodes n_frames frames q[f][N].
 *   p              block length of the partially parallel bit-choose, 1..N
 *   alpha_q, theta_q   per-pass weighting factor (x256) and flip threshold (x256)
 *                  of pass k of frame f at [f * sched_stride + k]; sched_stride = 0
 *                  shares one schedule between all frames (plain FWBF: alpha_q
 *                  constant, theta_q = 0).
 *   out_bits       [n_frames][ceil(N/32)] decisions z, bit n in word n/32 at n%32
 *   out_iters      [n_frames] k >= 0 converged after k passes, -max_iter failed
 * Optional single-frame trace (n_frames == 1, pointers may be NULL):
 *   trace_s        [max_iter + 1][M] syndrome at the start of each pass
 *   trace_E        [max_iter][N] metric E' of each pass
 *   trace_flip     [max_iter][N] 1 where the pass flipped the bit
 */
int oracle_fwbf_i8(int N, int M, int64_t nnz, const int32_t *rows, const int32_t *cols,
                   int32_t p, const int8_t *q, int64_t n_frames, int32_t max_iter,
                   const int32_t *alpha_q, const int32_t *theta_q, int64_t sched_stride,
                   uint32_t *out_bits, int32_t *out_iters,
                   uint8_t *trace_s, int64_t *trace_E, uint8_t *trace_flip) {
    if (p < 1 || p > N || max_iter < 1 || n_frames < 0) return ORACLE_EINVAL;
    ocode c;
    int rc = ocode_build(N, M, nnz, rows, cols, &c);
    if (rc) return rc;
    const int words = (N + 31) / 32;
    const int B = (N + p - 1) / p;
    int32_t *a = malloc(sizeof(int32_t) * (size_t)N);
    uint8_t *z = malloc((size_t)N);
    uint8_t *s = malloc((size_t)M);
    uint8_t *mark = malloc((size_t)N);
    int64_t *E = malloc(sizeof(int64_t) * (size_t)N);
    int32_t *w = malloc(sizeof(int32_t) * (size_t)nnz); /* w at row_bit positions */
    if (!a || !z || !s || !mark || !E || !w) {
        rc = ORACLE_ENOMEM;
        goto done;
    }
    for (int64_t f = 0; f < n_frames; ++f) {
        const int8_t *qf = q + f * (int64_t)N;
        /* Initialisation: z_0 and a_n */
        for (int n = 0; n < N; ++n) {
            const int32_t v = channel_q(qf[n]);
            a[n] = v < 0 ? -v : v;
            z[n] = v < 0 ? 1 : 0;
        }
        /* Initialisation: w_{n,m} = min over N(m)\n of a_i, directly */
        for (int m = 0; m < M; ++m) {
            for (int64_t e = c.row_ptr[m]; e < c.row_ptr[m + 1]; ++e) {
                int32_t best = INT32_MAX;
                for (int64_t e2 = c.row_ptr[m]; e2 < c.row_ptr[m + 1]; ++e2) {
                    if (e2 == e) continue;
                    if (a[c.row_bit[e2]] < best) best = a[c.row_bit[e2]];
                }
                w[e] = best;
            }
        }
        int k = 0;
        int32_t iters;
        for (;;) {
            /* Step 1: syndrome s_k = z_k H^T and its weight */
            int64_t wk = 0;
            for (int m = 0; m < M; ++m) {
                int par = 0;
                for (int64_t e = c.row_ptr[m]; e < c.row_ptr[m + 1]; ++e) par ^= z[c.row_bit[e]];
                s[m] = (uint8_t)par;
                wk += par;
            }
            if (trace_s && n_frames == 1 && k <= max_iter) memcpy(trace_s + (int64_t)k * M, s, (size_t)M);
            if (wk == 0) {
                iters = k;
                break;
            }
            if (k == max_iter) {
                iters = -max_iter;
                break;
            }
            const int64_t aq = alpha_q[f * sched_stride + k];
            const int64_t tq = theta_q[f * sched_stride + k];
            /* Step 2a: metric of Eq. 1 for every bit, scaled by 256 */
            for (int n = 0; n < N; ++n) {
                int64_t acc = 0;
                for (int64_t ce = c.col_ptr[n]; ce < c.col_ptr[n + 1]; ++ce) {
                    int m = c.col_chk[ce];
                    /* find w_{n,m}: the entry of bit n in row m */
                    int64_t e = c.row_ptr[m];
                    while (c.row_bit[e] != n) ++e;
                    acc += (2 * (int64_t)s[m] - 1) * (int64_t)w[e];
                }
                E[n] = 256 * acc - aq * (int64_t)a[n];
                if (E[n] > INT32_MAX || E[n] < INT32_MIN) {
                    rc = ORACLE_EOVERFLOW;
                    goto done;
                }
            }
            if (trace_E && n_frames == 1) memcpy(trace_E + (int64_t)k * N, E, sizeof(int64_t) * (size_t)N);
            /* Step 2b: one candidate per p-length block, first index wins ties */
            memset(mark, 0, (size_t)N);
            for (int i = 0; i < B; ++i) {
                int lo = i * p;
                int hi = lo + p < N ? lo + p : N; /* short last block: nulls never win */
                int b = lo;
                for (int n = lo + 1; n < hi; ++n)
                    if (E[n] > E[b]) b = n;
                if (E[b] > tq) mark[b] = 1;
            }
            if (trace_flip && n_frames == 1) memcpy(trace_flip + (int64_t)k * N, mark, (size_t)N);
            /* all blocks used s_k; apply their flips together */
            for (int n = 0; n < N; ++n) z[n] ^= mark[n];
            k = k + 1;
        }
        uint32_t *ob = out_bits + f * (int64_t)words;
        memset(ob, 0, sizeof(uint32_t) * (size_t)words);
        for (int n = 0; n < N; ++n)
            if (z[n]) ob[n / 32] |= 1u << (n % 32);
        out_iters[f] = iters;
    }
done:
    free(a);
    free(z);
    free(s);
    free(mark);
    free(E);
    free(w);
    ocode_free(&c);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* FWBF on real channel values, double precision                             */
/* ------------------------------------------------------------------------ */

/*
 * Same steps with a_n = |y_n|, z_0[n] = (y_n < 0) and E_n of Eq. 1 in double.
 *   out_margin   [n_frames] (may be NULL): smallest decision margin met on the
 *                way, over every pass and block: min(E_b - theta for the flip
 *                test (absolute), E_b - second largest E in the block).  A frame
 *                whose margin exceeds the rounding error of a lower-precision
 *                metric takes the same decisions at that precision.
 *   out_E0       [n_frames][N] (may be NULL): the metric of the first pass
 *                (k = 0), computed for every frame whether or not it converged.
 */
int oracle_fwbf_f64(int N, int M, int64_t nnz, const int32_t *rows, const int32_t *cols,
                    int32_t p, const float *y, int64_t n_frames, int32_t max_iter,
                    double alpha, double theta, uint32_t *out_bits, int32_t *out_iters,
                    double *out_margin, double *out_E0) {
    if (p < 1 || p > N || max_iter < 1 || n_frames < 0) return ORACLE_EINVAL;
    ocode c;
    int rc = ocode_build(N, M, nnz, rows, cols, &c);
    if (rc) return rc;
    const int words = (N + 31) / 32;
    const int B = (N + p - 1) / p;
    double *a = malloc(sizeof(double) * (size_t)N);
    uint8_t *z = malloc((size_t)N);
    uint8_t *s = malloc((size_t)M);
    uint8_t *mark = malloc((size_t)N);
    double *E = malloc(sizeof(double) * (size_t)N);
    double *w = malloc(sizeof(double) * (size_t)nnz);
    if (!a || !z || !s || !mark || !E || !w) {
        rc = ORACLE_ENOMEM;
        goto done;
    }
    for (int64_t f = 0; f < n_frames; ++f) {
        const float *yf = y + f * (int64_t)N;
        double margin = INFINITY;
        for (int n = 0; n < N; ++n) {
            a[n] = fabs((double)yf[n]);
            z[n] = yf[n] < 0.0f ? 1 : 0;
        }
        for (int m = 0; m < M; ++m)
            for (int64_t e = c.row_ptr[m]; e < c.row_ptr[m + 1]; ++e) {
                double best = INFINITY;
                for (int64_t e2 = c.row_ptr[m]; e2 < c.row_ptr[m + 1]; ++e2)
                    if (e2 != e && a[c.row_bit[e2]] < best) best = a[c.row_bit[e2]];
                w[e] = best;
            }
        int k = 0;
        int32_t iters;
        int have_E0 = 0;
        for (;;) {
            int64_t wk = 0;
            for (int m = 0; m < M; ++m) {
                int par = 0;
                for (int64_t e = c.row_ptr[m]; e < c.row_ptr[m + 1]; ++e) par ^= z[c.row_bit[e]];
                s[m] = (uint8_t)par;
                wk += par;
            }
            int stop = 0;
            if (wk == 0) {
                iters = k;
                stop = 1;
            } else if (k == max_iter) {
                iters = -max_iter;
                stop = 1;
            }
            if (stop && (!out_E0 || have_E0)) break;
            for (int n = 0; n < N; ++n) {
                double acc = 0.0;
                for (int64_t ce = c.col_ptr[n]; ce < c.col_ptr[n + 1]; ++ce) {
                    int m = c.col_chk[ce];
                    int64_t e = c.row_ptr[m];
                    while (c.row_bit[e] != n) ++e;
                    acc += (2.0 * s[m] - 1.0) * w[e];
                }
                E[n] = acc - alpha * a[n];
            }
            if (out_E0 && !have_E0) {
                memcpy(out_E0 + f * (int64_t)N, E, sizeof(double) * (size_t)N);
                have_E0 = 1;
            }
            if (stop) break;
            memset(mark, 0, (size_t)N);
            for (int i = 0; i < B; ++i) {
                int lo = i * p;
                int hi = lo + p < N ? lo + p : N;
                int b = lo;
                for (int n = lo + 1; n < hi; ++n)
                    if (E[n] > E[b]) b = n;
                double second = -INFINITY;
                for (int n = lo; n < hi; ++n)
                    if (n != b && E[n] > second) second = E[n];
                double mg = fabs(E[b] - theta);
                if (hi - lo > 1 && E[b] - second < mg) mg = E[b] - second;
                if (mg < margin) margin = mg;
                if (E[b] > theta) mark[b] = 1;
            }
            for (int n = 0; n < N; ++n) z[n] ^= mark[n];
            k = k + 1;
        }
        uint32_t *ob = out_bits + f * (int64_t)words;
        memset(ob, 0, sizeof(uint32_t) * (size_t)words);
        for (int n = 0; n < N; ++n)
            if (z[n]) ob[n / 32] |= 1u << (n % 32);
        out_iters[f] = iters;
        if (out_margin) out_margin[f] = margin;
    }
done:
    free(a);
    free(z);
    free(s);
    free(mark);
    free(E);
    free(w);
    ocode_free(&c);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Single-bit flipping (Sec. II, after Eq. 1), written on its own            */
/* ------------------------------------------------------------------------ */

/*
 * IMWBF-style decoding that flips only the bit with the globally largest
 * metric per pass, with FWBF's flip test (E > theta) and lowest-index ties.
 * It is FWBF with p = N; it is written separately (dense H, weights recomputed
 * from their definition on every use) so the two can be checked against each
 * other.  int8 channel values, fixed alpha_q, theta_q.
 */
int oracle_single_flip_i8(int N, int M, int64_t nnz, const int32_t *rows, const int32_t *cols,
                          const int8_t *q, int64_t n_frames, int32_t max_iter, int32_t alpha_q,
                          int32_t theta_q, uint32_t *out_bits, int32_t *out_iters) {
    if (N <= 0 || M <= 0 || max_iter < 1) return ORACLE_EINVAL;
    uint8_t *H = calloc((size_t)M * (size_t)N, 1);
    uint8_t *z = malloc((size_t)N);
    int32_t *a = malloc(sizeof(int32_t) * (size_t)N);
    uint8_t *s = malloc((size_t)M);
    if (!H || !z || !a || !s) {
        free(H);
        free(z);
        free(a);
        free(s);
        return ORACLE_ENOMEM;
    }
    for (int64_t e = 0; e < nnz; ++e) H[(size_t)rows[e] * N + cols[e]] = 1;
    const int words = (N + 31) / 32;
    for (int64_t f = 0; f < n_frames; ++f) {
        for (int n = 0; n < N; ++n) {
            int v = channel_q(q[f * N + n]);
            z[n] = v < 0;
            a[n] = v < 0 ? -v : v;
        }
        int32_t iters = 0;
        for (int k = 0;; ++k) {
            int weight = 0;
            for (int m = 0; m < M; ++m) {
                int par = 0;
                for (int n = 0; n < N; ++n)
                    if (H[(size_t)m * N + n]) par ^= z[n];
                s[m] = (uint8_t)par;
                weight += par;
            }
            if (weight == 0) {
                iters = k;
                break;
            }
            if (k == max_iter) {
                iters = -max_iter;
                break;
            }
            int64_t best = 0;
            int arg = -1;
            for (int n = 0; n < N; ++n) {
                int64_t sum = 0;
                for (int m = 0; m < M; ++m) {
                    if (!H[(size_t)m * N + n]) continue;
                    int wmin = 1 << 30;
                    for (int i = 0; i < N; ++i)
                        if (i != n && H[(size_t)m * N + i] && a[i] < wmin) wmin = a[i];
                    sum += s[m] ? wmin : -wmin;
                }
                int64_t metric = 256 * sum - (int64_t)alpha_q * a[n];
                if (arg < 0 || metric > best) {
                    best = metric;
                    arg = n;
                }
            }
            if (best > theta_q) z[arg] ^= 1;
        }
        uint32_t *ob = out_bits + f * (int64_t)words;
        memset(ob, 0, sizeof(uint32_t) * (size_t)words);
        for (int n = 0; n < N; ++n)
            if (z[n]) ob[n / 32] |= 1u << (n % 32);
        out_iters[f] = iters;
    }
    free(H);
    free(z);
    free(a);
    free(s);
    return ORACLE_OK;
}

/* ------------------------------------------------------------------------ */
/* lambda-largest selection (Sec. III, MLP-WBF's bit-choose), written on its  */
/* own                                                                       */
/* ------------------------------------------------------------------------ */

/*
 * Per pass: the IMWBF metric of Eq. 1 for every bit (x256, int8 path), then
 * the lambda bits with the largest metrics -- chosen one after another, each
 * the largest remaining, lowest index first among equals -- are flipped if
 * their metric is above theta_q.  All choices read the same syndrome.  lambda = 1
 * is single-bit flipping; lambda >= N flips every bit with a positive metric.
 */
int oracle_lambda_i8(int N, int M, int64_t nnz, const int32_t *rows, const int32_t *cols, int32_t lambda,
                     const int8_t *q, int64_t n_frames, int32_t max_iter, int32_t alpha_q, int32_t theta_q,
                     uint32_t *out_bits, int32_t *out_iters) {
    if (lambda < 1 || max_iter < 1) return ORACLE_EINVAL;
    ocode c;
    int rc = ocode_build(N, M, nnz, rows, cols, &c);
    if (rc) return rc;
    const int words = (N + 31) / 32;
    int32_t *a = malloc(sizeof(int32_t) * (size_t)N);
    uint8_t *z = malloc((size_t)N), *s = malloc((size_t)M), *taken = malloc((size_t)N);
    int64_t *E = malloc(sizeof(int64_t) * (size_t)N);
    if (!a || !z || !s || !taken || !E) {
        rc = ORACLE_ENOMEM;
        goto done;
    }
    for (int64_t f = 0; f < n_frames; ++f) {
        for (int n = 0; n < N; ++n) {
            int v = channel_q(q[f * N + n]);
            a[n] = v < 0 ? -v : v;
            z[n] = v < 0;
        }
        int32_t iters;
        for (int k = 0;; ++k) {
            int weight = 0;
            for (int m = 0; m < M; ++m) {
                int par = 0;
                for (int64_t e = c.row_ptr[m]; e < c.row_ptr[m + 1]; ++e) par ^= z[c.row_bit[e]];
                s[m] = (uint8_t)par;
                weight += par;
            }
            if (weight == 0) {
                iters = k;
                break;
            }
            if (k == max_iter) {
                iters = -max_iter;
                break;
            }
            for (int n = 0; n < N; ++n) {
                int64_t sum = 0;
                for (int64_t ce = c.col_ptr[n]; ce < c.col_ptr[n + 1]; ++ce) {
                    const int m = c.col_chk[ce];
                    int wmin = 1 << 30;
                    for (int64_t e = c.row_ptr[m]; e < c.row_ptr[m + 1]; ++e) {
                        const int i = c.row_bit[e];
                        if (i != n && a[i] < wmin) wmin = a[i];
                    }
                    sum += s[m] ? wmin : -wmin;
                }
                E[n] = 256 * sum - (int64_t)alpha_q * a[n];
            }
            memset(taken, 0, (size_t)N);
            for (int t = 0; t < lambda && t < N; ++t) {
                int best = -1;
                for (int n = 0; n < N; ++n)
                    if (!taken[n] && (best < 0 || E[n] > E[best])) best = n;
                if (best < 0 || E[best] <= theta_q) break;
                taken[best] = 1;
            }
            for (int n = 0; n < N; ++n) z[n] ^= taken[n];
        }
        uint32_t *ob = out_bits + f * (int64_t)words;
        memset(ob, 0, sizeof(uint32_t) * (size_t)words);
        for (int n = 0; n < N; ++n)
            if (z[n]) ob[n / 32] |= 1u << (n % 32);
        out_iters[f] = iters;
    }
done:
    free(a);
    free(z);
    free(s);
    free(taken);
    free(E);
    ocode_free(&c);
    return rc;
}
