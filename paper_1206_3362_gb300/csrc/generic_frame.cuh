// Per-frame body of the generic int8 FWBF decoder (any H, index lists or
// circulant lists), shared by the single-code kernel (decode_i8.cu) and the
// batched multi-code kernel (decode_batch.cu).  The reformulation it uses is
// described at the top of decode_i8.cu.
#pragma once

#include "device_common.cuh"
#include "fwbf_internal.h"

namespace fwbf {

struct I8Params {
    const uint32_t *table;  // global blob
    uint32_t table_words;
    int table_in_smem;
    int N, M, Z, MB, NB;
    uint32_t rptr_off, rent_off, cptr_off, cent_off;
    int p, B;
    uint32_t p_magic, z_magic;
    const int8_t *y;
    int64_t F;
    int max_iter, alpha_q, theta_q;
    uint32_t *out_bits;
    int32_t *out_iters;
    unsigned long long *counter;
    // per-warp shared-memory layout (bytes)
    uint32_t warp_bytes, off_T, off_crec, off_s, off_z, off_keys;
    uint32_t table_smem_bytes;
    // lambda-largest selection (MLP-WBF's bit-choose) in place of the p-blocks
    // when lambda > 0: candidates go to a per-frame list, the flip list holds
    // up to max(B, lambda) bits
    int lambda;
    int nkeys;
    uint32_t off_cand;
    uint32_t off_red;  // group sums: 2 halves x 4 ints x up to 8 warps
    int dc_max;        // largest row weight
};

// maximum of a 64-bit key over the warp
__device__ __forceinline__ unsigned long long warp_max_u64(unsigned long long v) {
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
        const unsigned long long o = __shfl_xor_sync(FULL, v, d);
        v = o > v ? o : v;
    }
    return v;
}

// Decodes frame f of P with a group of WPF warps (thread t of 32 * WPF); tbl
// is the code's table blob (shared or global memory), ws the group's
// shared-memory slice, bar_id its named barrier (WPF > 1).  Checks are taken
// 32 at a time per warp, bits and flip blocks strided over the group's
// threads.  lambda-largest selection (P.lambda > 0) runs with WPF = 1 only.
template <bool PLAIN, int WPF>  // PLAIN: Z == 1, the tables are plain CSR / CSC
__device__ __forceinline__ void generic_frame(const I8Params &P, const uint32_t *tbl, unsigned char *ws, int t,
                                              int bar_id, unsigned long long f) {
    constexpr int G = 32 * WPF;
    const int lane = t & 31, gw = t >> 5;
    const uint32_t *rptr = tbl + P.rptr_off;
    const uint32_t *rent = tbl + P.rent_off;
    const uint32_t *cptr = tbl + P.cptr_off;
    const uint32_t *cent = tbl + P.cent_off;
    int8_t *stage = reinterpret_cast<int8_t *>(ws);
    uint32_t *T = reinterpret_cast<uint32_t *>(ws + P.off_T);
    uint32_t *crec = reinterpret_cast<uint32_t *>(ws + P.off_crec);
    uint32_t *sbits = reinterpret_cast<uint32_t *>(ws + P.off_s);
    uint32_t *zbits = reinterpret_cast<uint32_t *>(ws + P.off_z);
    unsigned long long *keys = reinterpret_cast<unsigned long long *>(ws + P.off_keys);
    unsigned long long *cand = reinterpret_cast<unsigned long long *>(ws + P.off_cand);  // lambda mode
    uint32_t *ncand = reinterpret_cast<uint32_t *>(ws + P.off_cand + 8u * (uint32_t)P.N);
    int *red = reinterpret_cast<int *>(ws + P.off_red);
    int rhalf = 0;
    const int N = P.N, M = P.M;
    const uint32_t Z = (uint32_t)P.Z;
    const int Nw = (N + 31) >> 5, Mw = (M + 31) >> 5;
    const uintptr_t ybase = reinterpret_cast<uintptr_t>(P.y);
    const uintptr_t yend = ybase + (uintptr_t)(P.F * (int64_t)N);
    // row of check m: table row R and circulant index i
    auto row_of = [&](uint32_t m, uint32_t &R, uint32_t &i) {
        if (PLAIN) {
            R = m;
            i = 0;
        } else {
            R = div_small(m, Z, P.z_magic);
            i = m - R * Z;
        }
    };

    // ---- load the frame: aligned 16-byte chunks covering it --------------
    const uintptr_t fb = ybase + (uintptr_t)(f * (unsigned long long)N);
    const uintptr_t a0 = fb & ~(uintptr_t)15;
    const int off = (int)(fb - a0);
    const int nchunks = (off + N + 15) >> 4;
    for (int c = t; c < nchunks; c += G) {
        const uintptr_t src = a0 + (uintptr_t)c * 16;
        uint4 v;
        if (src + 16 <= yend) {
            v = __ldcs(reinterpret_cast<const uint4 *>(src));
        } else {  // tail of the buffer: byte loads, never past its end
            uint32_t wv[4] = {0u, 0u, 0u, 0u};
#pragma unroll
            for (int i = 0; i < 16; ++i)
                if (src + i < yend)
                    wv[i >> 2] |= (uint32_t)(*reinterpret_cast<const unsigned char *>(src + i)) << (8 * (i & 3));
            v = make_uint4(wv[0], wv[1], wv[2], wv[3]);
        }
        *reinterpret_cast<uint4 *>(stage + c * 16) = clamp_m127(v);  // -128 decodes as -127
    }
    for (int n = t; n < N; n += G) T[n] = 0u;
    group_sync<WPF>(bar_id);
    const int8_t *q = stage + off;

    // ---- initialisation: z_0, per-check (min1, min2, pos), s_0, tot, U ---
    for (int w = gw; w < Nw; w += WPF) {
        const int n = (w << 5) + lane;
        const uint32_t zb = __ballot_sync(FULL, n < N && q[n] < 0);
        if (lane == 0) zbits[w] = zb;
    }
    int W = 0;
    for (int base = 32 * gw; base < M; base += G) {
        const int m = base + lane;
        uint32_t s = 0;
        if (m < M) {
            uint32_t R, i;
            row_of(m, R, i);
            const uint32_t e0 = rptr[R], e1 = rptr[R + 1];
            uint32_t k1 = 0xffffu, k2 = 0xffffu, par = 0;
            for (uint32_t e = e0; e < e1; ++e) {
                const uint32_t n = PLAIN ? (rent[e] >> 16) : circ_index(rent[e], i, Z);
                const int v = q[n];
                const uint32_t key = ((uint32_t)abs(v) << 8) | (e - e0);
                par ^= (uint32_t)v;
                k2 = min(k2, max(k1, key));
                k1 = min(k1, key);
            }
            s = (par >> 7) & 1u;
            const uint32_t min1 = k1 >> 8, pos = k1 & 0xffu, min2 = k2 >> 8;
            crec[m] = min1 | (min2 << 8) | (pos << 16);
            const uint32_t mult = 65536u + s;  // tot in the high half, U in the low half
            for (uint32_t e = e0; e < e1; ++e) {
                const uint32_t n = PLAIN ? (rent[e] >> 16) : circ_index(rent[e], i, Z);
                const uint32_t wv = (e - e0 == pos) ? min2 : min1;
                atomicAdd(&T[n], wv * mult);
            }
        }
        const uint32_t sw = __ballot_sync(FULL, s);
        if (lane == 0) sbits[base >> 5] = sw;
        W += __popc(sw);
    }
    W = group_sum3<WPF>(make_int3(W, 0, 0), red, rhalf, lane, gw, bar_id).x;  // (meets the group if WPF > 1)
    if constexpr (WPF == 1) __syncwarp();

    // ---- iterations --------------------------------------------------------
    int iters;
    for (int k = 0;; ++k) {
        if (W == 0) {
            iters = k;
            break;
        }
        if (k == P.max_iter) {
            iters = -P.max_iter;
            break;
        }
        if (k > 0) {  // U_n from the unsatisfied checks of s_k
            if (P.dc_max >= 16) {
                // wide rows: the warp's 32 lanes share the edges of one unsatisfied check
                for (int wd = gw; wd < Mw; wd += WPF) {
                    uint32_t bits = sbits[wd];
                    while (bits) {
                        const int j = __ffs(bits) - 1;
                        bits &= bits - 1;
                        const uint32_t m = (wd << 5) + j;
                        const uint32_t rec = crec[m];
                        const uint32_t min1 = rec & 0xffu, min2 = (rec >> 8) & 0xffu, pos = rec >> 16;
                        uint32_t R, i;
                        row_of(m, R, i);
                        const uint32_t e0 = rptr[R], e1 = rptr[R + 1];
                        for (uint32_t e = e0 + lane; e < e1; e += 32) {
                            const uint32_t n = PLAIN ? (rent[e] >> 16) : circ_index(rent[e], i, Z);
                            atomicAdd(&T[n], (e - e0 == pos) ? min2 : min1);
                        }
                    }
                }
            } else {
                // narrow rows: a lane per syndrome word, its checks one after another
                for (int wd = t; wd < Mw; wd += G) {
                    uint32_t bits = sbits[wd];
                    while (bits) {
                        const int j = __ffs(bits) - 1;
                        bits &= bits - 1;
                        const uint32_t m = (wd << 5) + j;
                        const uint32_t rec = crec[m];
                        const uint32_t min1 = rec & 0xffu, min2 = (rec >> 8) & 0xffu, pos = rec >> 16;
                        uint32_t R, i;
                        row_of(m, R, i);
                        const uint32_t e0 = rptr[R], e1 = rptr[R + 1];
                        for (uint32_t e = e0; e < e1; ++e) {
                            const uint32_t n = PLAIN ? (rent[e] >> 16) : circ_index(rent[e], i, Z);
                            atomicAdd(&T[n], (e - e0 == pos) ? min2 : min1);
                        }
                    }
                }
            }
            group_sync<WPF>(bar_id);
        }
        // metric and per-block candidates
        for (int n = t; n < N; n += G) {
            const uint32_t tv = T[n];
            const uint32_t U = tv & 0xffffu;
            if (U) T[n] = tv & 0xffff0000u;
            const int tot = (int)(tv >> 16);
            const int E = (2 * (int)U - tot) * 256 - P.alpha_q * abs((int)q[n]);
            if (E > P.theta_q) {
                const unsigned long long key =
                    ((unsigned long long)((uint32_t)E ^ 0x80000000u) << 32) | (0xffffffffu - (uint32_t)n);
                if (WPF == 1 && P.lambda) {
                    cand[atomicAdd(ncand, 1u)] = key;
                } else {
                    const uint32_t blk = div_small((uint32_t)n, P.p, P.p_magic);
                    atomicMax(&keys[blk], key);
                }
            }
        }
        group_sync<WPF>(bar_id);
        if constexpr (WPF == 1) {
            if (P.lambda) {
                // the lambda largest candidates, one after another (largest
                // remaining, lowest index first among equals), into the flip list
                const int nc = (int)*ncand;
                int chosen = 0;
                for (; chosen < P.lambda && chosen < nc; ++chosen) {
                    unsigned long long best = 0ull;
                    for (int i = lane; i < nc; i += 32) best = cand[i] > best ? cand[i] : best;
                    best = warp_max_u64(best);
                    for (int i = lane; i < nc; i += 32)
                        if (cand[i] == best) cand[i] = 0ull;
                    if (lane == 0) keys[chosen] = best;
                    __syncwarp();
                }
                if (lane == 0) *ncand = 0u;
                __syncwarp();
            }
        }
        // flips: all blocks read s_k; apply together
        int dW = 0, nflip = 0;
        for (int b = t; b < P.nkeys; b += G) {
            const unsigned long long key = keys[b];
            if (key) {
                keys[b] = 0ull;
                ++nflip;
                const uint32_t n = 0xffffffffu - (uint32_t)key;
                atomicXor(&zbits[n >> 5], 1u << (n & 31));
                uint32_t C, j;
                if (PLAIN) {
                    C = n;
                    j = 0;
                } else {
                    C = div_small(n, Z, P.z_magic);
                    j = n - C * Z;
                }
                for (uint32_t e = cptr[C]; e < cptr[C + 1]; ++e) {
                    const uint32_t m = PLAIN ? (cent[e] >> 16) : circ_index(cent[e], j, Z);
                    const uint32_t bit = 1u << (m & 31);
                    const uint32_t old = atomicXor(&sbits[m >> 5], bit);
                    dW += (old & bit) ? -1 : 1;
                }
            }
        }
        const int3 tot3 = group_sum3<WPF>(make_int3(warp_sum(dW), warp_sum(nflip), 0), red, rhalf, lane, gw,
                                          bar_id);
        W += tot3.x;
        nflip = tot3.y;
        if constexpr (WPF == 1) __syncwarp();
        if (nflip == 0) {  // fixed point with a non-zero syndrome
            iters = -P.max_iter;
            break;
        }
    }

    // ---- outputs ---------------------------------------------------------
    uint32_t *ob = P.out_bits + f * (unsigned long long)Nw;
    for (int w = t; w < Nw; w += G) __stcs(ob + w, zbits[w]);
    if (t == 0) P.out_iters[f] = iters;
    group_sync<WPF>(bar_id);
}

// Host: fills the code-dependent fields and the per-warp shared-memory layout.
inline void generic_layout(const fwbf_code_s *c, I8Params &P) {
    auto a16 = [](uint32_t x) { return (x + 15u) & ~15u; };
    P.table = c->d_table;
    P.table_words = c->table_words;
    P.N = c->N;
    P.M = c->M;
    P.Z = c->Z;
    P.MB = c->MB;
    P.NB = c->NB;
    P.rptr_off = c->rptr_off;
    P.rent_off = c->rent_off;
    P.cptr_off = c->cptr_off;
    P.cent_off = c->cent_off;
    P.p = c->p;
    P.B = c->B;
    P.p_magic = c->p_magic;
    P.z_magic = c->z_magic;
    const uint32_t N = c->N, M = c->M;
    uint32_t o = a16(N + 32);
    P.off_T = o;
    o += a16(4 * N);
    P.off_crec = o;
    o += a16(4 * M);
    P.off_s = o;
    o += a16(4 * ((M + 31) / 32));
    P.off_z = o;
    o += a16(4 * ((N + 31) / 32));
    P.off_keys = o;
    P.nkeys = c->B;
    o += a16(8 * (uint32_t)c->B);
    P.off_red = o;
    o += 256;
    P.off_cand = o;
    P.warp_bytes = o;
    P.dc_max = c->dc_max;
}

// Host: adds the lambda-largest candidate list (and a flip list of at least
// lambda entries) to a layout made by generic_layout.
inline void generic_layout_lambda(const fwbf_code_s *c, I8Params &P, int lambda) {
    auto a16 = [](uint32_t x) { return (x + 15u) & ~15u; };
    P.lambda = lambda;
    P.nkeys = c->B > lambda ? c->B : lambda;
    uint32_t o = P.off_keys + a16(8 * (uint32_t)P.nkeys);
    P.off_red = o;
    o += 256;
    P.off_cand = o;
    o += a16(8 * (uint32_t)c->N + 4);
    P.warp_bytes = o;
}

}  // namespace fwbf
