// Per-frame body of the packed int8 FWBF decoder for cyclic codes, shared by
// the single-code kernel (decode_i8_cyclic.cu) and the batched multi-code
// kernel (decode_batch.cu).  The layout and reformulation it uses are
// described at the top of decode_i8_cyclic.cu.
#pragma once

#include "device_common.cuh"
#include "fwbf_internal.h"
#include "mlp_device.cuh"

namespace fwbf {

constexpr int kModePlain = 0, kModeSched = 1, kModeLearned = 2;
constexpr int kFeatures = FWBF_MLP_IN;

struct CyclicParams {
    const uint32_t *table;
    uint32_t table_words, table_smem_bytes;
    uint32_t rent_off, cent_off;
    int Z, H, DC;
    int p, B;
    uint32_t p_magic;
    const int8_t *y;
    int64_t F;
    int max_iter, alpha_q, theta_q;
    uint32_t *out_bits;
    int32_t *out_iters;
    unsigned long long *counter;
    // per-pass schedule (kModeSched): alpha_q / theta_q of pass k of frame f at [f * sched_stride + k]
    int mode;
    const int32_t *sched_a, *sched_t;
    long long sched_stride;
    // learned schedule (kModeLearned): network, learned passes, recorded schedule
    const unsigned char *mlp;
    int k_learn;
    int32_t *out_sched;   // [F][k_learn][2] (alpha_q, theta_q) used, or null
    float *out_feat;      // [F][feat_passes][kFeatures] features per pass, or null
    int feat_passes;
    uint32_t warp_bytes, off_X, off_crec, off_SC, off_s, off_z, off_keys;
};

__device__ __forceinline__ uint32_t vmin_u16x2(uint32_t a, uint32_t b) {
    uint32_t d;
    asm("min.u16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
    return d;
}
__device__ __forceinline__ uint32_t vmax_u16x2(uint32_t a, uint32_t b) {
    uint32_t d;
    asm("max.u16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
    return d;
}

// packed check key of one int8 value: |q| << 8 | (q < 0) << 7
__device__ __forceinline__ uint32_t qkey(int v) { return ((uint32_t)abs(v) << 8) | (((uint32_t)v >> 24) & 0x80u); }

// pair slot of position n: (n, lo) for n < H, (n - H, hi) otherwise
__device__ __forceinline__ void pair_slot(int n, int H, int &idx, int &shift) {
    const bool hi = n >= H;
    idx = hi ? n - H : n;
    shift = hi ? 16 : 0;
}

// Rebuilds the doubled array X2[j] = v(j mod Z) | v((j + H) mod Z) << 16,
// j < XJ = Z + H - 1, in three index ranges without modulo arithmetic:
// j < Z - H: (j, j + H); Z - H <= j < Z: (j, j + H - Z); j >= Z: (j - Z, j - Z + H).
template <typename F>
__device__ __forceinline__ void build_doubled(uint32_t *X2, int Z, int H, int XJ, int lane, F v) {
    const int zh = Z - H;
    for (int j = lane; j < zh; j += 32) X2[j] = v(j) | (v(j + H) << 16);
    for (int j = zh + lane; j < Z; j += 32) X2[j] = v(j) | (v(j - zh) << 16);
    for (int j = Z + lane; j < XJ; j += 32) X2[j] = v(j - Z) | (v(j - zh) << 16);
}

// Adds delta to every half-word of the doubled array that holds position m
// (the half-words stay in [1, 255], so no carry or borrow crosses halves).
__device__ __forceinline__ void doubled_add(uint32_t *X2, int m, int delta, int Z, int H, int XJ) {
    const uint32_t lo = (uint32_t)delta, hi = (uint32_t)delta * 65536u;
    atomicAdd(&X2[m], lo);
    if (m + Z < XJ) atomicAdd(&X2[m + Z], lo);
    int jh = m - H;
    if (jh < 0) jh += Z;
    atomicAdd(&X2[jh], hi);
    if (jh + Z < XJ) atomicAdd(&X2[jh + Z], hi);
}

// Decodes frame f of P with the calling warp; d_off / u_off are the code's
// row / column offsets (shared memory), ws the warp's shared-memory slice.
template <int R>  // pairs per lane per chunk
__device__ __forceinline__ void cyclic_frame(const CyclicParams &P, const uint32_t *d_off, const uint32_t *u_off,
                                             unsigned char *ws, int lane, unsigned long long f) {
    int8_t *stage = reinterpret_cast<int8_t *>(ws);
    uint32_t *X2 = reinterpret_cast<uint32_t *>(ws + P.off_X);
    uint32_t *crec = reinterpret_cast<uint32_t *>(ws + P.off_crec);
    // SC_n = sum of (2 s_m - 1) diff_m over the checks whose arg-min bit is n,
    // packed in pairs, each half biased by 0x4000 (|SC| <= 127 d_c < 0x4000)
    uint32_t *SC = reinterpret_cast<uint32_t *>(ws + P.off_SC);
    uint32_t *sbits = reinterpret_cast<uint32_t *>(ws + P.off_s);
    uint32_t *zbits = reinterpret_cast<uint32_t *>(ws + P.off_z);
    unsigned long long *keys = reinterpret_cast<unsigned long long *>(ws + P.off_keys);
    const int Z = P.Z, H = P.H, DC = P.DC;
    const int Zw = (Z + 31) >> 5;
    const int XJ = Z + H - 1;  // doubled-array words used: i + r <= H - 1 + Z - 1
    const int chunks = H / (32 * R);
    const uintptr_t ybase = reinterpret_cast<uintptr_t>(P.y);
    const uintptr_t yend = ybase + (uintptr_t)(P.F * (int64_t)Z);
    const uint32_t my_u = lane < DC ? u_off[lane] : 0u;  // column offset of row position e = lane
    const int bias = 128 * DC + 0x4000;
    const uint32_t dfilter = (uint32_t)(0x8000 - bias - 1) * 0x10001u;
    const float inv_Z = 1.0f / (float)Z, inv_B = 1.0f / (float)P.B;

    // ---- frame load (aligned 16-byte chunks; byte loads at the buffer end)
    const uintptr_t fb = ybase + (uintptr_t)(f * (unsigned long long)Z);
    const uintptr_t a0 = fb & ~(uintptr_t)15;
    const int off = (int)(fb - a0);
    const int nchunks = (off + Z + 15) >> 4;
    for (int c = lane; c < nchunks; c += 32) {
        const uintptr_t src = a0 + (uintptr_t)c * 16;
        uint4 v;
        if (src + 16 <= yend) {
            v = __ldcs(reinterpret_cast<const uint4 *>(src));
        } else {
            uint32_t wv[4] = {0u, 0u, 0u, 0u};
            for (int i = 0; i < 16; ++i)
                if (src + i < yend)
                    wv[i >> 2] |= (uint32_t)(*reinterpret_cast<const unsigned char *>(src + i)) << (8 * (i & 3));
            v = make_uint4(wv[0], wv[1], wv[2], wv[3]);
        }
        *reinterpret_cast<uint4 *>(stage + c * 16) = v;
    }
    __syncwarp();
    const int8_t *q = stage + off;
    // frame statistics for the features of scheduled and learned decoding
    float mean_a = 0.0f, weak_frac = 0.0f;
    if (P.mode != kModePlain || P.out_feat) {
        int sa = 0, sw = 0;
        for (int n = lane; n < Z; n += 32) {
            const int a = abs((int)q[n]);
            sa += a;
            sw += a < 8;
        }
        mean_a = (float)warp_sum(sa) / (127.0f * (float)Z);
        weak_frac = (float)warp_sum(sw) / (float)Z;
    }
    int iters = 0, passes_before = 0, mode = P.mode;
    for (;;) {  // attempts: the requested mode, then plain FWBF as fallback
    for (int i = lane; i < H; i += 32) SC[i] = 0x40004000u;

    for (int w = 0; w < Zw; ++w) {
        const int n = (w << 5) + lane;
        const uint32_t zb = __ballot_sync(FULL, n < Z && q[n] < 0);
        if (lane == 0) zbits[w] = zb;
    }
    build_doubled(X2, Z, H, XJ, lane, [&](int n) { return qkey(q[n]); });
    __syncwarp();

    // ---- check pass: min1/pos, min2 and parity of every check pair; the
    //      signed arg-min corrections (into SC) ----------------------------
    int W = 0;
    for (int c = 0; c < chunks; ++c) {
        uint32_t k1[R], k2[R], par[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            k1[r] = 0xffffffffu;
            k2[r] = 0xffffffffu;
            par[r] = 0u;
        }
        const uint32_t *xb = X2 + lane + 32 * R * c;
        uint32_t ek = 0u;  // the row position e in both halves
#pragma unroll 2
        for (int e = 0; e < DC; ++e, ek += 0x10001u) {
            const uint32_t *p = xb + d_off[e];
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const uint32_t v = p[32 * r];
                const uint32_t key = v | ek;
                k2[r] = vmin_u16x2(k2[r], vmax_u16x2(k1[r], key));
                k1[r] = vmin_u16x2(k1[r], key);
                par[r] ^= v;
            }
        }
        for (int r = 0; r < R; ++r) {
            const int i = lane + 32 * (R * c + r);
            const bool hi_ok = i + H < Z;
            const uint32_t s_lo = (par[r] >> 7) & 1u;
            const uint32_t s_hi = hi_ok ? (par[r] >> 23) & 1u : 0u;
#pragma unroll
            for (int half = 0; half < 2; ++half) {
                if (half && !hi_ok) break;
                const int m = i + half * H;
                const uint32_t a1 = k1[r] >> (16 * half), a2 = k2[r] >> (16 * half);
                const uint32_t min1 = (a1 >> 8) & 0x7fu, pos = a1 & 0x7fu, min2 = (a2 >> 8) & 0x7fu;
                const uint32_t diff = min2 - min1;
                int n = m + (int)d_off[pos];
                n = n >= Z ? n - Z : n;
                crec[m] = min1 | (diff << 8) | ((uint32_t)n << 16);  // min1, diff, arg-min bit
                if (diff) {
                    int idx, sh;
                    pair_slot(n, H, idx, sh);
                    const int d = (half ? s_hi : s_lo) ? (int)diff : -(int)diff;
                    atomicAdd(&SC[idx], sh ? (uint32_t)d * 65536u : (uint32_t)d);
                }
            }
            const uint32_t slo = __ballot_sync(FULL, s_lo);
            const uint32_t shi = __ballot_sync(FULL, s_hi);
            if (lane == 0) {
                sbits[R * c + r] = slo;
                sbits[(H >> 5) + R * c + r] = shi;
            }
            W += __popc(slo) + __popc(shi);
        }
    }
    __syncwarp();

    // the doubled array of V'_m = (2 s_m - 1) min1_m + 128, kept current
    build_doubled(X2, Z, H, XJ, lane, [&](int n) {
        const uint32_t mn = crec[n] & 0x7fu;
        return ((sbits[n >> 5] >> (n & 31)) & 1u) ? 128u + mn : 128u - mn;
    });
    __syncwarp();

    // ---- iterations ------------------------------------------------------
    const int W0 = W;
    int Wprev = W, nflip_prev = 0, ncand_prev = 0;
    bool give_up = false;  // learned passes exhausted: fall back to plain FWBF
    for (int k = 0;; ++k) {
        if (W == 0) {
            iters = passes_before + k;
            break;
        }
        if (mode == kModeLearned && k == P.k_learn) {
            give_up = true;
            break;
        }
        if (k == P.max_iter) {
            iters = -P.max_iter;
            break;
        }
        // weighting factor and threshold of this pass (fixed point, x256)
        int aq = P.alpha_q, tq = P.theta_q;
        if (mode != kModePlain || P.out_feat) {
            float feat[kFeatures];
            feat[0] = (float)W * inv_Z;
            feat[1] = (float)Wprev * inv_Z;
            feat[2] = (float)W0 * inv_Z;
            feat[3] = (float)k * (1.0f / 16.0f);
            feat[4] = (float)nflip_prev * inv_B;
            feat[5] = (float)ncand_prev * inv_Z;
            feat[6] = mean_a;
            feat[7] = weak_frac;
            const int kk = passes_before + k;
            if (P.out_feat && kk < P.feat_passes && lane == 0) {
                float *o = P.out_feat + (f * (unsigned long long)P.feat_passes + kk) * kFeatures;
#pragma unroll
                for (int j = 0; j < kFeatures; ++j) o[j] = feat[j];
            }
            if (mode == kModeSched) {
                const long long o = (long long)f * P.sched_stride + kk;
                aq = P.sched_a[o];
                tq = P.sched_t[o];
            } else if (mode == kModeLearned) {
                float al, th;
                mlp_eval(P.mlp, feat, lane, al, th);
                th *= 16.0f;
                aq = __float2int_rn(fminf(fmaxf(al, 0.0f), 64.0f) * 256.0f);
                tq = __float2int_rn(fminf(fmaxf(th, 0.0f), 4096.0f) * 256.0f);
                if (P.out_sched && lane == 0) {
                    const unsigned long long o = (f * (unsigned long long)P.k_learn + k) * 2;
                    P.out_sched[o] = aq;
                    P.out_sched[o + 1] = tq;
                }
            }
            aq = min(max(aq, 0), 16384);
            tq = max(tq, 0);
        }
        int ncand = 0;
        // D_n = sum (2 s_m - 1) w_{n,m} = G_n - 128 d_c + 2 UC_n - TC_n with
        // G the gather of V' over M(n); metric E' = 256 D_n - alpha_q a_n
        for (int c = 0; c < chunks; ++c) {
            uint32_t acc[R];
#pragma unroll
            for (int r = 0; r < R; ++r) acc[r] = 0u;
            const uint32_t *xb = X2 + lane + 32 * R * c;
            int e = 0;
            for (; e + 1 < DC; e += 2) {
                const uint32_t *p0 = xb + u_off[e];
                const uint32_t *p1 = xb + u_off[e + 1];
#pragma unroll
                for (int r = 0; r < R; ++r) acc[r] += p0[32 * r] + p1[32 * r];
            }
            if (e < DC) {
                const uint32_t *p0 = xb + u_off[e];
#pragma unroll
                for (int r = 0; r < R; ++r) acc[r] += p0[32 * r];
            }
            for (int r = 0; r < R; ++r) {
                const int i = lane + 32 * (R * c + r);
                const uint32_t G2 = acc[r], SC2 = SC[i];
                // D_n >= 1 is necessary for E' > theta >= 0: test both halves of
                // G + SC at once (0x8000 + (G + SC - bias) - 1 has bit 15 set iff
                // D_n >= 1; the half-words stay in [0, 65535])
                uint32_t cmask = (G2 + SC2 + dfilter) & 0x80008000u;
                if (i + H >= Z) cmask &= 0x8000u;  // the duplicated position
                if (cmask == 0u) continue;
                ncand += __popc(cmask);
#pragma unroll
                for (int half = 0; half < 2; ++half) {
                    const int n = i + half * H;
                    const int G = (int)((G2 >> (16 * half)) & 0xffffu);
                    const int sc = (int)((SC2 >> (16 * half)) & 0xffffu);
                    const int a = abs((int)q[n < Z ? n : 0]);
                    const int E = (G + sc - bias) * 256 - aq * a;
                    if (E > tq && n < Z) {
                        const uint32_t blk = div_small((uint32_t)n, P.p, P.p_magic);
                        const unsigned long long key =
                            ((unsigned long long)((uint32_t)E ^ 0x80000000u) << 32) | (0xffffffffu - (uint32_t)n);
                        atomicMax(&keys[blk], key);
                    }
                }
            }
        }
        __syncwarp();
        // flips: the warp toggles the checks of one flipped bit at a time and
        // keeps the syndrome, the doubled V array and the corrections current
        int dW = 0, nflip = 0;
        for (int b0 = 0; b0 < P.B; b0 += 32) {
            const int b = b0 + lane;
            unsigned long long key = 0ull;
            if (b < P.B) {
                key = keys[b];
                if (key) keys[b] = 0ull;
            }
            uint32_t pend = __ballot_sync(FULL, key != 0ull);
            nflip += __popc(pend);
            while (pend) {
                const int src = __ffs(pend) - 1;
                pend &= pend - 1;
                const uint32_t n = 0xffffffffu - (uint32_t)__shfl_sync(FULL, key, src);
                if (lane == 0) zbits[n >> 5] ^= 1u << (n & 31);
                for (int e = lane; e < DC; e += 32) {
                    uint32_t m = n + (e < 32 ? my_u : u_off[e]);
                    m = m >= (uint32_t)Z ? m - Z : m;
                    const uint32_t bit = 1u << (m & 31);
                    const uint32_t old = atomicXor(&sbits[m >> 5], bit);
                    const bool now_set = !(old & bit);
                    dW += now_set ? 1 : -1;
                    const uint32_t rec = crec[m];
                    const uint32_t min1 = rec & 0x7fu, diff = (rec >> 8) & 0x7fu;
                    doubled_add(X2, (int)m, now_set ? 2 * (int)min1 : -2 * (int)min1, Z, H, XJ);
                    if (diff) {
                        int idx, sh;
                        pair_slot((int)(rec >> 16), H, idx, sh);
                        const int d = now_set ? 2 * (int)diff : -2 * (int)diff;
                        atomicAdd(&SC[idx], sh ? (uint32_t)d * 65536u : (uint32_t)d);
                    }
                }
            }
        }
        Wprev = W;
        W += warp_sum(dW);
        nflip_prev = nflip;
        ncand_prev = warp_sum(ncand);
        __syncwarp();
        if (nflip == 0 && mode == kModePlain) {  // fixed point: every later pass repeats this one
            iters = -P.max_iter;
            break;
        }
    }
    if (!give_up) break;
    passes_before = P.k_learn;
    mode = kModePlain;
    }  // attempts

    uint32_t *ob = P.out_bits + f * (unsigned long long)Zw;
    for (int w = lane; w < Zw; w += 32) __stcs(ob + w, zbits[w]);
    if (lane == 0) P.out_iters[f] = iters;
    __syncwarp();
}

bool cyclic_eligible(const fwbf_code_s *c);

// Host: fills the code-dependent fields and the per-warp shared-memory layout.
inline void cyclic_layout(const fwbf_code_s *c, CyclicParams &P) {
    auto a16 = [](uint32_t x) { return (x + 15u) & ~15u; };
    P.table = c->d_table;
    P.table_words = c->table_words;
    P.rent_off = c->rent_off;
    P.cent_off = c->cent_off;
    P.Z = c->Z;
    P.H = (c->Z + 1) / 2;
    P.DC = c->dc_max;
    P.p = c->p;
    P.B = c->B;
    P.p_magic = c->p_magic;
    const uint32_t Z = c->Z, H = P.H;
    uint32_t o = a16(Z + 32);
    P.off_X = o;
    o += a16(4 * (Z + H));
    P.off_crec = o;
    o += a16(4 * Z);
    P.off_SC = o;
    o += a16(4 * H);
    P.off_s = o;
    o += a16(4 * ((Z + 31) / 32));
    P.off_z = o;
    o += a16(4 * ((Z + 31) / 32));
    P.off_keys = o;
    o += a16(8 * (uint32_t)c->B);
    P.warp_bytes = o;
    P.table_smem_bytes = a16(c->table_words * 4u);
}

// pairs per lane per chunk of the packed kernel (a divisor of H / 32)
inline int cyclic_R(const fwbf_code_s *c) {
    const int ppl = ((c->Z + 1) / 2) / 32;
    return ppl % 8 == 0 ? 8 : ppl % 4 == 0 ? 4 : ppl % 2 == 0 ? 2 : 1;
}

}  // namespace fwbf
