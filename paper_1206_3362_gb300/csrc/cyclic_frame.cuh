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
// what a compiled body of the frame decoder handles (smaller bodies stay in the
// instruction cache): plain FWBF alone; learned decoding without recording;
// every mode (schedules, learned, feature and schedule recording)
constexpr int kVarPlain = 0, kVarLearned = 1, kVarAll = 2;

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
    uint32_t warp_bytes, off_X, off_crec, off_SC, off_s, off_z, off_keys, off_red;
    uint32_t off_h;       // 64 floats of layer-1 outputs of the network (kModeLearned)
    float inv_Z, inv_B;   // 1 / Z and 1 / B (features)
    // block arg-max keys: 32-bit keys (E' << ksh | (2^ksh - 1 - offset in the
    // block)) when every positive E' fits beside the offset, else (ksh = -1)
    // 64-bit keys ((E' ^ 2^31) << 32 | (2^32 - 1 - n)); key_words uint32 words
    int ksh;
    uint32_t key_words;
    int gate_dv;          // learned passes with W < gate_dv d_v use the fallback parameters
    int w_gate;           // gate_dv d_v (set by cyclic_layout)
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
// Thread t of a group of G threads writes every G-th word.
template <typename F>
__device__ __forceinline__ void build_doubled(uint32_t *X2, int Z, int H, int XJ, int t, int G, F v) {
    const int zh = Z - H;
    for (int j = t; j < zh; j += G) X2[j] = v(j) | (v(j + H) << 16);
    for (int j = zh + t; j < Z; j += G) X2[j] = v(j) | (v(j - zh) << 16);
    for (int j = Z + t; j < XJ; j += G) X2[j] = v(j - Z) | (v(j - zh) << 16);
}

// Writes a = v(i) and b = v(i + H) (pair i < H; b only if i + H < Z) into every
// half-word of the doubled array that holds them.  v(x) is the low half of
// words x and x + Z, the high half of words (x - H) mod Z and that + Z (each
// while < XJ); for pair i that is: words i and i + Z (i < H - 1) whole, the low
// half of word i + H and the high half of word i + Z - H.  Over all pairs the
// whole-word stores ([0, H - 1) or [0, H), and [Z, XJ)) and the half-word
// stores ([Z - H, Z)) touch disjoint words, so no two stores overlap.
__device__ __forceinline__ void doubled_pair_store(uint32_t *X2, int i, uint32_t a, uint32_t b, bool has_b, int Z,
                                                   int H) {
    uint16_t *X16 = reinterpret_cast<uint16_t *>(X2);
    if (has_b) {
        const uint32_t w = a | (b << 16);
        X2[i] = w;
        if (i < H - 1) X2[i + Z] = w;
        X16[2 * (i + H)] = (uint16_t)b;
    } else {
        X16[2 * i] = (uint16_t)a;  // the high half is v(0), stored by pair 0
    }
    X16[2 * (i + Z - H) + 1] = (uint16_t)a;
}

// Adds delta to every half-word of the doubled array that holds position m
// (after all updates of a pass the half-words are back in [1, 255]; the
// additions commute, so updates of several flips may interleave).
__device__ __forceinline__ void doubled_add(uint32_t *X2, int m, int delta, int Z, int H, int XJ) {
    const uint32_t lo = (uint32_t)delta, hi = (uint32_t)delta * 65536u;
    atomicAdd(&X2[m], lo);
    if (m + Z < XJ) atomicAdd(&X2[m + Z], lo);
    int jh = m - H;
    if (jh < 0) jh += Z;
    atomicAdd(&X2[jh], hi);
    if (jh + Z < XJ) atomicAdd(&X2[jh + Z], hi);
}

// Flip updates of check m for one flipped bit: syndrome toggle (returns the
// change of the syndrome weight), V' in the doubled array, and the arg-min
// correction; `old` is the syndrome word before the toggle.
__device__ __forceinline__ int flip_check(uint32_t *X2, uint32_t *SC, uint32_t rec, uint32_t m, uint32_t old, int Z,
                                          int H, int XJ) {
    const uint32_t bit = 1u << (m & 31);
    const bool now_set = !(old & bit);
    const uint32_t min1 = rec & 0x7fu, diff = (rec >> 8) & 0x7fu;
    doubled_add(X2, (int)m, now_set ? 2 * (int)min1 : -2 * (int)min1, Z, H, XJ);
    if (diff) {
        int idx, sh;
        pair_slot((int)(rec >> 16), H, idx, sh);
        const int d = now_set ? 2 * (int)diff : -2 * (int)diff;
        atomicAdd(&SC[idx], sh ? (uint32_t)d * 65536u : (uint32_t)d);
    }
    return now_set ? 1 : -1;
}

// Decodes frame f of P with a group of WPF warps (thread t of 32 * WPF);
// d_off / u_off are the code's row / column offsets (shared memory), ws the
// group's shared-memory slice, bar_id the group's named barrier (WPF > 1).
// The check pass and the gather split their chunks over the warps, the flips
// their blocks; every other loop strides over the group's threads.
// VAR selects the compiled body (kVarPlain: plain FWBF alone, no schedules,
// network or features, 3.5 % faster on EG(1023) than the full body;
// kVarLearned: P.mode is kModeLearned and nothing is recorded; kVarAll: any mode).
template <int R, int WPF, int VAR>  // pairs per lane per chunk, warps per frame, body
__device__ __forceinline__ void cyclic_frame(const CyclicParams &P, const uint32_t *d_off, const uint32_t *u_off,
                                             unsigned char *ws, int t, int bar_id, unsigned long long f) {
    constexpr int G = 32 * WPF;
    const int lane = t & 31, gw = t >> 5;
    int8_t *stage = reinterpret_cast<int8_t *>(ws);
    uint32_t *X2 = reinterpret_cast<uint32_t *>(ws + P.off_X);
    uint32_t *crec = reinterpret_cast<uint32_t *>(ws + P.off_crec);
    // SC_n = sum of (2 s_m - 1) diff_m over the checks whose arg-min bit is n,
    // packed in pairs, each half biased by 0x4000 (|SC| <= 127 d_c < 0x4000)
    uint32_t *SC = reinterpret_cast<uint32_t *>(ws + P.off_SC);
    uint32_t *sbits = reinterpret_cast<uint32_t *>(ws + P.off_s);
    uint32_t *zbits = reinterpret_cast<uint32_t *>(ws + P.off_z);
    unsigned long long *keys = reinterpret_cast<unsigned long long *>(ws + P.off_keys);
    uint32_t *keys32 = reinterpret_cast<uint32_t *>(ws + P.off_keys);
    const uint32_t kmask = P.ksh >= 0 ? (1u << P.ksh) - 1u : 0u;
    int *red = reinterpret_cast<int *>(ws + P.off_red);
    float *mlp_slot = reinterpret_cast<float *>(ws + P.off_red + 32 * WPF);  // network halves (WPF > 1)
    float *mlp_h = reinterpret_cast<float *>(ws + P.off_h);                    // network layer 1 (learned)
    int rhalf = 0;
    const int Z = P.Z, H = P.H, DC = P.DC;
    const int Zw = (Z + 31) >> 5;
    const int XJ = Z + H - 1;  // doubled-array words used: i + r <= H - 1 + Z - 1
    const int chunks = H / (32 * R);
    const uintptr_t ybase = reinterpret_cast<uintptr_t>(P.y);
    const uintptr_t yend = ybase + (uintptr_t)(P.F * (int64_t)Z);
    const uint32_t my_u = lane < DC ? u_off[lane] : 0u;  // column offset of row position e = lane
    const int bias = 128 * DC + 0x4000;
    const uint32_t dfilter = (uint32_t)(0x8000 - bias - 1) * 0x10001u;

    // ---- frame load (aligned 16-byte chunks; byte loads at the buffer end)
    const uintptr_t fb = ybase + (uintptr_t)(f * (unsigned long long)Z);
    const uintptr_t a0 = fb & ~(uintptr_t)15;
    const int off = (int)(fb - a0);
    const int nchunks = (off + Z + 15) >> 4;
    // frame statistics for the features of scheduled decoding and of recorded
    // runs, taken from the loaded chunks (bytes outside the frame masked) and
    // summed over the group with the check pass's syndrome weight; the learned
    // body takes them from the staged bytes when a pass first consults the
    // network (about one frame in six at the usual gates: 2.4 % of the frame
    // time when taken for every frame)
    const bool stats = VAR == kVarAll && (P.mode != kModePlain || P.out_feat);
    int sa = 0, sw = 0;  // sum of |q_n|, count of |q_n| < 8
    for (int c = t; c < nchunks; c += G) {
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
        v = clamp_m127(v);
        *reinterpret_cast<uint4 *>(stage + c * 16) = v;
        if (stats) {
            const int lo = off - 16 * c, hi = off + Z - 16 * c;  // frame bytes of the chunk: [lo, hi)
            const uint32_t wv[4] = {v.x, v.y, v.z, v.w};
            const bool edge = lo > 0 || hi < 16;
            uint32_t wc = 0u;  // per byte lane: values with |q| < 8 (at most 4)
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                uint32_t keep = 0xffffffffu;
                if (edge) {
                    const int l = lo - 4 * i, h = hi - 4 * i;  // frame bytes of word i: [l, h)
                    keep = l >= 4 || h <= 0 ? 0u : keep;
                    if (l > 0 && l < 4) keep <<= 8 * l;
                    if (h > 0 && h < 4) keep &= 0xffffffffu >> (8 * (4 - h));
                }
                const uint32_t a = __vabsss4(wv[i]) & keep;  // |q| per byte (q >= -127)
                sa += (int)__vsadu4(a, 0u);
                wc += __vcmpltu4(a, 0x08080808u) & keep & 0x01010101u;
            }
            sw += (int)__vsadu4(wc, 0u);
        }
    }
    if (stats) {
        sa = warp_sum(sa);
        sw = warp_sum(sw);
        if (WPF > 1 && lane == 0) {
            red[4 * gw] = sa;
            red[4 * gw + 1] = sw;
        }
    }
    group_sync<WPF>(bar_id);
    const int8_t *q = stage + off;
    // frame-constant features in shared memory: mean |q| / 127, fraction of
    // |q| < 8, W_0 / Z (read by every pass; written before the group's next meeting)
    float *fstate = reinterpret_cast<float *>(ws + P.off_red + 32 * WPF + 16);
    if (stats) {
        if (t == 0) {
            if (WPF > 1) {
                sa = sw = 0;
#pragma unroll
                for (int w = 0; w < WPF; ++w) {
                    sa += red[4 * w];
                    sw += red[4 * w + 1];
                }
            }
            fstate[0] = (float)sa / (127.0f * (float)Z);
            fstate[1] = (float)sw / (float)Z;
        }
        rhalf = 1;  // half 0 of the group scratch held the statistics
    }
    int iters = 0, mode = VAR == kVarPlain ? kModePlain : VAR == kVarLearned ? kModeLearned : P.mode;
    bool have_stats = stats;  // fstate[0..1] hold this frame's statistics
    for (;;) {  // attempts: the requested mode, then plain FWBF as fallback
    // per pair i (a warp's 32 pairs lie in one 32-bit word of decisions, as
    // H % 32 == 0): the check keys of both positions into the doubled array,
    // the hard decisions, the cleared corrections
    for (int i = t; i < H; i += G) {
        const bool has_b = i + H < Z;
        const int qa = q[i], qb = has_b ? q[i + H] : 0;
        doubled_pair_store(X2, i, qkey(qa), qkey(qb), has_b, Z, H);
        SC[i] = 0x40004000u;
        const uint32_t za = __ballot_sync(FULL, qa < 0), zb = __ballot_sync(FULL, qb < 0);
        if (lane == 0) {
            zbits[i >> 5] = za;
            zbits[(i + H) >> 5] = zb;  // (i + H < Z for lane 0: Z >= 2H - 1)
        }
    }
    group_sync<WPF>(bar_id);

    // ---- check pass: min1/pos, min2 and parity of every check pair; the
    //      signed arg-min corrections (into SC) ----------------------------
    int W = 0;
    for (int c = gw; c < chunks; c += WPF) {
        uint32_t k1[R], k2[R], par[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            k1[r] = 0xffffffffu;
            k2[r] = 0xffffffffu;
            par[r] = 0u;
        }
        const uint32_t *xb = X2 + lane + 32 * R * c;
        uint32_t ek = 0u;  // the row position e in both halves
        if constexpr (VAR == kVarPlain) {
            // two row positions per step: with lo <= hi the step's two keys and
            // k1 <= k2 the two smallest so far, the new two smallest are
            // min(k1, lo) and min(k2, max(k1, lo), hi); the parity (bit 7 of each
            // half) is the XOR of the keys, whose position bits lie below it.
            // (2 % faster plain FWBF on EG(1023); the learned body, with more
            // state live, ran 3.5 % slower with it and keeps one position per step.)
            int e = 0;
            for (; e + 1 < DC; e += 2, ek += 0x20002u) {
                const uint32_t *pa = xb + d_off[e], *pb = xb + d_off[e + 1];
                const uint32_t ek1 = ek + 0x10001u;
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const uint32_t a = pa[32 * r] | ek, b = pb[32 * r] | ek1;
                    const uint32_t lo = vmin_u16x2(a, b), hi = vmax_u16x2(a, b);
                    k2[r] = __vimin3_u16x2(k2[r], vmax_u16x2(k1[r], lo), hi);
                    k1[r] = vmin_u16x2(k1[r], lo);
                    par[r] ^= a ^ b;
                }
            }
            if (e < DC) {
                const uint32_t *p = xb + d_off[e];
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const uint32_t key = p[32 * r] | ek;
                    k2[r] = vmin_u16x2(k2[r], vmax_u16x2(k1[r], key));
                    k1[r] = vmin_u16x2(k1[r], key);
                    par[r] ^= key;
                }
            }
        } else {
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
                // min1, the syndrome bit at the check pass (read only by the V'
                // build below), diff, arg-min bit
                crec[m] = min1 | ((half ? s_hi : s_lo) << 7) | (diff << 8) | ((uint32_t)n << 16);
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
    W = group_sum3<WPF>(make_int3(W, 0, 0), red, rhalf, lane, gw, bar_id).x;  // (meets the group if WPF > 1)
    if ((stats || VAR == kVarLearned) && t == 0) fstate[2] = (float)W * P.inv_Z;
    if constexpr (WPF == 1) __syncwarp();

    // the doubled array of V'_m = (2 s_m - 1) min1_m + 128, kept current
    for (int i = t; i < H; i += G) {
        const bool has_b = i + H < Z;
        const uint32_t ra = crec[i], rb = has_b ? crec[i + H] : 0u;
        const uint32_t va = (ra & 0x80u) ? 128u + (ra & 0x7fu) : 128u - (ra & 0x7fu);
        const uint32_t vb = (rb & 0x80u) ? 128u + (rb & 0x7fu) : 128u - (rb & 0x7fu);
        doubled_pair_store(X2, i, va, vb, has_b, Z, H);
    }
    group_sync<WPF>(bar_id);

    // ---- iterations ------------------------------------------------------
    bool give_up = false;   // learned passes exhausted: fall back to plain FWBF
    bool deviated = false;  // a learned pass used parameters other than plain FWBF's
    for (int k = 0;; ++k) {
        if (W == 0) {
            iters = k;
            break;
        }
        if (VAR != kVarPlain && mode == kModeLearned && k == P.k_learn) {
            // every pass so far used plain FWBF's parameters: the state is plain
            // FWBF's after k passes, so plain decoding continues from it
            if (!deviated) {
                mode = kModePlain;
            } else {
                give_up = true;
                break;
            }
        }
        if (k == P.max_iter) {
            iters = -P.max_iter;
            break;
        }
        // weighting factor and threshold of this pass (fixed point, x256)
        int aq = P.alpha_q, tq = P.theta_q;
        bool gated = false;  // a learned pass that used the fallback parameters
        if (VAR != kVarPlain && mode != kModePlain) {
            if (mode == kModeLearned) gated = W < P.w_gate;
            // features of this pass (feat[0..3], feat[4..7]), where something uses them
            float4 fa = make_float4(0.0f, 0.0f, 0.0f, 0.0f), fb = fa;
            if (!gated || (VAR == kVarAll && P.out_feat)) {
                // the previous pass's (syndrome change, flips, candidates), summed
                // over the group, are still in the group scratch its sum used
                // (kept out of registers: the gather runs under a 64-register cap)
                int Wprev = W, nflip_prev = 0, ncand_prev = 0;
                if (k > 0) {
                    const int *r = red + (WPF == 1 ? 0 : (rhalf ^ 1) * 4 * WPF);
                    int dW = 0;
#pragma unroll
                    for (int w = 0; w < WPF; ++w) {
                        dW += r[4 * w];
                        nflip_prev += r[4 * w + 1];
                        ncand_prev += r[4 * w + 2];
                    }
                    Wprev = W - dW;
                }
                float mean_a, weak;
                if (VAR == kVarLearned && !have_stats) {
                    // sum |q| and count |q| < 8 over the frame's staged values; the
                    // group's partial sums pass through the free half of the scratch
                    // (the other half holds the previous pass's sums read above)
                    int sa = 0, sw = 0;
                    for (int n = t; n < Z; n += G) {
                        const int a = abs((int)q[n]);
                        sa += a;
                        sw += a < 8 ? 1 : 0;
                    }
                    sa = warp_sum(sa);
                    sw = warp_sum(sw);
                    if constexpr (WPF > 1) {
                        int *r = red + rhalf * 4 * WPF;
                        if (lane == 0) {
                            r[4 * gw] = sa;
                            r[4 * gw + 1] = sw;
                        }
                        group_sync<WPF>(bar_id);
                        sa = sw = 0;
#pragma unroll
                        for (int w = 0; w < WPF; ++w) {
                            sa += r[4 * w];
                            sw += r[4 * w + 1];
                        }
                    }
                    mean_a = (float)sa / (127.0f * (float)Z);  // (the same arithmetic as at the load)
                    weak = (float)sw / (float)Z;
                    if (t == 0) {
                        fstate[0] = mean_a;
                        fstate[1] = weak;
                    }
                    have_stats = true;
                } else {
                    mean_a = fstate[0];
                    weak = fstate[1];
                }
                fa = make_float4((float)W * P.inv_Z, (float)Wprev * P.inv_Z, fstate[2], (float)k * (1.0f / 16.0f));
                fb = make_float4((float)nflip_prev * P.inv_B, (float)ncand_prev * P.inv_Z, mean_a, weak);
            }
            if (VAR == kVarAll && P.out_feat && k < P.feat_passes && t == 0) {
                float *o = P.out_feat + (f * (unsigned long long)P.feat_passes + k) * kFeatures;
                o[0] = fa.x, o[1] = fa.y, o[2] = fa.z, o[3] = fa.w;
                o[4] = fb.x, o[5] = fb.y, o[6] = fb.z, o[7] = fb.w;
            }
            if (VAR == kVarAll && mode == kModeSched) {
                const long long o = (long long)f * P.sched_stride + k;
                aq = P.sched_a[o];
                tq = P.sched_t[o];
            } else if (mode == kModeLearned) {
                if (!gated) {
                    const float2 o = mlp_eval<WPF>(P.mlp, fa, fb, lane, gw, mlp_h, mlp_slot, bar_id);
                    const float al = o.x, th = o.y;
                    // the layer-1 outputs may share the (idle, all-zero) key array:
                    // clear them, and meet, before this pass's keys are written
                    if (WPF == 1 || gw < 2) mlp_h[32 * gw + lane] = 0.0f;
                    if constexpr (WPF == 1) mlp_h[32 + lane] = 0.0f;
                    group_sync<WPF>(bar_id);
                    // alpha in steps of 1/2 in [0, 64], theta = 16 o1 in steps of 4 in [0, 4096]
                    aq = 128 * __float2int_rn(fminf(fmaxf(al, 0.0f), 64.0f) * 2.0f);
                    tq = 1024 * __float2int_rn(fminf(fmaxf(th * 4.0f, 0.0f), 1024.0f));
                    deviated |= aq != P.alpha_q || tq != 0;
                }
                if (VAR == kVarAll && P.out_sched && t == 0) {
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
        for (int c = gw; c < chunks; c += WPF) {
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
                if (VAR != kVarPlain) ncand += __popc(cmask);  // a feature of the next pass
#pragma unroll
                for (int half = 0; half < 2; ++half) {
                    const int n = i + half * H;
                    const int Gv = (int)((G2 >> (16 * half)) & 0xffffu);
                    const int sc = (int)((SC2 >> (16 * half)) & 0xffffu);
                    const int a = abs((int)q[n < Z ? n : 0]);
                    const int E = (Gv + sc - bias) * 256 - aq * a;
                    if (E > tq && n < Z) {  // E >= 1: a 32-bit key is never 0
                        const uint32_t blk = div_small((uint32_t)n, P.p, P.p_magic);
                        if (P.ksh >= 0) {
                            const uint32_t off = (uint32_t)n - blk * (uint32_t)P.p;
                            atomicMax(&keys32[blk], ((uint32_t)E << P.ksh) | (kmask - off));
                        } else {
                            const unsigned long long key = ((unsigned long long)((uint32_t)E ^ 0x80000000u) << 32) |
                                                           (0xffffffffu - (uint32_t)n);
                            atomicMax(&keys[blk], key);
                        }
                    }
                }
            }
        }
        group_sync<WPF>(bar_id);
        // flips: warp gw takes the blocks b = gw (mod WPF); a warp toggles the
        // checks of two flipped bits at a time and keeps the syndrome, the
        // doubled V array and the corrections current (all by atomics, so the
        // warps of the group may touch the same words)
        int dW = 0, nflip = 0;
        for (int b0 = 0; b0 < P.B; b0 += G) {
            const int b = b0 + WPF * lane + gw;
            bool has = false;
            uint32_t nmine = 0u;
            if (b < P.B) {
                if (P.ksh >= 0) {
                    const uint32_t key = keys32[b];
                    has = key != 0u;
                    if (has) keys32[b] = 0u;
                    nmine = (uint32_t)b * (uint32_t)P.p + (kmask - (key & kmask));
                } else {
                    const unsigned long long key = keys[b];
                    has = key != 0ull;
                    if (has) keys[b] = 0ull;
                    nmine = 0xffffffffu - (uint32_t)key;
                }
            }
            if (has) atomicXor(&zbits[nmine >> 5], 1u << (nmine & 31));
            uint32_t pend = __ballot_sync(FULL, has);
            nflip += __popc(pend);
            while (pend) {
                const int s0 = __ffs(pend) - 1;
                pend &= pend - 1;
                const bool two = pend != 0u;
                const int s1 = two ? __ffs(pend) - 1 : s0;
                if (two) pend &= pend - 1;
                const uint32_t n0 = __shfl_sync(FULL, nmine, s0);
                const uint32_t n1 = __shfl_sync(FULL, nmine, s1);
                for (int e = lane; e < DC; e += 32) {
                    const uint32_t u = e < 32 ? my_u : u_off[e];
                    uint32_t m0 = n0 + u, m1 = n1 + u;
                    m0 = m0 >= (uint32_t)Z ? m0 - Z : m0;
                    m1 = m1 >= (uint32_t)Z ? m1 - Z : m1;
                    const uint32_t old0 = atomicXor(&sbits[m0 >> 5], 1u << (m0 & 31));
                    const uint32_t old1 = two ? atomicXor(&sbits[m1 >> 5], 1u << (m1 & 31)) : 0u;
                    const uint32_t rec0 = crec[m0], rec1 = crec[m1];
                    dW += flip_check(X2, SC, rec0, m0, old0, Z, H, XJ);
                    if (two) dW += flip_check(X2, SC, rec1, m1, old1, Z, H, XJ);
                }
            }
        }
        const int3 tot = group_sum3<WPF>(make_int3(warp_sum(dW), nflip, warp_sum(ncand)), red, rhalf, lane, gw,
                                         bar_id);
        W += tot.x;
        nflip = tot.y;
        if constexpr (WPF == 1) {  // (one warp: the sums are kept where a group's would be)
            if (VAR != kVarPlain && lane == 0) {
                red[0] = tot.x;
                red[1] = tot.y;
                red[2] = tot.z;
            }
            __syncwarp();
        }
        if (nflip == 0 && mode == kModePlain) {  // fixed point: every later pass repeats this one
            iters = -P.max_iter;
            break;
        }
        if (VAR != kVarPlain && nflip == 0 && gated) {
            // W is unchanged, so every later learned pass is gated too and repeats
            // this one: plain FWBF's fixed point if no pass deviated (and so its
            // result), else the frame goes to the fallback now, as at k_learn
            if (!deviated) {
                iters = -P.max_iter;
                break;
            }
            give_up = true;
            break;
        }
    }
    if (!give_up) break;
    mode = kModePlain;  // plain FWBF from the channel values; its result is the frame's
    }  // attempts

    uint32_t *ob = P.out_bits + f * (unsigned long long)Zw;
    for (int w = t; w < Zw; w += G) __stcs(ob + w, zbits[w]);
    if (t == 0) P.out_iters[f] = iters;
    group_sync<WPF>(bar_id);
}

bool cyclic_eligible(const fwbf_code_s *c);

// Host: fills the code-dependent fields and the per-warp shared-memory layout.
// bytes of a frame's group scratch for wpf warps (the last item of the slice)
// (2 x 4 ints per warp of group sums, 4 floats of network halves, 4 floats of
// frame-constant features)
inline uint32_t cyclic_red_bytes(int wpf) { return 32u * (uint32_t)wpf + 32u; }

// Sizes the frame's slice for groups of wpf warps (cyclic_layout assumes 4);
// learned decoding adds the network's 64 layer-1 outputs (P.mode must be set).
inline void cyclic_set_wpf(CyclicParams &P, int wpf) {
    const bool in_keys = 4u * P.key_words >= 256u;  // the key array is all zero between passes
    P.off_h = in_keys ? P.off_keys : P.off_red + cyclic_red_bytes(wpf);
    P.warp_bytes = P.off_red + cyclic_red_bytes(wpf) + (P.mode == kModeLearned && !in_keys ? 256u : 0u);
}

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
    P.inv_Z = 1.0f / (float)c->Z;
    P.inv_B = 1.0f / (float)c->B;
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
    {
        int sh = 0;
        while ((1 << sh) < c->p) ++sh;
        const uint64_t emax = 256ull * 127ull * (uint64_t)c->dv_max;  // largest positive E'
        P.ksh = (emax << sh) < (1ull << 32) ? sh : -1;
        P.key_words = (uint32_t)c->B * (P.ksh >= 0 ? 1u : 2u);
        P.w_gate = P.gate_dv * c->dv_max;
    }
    o += a16(4 * P.key_words);
    P.off_red = o;  // group sums: 2 halves x 4 ints per warp of the group; then 4 floats for the network
    cyclic_set_wpf(P, 4);
    P.table_smem_bytes = a16(c->table_words * 4u);
}

// pairs per lane per chunk of the packed kernel: the largest of 8 (or of 4
// with two warps per frame: at 32 warps per SM the smaller unrolled body
// stays in the instruction cache, 7 % faster on EG(1023); with four warps R = 8
// is 3 % faster on EG(4095)), then 2, 1, that divides H / 32 and still gives
// each of the frame's wpf warps a chunk
inline int cyclic_R(const fwbf_code_s *c, int wpf = 1) {
    const int ppl = ((c->Z + 1) / 2) / 32;
    for (int r = wpf == 2 ? 4 : 8; r > 1; r >>= 1)
        if (ppl % r == 0 && ppl / r >= wpf) return r;
    return 1;
}

}  // namespace fwbf
