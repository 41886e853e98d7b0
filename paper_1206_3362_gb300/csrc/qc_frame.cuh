// Per-frame body of the packed int8 FWBF decoder for quasi-cyclic codes: H
// made of MB x NB blocks of Z x Z circulants (each block a sum of circulant
// permutations), Z a multiple of 64.  The same exact reformulation as the
// cyclic decoder (paper Sec. III, Eq. 1 in fixed point), carried over to
// several circulant blocks:
//
//   * bit n = (block column c, j), check m = (block row r, i); positions j and
//     j + H (H = Z/2) of a block column, and checks i and i + H of a block
//     row, share one 32-bit word (two 16-bit halves).
//   * check pass (once per frame): for four consecutive checks i .. i + 3 of
//     a block row at once, over the row's entries (c, t) -- bits
//     (c, (i + t) mod Z) .. -- the packed key |q| << 8 | sign << 7 | entry
//     gives min1 / arg-min and min2 by packed min/max, the sign bits the
//     parity; records crec[m] = min1 | diff << 8 | arg-min bit << 16, and the
//     signed arg-min corrections per bit in SC.
//   * per pass: V'_m = (2 s_m - 1) min1_m + 128 lives in a doubled pair array
//     per block row (X2r[k] = V'(r, k mod Z) | V'(r, (k + H) mod Z) << 16), so
//     a bit pair gathers over its column's entries (r, t') with one aligned,
//     conflict-free load each: D_n = G_n - 128 d_v(c) + SC_n + T_n - 0x8000,
//     metric E' = 256 D_n - alpha_q |q_n|.  SC holds the corrections less the
//     frame-constant T_n = floor((alpha_q |q_n| + theta_q) / 256) (capped at
//     127 * 127, above any D_n): E' > theta_q iff D_n - T_n >= 1, so one packed
//     test per bit pair selects exactly the candidates.
//   * flips toggle the syndrome and keep V' and SC current with atomics; a
//     pass without flips ends the frame (its state would repeat to K_max).
#pragma once

#include "cyclic_frame.cuh"

namespace fwbf {

struct QcParams {
    const uint32_t *table;
    uint32_t table_words, table_smem_bytes;
    uint32_t rptr_off, rent_off, cptr_off, cent_off;
    int Z, H, MB, NB, XJ;  // XJ = Z + H - 1 words of the doubled array per block row
    int p, B;
    uint32_t p_magic, z_magic, h_magic;
    const int8_t *y;
    int64_t F;
    int max_iter, alpha_q, theta_q;
    uint32_t *out_bits;
    int32_t *out_iters;
    unsigned long long *counter;
    uint32_t warp_bytes, off_X, off_crec, off_SC, off_s, off_z, off_keys, off_mbar, off_red;
    int lane_shift; // 2^lane_shift lanes per flipped bit: the largest column weight, up to 32
};

// Before a group's first frame: its frame-load mbarrier (thread t == 0; the
// group meets before the first wait) and its load-timeout flag.
template <int WPF>
__device__ __forceinline__ void qc_group_init(const QcParams &P, unsigned char *ws, int t) {
    if (t == 0) {
        mbar_init(reinterpret_cast<uint64_t *>(ws + P.off_mbar), 1);
        *reinterpret_cast<int *>(ws + P.off_mbar + 8) = 0;
    }
}

// After a group's last frame (every copy waited for): ends its mbarrier, whose
// shared memory the block may use for another job's slices.
__device__ __forceinline__ void qc_group_done(const QcParams &P, unsigned char *ws, int t) {
    if (t == 0) mbar_inval(reinterpret_cast<uint64_t *>(ws + P.off_mbar));
}

// arg-min correction slot of bit (c, a): pair word c * H + (a mod H), half a >= H
__device__ __forceinline__ void qc_pair_slot(uint32_t c, uint32_t a, uint32_t H, uint32_t &idx, uint32_t &shift) {
    const bool hi = a >= H;
    idx = c * H + (hi ? a - H : a);
    shift = hi ? 16u : 0u;
}

// Decodes frame f of P with a group of WPF warps (thread t of 32 * WPF); tbl
// is the code's table blob staged in shared memory, ws the group's slice,
// bar_id its named barrier (WPF > 1).
// Returns false (for every thread of the group) if the frame's bulk copy did
// not arrive within the wait limit; lpar is the group's mbarrier phase.
template <int R, int WPF>  // pairs per lane per gather chunk, warps per frame
__device__ __forceinline__ bool qc_frame(const QcParams &P, const uint32_t *tbl, unsigned char *ws, int t, int bar_id,
                                         unsigned long long f, uint32_t &lpar) {
    constexpr int G = 32 * WPF;
    const int lane = t & 31, gw = t >> 5;
    const uint32_t *rptr = tbl + P.rptr_off;
    const uint32_t *rent = tbl + P.rent_off;
    const uint32_t *cptr = tbl + P.cptr_off;
    const uint32_t *cent = tbl + P.cent_off;
    int8_t *stage = reinterpret_cast<int8_t *>(ws);
    uint32_t *X2 = reinterpret_cast<uint32_t *>(ws + P.off_X);
    uint32_t *crec = reinterpret_cast<uint32_t *>(ws + P.off_crec);
    uint32_t *SC = reinterpret_cast<uint32_t *>(ws + P.off_SC);  // per bit pair, halves biased by 0x8000
    uint32_t *sbits = reinterpret_cast<uint32_t *>(ws + P.off_s);
    uint32_t *zbits = reinterpret_cast<uint32_t *>(ws + P.off_z);
    unsigned long long *keys = reinterpret_cast<unsigned long long *>(ws + P.off_keys);
    int *red = reinterpret_cast<int *>(ws + P.off_red);
    int rhalf = 0;
    const uint32_t Z = (uint32_t)P.Z, H = (uint32_t)P.H;
    const int MB = P.MB, NB = P.NB, XJ = P.XJ;
    const int N = NB * (int)Z;
    const int Nw = N >> 5;
    const uintptr_t ybase = reinterpret_cast<uintptr_t>(P.y);

    // ---- frame load: one bulk copy (TMA) of the frame's N bytes (y is
    // 16-byte aligned and N a multiple of 64), thread t == 0 issuing it and
    // the group waiting on its mbarrier (bounded)
    const uintptr_t fb = ybase + (uintptr_t)(f * (unsigned long long)N);
    const int nwords = N >> 2;
    int *lflag = reinterpret_cast<int *>(ws + P.off_mbar + 8);
    {
        uint64_t *mbar = reinterpret_cast<uint64_t *>(ws + P.off_mbar);
        if (t == 0) {
            // the previous frame's generic-proxy accesses of the stage (ordered
            // before this thread by the group's last meeting) before the copy
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            mbar_expect_tx(mbar, (uint32_t)N);
            for (uint32_t o = 0; o < (uint32_t)N; o += kBulkChunk)
                bulk_g2s(stage + o, reinterpret_cast<const void *>(fb + o),
                         (uint32_t)N - o < kBulkChunk ? (uint32_t)N - o : kBulkChunk, mbar);
        }
        if (!mbar_wait_bounded(mbar, lpar, kWaitLimitNs)) {
            mbar_wait_bounded(mbar, lpar, kWaitLimitNs);  // let a late copy land before leaving
            atomicOr(lflag, 1);
        }
        lpar ^= 1u;
    }
    group_sync<WPF>(bar_id);
    if (*lflag) return false;  // (read by every thread after the meeting)
    // the staged bytes become sign-magnitude bytes sm = |q| << 1 | (q < 0),
    // four per word, -128 read as -127 (per byte: |q| = (q ^ 0xff) + 1 for
    // q < 0, no carry across bytes since |q| <= 127); sm << 7 is the packed
    // check-pass key
    {
        uint32_t *w32 = reinterpret_cast<uint32_t *>(stage);
        for (int w = t; w < nwords; w += G) {
            const uint32_t x = __vmaxs4(w32[w], 0x81818181u);
            const uint32_t sg = (x >> 7) & 0x01010101u;
            w32[w] = (((x ^ (sg * 0xffu)) + sg) << 1) | sg;
        }
    }
    group_sync<WPF>(bar_id);
    const uint8_t *sm = reinterpret_cast<const uint8_t *>(stage);
    for (int w = gw; w < Nw; w += WPF) {
        const int n = (w << 5) + lane;
        const uint32_t zb = __ballot_sync(FULL, sm[n] & 1u);
        if (lane == 0) zbits[w] = zb;
    }
    // corrections of bit pair (c, j), (c, j + H): 0x8000 - T_n per half, T_n
    // capped at 127 * 127 (|SC_n| <= 127 d_v and |D_n| <= 127 d_v, d_v <= 127:
    // a half stays in [510, 65025] and the pass's packed test exact)
    {
        const uint32_t aq = (uint32_t)P.alpha_q, tq = (uint32_t)P.theta_q;
        auto tn = [&](uint32_t n) {
            const uint32_t v = (aq * (uint32_t)(sm[n] >> 1) + tq) >> 8;
            return v < 16129u ? v : 16129u;
        };
        for (int i = t; i < NB * (int)H; i += G) {
            const uint32_t c = div_small((uint32_t)i, H, P.h_magic);
            const uint32_t n = c * Z + ((uint32_t)i - c * H);
            SC[i] = 0x80008000u - (tn(n) | (tn(n + H) << 16));
        }
    }
    group_sync<WPF>(bar_id);  // (the check pass adds into any pair's corrections)

    // ---- check pass: a lane takes four consecutive checks 4 qd .. 4 qd + 3
    //      of block row r (a warp 32 consecutive quads of one row).  For a
    //      row entry (c, t) their bits are the four bytes at (4 qd + t) mod Z
    //      of column c's sign-magnitude bytes: two aligned words of the
    //      column, funnel-shifted by (t mod 4) bytes, give all four; byte
    //      permutes spread them over two packed key pairs ----------------------
    int W = 0;
    {
        const uint32_t Zq = Z >> 2;                  // quads per row (a multiple of 16)
        const int tpr = (int)((Zq + 31u) >> 5);      // warp tasks per row
        const uint32_t *w32 = reinterpret_cast<const uint32_t *>(sm);
        int rr = 0, tk = gw;                         // task = rr * tpr + tk, stepped by WPF
        while (tk >= tpr) tk -= tpr, ++rr;
        for (int task = gw; task < MB * tpr; task += WPF) {
            const uint32_t r = (uint32_t)rr;
            const uint32_t qd = (uint32_t)tk * 32u + (uint32_t)lane;
            for (tk += WPF; tk >= tpr; tk -= tpr) ++rr;
            const bool ok = qd < Zq;                  // (groups of 8 lanes all or none: Zq % 16 == 0)
            const uint32_t qv = ok ? qd : 0u;
            const uint32_t e0 = rptr[r], e1 = rptr[r + 1];
            uint32_t k1a = 0xffffffffu, k2a = 0xffffffffu, k1b = 0xffffffffu, k2b = 0xffffffffu, par = 0u;
            uint32_t ek = 0u;  // the entry index in both halves
            for (uint32_t e = e0; e < e1; ++e, ek += 0x10001u) {
                const uint32_t ent = rent[e];
                const uint32_t tt = ent & 0xffffu;
                const uint32_t *col = w32 + (ent >> 16) * Zq;
                uint32_t wq = qv + (tt >> 2);
                wq = wq >= Zq ? wq - Zq : wq;
                const uint32_t wq1 = wq + 1u == Zq ? 0u : wq + 1u;
                const uint32_t v = __funnelshift_r(col[wq], col[wq1], 8u * (tt & 3u));
                // |q| << 8 | sign << 7 | entry for checks (0, 1) and (2, 3)
                const uint32_t ka = __byte_perm(v, 0u, 0x4140) * 128u + ek;
                const uint32_t kb = __byte_perm(v, 0u, 0x4342) * 128u + ek;
                k2a = vmin_u16x2(k2a, vmax_u16x2(k1a, ka));
                k1a = vmin_u16x2(k1a, ka);
                k2b = vmin_u16x2(k2b, vmax_u16x2(k1b, kb));
                k1b = vmin_u16x2(k1b, kb);
                par ^= v;
            }
            uint32_t nib = 0u;  // the four syndrome bits
#pragma unroll
            for (int sidx = 0; sidx < 4; ++sidx) {
                const uint32_t k1 = sidx < 2 ? k1a : k1b, k2 = sidx < 2 ? k2a : k2b;
                const uint32_t a1 = k1 >> (16 * (sidx & 1)), a2 = k2 >> (16 * (sidx & 1));
                const uint32_t min1 = (a1 >> 8) & 0x7fu, pos = a1 & 0x7fu, min2 = (a2 >> 8) & 0x7fu;
                const uint32_t diff = min2 - min1;
                const uint32_t sb = (par >> (8 * sidx)) & 1u;
                nib |= sb << sidx;
                const uint32_t ii = 4u * qv + (uint32_t)sidx;
                const uint32_t ent = rent[e0 + pos];
                const uint32_t c = ent >> 16;
                uint32_t a = ii + (ent & 0xffffu);
                a = a >= Z ? a - Z : a;
                if (ok) {
                    crec[r * Z + ii] = min1 | (diff << 8) | ((c * Z + a) << 16);  // min1, diff, arg-min bit
                    if (diff) {
                        uint32_t idx, sh;
                        qc_pair_slot(c, a, H, idx, sh);
                        const int d = sb ? (int)diff : -(int)diff;
                        atomicAdd(&SC[idx], (uint32_t)d << sh);
                    }
                }
            }
            if (!ok) nib = 0u;
            // 8 lanes' nibbles make one 32-bit word of syndrome bits
            uint32_t wv = nib << (4 * (lane & 7));
            wv |= __shfl_xor_sync(FULL, wv, 1);
            wv |= __shfl_xor_sync(FULL, wv, 2);
            wv |= __shfl_xor_sync(FULL, wv, 4);
            if (ok && (lane & 7) == 0) sbits[(r * Z + 4u * qv) >> 5] = wv;
            W += __popc(nib);
        }
        W = warp_sum(W);  // (per lane so far; the group sum takes lane 0's)
    }
    W = group_sum3<WPF>(make_int3(W, 0, 0), red, rhalf, lane, gw, bar_id).x;  // (meets the group if WPF > 1)
    if constexpr (WPF == 1) __syncwarp();

    // the doubled arrays of V'_m = (2 s_m - 1) min1_m + 128, one per block row
    for (int r = 0; r < MB; ++r) {
        const uint32_t base = (uint32_t)r * Z;
        build_doubled(X2 + r * XJ, (int)Z, (int)H, XJ, t, G, [&](int k) {
            const uint32_t m = base + (uint32_t)k;
            const uint32_t mn = crec[m] & 0x7fu;
            return ((sbits[m >> 5] >> (m & 31)) & 1u) ? 128u + mn : 128u - mn;
        });
    }
    group_sync<WPF>(bar_id);

    // ---- iterations ------------------------------------------------------
    int iters;
    const int aq = P.alpha_q, tq = P.theta_q;
    for (int k = 0;; ++k) {
        if (W == 0) {
            iters = k;
            break;
        }
        if (k == P.max_iter) {
            iters = -P.max_iter;
            break;
        }
        // gather over the column's entries, then the per-block candidates:
        // chunks of 32 R consecutive pairs of one block column, R per lane
        // (the column's entries and addresses shared by the lane's R pairs)
        const int cpc = (int)H / (32 * R);  // chunks per block column
        // chunk ch = c * cpc + k of this warp, (c, k) stepped along with ch
        int cc = 0, ck = gw;
        while (ck >= cpc) ck -= cpc, ++cc;
        for (int ch = gw; ch < NB * cpc; ch += WPF) {
            const uint32_t c = (uint32_t)cc;
            const uint32_t j0 = (uint32_t)ck * 32u * R + (uint32_t)lane;
            for (ck += WPF; ck >= cpc; ck -= cpc) ++cc;
            // D_n - T_n = G_n - 128 d_v(c) + SC_n - 0x8000: the block column's
            // own weight d_v(c) (block columns may differ in weight)
            const uint32_t e0 = cptr[c], e1 = cptr[c + 1];
            const int bias = 128 * (int)(e1 - e0) + 0x8000;
            const uint32_t dfilter = (uint32_t)(0x8000 - bias - 1) * 0x10001u;
            uint32_t acc[R];
#pragma unroll
            for (int r = 0; r < R; ++r) acc[r] = 0u;
            for (uint32_t e = e0; e < e1; ++e) {
                const uint32_t ent = cent[e];
                const uint32_t *xb = X2 + (ent >> 16) * (uint32_t)XJ + j0 + (ent & 0xffffu);
#pragma unroll
                for (int r = 0; r < R; ++r) acc[r] += xb[32 * r];
            }
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const uint32_t j = j0 + 32u * r;
                const uint32_t SC2 = SC[c * H + j];
                // D_n - T_n >= 1, i.e. E' > theta: both halves at once (per half
                // 0x8000 + D_n - T_n - 1 in [0, 65535], so the 32-bit sum is the
                // packed pair exactly)
                const uint32_t cmask = (acc[r] + SC2 + dfilter) & 0x80008000u;
                if (cmask == 0u) continue;
#pragma unroll
                for (int half = 0; half < 2; ++half) {
                    const uint32_t n = c * Z + j + (half ? H : 0u);
                    const int Gv = (int)((acc[r] >> (16 * half)) & 0xffffu);
                    const int sc = (int)((SC2 >> (16 * half)) & 0xffffu);
                    const int a = (int)(sm[n] >> 1);
                    const uint32_t tnv = ((uint32_t)aq * (uint32_t)a + (uint32_t)tq) >> 8;
                    const int E = (Gv + sc - bias + (int)(tnv < 16129u ? tnv : 16129u)) * 256 - aq * a;
                    if (E > tq) {
                        const uint32_t blk = div_small(n, P.p, P.p_magic);
                        const unsigned long long key =
                            ((unsigned long long)((uint32_t)E ^ 0x80000000u) << 32) | (0xffffffffu - n);
                        atomicMax(&keys[blk], key);
                    }
                }
            }
        }
        group_sync<WPF>(bar_id);
        // flips: warp gw reads the keys of 32 blocks at a time (b = b0 + lane);
        // the flipped bits' positions go, in lane order, into the slots of
        // those keys (read, so free), and 2^lsh lanes per flipped bit then
        // update its checks (the column's entries e = lane mod 2^lsh, stepping
        // by 2^lsh): 32 >> lsh flipped bits per step, every update by atomics
        int dW = 0, nflip = 0;
        const int lsh = P.lane_shift, lpf = 1 << lsh;
        for (int b0 = 32 * gw; b0 < P.B; b0 += G) {
            const int b = b0 + lane;
            const unsigned long long key = b < P.B ? keys[b] : 0ull;
            const uint32_t pend = __ballot_sync(FULL, key != 0ull);
            if (pend == 0u) continue;
            const int nf = __popc(pend);
            nflip += nf;  // (warp-uniform)
            uint32_t *slot = reinterpret_cast<uint32_t *>(keys + b0);  // nf < 2 (B - b0) words
            if (key) {
                const uint32_t n = 0xffffffffu - (uint32_t)key;
                atomicXor(&zbits[n >> 5], 1u << (n & 31));
                slot[__popc(pend & ((1u << lane) - 1u))] = n;  // (after the warp's key reads: the ballot)
            }
            __syncwarp();
            for (int k = lane >> lsh; k < nf; k += 32 >> lsh) {
                const uint32_t n = slot[k];
                const uint32_t c = div_small(n, Z, P.z_magic);
                const uint32_t j = n - c * Z;
                const uint32_t e1 = cptr[c + 1];
                for (uint32_t e = cptr[c] + (uint32_t)(lane & (lpf - 1)); e < e1; e += (uint32_t)lpf) {
                    const uint32_t ent = cent[e];
                    const uint32_t r = ent >> 16;
                    uint32_t a = j + (ent & 0xffffu);
                    a = a >= Z ? a - Z : a;
                    const uint32_t m = r * Z + a;
                    const uint32_t bit = 1u << (m & 31);
                    const uint32_t old = atomicXor(&sbits[m >> 5], bit);
                    const bool now_set = !(old & bit);
                    dW += now_set ? 1 : -1;
                    const uint32_t rec = crec[m];
                    const int min1 = (int)(rec & 0x7fu), diff = (int)((rec >> 8) & 0x7fu);
                    doubled_add(X2 + r * XJ, (int)a, now_set ? 2 * min1 : -2 * min1, (int)Z, (int)H, XJ);
                    if (diff) {
                        const uint32_t na = rec >> 16;
                        const uint32_t ca = div_small(na, Z, P.z_magic);
                        uint32_t idx, sh;
                        qc_pair_slot(ca, na - ca * Z, H, idx, sh);
                        const int d = now_set ? 2 * diff : -2 * diff;
                        atomicAdd(&SC[idx], (uint32_t)d << sh);
                    }
                }
            }
            __syncwarp();
            if (b < P.B) keys[b] = 0ull;  // the slots and the read keys, for the next pass
        }
        const int3 tot = group_sum3<WPF>(make_int3(warp_sum(dW), nflip, 0), red, rhalf, lane, gw, bar_id);
        W += tot.x;
        if constexpr (WPF == 1) __syncwarp();
        if (tot.y == 0) {  // fixed point: every later pass repeats this one
            iters = -P.max_iter;
            break;
        }
    }

    uint32_t *ob = P.out_bits + f * (unsigned long long)Nw;
    for (int w = t; w < Nw; w += G) __stcs(ob + w, zbits[w]);
    if (t == 0) P.out_iters[f] = iters;
    group_sync<WPF>(bar_id);
    return true;
}

inline uint32_t qc_magic(uint32_t d) { return d <= 1 ? 0u : (uint32_t)((0x100000000ull + d - 1) / d); }

// Host: the code-dependent fields and the per-frame shared-memory layout.
inline void qc_layout(const fwbf_code_s *c, QcParams &P) {
    auto a16 = [](uint32_t x) { return (x + 15u) & ~15u; };
    P.table = c->d_table;
    P.table_words = c->table_words;
    P.table_smem_bytes = a16(c->table_words * 4u);
    P.rptr_off = c->rptr_off;
    P.rent_off = c->rent_off;
    P.cptr_off = c->cptr_off;
    P.cent_off = c->cent_off;
    P.Z = c->Z;
    P.H = c->Z / 2;
    P.MB = c->MB;
    P.NB = c->NB;
    P.XJ = P.Z + P.H - 1;
    P.p = c->p;
    P.B = c->B;
    P.p_magic = c->p_magic;
    P.z_magic = c->z_magic;
    P.h_magic = qc_magic((uint32_t)P.H);
    P.lane_shift = 0;
    while ((1 << P.lane_shift) < c->dv_max && P.lane_shift < 5) ++P.lane_shift;
    const uint32_t N = (uint32_t)c->N, M = (uint32_t)c->M;
    uint32_t o = a16(N + 32);
    P.off_X = o;
    o += a16(4u * (uint32_t)(P.MB * P.XJ));
    P.off_crec = o;
    o += a16(4u * M);
    P.off_SC = o;
    o += a16(4u * (uint32_t)(P.NB * P.H));
    P.off_s = o;
    o += a16(M / 8u);
    P.off_z = o;
    o += a16(N / 8u);
    P.off_keys = o;
    o += a16(8u * (uint32_t)P.B);
    P.off_mbar = o;  // the frame-load mbarrier (8 bytes) and the load-timeout flag
    o += 16u;
    P.off_red = o;  // group sums: 2 halves x 4 ints x up to 8 warps (qc_set_wpf: 16)
    P.warp_bytes = o + 256u;
}

// Sizes the frame's slice for groups of wpf warps (qc_layout assumes up to 8).
inline void qc_set_wpf(QcParams &P, int wpf) { P.warp_bytes = P.off_red + (wpf > 8 ? 512u : 256u); }

// R pairs per lane per gather chunk: the largest of 8, 4, 2, 1 that divides a
// block column's H / 32 = Z / 64 groups of 32 pairs (odd for Z = 64, 192, ...)
inline int qc_R(const QcParams &P) {
    const int groups = P.H / 32;
    return groups % 8 == 0 ? 8 : groups % 4 == 0 ? 4 : groups % 2 == 0 ? 2 : 1;
}

}  // namespace fwbf
