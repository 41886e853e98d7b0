// FWBF decoding of real (float32) channel values on sm_103a, and the first-pass
// metric of Eq. 1 for every bit.
//
// Same execution model as the int8 decoder (persistent grid, one warp per
// frame, code tables staged into shared memory by bulk copies), but the
// metric is recomputed for every bit on every pass by gathering over M(n) in
// a fixed order, so that results do not depend on the order of floating-point
// additions between runs:
//   E_n = sum_{m in M(n)} (s_m ? w_{n,m} : -w_{n,m}) - alpha |y_n|,
//   w_{n,m} = min2_m if n is the bit holding min1_m, else min1_m.
#include <math.h>

#include "device_common.cuh"
#include "fwbf_internal.h"

namespace fwbf {

__device__ int g_status_f32;

struct F32Params {
    const uint32_t *table;
    uint32_t table_words;
    int table_in_smem;
    int N, M, Z;
    uint32_t rptr_off, rent_off, cptr_off, cent_off;
    int p, B;
    uint32_t p_magic, z_magic;
    const float *y;
    int64_t F;
    int max_iter;
    float alpha, theta;
    uint32_t *out_bits;
    int32_t *out_iters;
    float *out_E;  // metric-only mode when non-null
    unsigned long long *counter;
    uint32_t warp_bytes, off_min1, off_min2, off_arg, off_s, off_z, off_keys;
    uint32_t table_smem_bytes;
};

// order-preserving map of a float to uint32 (larger float -> larger key)
__device__ __forceinline__ uint32_t float_key(float x) {
    const uint32_t u = __float_as_uint(x);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

template <bool PLAIN>
__global__ void __launch_bounds__(768, 1) fwbf_decode_f32_kernel(const F32Params P) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ uint64_t bar;
    __shared__ int flag;

    const uint32_t *tbl = P.table;
    if (P.table_in_smem) {
        uint32_t *st = reinterpret_cast<uint32_t *>(smem);
        if (!stage_table(st, P.table, P.table_words, &bar, &flag)) {
            if (threadIdx.x == 0) atomicOr(&g_status_f32, 1);
            return;
        }
        tbl = st;
    }
    const uint32_t *rptr = tbl + P.rptr_off;
    const uint32_t *rent = tbl + P.rent_off;
    const uint32_t *cptr = tbl + P.cptr_off;
    const uint32_t *cent = tbl + P.cent_off;

    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    unsigned char *ws = smem + P.table_smem_bytes + warp * P.warp_bytes;
    float *a = reinterpret_cast<float *>(ws);
    float *min1 = reinterpret_cast<float *>(ws + P.off_min1);
    float *min2 = reinterpret_cast<float *>(ws + P.off_min2);
    uint32_t *arg = reinterpret_cast<uint32_t *>(ws + P.off_arg);
    uint32_t *sbits = reinterpret_cast<uint32_t *>(ws + P.off_s);
    uint32_t *zbits = reinterpret_cast<uint32_t *>(ws + P.off_z);
    unsigned long long *keys = reinterpret_cast<unsigned long long *>(ws + P.off_keys);

    const int N = P.N, M = P.M;
    const uint32_t Z = (uint32_t)P.Z;
    const int Nw = (N + 31) >> 5;
    const bool metric_only = P.out_E != nullptr;

    for (int b = lane; b < P.B; b += 32) keys[b] = 0ull;

    for (;;) {
        unsigned long long f = 0;
        if (lane == 0) f = atomicAdd(P.counter, 1ull);
        f = __shfl_sync(FULL, f, 0);
        if (f >= (unsigned long long)P.F) break;
        const float *yf = P.y + f * (unsigned long long)N;

        for (int w = 0; w < Nw; ++w) {
            const int n = (w << 5) + lane;
            float v = 0.0f;
            if (n < N) {
                v = __ldcs(yf + n);
                a[n] = fabsf(v);
            }
            const uint32_t zb = __ballot_sync(FULL, n < N && v < 0.0f);
            if (lane == 0) zbits[w] = zb;
        }
        __syncwarp();

        int W = 0;
        for (int base = 0; base < M; base += 32) {
            const int m = base + lane;
            uint32_t s = 0;
            if (m < M) {
                uint32_t R, i;
                if (PLAIN) {
                    R = m;
                    i = 0;
                } else {
                    R = div_small(m, Z, P.z_magic);
                    i = m - R * Z;
                }
                float m1 = INFINITY, m2 = INFINITY;
                uint32_t am = 0, par = 0;
                for (uint32_t e = rptr[R]; e < rptr[R + 1]; ++e) {
                    const uint32_t n = PLAIN ? (rent[e] >> 16) : circ_index(rent[e], i, Z);
                    const float v = a[n];
                    par ^= zbits[n >> 5] >> (n & 31);
                    if (v < m1) {
                        m2 = m1;
                        m1 = v;
                        am = n;
                    } else if (v < m2) {
                        m2 = v;
                    }
                }
                s = par & 1u;
                min1[m] = m1;
                min2[m] = m2;
                arg[m] = am;
            }
            const uint32_t sw = __ballot_sync(FULL, s);
            if (lane == 0) sbits[base >> 5] = sw;
            W += __popc(sw);
        }
        __syncwarp();

        int iters = 0;
        for (int k = 0;; ++k) {
            if (!metric_only) {
                if (W == 0) {
                    iters = k;
                    break;
                }
                if (k == P.max_iter) {
                    iters = -P.max_iter;
                    break;
                }
            }
            for (int n = lane; n < N; n += 32) {
                uint32_t C, j;
                if (PLAIN) {
                    C = n;
                    j = 0;
                } else {
                    C = div_small(n, Z, P.z_magic);
                    j = n - C * Z;
                }
                float E = 0.0f;
                for (uint32_t e = cptr[C]; e < cptr[C + 1]; ++e) {
                    const uint32_t m = PLAIN ? (cent[e] >> 16) : circ_index(cent[e], j, Z);
                    const float w = (arg[m] == (uint32_t)n) ? min2[m] : min1[m];
                    E += ((sbits[m >> 5] >> (m & 31)) & 1u) ? w : -w;
                }
                E = __fsub_rn(E, __fmul_rn(P.alpha, a[n]));
                if (metric_only) {
                    __stcs(P.out_E + f * (unsigned long long)N + n, E);
                } else if (E > P.theta) {
                    const uint32_t blk = div_small(n, P.p, P.p_magic);
                    const unsigned long long key =
                        ((unsigned long long)float_key(E) << 32) | (0xffffffffu - (uint32_t)n);
                    atomicMax(&keys[blk], key);
                }
            }
            __syncwarp();
            if (metric_only) break;
            int dW = 0, nflip = 0;
            for (int b = lane; b < P.B; b += 32) {
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
            W += warp_sum(dW);
            nflip = warp_sum(nflip);
            __syncwarp();
            if (nflip == 0) {
                iters = -P.max_iter;
                break;
            }
        }
        if (!metric_only) {
            uint32_t *ob = P.out_bits + f * (unsigned long long)Nw;
            for (int w = lane; w < Nw; w += 32) __stcs(ob + w, zbits[w]);
            if (lane == 0) P.out_iters[f] = iters;
        }
        __syncwarp();
    }
}

static inline uint32_t align16(uint32_t x) { return (x + 15u) & ~15u; }

int read_and_clear_status_f32(cudaStream_t s, int *out) {
    int v = 0, zero = 0;
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    e = cudaMemcpyFromSymbol(&v, g_status_f32, sizeof(int));
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyFromSymbol(status)");
    if (v) {
        e = cudaMemcpyToSymbol(g_status_f32, &zero, sizeof(int));
        if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyToSymbol(status)");
    }
    *out = v;
    return 0;
}

int launch_decode_f32(const fwbf_code_s *c, const float *y, int64_t n_frames, int max_iter, float alpha,
                      float theta, uint32_t *out_bits, int32_t *out_iters, float *out_E, cudaStream_t s) {
    F32Params P{};
    P.table = c->d_table;
    P.table_words = c->table_words;
    P.N = c->N;
    P.M = c->M;
    P.Z = c->Z;
    P.rptr_off = c->rptr_off;
    P.rent_off = c->rent_off;
    P.cptr_off = c->cptr_off;
    P.cent_off = c->cent_off;
    P.p = c->p;
    P.B = c->B;
    P.p_magic = c->p_magic;
    P.z_magic = c->z_magic;
    P.y = y;
    P.F = n_frames;
    P.max_iter = max_iter;
    P.alpha = alpha;
    P.theta = theta;
    P.out_bits = out_bits;
    P.out_iters = out_iters;
    P.out_E = out_E;

    const uint32_t N = c->N, M = c->M;
    uint32_t o = align16(4 * N);
    P.off_min1 = o;
    o += align16(4 * M);
    P.off_min2 = o;
    o += align16(4 * M);
    P.off_arg = o;
    o += align16(4 * M);
    P.off_s = o;
    o += align16(4 * ((M + 31) / 32));
    P.off_z = o;
    o += align16(4 * ((N + 31) / 32));
    P.off_keys = o;
    o += align16(8 * (uint32_t)c->B);
    P.warp_bytes = o;

    const uint32_t tbytes = c->table_words * 4u;
    const uint32_t optin = (uint32_t)c->smem_optin;
    P.table_in_smem = (tbytes + P.warp_bytes + 256u <= optin && tbytes <= 96u * 1024u) ? 1 : 0;
    P.table_smem_bytes = P.table_in_smem ? tbytes : 0;
    const uint32_t avail = optin - 256u - P.table_smem_bytes;
    if (P.warp_bytes > avail) return fail(FWBF_EUNSUPPORTED, "code too large for one warp's shared memory");
    int warps = (int)(avail / P.warp_bytes);
    if (warps > 24) warps = 24;
    const uint32_t dyn = P.table_smem_bytes + warps * P.warp_bytes;

    auto kern = c->Z == 1 ? fwbf_decode_f32_kernel<true> : fwbf_decode_f32_kernel<false>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute");
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, warps * 32, dyn);
    if (e != cudaSuccess) return cuda_fail(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
    if (per_sm < 1) return fail(FWBF_EUNSUPPORTED, "decode kernel does not fit on an SM");
    int64_t blocks = (int64_t)per_sm * c->num_sms;
    const int64_t need = (n_frames + warps - 1) / warps;
    if (blocks > need) blocks = need;

    CounterLease ctr;
    int rc = acquire_counter(c, s, &ctr);
    if (rc) return rc;
    P.counter = ctr.ptr;
    kern<<<(unsigned)blocks, warps * 32, dyn, s>>>(P);
    e = cudaGetLastError();
    const int rc2 = release_counter(ctr, s);
    if (e != cudaSuccess) return cuda_fail(e, "decode_f32 launch");
    return rc2;
}

}  // namespace fwbf
