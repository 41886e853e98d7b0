// FWBF decoding of int8 channel values on sm_103a (paper Sec. III with the
// metric of Eq. 1 in fixed point).
//
// Execution model: a persistent grid, one warp per frame.  A warp takes the
// next frame from a global counter, decodes it entirely in its own slice of
// shared memory and writes the bit-packed decisions and the pass count.  The
// code's index tables are staged into shared memory once per CTA with bulk
// copies (TMA).
//
// Exact reformulation used on the device (every step gives the same integers
// as the definition):
//   * per check m: min1 = smallest |q| of N(m), pos = its position in the row,
//     min2 = second smallest (with multiplicity).  w_{n,m} = min2 for the bit at
//     pos and min1 for every other bit of the row -- the minimum over N(m)\n.
//   * per bit n: tot_n = sum_{m in M(n)} w_{n,m} (fixed) and
//     U_n = sum_{m in M(n), s_m = 1} w_{n,m}; then
//     E'_n = 256 sum (2 s_m - 1) w_{n,m} - alpha_q a_n = 256 (2 U_n - tot_n) - alpha_q a_n.
//     U_n is rebuilt each pass by scattering w from the unsatisfied checks only
//     (satisfied checks add nothing to U).
//   * block arg-max: a bit with E' <= theta can neither win a block whose
//     maximum exceeds theta nor be flipped, so only bits with E' > theta compete;
//     a 64-bit key (E' biased, then ~n) max-reduced per block keeps the largest
//     metric and, among equals, the lowest index.
//   * the syndrome is updated by toggling the checks of each flipped bit; its
//     weight follows from the toggles.
//   * a pass that flips nothing leaves the state unchanged, so every later pass
//     repeats it: the frame ends as "not converged" (-max_iter) at once with the
//     same z.
#include <mutex>
#include <string>

#include "device_common.cuh"
#include "fwbf_internal.h"

namespace fwbf {

__device__ int g_status_i8;

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
};

template <bool PLAIN>  // PLAIN: Z == 1, the tables are plain CSR / CSC
__global__ void __launch_bounds__(768, 1) fwbf_decode_i8_kernel(const I8Params P) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ uint64_t bar;
    __shared__ int flag;

    const uint32_t *tbl = P.table;
    if (P.table_in_smem) {
        uint32_t *st = reinterpret_cast<uint32_t *>(smem);
        if (!stage_table(st, P.table, P.table_words, &bar, &flag)) {
            if (threadIdx.x == 0) atomicOr(&g_status_i8, 1);
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
    int8_t *stage = reinterpret_cast<int8_t *>(ws);
    uint32_t *T = reinterpret_cast<uint32_t *>(ws + P.off_T);
    uint32_t *crec = reinterpret_cast<uint32_t *>(ws + P.off_crec);
    uint32_t *sbits = reinterpret_cast<uint32_t *>(ws + P.off_s);
    uint32_t *zbits = reinterpret_cast<uint32_t *>(ws + P.off_z);
    unsigned long long *keys = reinterpret_cast<unsigned long long *>(ws + P.off_keys);

    const int N = P.N, M = P.M;
    const uint32_t Z = (uint32_t)P.Z;
    const int Nw = (N + 31) >> 5, Mw = (M + 31) >> 5;
    const uintptr_t ybase = reinterpret_cast<uintptr_t>(P.y);
    const uintptr_t yend = ybase + (uintptr_t)(P.F * (int64_t)N);

    for (int b = lane; b < P.B; b += 32) keys[b] = 0ull;

    for (;;) {
        unsigned long long f = 0;
        if (lane == 0) f = atomicAdd(P.counter, 1ull);
        f = __shfl_sync(FULL, f, 0);
        if (f >= (unsigned long long)P.F) break;

        // ---- load the frame: aligned 16-byte chunks covering it --------------
        const uintptr_t fb = ybase + (uintptr_t)(f * (unsigned long long)N);
        const uintptr_t a0 = fb & ~(uintptr_t)15;
        const int off = (int)(fb - a0);
        const int nchunks = (off + N + 15) >> 4;
        for (int c = lane; c < nchunks; c += 32) {
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
            *reinterpret_cast<uint4 *>(stage + c * 16) = v;
        }
        for (int n = lane; n < N; n += 32) T[n] = 0u;
        __syncwarp();
        const int8_t *q = stage + off;

        // ---- initialisation: z_0, per-check (min1, min2, pos), s_0, tot, U ---
        for (int w = 0; w < Nw; ++w) {
            const int n = (w << 5) + lane;
            const uint32_t zb = __ballot_sync(FULL, n < N && q[n] < 0);
            if (lane == 0) zbits[w] = zb;
        }
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
        __syncwarp();

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
                for (int wd = lane; wd < Mw; wd += 32) {
                    uint32_t bits = sbits[wd];
                    while (bits) {
                        const int j = __ffs(bits) - 1;
                        bits &= bits - 1;
                        const uint32_t m = (wd << 5) + j;
                        const uint32_t rec = crec[m];
                        const uint32_t min1 = rec & 0xffu, min2 = (rec >> 8) & 0xffu, pos = rec >> 16;
                        uint32_t R, i;
                        if (PLAIN) {
                            R = m;
                            i = 0;
                        } else {
                            R = div_small(m, Z, P.z_magic);
                            i = m - R * Z;
                        }
                        const uint32_t e0 = rptr[R], e1 = rptr[R + 1];
                        for (uint32_t e = e0; e < e1; ++e) {
                            const uint32_t n = PLAIN ? (rent[e] >> 16) : circ_index(rent[e], i, Z);
                            atomicAdd(&T[n], (e - e0 == pos) ? min2 : min1);
                        }
                    }
                }
                __syncwarp();
            }
            // metric and per-block candidates
            for (int n = lane; n < N; n += 32) {
                const uint32_t t = T[n];
                const uint32_t U = t & 0xffffu;
                if (U) T[n] = t & 0xffff0000u;
                const int tot = (int)(t >> 16);
                const int E = (2 * (int)U - tot) * 256 - P.alpha_q * abs((int)q[n]);
                if (E > P.theta_q) {
                    const uint32_t blk = div_small(n, P.p, P.p_magic);
                    const unsigned long long key =
                        ((unsigned long long)((uint32_t)E ^ 0x80000000u) << 32) | (0xffffffffu - (uint32_t)n);
                    atomicMax(&keys[blk], key);
                }
            }
            __syncwarp();
            // flips: all blocks read s_k; apply together
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
            if (nflip == 0) {  // fixed point with a non-zero syndrome
                iters = -P.max_iter;
                break;
            }
        }

        // ---- outputs ---------------------------------------------------------
        uint32_t *ob = P.out_bits + f * (unsigned long long)Nw;
        for (int w = lane; w < Nw; w += 32) __stcs(ob + w, zbits[w]);
        if (lane == 0) P.out_iters[f] = iters;
        __syncwarp();
    }
}

int read_and_clear_status_i8(cudaStream_t s, int *out) {
    int v = 0, zero = 0;
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    e = cudaMemcpyFromSymbol(&v, g_status_i8, sizeof(int));
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyFromSymbol(status)");
    if (v) {
        e = cudaMemcpyToSymbol(g_status_i8, &zero, sizeof(int));
        if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyToSymbol(status)");
    }
    *out = v;
    return 0;
}

static inline uint32_t align16(uint32_t x) { return (x + 15u) & ~15u; }

// Generic (any H) int8 decoder launch with a caller-provided frame counter
// that is already zero on the stream.
static int launch_generic_i8(const fwbf_code_s *c, const int8_t *y, int64_t n_frames, int max_iter, int alpha_q,
                             int theta_q, uint32_t *out_bits, int32_t *out_iters, unsigned long long *counter,
                             cudaStream_t s) {
    I8Params P{};
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
    P.y = y;
    P.F = n_frames;
    P.max_iter = max_iter;
    P.alpha_q = alpha_q;
    P.theta_q = theta_q;
    P.out_bits = out_bits;
    P.out_iters = out_iters;
    P.counter = counter;

    const uint32_t N = c->N, M = c->M;
    uint32_t o = align16(N + 32);
    P.off_T = o;
    o += align16(4 * N);
    P.off_crec = o;
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
    const uint32_t avail = optin - 256u - P.table_smem_bytes;  // static shared memory margin
    if (P.warp_bytes > avail) return fail(FWBF_EUNSUPPORTED, "code too large for one warp's shared memory");
    int warps = (int)(avail / P.warp_bytes);
    if (warps > 24) warps = 24;
    const uint32_t dyn = P.table_smem_bytes + warps * P.warp_bytes;

    auto kern = c->Z == 1 ? fwbf_decode_i8_kernel<true> : fwbf_decode_i8_kernel<false>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute");
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, warps * 32, dyn);
    if (e != cudaSuccess) return cuda_fail(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
    if (per_sm < 1) return fail(FWBF_EUNSUPPORTED, "decode kernel does not fit on an SM");
    int64_t blocks = (int64_t)per_sm * c->num_sms;
    const int64_t need = (n_frames + warps - 1) / warps;
    if (blocks > need) blocks = need;
    kern<<<(unsigned)blocks, warps * 32, dyn, s>>>(P);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "decode_i8 launch");
    return 0;
}

// Picks the decoder for the code: the packed cyclic kernel when H is a single
// circulant it handles, the generic kernel otherwise.
static int launch_i8_with_counter(const fwbf_code_s *c, const int8_t *y, int64_t n_frames, int max_iter,
                                  int alpha_q, int theta_q, uint32_t *out_bits, int32_t *out_iters,
                                  unsigned long long *counter, cudaStream_t s) {
    if (cyclic_eligible(c))
        return launch_decode_i8_cyclic(c, y, n_frames, max_iter, alpha_q, theta_q, out_bits, out_iters, counter, s);
    return launch_generic_i8(c, y, n_frames, max_iter, alpha_q, theta_q, out_bits, out_iters, counter, s);
}

int launch_decode_i8(const fwbf_code_s *c, const int8_t *y, int64_t n_frames, int max_iter, int alpha_q,
                     int theta_q, uint32_t *out_bits, int32_t *out_iters, cudaStream_t s) {
    unsigned long long *counter = nullptr;
    cudaError_t e = cudaMallocAsync(reinterpret_cast<void **>(&counter), sizeof(unsigned long long), s);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMallocAsync(frame counter)");
    e = cudaMemsetAsync(counter, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) {
        cudaFreeAsync(counter, s);
        return cuda_fail(e, "cudaMemsetAsync");
    }
    const int rc = launch_i8_with_counter(c, y, n_frames, max_iter, alpha_q, theta_q, out_bits, out_iters, counter, s);
    e = cudaFreeAsync(counter, s);
    if (rc) return rc;
    if (e != cudaSuccess) return cuda_fail(e, "cudaFreeAsync(frame counter)");
    return 0;
}

// ---------------------------------------------------------------------------
// Decoding without any device allocation (fwbf_decode_noalloc).
//
// The decoder's only scratch is its frame work counter (8 bytes).  For callers
// that must not allocate device memory once they are running, the counter is
// taken from a fixed array that every GPU loading this library holds until the
// process exits.  All such calls share the array: it is cleared on the stream
// before each launch, and calls that overlap on the GPU race on it.
// ---------------------------------------------------------------------------

constexpr size_t kNoAllocScratchBytes = 256;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 64;
static std::mutex g_noalloc_mu;
static void *g_noalloc_addr[kMaxDevices];

// Device address of g_noalloc_scratch on the current device, looked up once
// per device.  (In host code the array's name is only a host-side stand-in.)
static int noalloc_scratch(void **out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) return fail(FWBF_EUNSUPPORTED, "device index above 63");
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(no-allocation scratch)");
        g_noalloc_addr[dev] = p;
    }
    *out = g_noalloc_addr[dev];
    return 0;
}

int launch_decode_i8_noalloc(const fwbf_code_s *c, const int8_t *y, int64_t n_frames, int max_iter, int alpha_q,
                             int theta_q, uint32_t *out_bits, int32_t *out_iters, cudaStream_t s) {
    const size_t need = sizeof(unsigned long long);
    if (need > kNoAllocScratchBytes)
        return fail(FWBF_EUNSUPPORTED, "no-allocation decode needs " + std::to_string(need) +
                                           " bytes of scratch, above its fixed " +
                                           std::to_string(kNoAllocScratchBytes) + "-byte array");
    void *scratch = nullptr;
    int rc = noalloc_scratch(&scratch);
    if (rc) return rc;

    // the counter must start at zero; the array keeps the previous call's value
    cudaError_t e = cudaMemsetAsync(scratch, 0, need, s);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync(no-allocation scratch)");
    return launch_i8_with_counter(c, y, n_frames, max_iter, alpha_q, theta_q, out_bits, out_iters,
                                  static_cast<unsigned long long *>(scratch), s);
}

}  // namespace fwbf
