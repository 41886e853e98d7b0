// FWBF decoding of int8 channel values for quasi-cyclic codes on sm_103a
// (paper Sec. III with the metric of Eq. 1 in fixed point): the packed layout
// of the cyclic decoder carried over to H made of several circulant blocks
// (qc_frame.cuh).  A frame is decoded by a group of warps from its own slice
// of shared memory; the code's tables are staged once per block with bulk
// copies (TMA) on a bounded mbarrier wait.  All integer results equal the
// definition exactly.
#include "qc_frame.cuh"

namespace fwbf {

__device__ int g_status_i8_qc;

template <int R, int WPF>  // pairs per lane per gather chunk, warps per frame
__global__ void __launch_bounds__(768, 1) fwbf_decode_i8_qc_kernel(const __grid_constant__ QcParams P) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ uint64_t bar;
    __shared__ int flag;
    __shared__ unsigned long long fslot[24];

    uint32_t *st = reinterpret_cast<uint32_t *>(smem);
    if (!stage_table(st, P.table, P.table_words, &bar, &flag)) {
        if (threadIdx.x == 0) atomicOr(&g_status_i8_qc, 1);
        return;
    }
    // groups of WPF warps, one frame each; group g meets at named barrier 1 + g
    constexpr int G = 32 * WPF;
    const int t = threadIdx.x % G;
    const int grp = threadIdx.x / G;
    const int bar_id = 1 + grp;
    unsigned char *ws = smem + P.table_smem_bytes + grp * P.warp_bytes;
    unsigned long long *keys = reinterpret_cast<unsigned long long *>(ws + P.off_keys);
    for (int b = t; b < P.B; b += G) keys[b] = 0ull;
    qc_group_init<WPF>(P, ws, t);
    uint32_t lpar = 0;  // phase of the group's frame-load mbarrier
    for (;;) {
        if (t == 0) fslot[grp] = atomicAdd(P.counter, 1ull);
        group_sync<WPF>(bar_id);
        const unsigned long long f = fslot[grp];  // rewritten only after the frame's last meeting
        if (f >= (unsigned long long)P.F) break;
        if (!qc_frame<R, WPF>(P, st, ws, t, bar_id, f, lpar)) {
            if (t == 0) atomicOr(&g_status_i8_qc, 2);
            return;  // (the frame's copy did not arrive: the group leaves)
        }
    }
    qc_group_done(P, ws, t);
}

constexpr uint32_t kQcReserve = 1024u;  // static shared memory of the kernel

// Quasi-cyclic H (several blocks, circulants of a multiple of 64) whose frame
// state fits one block's shared memory; rows up to 127 bits (the arg-min
// position is 7 bits of the packed key), columns up to 127 checks.
bool qc_eligible(const fwbf_code_s *c) {
    if (c->Z <= 1 || c->Z % 64 != 0 || (c->MB == 1 && c->NB == 1)) return false;
    if (c->dc_max > 127 || c->dv_max > 127) return false;
    QcParams P{};
    qc_layout(c, P);
    return P.table_smem_bytes + P.warp_bytes + kQcReserve <= (uint32_t)c->smem_optin;
}

int read_and_clear_status_i8_qc(cudaStream_t s, int *out) {
    int v = 0, zero = 0;
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    e = cudaMemcpyFromSymbol(&v, g_status_i8_qc, sizeof(int));
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyFromSymbol(status)");
    if (v) {
        e = cudaMemcpyToSymbol(g_status_i8_qc, &zero, sizeof(int));
        if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyToSymbol(status)");
    }
    *out = v;
    return 0;
}

int launch_decode_i8_qc(const fwbf_code_s *c, const int8_t *y, int64_t n_frames, int max_iter, int alpha_q,
                        int theta_q, uint32_t *out_bits, int32_t *out_iters, unsigned long long *counter,
                        cudaStream_t s) {
    QcParams P{};
    qc_layout(c, P);
    P.y = y;
    P.F = n_frames;
    P.max_iter = max_iter;
    P.alpha_q = alpha_q;
    P.theta_q = theta_q;
    P.out_bits = out_bits;
    P.out_iters = out_iters;
    P.counter = counter;
    const uint32_t optin = (uint32_t)c->smem_optin;
    if (P.table_smem_bytes + P.warp_bytes + kQcReserve > optin)
        return fail(FWBF_EUNSUPPORTED, "quasi-cyclic code too large for one block's shared memory");
    int frames = (int)((optin - kQcReserve - P.table_smem_bytes) / P.warp_bytes);
    if (frames > 24) frames = 24;
    // up to 24 warps per block: 2, 4 or 8 warps per frame when fewer frames fit
    int wpf = 1;
    while (wpf < 8 && frames * wpf * 2 <= 24) wpf *= 2;
    const int R = qc_R(P);
    void (*kern)(const QcParams);
    if (R == 8)
        kern = wpf == 1 ? fwbf_decode_i8_qc_kernel<8, 1> : wpf == 2 ? fwbf_decode_i8_qc_kernel<8, 2>
             : wpf == 4 ? fwbf_decode_i8_qc_kernel<8, 4> : fwbf_decode_i8_qc_kernel<8, 8>;
    else if (R == 4)
        kern = wpf == 1 ? fwbf_decode_i8_qc_kernel<4, 1> : wpf == 2 ? fwbf_decode_i8_qc_kernel<4, 2>
             : wpf == 4 ? fwbf_decode_i8_qc_kernel<4, 4> : fwbf_decode_i8_qc_kernel<4, 8>;
    else if (R == 2)
        kern = wpf == 1 ? fwbf_decode_i8_qc_kernel<2, 1> : wpf == 2 ? fwbf_decode_i8_qc_kernel<2, 2>
             : wpf == 4 ? fwbf_decode_i8_qc_kernel<2, 4> : fwbf_decode_i8_qc_kernel<2, 8>;
    else
        kern = wpf == 1 ? fwbf_decode_i8_qc_kernel<1, 1> : wpf == 2 ? fwbf_decode_i8_qc_kernel<1, 2>
             : wpf == 4 ? fwbf_decode_i8_qc_kernel<1, 4> : fwbf_decode_i8_qc_kernel<1, 8>;
    int per_sm = 0;
    uint32_t dyn = 0;
    cudaError_t e = cudaSuccess;
    for (; frames >= 1; --frames) {
        dyn = P.table_smem_bytes + frames * P.warp_bytes;
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
        if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute");
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, frames * wpf * 32, dyn);
        if (e != cudaSuccess) return cuda_fail(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
        if (per_sm >= 1) break;
    }
    if (frames < 1 || per_sm < 1) return fail(FWBF_EUNSUPPORTED, "quasi-cyclic kernel does not fit on an SM");
    int64_t blocks = (int64_t)per_sm * c->num_sms;
    const int64_t need = (n_frames + frames - 1) / frames;
    if (blocks > need) blocks = need;
    kern<<<(unsigned)blocks, frames * wpf * 32, dyn, s>>>(P);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "decode_i8_qc launch");
    return 0;
}

}  // namespace fwbf
