// FWBF decoding of int8 channel values for cyclic codes (H a single Z x Z
// circulant: N = M = Z, N(m) = {(m + d_e) mod Z}, M(n) = {(n + u_e) mod Z},
// u_e = -d_e mod Z), e.g. the type-I EG(2, 2^s) codes of the paper's Sec. V.
//
// Same persistent warp-per-frame model as the generic int8 decoder; what
// changes is the data layout, which turns every edge loop into aligned,
// conflict-free shared-memory loads and packed 2 x 16-bit integer arithmetic:
//
//   * positions are paired as (i, i + H), H = ceil(Z / 2), i in [0, H).  A
//     rotation by r maps the pair (i, i + H) onto the positions
//     (i + r, i + H + r) mod Z, which form again a pair of the "doubled" array
//     X2[j] = x[j mod Z] | x[(j + H) mod Z] << 16 (j < Z + H).  So for pair i
//     and offset r the two values are the single word X2[i + r].
//   * check pass (once per frame): per check pair and row offset, the packed
//     key |q| << 8 | sign << 7 | e is min/max-reduced with min.u16x2/max.u16x2
//     into (min1, pos) and min2, and the sign bits XOR into the parity.
//   * w_{n,m} = min1_m except w = min2_m at the row position pos_m holding
//     min1 (the minimum over N(m)\n).  With diff_m = min2_m - min1_m,
//       D_n = sum_{m in M(n)} (2 s_m - 1) w_{n,m}
//           = sum_{m in M(n)} V'_m - 128 d_c + 2 UC_n - TC_n,
//     V'_m = (2 s_m - 1) min1_m + 128 (in [1, 255], so packed sums never carry),
//     TC_n = sum of diff_m over the checks whose arg-min bit is n (fixed) and
//     UC_n = the same sum over those checks with s_m = 1; the kernel keeps
//     SC_n = 2 UC_n - TC_n = sum of (2 s_m - 1) diff_m over those checks.  The sum over M(n)
//     is a gather over the doubled array of V': one load and one packed add per
//     two edges.  Every syndrome toggle updates V' (+-2 min1) and SC (+-2 diff)
//     in place, so a pass is one gather plus its metric epilogue.
//   * E'_n = 256 D_n - alpha_q a_n (Eq. 1 times 256); block arg-max, flips and
//     the no-flip shortcut are those of the generic decoder.
// All integer results equal the definition (Sec. III, Eq. 1) exactly.
#include "cyclic_frame.cuh"

namespace fwbf {

__device__ int g_status_i8_cyclic;

template <int R, int WPF, int VAR>  // pairs per lane per chunk, warps per frame, body (kVar*)
__global__ void __launch_bounds__(512, WPF == 2 ? 2 : 1) fwbf_decode_i8_cyclic_kernel(const CyclicParams P) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ uint64_t bar;
    __shared__ int flag;
    __shared__ __align__(16) uint32_t d_off[128], u_off[128];  // read as 8- and 16-byte vectors
    __shared__ unsigned long long fslot[16];

    {
        uint32_t *st = reinterpret_cast<uint32_t *>(smem);
        if (!stage_table(st, P.table, P.table_words, &bar, &flag)) {
            if (threadIdx.x == 0) atomicOr(&g_status_i8_cyclic, 1);
            return;
        }
        for (int e = threadIdx.x; e < 128; e += blockDim.x) {  // zeros past d_c
            d_off[e] = e < P.DC ? st[P.rent_off + e] & 0xffffu : 0u;
            u_off[e] = e < P.DC ? st[P.cent_off + e] & 0xffffu : 0u;
        }
        __syncthreads();
    }
    // groups of WPF warps, one frame each; group g meets at named barrier 1 + g
    constexpr int G = 32 * WPF;
    const int t = threadIdx.x % G;
    const int grp = threadIdx.x / G;
    const int bar_id = 1 + grp;
    unsigned char *ws = smem + P.table_smem_bytes + grp * P.warp_bytes;
    uint32_t *keys = reinterpret_cast<uint32_t *>(ws + P.off_keys);
    for (uint32_t b = t; b < P.key_words; b += G) keys[b] = 0u;
    for (;;) {
        if (t == 0) fslot[grp] = atomicAdd(P.counter, 1ull);
        group_sync<WPF>(bar_id);
        const unsigned long long f = fslot[grp];  // rewritten only after the frame's last meeting
        if (f >= (unsigned long long)P.F) break;
        cyclic_frame<R, WPF, VAR>(P, d_off, u_off, ws, t, bar_id, f);
    }
}

template <int WPF, int VAR>
static void (*cyclic_kernel_r(int R))(const CyclicParams) {
    return R == 8 ? fwbf_decode_i8_cyclic_kernel<8, WPF, VAR> : R == 4 ? fwbf_decode_i8_cyclic_kernel<4, WPF, VAR>
         : R == 2 ? fwbf_decode_i8_cyclic_kernel<2, WPF, VAR> : fwbf_decode_i8_cyclic_kernel<1, WPF, VAR>;
}

template <int WPF>
static void (*cyclic_kernel_for(int R, int var))(const CyclicParams) {
    return var == kVarPlain ? cyclic_kernel_r<WPF, kVarPlain>(R)
         : var == kVarLearned ? cyclic_kernel_r<WPF, kVarLearned>(R) : cyclic_kernel_r<WPF, kVarAll>(R);
}

bool cyclic_eligible(const fwbf_code_s *c) {
    if (c->Z != c->N || c->N != c->M || c->MB != 1 || c->NB != 1) return false;
    const int H = (c->Z + 1) / 2;
    if (H % 32 != 0) return false;
    if (c->dc_max > 127 || c->dc_max != c->dv_max) return false;
    return true;
}

int read_and_clear_status_i8_cyclic(cudaStream_t s, int *out) {
    int v = 0, zero = 0;
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    e = cudaMemcpyFromSymbol(&v, g_status_i8_cyclic, sizeof(int));
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyFromSymbol(status)");
    if (v) {
        e = cudaMemcpyToSymbol(g_status_i8_cyclic, &zero, sizeof(int));
        if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyToSymbol(status)");
    }
    *out = v;
    return 0;
}

int launch_decode_i8_cyclic(const fwbf_code_s *c, const int8_t *y, int64_t n_frames, int max_iter, int alpha_q,
                            int theta_q, uint32_t *out_bits, int32_t *out_iters, unsigned long long *counter,
                            cudaStream_t s, const CyclicModes *modes) {
    CyclicParams P{};
    if (modes) {
        P.mode = modes->mode;
        P.sched_a = modes->sched_a;
        P.sched_t = modes->sched_t;
        P.sched_stride = modes->sched_stride;
        P.mlp = modes->mlp;
        P.k_learn = modes->k_learn;
        P.gate_dv = modes->gate_dv;
        P.out_sched = modes->out_sched;
        P.out_feat = modes->out_feat;
        P.feat_passes = modes->feat_passes;
    }
    cyclic_layout(c, P);
    P.y = y;
    P.F = n_frames;
    P.max_iter = max_iter;
    P.alpha_q = alpha_q;
    P.theta_q = theta_q;
    P.out_bits = out_bits;
    P.out_iters = out_iters;
    P.counter = counter;

    const uint32_t optin = (uint32_t)c->smem_optin;
    const uint32_t reserve = 2048u;  // static shared memory of the kernel
    if (P.table_smem_bytes + P.warp_bytes + reserve > optin)
        return fail(FWBF_EUNSUPPORTED, "cyclic code too large for one block's shared memory");
    // frames whose slices fit in one block; with 16 or more, two blocks of 8
    // frames per SM and two warps per frame (32 warps, 64 registers each);
    // otherwise one block and four warps per frame
    const int fmax = (int)((optin - reserve - P.table_smem_bytes) / P.warp_bytes);
    const int wpf = fmax >= 8 ? 2 : 4;
    cyclic_set_wpf(P, wpf);
    int frames = wpf == 2 ? (fmax >= 16 ? 8 : fmax / 2) : (fmax < 4 ? fmax : 4);
    const int R = cyclic_R(c, wpf);
    const int var = P.mode == kModePlain && !P.out_feat ? kVarPlain
                  : P.mode == kModeLearned && !P.out_feat && !P.out_sched ? kVarLearned : kVarAll;
    void (*kern)(const CyclicParams) = wpf == 2 ? cyclic_kernel_for<2>(R, var) : cyclic_kernel_for<4>(R, var);
    int per_sm = 0;
    uint32_t dyn = 0;
    cudaError_t e = cudaSuccess;
    for (; frames >= 1; --frames) {  // shrink the block until the occupancy calculator places one
        dyn = P.table_smem_bytes + frames * P.warp_bytes;
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
        if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute");
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, frames * wpf * 32, dyn);
        if (e != cudaSuccess) return cuda_fail(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
        if (per_sm >= 1) break;
    }
    if (frames < 1 || per_sm < 1) return fail(FWBF_EUNSUPPORTED, "cyclic decode kernel does not fit on an SM");
    int64_t blocks = (int64_t)per_sm * c->num_sms;
    const int64_t need = (n_frames + frames - 1) / frames;
    if (blocks > need) blocks = need;
    kern<<<(unsigned)blocks, frames * wpf * 32, dyn, s>>>(P);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "decode_i8_cyclic launch");
    return 0;
}

}  // namespace fwbf

namespace fwbf {

// Scheduled and learned decoding: the cyclic kernel with the handle's frame
// counter for the stream.
int launch_decode_i8_modes(const fwbf_code_s *c, const int8_t *y, int64_t n_frames, int max_iter, int alpha_q,
                           uint32_t *out_bits, int32_t *out_iters, const CyclicModes &modes, cudaStream_t s) {
    if (!cyclic_eligible(c)) return fail(FWBF_EUNSUPPORTED, "per-pass schedules need a cyclic code");
    CounterLease ctr;
    int rc = acquire_counter(c, s, &ctr);
    if (rc) return rc;
    rc = launch_decode_i8_cyclic(c, y, n_frames, max_iter, alpha_q, 0, out_bits, out_iters, ctr.ptr, s, &modes);
    const int rc2 = release_counter(ctr, s);
    return rc ? rc : rc2;
}

}  // namespace fwbf
