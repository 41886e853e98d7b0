// Batched FWBF decoding: one persistent launch over several codes, each with
// its own frames and outputs (codes of different N, M and row / column
// weight in the same launch).
//
// The batch handle holds the table of jobs (one per code; passed whole as the
// launch's parameter block) and one device frame counter per job.  Every CTA
// walks the jobs, starting at job blockIdx.x mod n_jobs so that CTAs spread
// over the codes: for each job with frames left it stages that code's index
// tables with a bulk copy (TMA) on a fresh mbarrier, lays its warps' shared-
// memory slices out for that code and lets each warp (or warp group) pull
// frames from the job's counter until the job is exhausted; then the CTA moves on.
// Per frame a warp (or warp group) runs the packed cyclic decoder (cyclic
// codes), the packed quasi-cyclic decoder (codes of circulant blocks, groups
// of 4 or 8 warps, Z a multiple of 256) or the generic list decoder (every
// other code) -- the same device code as the single-code kernels, so results
// are identical to fwbf_decode.
//
// A decode call is a memset of the counters plus one launch on the caller's
// stream; it allocates nothing, so it can be captured in a CUDA graph.
#include <math.h>

#include <vector>

#include "generic_frame.cuh"
#include "qc_frame.cuh"

namespace fwbf {

__device__ int g_status_batch;

enum JobKind : int { kJobGenericPlain = 0, kJobGenericCirc = 1, kJobCyclic4 = 2, kJobCyclic8 = 3, kJobCyclic2 = 4,
                     kJobCyclic1 = 5, kJobCyclic4W2 = 6, kJobCyclic8W4 = 7, kJobCyclic4W4 = 8,
                     kJobQc8 = 9, kJobQc4 = 10 };  // QC: R pairs per lane per chunk

__host__ __device__ inline bool job_is_cyclic(int kind) { return kind >= kJobCyclic4 && kind <= kJobCyclic4W4; }
__host__ __device__ inline bool job_is_qc(int kind) { return kind >= kJobQc8; }

struct BatchJob {
    int kind;
    int warps;  // warps of a CTA that decode this job (shared memory permitting)
    int wpf;    // warps per frame (codes whose frames fill the CTA's shared memory before its warps)
    uint32_t table_smem_bytes;
    uint32_t warp_bytes;
    unsigned long long *counter;
    long long F;
    I8Params gp;
    CyclicParams cp;
    QcParams qp;
};

constexpr int kMaxJobs = 16;

// The whole job table travels as the launch's parameter block (constant
// space, 16 jobs of under 600 bytes): the frame code reads its job's fields
// without touching shared memory, which the decoders keep busy.
struct BatchParams {
    BatchJob jobs[kMaxJobs];
    int n_jobs;
};
static_assert(sizeof(BatchParams) <= 32764, "kernel parameter block limit");

// The CTA's frames of a cyclic job decoded by groups of WPF warps, R pairs
// per lane per chunk (group g meets at named barrier 1 + g; the CTA-wide
// barrier 0 is not used meanwhile).  BODIES: the decoder bodies compiled in
// (1: plain only, 2: learned only, 3: both, chosen per job).
template <int R, int WPF, int BODIES = 3>
__device__ __forceinline__ void batch_cyclic_groups(const BatchJob &J, const uint32_t *d_off, const uint32_t *u_off,
                                                    unsigned char *smem, unsigned long long *fslot) {
    constexpr int G = 32 * WPF;
    const int t = threadIdx.x % G, grp = threadIdx.x / G, bar_id = 1 + grp;
    unsigned char *ws = smem + J.table_smem_bytes + grp * J.warp_bytes;
    uint32_t *keys = reinterpret_cast<uint32_t *>(ws + J.cp.off_keys);
    for (uint32_t b = t; b < J.cp.key_words; b += G) keys[b] = 0u;
    for (;;) {
        if (t == 0) fslot[grp] = atomicAdd(J.counter, 1ull);
        group_sync<WPF>(bar_id);
        const unsigned long long f = fslot[grp];
        if (f >= (unsigned long long)J.F) break;
        if (BODIES == 1 || (BODIES == 3 && J.cp.mode == kModePlain))
            cyclic_frame<R, WPF, kVarPlain>(J.cp, d_off, u_off, ws, t, bar_id, f);
        else
            cyclic_frame<R, WPF, kVarLearned>(J.cp, d_off, u_off, ws, t, bar_id, f);
    }
}

// The same for a job of the list decoder (tbl: the code's staged tables).
template <bool PLAIN, int WPF>
__device__ __forceinline__ void batch_generic_groups(const BatchJob &J, const uint32_t *tbl, unsigned char *smem,
                                                     unsigned long long *fslot) {
    constexpr int G = 32 * WPF;
    const int t = threadIdx.x % G, grp = threadIdx.x / G, bar_id = 1 + grp;
    unsigned char *ws = smem + J.table_smem_bytes + grp * J.warp_bytes;
    unsigned long long *keys = reinterpret_cast<unsigned long long *>(ws + J.gp.off_keys);
    for (int b = t; b < J.gp.nkeys; b += G) keys[b] = 0ull;
    for (;;) {
        if (t == 0) fslot[grp] = atomicAdd(J.counter, 1ull);
        group_sync<WPF>(bar_id);
        const unsigned long long f = fslot[grp];
        if (f >= (unsigned long long)J.F) break;
        generic_frame<PLAIN, WPF>(J.gp, tbl, ws, t, bar_id, f);
    }
}

// The same for a quasi-cyclic job (plain FWBF only).
template <int R, int WPF>
__device__ __forceinline__ void batch_qc_groups(const BatchJob &J, const uint32_t *tbl, unsigned char *smem,
                                                unsigned long long *fslot) {
    constexpr int G = 32 * WPF;
    const int t = threadIdx.x % G, grp = threadIdx.x / G, bar_id = 1 + grp;
    unsigned char *ws = smem + J.table_smem_bytes + grp * J.warp_bytes;
    unsigned long long *keys = reinterpret_cast<unsigned long long *>(ws + J.qp.off_keys);
    for (int b = t; b < J.qp.B; b += G) keys[b] = 0ull;
    qc_group_init<WPF>(J.qp, ws, t);
    uint32_t lpar = 0;  // phase of the group's frame-load mbarrier
    for (;;) {
        if (t == 0) fslot[grp] = atomicAdd(J.counter, 1ull);
        group_sync<WPF>(bar_id);
        const unsigned long long f = fslot[grp];
        if (f >= (unsigned long long)J.F) break;
        if (!qc_frame<R, WPF>(J.qp, tbl, ws, t, bar_id, f, lpar)) {
            if (t == 0) atomicOr(&g_status_batch, 2);
            return;  // (the frame's copy did not arrive: the group leaves)
        }
    }
    qc_group_done(J.qp, ws, t);
}

template <int WPF>
__device__ __forceinline__ void batch_qc_dispatch(const BatchJob &J, const uint32_t *tbl, unsigned char *smem,
                                                  unsigned long long *fslot) {
    if (J.kind == kJobQc8)
        batch_qc_groups<8, WPF>(J, tbl, smem, fslot);
    else
        batch_qc_groups<4, WPF>(J, tbl, smem, fslot);
}

// One frame of a cyclic job by one warp (plain jobs run the plain-only body,
// learned jobs the learned body: batch jobs record nothing).
template <int R>
__device__ __forceinline__ void cyclic_frame_job(const BatchJob &J, const uint32_t *d_off, const uint32_t *u_off,
                                                 unsigned char *ws, int lane, unsigned long long f) {
    if (J.cp.mode == kModePlain)
        cyclic_frame<R, 1, kVarPlain>(J.cp, d_off, u_off, ws, lane, 0, f);
    else
        cyclic_frame<R, 1, kVarLearned>(J.cp, d_off, u_off, ws, lane, 0, f);
}

template <bool PLAIN>
__device__ __forceinline__ void batch_generic_dispatch(const BatchJob &J, const uint32_t *tbl, unsigned char *smem,
                                                       unsigned long long *fslot) {
    if (J.wpf == 2)
        batch_generic_groups<PLAIN, 2>(J, tbl, smem, fslot);
    else if (J.wpf == 4)
        batch_generic_groups<PLAIN, 4>(J, tbl, smem, fslot);
    else
        batch_generic_groups<PLAIN, 8>(J, tbl, smem, fslot);
}

// GROUPED: every job runs warp groups (two blocks of 512 threads per SM, 64
// registers); otherwise any mix of one-warp and group jobs (one block per SM).
// CYCLIC_ONLY (grouped launches whose jobs are all cyclic codes): only the
// cyclic decoder bodies are compiled in, a smaller kernel for the instruction
// cache and the register allocator; BODIES of them (1: plain, 2: learned, 3:
// both).  ONE_JOB (a cyclic-only launch of one job): the job's fields sit at
// fixed offsets of the parameter block, operands of the instructions that use
// them instead of loads through a job index (plain jobs 1.4 %, learned jobs
// 1.1 % faster on EG(1023) together with BODIES).
template <bool GROUPED, bool CYCLIC_ONLY = false, bool ONE_JOB = false, int BODIES = 3>
__global__ void __launch_bounds__(512, GROUPED ? 2 : 1) fwbf_decode_batch_kernel(const __grid_constant__ BatchParams bp) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ uint64_t bars[kMaxJobs];
    __shared__ int flag;
    __shared__ __align__(16) uint32_t d_off[128], u_off[128];  // read as 8- and 16-byte vectors
    __shared__ int live;
    __shared__ unsigned long long fslot[16];

    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int n_jobs = ONE_JOB ? 1 : bp.n_jobs;
    for (int t = 0; t < n_jobs; ++t) {
        const int j = ONE_JOB ? 0 : (blockIdx.x + t) % n_jobs;
        const BatchJob &J = bp.jobs[j];
        if (threadIdx.x == 0) live = atomicAdd(J.counter, 0ull) < (unsigned long long)J.F;
        __syncthreads();
        if (!live) {
            __syncthreads();
            continue;
        }
        const bool qc = job_is_qc(J.kind), cyc = job_is_cyclic(J.kind);
        const uint32_t words = qc ? J.qp.table_words : cyc ? J.cp.table_words : J.gp.table_words;
        const uint32_t *gtab = qc ? J.qp.table : cyc ? J.cp.table : J.gp.table;
        uint32_t *st = reinterpret_cast<uint32_t *>(smem);
        if (!stage_table(st, gtab, words, &bars[t], &flag)) {
            if (threadIdx.x == 0) atomicOr(&g_status_batch, 1);
            return;
        }
        if (cyc) {
            for (int e = threadIdx.x; e < 128; e += blockDim.x) {  // zeros past d_c
                d_off[e] = e < J.cp.DC ? st[J.cp.rent_off + e] & 0xffffu : 0u;
                u_off[e] = e < J.cp.DC ? st[J.cp.cent_off + e] & 0xffffu : 0u;
            }
        }
        __syncthreads();
        if (warp < J.warps && J.wpf > 1) {
            if (J.kind == kJobCyclic4W2) {
                batch_cyclic_groups<4, 2, BODIES>(J, d_off, u_off, smem, fslot);
            } else if (J.kind == kJobCyclic8W4 || J.kind == kJobCyclic4W4) {
                if constexpr (GROUPED)
                    batch_cyclic_groups<4, 4, BODIES>(J, d_off, u_off, smem, fslot);
                else
                    batch_cyclic_groups<8, 4, BODIES>(J, d_off, u_off, smem, fslot);
            } else if constexpr (CYCLIC_ONLY) {
                // (no other job kind in this launch)
            } else if (qc) {
                if (J.wpf == 16) {
                    if constexpr (GROUPED) batch_qc_dispatch<16>(J, st, smem, fslot);
                } else if (J.wpf == 8) {
                    batch_qc_dispatch<8>(J, st, smem, fslot);
                } else {
                    batch_qc_dispatch<4>(J, st, smem, fslot);
                }
            } else if (J.kind == kJobGenericPlain) {
                batch_generic_dispatch<true>(J, st, smem, fslot);
            } else {
                batch_generic_dispatch<false>(J, st, smem, fslot);
            }
        } else if (!GROUPED && warp < J.warps) {
            unsigned char *ws = smem + J.table_smem_bytes + warp * J.warp_bytes;
            // key array in uint32 words: 64-bit keys in the list decoder, 32- or
            // 64-bit keys in the cyclic decoder
            const uint32_t kw = J.kind <= kJobGenericCirc ? 2u * (uint32_t)J.gp.nkeys : J.cp.key_words;
            const uint32_t off_keys = J.kind <= kJobGenericCirc ? J.gp.off_keys : J.cp.off_keys;
            uint32_t *keys = reinterpret_cast<uint32_t *>(ws + off_keys);
            for (uint32_t b = lane; b < kw; b += 32) keys[b] = 0u;
            __syncwarp();
            for (;;) {
                unsigned long long f = 0;
                if (lane == 0) f = atomicAdd(J.counter, 1ull);
                f = __shfl_sync(FULL, f, 0);
                if (f >= (unsigned long long)J.F) break;
                switch (J.kind) {
                    case kJobGenericPlain: generic_frame<true, 1>(J.gp, st, ws, lane, 0, f); break;
                    case kJobGenericCirc: generic_frame<false, 1>(J.gp, st, ws, lane, 0, f); break;
                    case kJobCyclic8: cyclic_frame_job<8>(J, d_off, u_off, ws, lane, f); break;
                    case kJobCyclic4: cyclic_frame_job<4>(J, d_off, u_off, ws, lane, f); break;
                    case kJobCyclic2: cyclic_frame_job<2>(J, d_off, u_off, ws, lane, f); break;
                    default: cyclic_frame_job<1>(J, d_off, u_off, ws, lane, f); break;
                }
            }
        }
        __syncthreads();
    }
}

}  // namespace fwbf

using namespace fwbf;

struct fwbf_batch_s {
    int n_jobs = 0;
    bool grouped = false;
    bool cyclic_only = false;  // grouped launch of cyclic jobs only
    void (*kern)(const BatchParams) = nullptr;  // the kernel instance for these jobs
    BatchParams params{};
    unsigned long long *d_counters = nullptr;
    int blocks = 0, threads = 0;
    uint32_t dyn = 0;
    int device = 0;
};

extern "C" {

int fwbf_batch_create(const fwbf_batch_job *jobs, int32_t n_jobs, int32_t warps_per_cta, int32_t packed,
                      fwbf_batch *out) {
    TraceRange trace("fwbf_batch_create");
    if (!out) return fail(FWBF_EINVAL, "out is NULL");
    *out = nullptr;
    if (!jobs || n_jobs < 1 || n_jobs > kMaxJobs) return fail(FWBF_EINVAL, "n_jobs must be in [1, 16]");
    if (warps_per_cta < 1 || warps_per_cta > 16) return fail(FWBF_EINVAL, "warps_per_cta must be in [1, 16]");
    if (packed < 0 || packed > 2) return fail(FWBF_EINVAL, "packed must be 0, 1 or 2");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    std::vector<BatchJob> hj((size_t)n_jobs);
    int optin = 0, sms = 0;
    e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return cuda_fail(e, "device query");
    const uint32_t reserve = 4096u;  // static shared memory of the kernel
    uint32_t dyn = 0;
    for (int j = 0; j < n_jobs; ++j) {
        const fwbf_batch_job &in = jobs[j];
        const fwbf_code_s *c = in.code;
        if (!c) return fail(FWBF_EINVAL, "job code is NULL");
        if (c->device != dev) return fail(FWBF_EINVAL, "job code was created on another device");
        if (in.n_frames < 0 || in.max_iter < 1 || !(in.alpha >= 0.0f && in.alpha <= 64.0f))
            return fail(FWBF_EINVAL, "bad job frames / max_iter / alpha");
        if (in.n_frames > 0 && (!in.y || !in.out_bits || !in.out_iters)) return fail(FWBF_EINVAL, "NULL job buffer");
        if (reinterpret_cast<uintptr_t>(in.y) % 16) return fail(FWBF_EINVAL, "job y must be 16-byte aligned");
        if (in.mlp && (!packed || !cyclic_eligible(c)))
            return fail(FWBF_EUNSUPPORTED, "a learned job needs a cyclic code and the packed decoder");
        if (in.mlp && (in.k_learn < 1 || in.gate_dv < 0 || in.gate_dv > 65535 ||
                       reinterpret_cast<uintptr_t>(in.mlp) % 16))
            return fail(FWBF_EINVAL, "learned job: k_learn < 1, gate_dv outside [0, 65535] or unaligned network blob");
        BatchJob &b = hj[j];
        b = BatchJob{};
        const int aq = (int)nearbyint((double)in.alpha * 256.0);
        // quasi-cyclic codes with Z a multiple of 256 (R = 8 or 4 pairs per lane
        // per chunk): the packed QC decoder (groups of 4 or 8 warps) when a
        // group fits, else (and for other Z) the list decoder
        bool qc_ok = packed && !cyclic_eligible(c) && !in.mlp && warps_per_cta >= 4 && qc_eligible(c);
        if (qc_ok) {
            qc_layout(c, b.qp);
            qc_ok = qc_R(b.qp) >= 4 && b.qp.table_smem_bytes + b.qp.warp_bytes + reserve <= (uint32_t)optin;
        }
        if (packed && cyclic_eligible(c)) {
            if (in.mlp) {  // (before the layout: a learned frame's slice holds the network's layer 1)
                b.cp.mode = kModeLearned;
                b.cp.mlp = static_cast<const unsigned char *>(in.mlp);
                b.cp.k_learn = in.k_learn;
                b.cp.gate_dv = in.gate_dv;
            }
            cyclic_layout(c, b.cp);
            const int R = cyclic_R(c);
            b.kind = R == 8 ? kJobCyclic8 : R == 4 ? kJobCyclic4 : R == 2 ? kJobCyclic2 : kJobCyclic1;
            b.cp.y = in.y;
            b.cp.F = in.n_frames;
            b.cp.max_iter = in.max_iter;
            b.cp.alpha_q = aq;
            b.cp.out_bits = in.out_bits;
            b.cp.out_iters = in.out_iters;
            b.table_smem_bytes = b.cp.table_smem_bytes;
            b.warp_bytes = b.cp.warp_bytes;
        } else if (qc_ok) {
            b.kind = qc_R(b.qp) == 8 ? kJobQc8 : kJobQc4;
            b.qp.y = in.y;
            b.qp.F = in.n_frames;
            b.qp.max_iter = in.max_iter;
            b.qp.alpha_q = aq;
            b.qp.theta_q = 0;
            b.qp.out_bits = in.out_bits;
            b.qp.out_iters = in.out_iters;
            b.table_smem_bytes = b.qp.table_smem_bytes;
            b.warp_bytes = b.qp.warp_bytes;
        } else {
            generic_layout(c, b.gp);
            b.kind = c->Z == 1 ? kJobGenericPlain : kJobGenericCirc;
            b.gp.y = in.y;
            b.gp.F = in.n_frames;
            b.gp.max_iter = in.max_iter;
            b.gp.alpha_q = aq;
            b.gp.out_bits = in.out_bits;
            b.gp.out_iters = in.out_iters;
            b.table_smem_bytes = (c->table_words * 4u + 15u) & ~15u;
            b.gp.table_in_smem = 1;
            b.gp.table_smem_bytes = b.table_smem_bytes;
            b.warp_bytes = b.gp.warp_bytes;
        }
        b.F = in.n_frames;
        if (b.table_smem_bytes + b.warp_bytes + reserve > (uint32_t)optin)
            return fail(FWBF_EUNSUPPORTED, "a job's code does not fit one warp's shared memory");
        int frames = (int)(((uint32_t)optin - reserve - b.table_smem_bytes) / b.warp_bytes);
        if (frames > warps_per_cta) frames = warps_per_cta;
        // codes whose frames fill the shared memory before the warps run out:
        // 4 warps per frame (packed decoder, R = 8) or 2 (R = 4) when H / 32
        // gives every warp a chunk; 2, 4 or 8 (list decoder)
        b.wpf = 1;
        if (job_is_qc(b.kind) && frames > warps_per_cta / 4) frames = warps_per_cta / 4;
        const int spare = warps_per_cta / frames;
        if (job_is_qc(b.kind)) {
            b.wpf = spare >= 8 ? 8 : 4;
        } else if (job_is_cyclic(b.kind)) {
            const int ppl = b.cp.H / 32;
            b.wpf = spare >= 4 && ppl % 8 == 0 && ppl / 8 >= 4 ? 4 : spare >= 2 && ppl % 4 == 0 && ppl / 4 >= 2 ? 2 : 1;
            if (b.wpf > 1) b.kind = b.wpf == 4 ? kJobCyclic8W4 : kJobCyclic4W2;
            cyclic_set_wpf(b.cp, b.wpf);  // (frames were counted with the largest scratch)
            b.warp_bytes = b.cp.warp_bytes;
        } else if (b.kind <= kJobGenericCirc) {
            b.wpf = spare >= 8 ? 8 : spare >= 4 ? 4 : spare >= 2 ? 2 : 1;
        }
        b.warps = frames * b.wpf;
        const uint32_t need = b.table_smem_bytes + frames * b.warp_bytes;
        if (need > dyn) dyn = need;
    }
    // packed = 2: the grouped kernel (two 512-thread blocks per SM) when every
    // job can run warp groups in half an SM's shared memory: up to 8 frames per
    // block, two warps per frame (four when at most 4 frames fit, R = 4) for
    // the packed cyclic decoder, 4, 8 or 16 (up to 4 frames; 16 when one fits)
    // for the packed QC decoder, 2, 4 or 8 for the list decoder
    bool grouped = false;
    if (packed == 2) {
        int smem_sm = 0;
        cudaFuncAttributes fa{};
        e = cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
        if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, fwbf_decode_batch_kernel<true>);
        if (e != cudaSuccess) return cuda_fail(e, "grouped batch query");
        const int64_t half = (int64_t)smem_sm / 2 - 1024 - (int64_t)fa.sharedSizeBytes;
        std::vector<BatchJob> gj = hj;
        uint32_t gdyn = 0;
        grouped = true;
        for (int j = 0; j < n_jobs && grouped; ++j) {
            BatchJob &b = gj[j];
            const int64_t avail = half - (int64_t)b.table_smem_bytes;
            int frames = avail > 0 ? (int)(avail / b.warp_bytes) : 0;
            if (frames > 8) frames = 8;
            if (frames < 1) {
                grouped = false;
                break;
            }
            if (b.kind <= kJobGenericCirc) {
                int w = 2;
                while (w < 8 && frames * w * 2 <= 16) w *= 2;
                b.wpf = w;
            } else if (job_is_qc(b.kind)) {
                if (frames > 4) frames = 4;
                b.wpf = frames <= 2 ? 8 : 4;
                if (frames == 1) {  // the whole block on the one frame that fits
                    QcParams q16 = b.qp;
                    qc_set_wpf(q16, 16);
                    if ((int64_t)q16.warp_bytes <= avail) {
                        b.qp = q16;
                        b.warp_bytes = q16.warp_bytes;
                        b.wpf = 16;
                    }
                }
            } else {
                const int ppl = b.cp.H / 32;
                if (ppl % 4 != 0 || ppl / 4 < 2) {
                    grouped = false;
                    break;
                }
                if (frames <= 4 && ppl / 4 >= 4) {
                    b.wpf = 4;
                    b.kind = kJobCyclic4W4;
                } else {
                    b.wpf = 2;
                    b.kind = kJobCyclic4W2;
                }
                cyclic_set_wpf(b.cp, b.wpf);  // the slice shrinks to the group's scratch
                b.warp_bytes = b.cp.warp_bytes;
                frames = (int)(avail / b.warp_bytes);
                if (frames > (b.wpf == 4 ? 4 : 8)) frames = b.wpf == 4 ? 4 : 8;
            }
            b.warps = frames * b.wpf;
            const uint32_t need = b.table_smem_bytes + frames * b.warp_bytes;
            if (need > gdyn) gdyn = need;
        }
        if (grouped) {
            hj = gj;
            dyn = gdyn;
        }
    }
    fwbf_batch_s *bh = new (std::nothrow) fwbf_batch_s();
    if (!bh) return fail(FWBF_ENOMEM, "host allocation");
    bh->n_jobs = n_jobs;
    bh->device = dev;
    bh->grouped = grouped;
    bh->threads = grouped ? 512 : 32 * warps_per_cta;
    bh->dyn = dyn;
    e = cudaMalloc(reinterpret_cast<void **>(&bh->d_counters), sizeof(unsigned long long) * n_jobs);
    if (e != cudaSuccess) {
        cudaFree(bh->d_counters);
        delete bh;
        return e == cudaErrorMemoryAllocation ? fail(FWBF_ENOMEM, "cudaMalloc(batch)") : cuda_fail(e, "cudaMalloc");
    }
    for (int j = 0; j < n_jobs; ++j) {
        hj[j].counter = bh->d_counters + j;
        hj[j].gp.counter = hj[j].counter;
        hj[j].cp.counter = hj[j].counter;
        hj[j].qp.counter = hj[j].counter;
        bh->params.jobs[j] = hj[j];
    }
    bh->params.n_jobs = n_jobs;
    bool cyclic_only = grouped;
    int bodies = 0;  // cyclic bodies the jobs need: 1 plain, 2 learned
    for (int j = 0; j < n_jobs; ++j) {
        cyclic_only = cyclic_only && job_is_cyclic(hj[j].kind);
        bodies |= hj[j].cp.mode == kModePlain ? 1 : 2;
    }
    bh->cyclic_only = cyclic_only;
    void (*kern)(const BatchParams) =
        cyclic_only && n_jobs == 1 ? (bodies == 1 ? fwbf_decode_batch_kernel<true, true, true, 1>
                                                  : fwbf_decode_batch_kernel<true, true, true, 2>)
        : cyclic_only ? fwbf_decode_batch_kernel<true, true>
        : grouped     ? fwbf_decode_batch_kernel<true, false>
                      : fwbf_decode_batch_kernel<false, false>;
    bh->kern = kern;
    if (e == cudaSuccess) e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
    int per_sm = 0;
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, bh->threads, dyn);
    if (e != cudaSuccess || per_sm < 1) {
        cudaFree(bh->d_counters);
        delete bh;
        return e != cudaSuccess ? cuda_fail(e, "batch set-up") : fail(FWBF_EUNSUPPORTED, "batch kernel does not fit");
    }
    bh->blocks = per_sm * sms;
    *out = bh;
    return FWBF_OK;
}

int fwbf_decode_batch(fwbf_batch b, void *stream) {
    TraceRange trace("fwbf_decode_batch");
    if (!b) return fail(FWBF_EINVAL, "batch is NULL");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemsetAsync(b->d_counters, 0, sizeof(unsigned long long) * b->n_jobs, s);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync(batch counters)");
    b->kern<<<b->blocks, b->threads, b->dyn, s>>>(b->params);
    e = cudaGetLastError();
    return e == cudaSuccess ? FWBF_OK : cuda_fail(e, "decode_batch launch");
}

int fwbf_batch_query(fwbf_batch b, int32_t job, fwbf_batch_job_info *out) {
    if (!b || !out) return fail(FWBF_EINVAL, "batch or out is NULL");
    if (job < 0 || job >= b->n_jobs) return fail(FWBF_EINVAL, "job index out of range");
    const BatchJob &J = b->params.jobs[job];
    out->decoder = job_is_qc(J.kind) ? FWBF_DECODER_QC : job_is_cyclic(J.kind) ? FWBF_DECODER_CYCLIC
                                                                             : FWBF_DECODER_LIST;
    out->warps_per_frame = J.wpf;
    out->frames_per_cta = J.wpf > 0 ? J.warps / J.wpf : 0;
    out->grouped = b->grouped ? 1 : 0;
    return FWBF_OK;
}

int fwbf_batch_destroy(fwbf_batch b) {
    if (!b) return FWBF_OK;
    cudaError_t e = cudaDeviceSynchronize();
    cudaFree(b->d_counters);
    delete b;
    return e == cudaSuccess ? FWBF_OK : cuda_fail(e, "cudaDeviceSynchronize");
}

int fwbf_batch_status(void *stream) {
    int v = 0, zero = 0;
    cudaError_t e = cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
    if (e == cudaSuccess) e = cudaMemcpyFromSymbol(&v, g_status_batch, sizeof(int));
    if (e == cudaSuccess && v) e = cudaMemcpyToSymbol(g_status_batch, &zero, sizeof(int));
    if (e != cudaSuccess) return cuda_fail(e, "batch status");
    return v ? fail(FWBF_ETIMEOUT, "the batch kernel gave up waiting for a table copy") : FWBF_OK;
}

}  // extern "C"
