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

#include "generic_frame.cuh"

namespace fwbf {

__device__ int g_status_i8;

template <bool PLAIN, int WPF>  // PLAIN: Z == 1, the tables are plain CSR / CSC; warps per frame
__global__ void __launch_bounds__(768, 1) fwbf_decode_i8_kernel(const I8Params P) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ uint64_t bar;
    __shared__ int flag;
    __shared__ unsigned long long fslot[24];

    const uint32_t *tbl = P.table;
    if (P.table_in_smem) {
        uint32_t *st = reinterpret_cast<uint32_t *>(smem);
        if (!stage_table(st, P.table, P.table_words, &bar, &flag)) {
            if (threadIdx.x == 0) atomicOr(&g_status_i8, 1);
            return;
        }
        tbl = st;
    }
    // groups of WPF warps, one frame each; group g meets at named barrier 1 + g
    constexpr int G = 32 * WPF;
    const int t = threadIdx.x % G;
    const int grp = threadIdx.x / G;
    const int bar_id = 1 + grp;
    unsigned char *ws = smem + P.table_smem_bytes + grp * P.warp_bytes;
    unsigned long long *keys = reinterpret_cast<unsigned long long *>(ws + P.off_keys);
    for (int b = t; b < P.nkeys; b += G) keys[b] = 0ull;
    if (P.lambda && t == 0) *reinterpret_cast<uint32_t *>(ws + P.off_cand + 8u * (uint32_t)P.N) = 0u;
    for (;;) {
        if (t == 0) fslot[grp] = atomicAdd(P.counter, 1ull);
        group_sync<WPF>(bar_id);
        const unsigned long long f = fslot[grp];  // rewritten only after the frame's last meeting
        if (f >= (unsigned long long)P.F) break;
        generic_frame<PLAIN, WPF>(P, tbl, ws, t, bar_id, f);
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

// Generic (any H) int8 decoder launch with a caller-provided frame counter
// that is already zero on the stream.
static int launch_generic_i8(const fwbf_code_s *c, const int8_t *y, int64_t n_frames, int max_iter, int alpha_q,
                             int theta_q, uint32_t *out_bits, int32_t *out_iters, unsigned long long *counter,
                             cudaStream_t s, int lambda = 0) {
    I8Params P{};
    generic_layout(c, P);
    if (lambda > 0) generic_layout_lambda(c, P, lambda);
    P.y = y;
    P.F = n_frames;
    P.max_iter = max_iter;
    P.alpha_q = alpha_q;
    P.theta_q = theta_q;
    P.out_bits = out_bits;
    P.out_iters = out_iters;
    P.counter = counter;

    const uint32_t tbytes = c->table_words * 4u;
    const uint32_t optin = (uint32_t)c->smem_optin;
    const uint32_t margin = 512u;  // static shared memory of the kernel
    P.table_in_smem = (tbytes + P.warp_bytes + margin <= optin && tbytes <= 96u * 1024u) ? 1 : 0;
    P.table_smem_bytes = P.table_in_smem ? tbytes : 0;
    const uint32_t avail = optin - margin - P.table_smem_bytes;
    if (P.warp_bytes > avail) return fail(FWBF_EUNSUPPORTED, "code too large for one block's shared memory");
    int frames = (int)(avail / P.warp_bytes);
    if (frames > 24) frames = 24;
    // up to 24 warps per block: codes with fewer frames per block than that
    // get 2, 4 or 8 warps per frame (lambda-largest selection keeps one)
    int wpf = 1;
    while (lambda == 0 && wpf < 8 && frames * wpf * 2 <= 24) wpf *= 2;
    const uint32_t dyn = P.table_smem_bytes + frames * P.warp_bytes;

    void (*kern)(const I8Params);
    if (c->Z == 1)
        kern = wpf == 1 ? fwbf_decode_i8_kernel<true, 1> : wpf == 2 ? fwbf_decode_i8_kernel<true, 2>
             : wpf == 4 ? fwbf_decode_i8_kernel<true, 4> : fwbf_decode_i8_kernel<true, 8>;
    else
        kern = wpf == 1 ? fwbf_decode_i8_kernel<false, 1> : wpf == 2 ? fwbf_decode_i8_kernel<false, 2>
             : wpf == 4 ? fwbf_decode_i8_kernel<false, 4> : fwbf_decode_i8_kernel<false, 8>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute");
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, frames * wpf * 32, dyn);
    if (e != cudaSuccess) return cuda_fail(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
    if (per_sm < 1) return fail(FWBF_EUNSUPPORTED, "decode kernel does not fit on an SM");
    int64_t blocks = (int64_t)per_sm * c->num_sms;
    const int64_t need = (n_frames + frames - 1) / frames;
    if (blocks > need) blocks = need;
    kern<<<(unsigned)blocks, frames * wpf * 32, dyn, s>>>(P);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "decode_i8 launch");
    return 0;
}

// Picks the decoder for the code: the packed cyclic kernel when H is a single
// circulant it handles, the packed quasi-cyclic kernel when H is made of
// circulant blocks it handles, the generic (list) kernel otherwise.
static int launch_i8_with_counter(const fwbf_code_s *c, const int8_t *y, int64_t n_frames, int max_iter,
                                  int alpha_q, int theta_q, uint32_t *out_bits, int32_t *out_iters,
                                  unsigned long long *counter, cudaStream_t s) {
    if (cyclic_eligible(c))
        return launch_decode_i8_cyclic(c, y, n_frames, max_iter, alpha_q, theta_q, out_bits, out_iters, counter, s);
    if (qc_eligible(c))
        return launch_decode_i8_qc(c, y, n_frames, max_iter, alpha_q, theta_q, out_bits, out_iters, counter, s);
    return launch_generic_i8(c, y, n_frames, max_iter, alpha_q, theta_q, out_bits, out_iters, counter, s);
}

int launch_decode_i8_with(const fwbf_code_s *c, const int8_t *y, int64_t n_frames, int max_iter, int alpha_q,
                          int theta_q, uint32_t *out_bits, int32_t *out_iters, unsigned long long *counter,
                          cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync(frame counter)");
    return launch_i8_with_counter(c, y, n_frames, max_iter, alpha_q, theta_q, out_bits, out_iters, counter, s);
}

int launch_decode_i8(const fwbf_code_s *c, const int8_t *y, int64_t n_frames, int max_iter, int alpha_q,
                     int theta_q, uint32_t *out_bits, int32_t *out_iters, cudaStream_t s) {
    CounterLease ctr;
    int rc = acquire_counter(c, s, &ctr);
    if (rc) return rc;
    rc = launch_i8_with_counter(c, y, n_frames, max_iter, alpha_q, theta_q, out_bits, out_iters, ctr.ptr, s);
    const int rc2 = release_counter(ctr, s);
    return rc ? rc : rc2;
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

namespace fwbf {

// lambda-largest selection: the list decoder with a per-frame candidate list
int launch_decode_i8_lambda(const fwbf_code_s *c, const int8_t *y, int64_t n_frames, int max_iter, int alpha_q,
                            int lambda, uint32_t *out_bits, int32_t *out_iters, cudaStream_t s) {
    CounterLease ctr;
    int rc = acquire_counter(c, s, &ctr);
    if (rc) return rc;
    rc = launch_generic_i8(c, y, n_frames, max_iter, alpha_q, 0, out_bits, out_iters, ctr.ptr, s, lambda);
    const int rc2 = release_counter(ctr, s);
    return rc ? rc : rc2;
}

}  // namespace fwbf
