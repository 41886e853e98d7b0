// Integer issue-rate microbenchmark (include/fwbf_peak.h).  Every thread runs
// eight chains of dependent 32-bit integer instructions; the chains are
// coupled (each step reads its neighbour) and non-linear, so the compiler can
// neither fold a chain into a closed form nor merge consecutive steps.  With
// 64 warps per SM the dependency latency is hidden and the launch measures
// issue throughput.
#include <cuda_runtime.h>

#include "device_common.cuh"
#include "fwbf.h"
#include "fwbf_internal.h"
#include "fwbf_peak.h"

namespace fwbf {
namespace {

constexpr int kChains = 8;
constexpr int kRounds = 8;  // unrolled rounds per loop iteration
constexpr int kThreads = 256;
constexpr int kBlocksPerSm = 8;

template <int MIX>
__global__ void __launch_bounds__(kThreads, kBlocksPerSm)
    int_issue_kernel(uint32_t *sink, uint32_t seed, int iters) {
    uint32_t v[kChains];
#pragma unroll
    for (int i = 0; i < kChains; ++i) v[i] = seed * (threadIdx.x + 1u) + 0x9e3779b9u * (i + 1u) + blockIdx.x;
    const uint32_t c = seed ^ 0x5bd1e995u;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int r = 0; r < kRounds; ++r) {
#pragma unroll
            for (int i = 0; i < kChains; ++i) {
                if (MIX == 0 || (i & 1) == 0)  // v_i ^= v_{i+1} & c
                    asm volatile("lop3.b32 %0, %0, %1, %2, 0x78;" : "+r"(v[i]) : "r"(v[(i + 1) % kChains]), "r"(c));
                else  // v_i = v_i * v_i + v_{i+1}
                    asm volatile("mad.lo.u32 %0, %0, %0, %1;" : "+r"(v[i]) : "r"(v[(i + 1) % kChains]));
            }
        }
    }
    uint32_t acc = 0;
#pragma unroll
    for (int i = 0; i < kChains; ++i) acc ^= v[i];
    if (acc == 0x2545f491u) sink[0] = acc;  // keeps every chain live
}

// The table-staging wait of the decoders on a barrier expecting bytes that no
// copy delivers (expect_bytes > 0): the bounded wait gives up and the status
// records the timeout.
__global__ void bounded_wait_probe_kernel(int *status, uint32_t expect_bytes) {
    __shared__ uint64_t bar;
    __shared__ int flag;
    if (threadIdx.x == 0) {
        flag = 0;
        mbar_init(&bar, 1);
    }
    __syncthreads();
    if (threadIdx.x == 0) mbar_expect_tx(&bar, expect_bytes);
    if (!mbar_wait_bounded(&bar, 0, kWaitLimitNs)) atomicOr(&flag, 1);
    __syncthreads();
    if (threadIdx.x == 0) *status = flag ? FWBF_ETIMEOUT : FWBF_OK;
}

}  // namespace
}  // namespace fwbf

using namespace fwbf;

extern "C" int fwbf_probe_bounded_wait(uint32_t expect_bytes, void *stream, int *out_status) {
    if (expect_bytes > 65536u || !out_status)
        return fail(FWBF_EINVAL, "fwbf_probe_bounded_wait: expect_bytes <= 65536 and a result pointer");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int *d_status = nullptr;
    cudaError_t e = cudaMallocAsync(reinterpret_cast<void **>(&d_status), sizeof(int), s);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMallocAsync(status)");
    bounded_wait_probe_kernel<<<1, 32, 0, s>>>(d_status, expect_bytes);
    e = cudaGetLastError();
    int h = -1;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, d_status, sizeof(int), cudaMemcpyDeviceToHost, s);
    cudaFreeAsync(d_status, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "bounded-wait probe");
    *out_status = h;
    return FWBF_OK;
}

extern "C" int fwbf_peak_int_issue(int mix, double ms, void *stream, double *out_ops_per_s, double *out_ops) {
    if ((mix != 0 && mix != 1) || !(ms >= 1.0 && ms <= 10000.0) || !out_ops_per_s)
        return fail(FWBF_EINVAL, "fwbf_peak_int_issue: mix must be 0/1, 1 <= ms <= 10000, result pointer set");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return cuda_fail(e, "device query");
    uint32_t *sink = nullptr;
    cudaEvent_t t0 = nullptr, t1 = nullptr;
    e = cudaMallocAsync(reinterpret_cast<void **>(&sink), 16, s);
    if (e == cudaSuccess) e = cudaEventCreate(&t0);
    if (e == cudaSuccess) e = cudaEventCreate(&t1);
    const int blocks = sms * kBlocksPerSm;
    auto run = [&](int iters, float *elapsed) -> cudaError_t {
        cudaError_t r = cudaEventRecord(t0, s);
        if (r != cudaSuccess) return r;
        if (mix == 0)
            int_issue_kernel<0><<<blocks, kThreads, 0, s>>>(sink, 0x1234567u, iters);
        else
            int_issue_kernel<1><<<blocks, kThreads, 0, s>>>(sink, 0x1234567u, iters);
        r = cudaGetLastError();
        if (r == cudaSuccess) r = cudaEventRecord(t1, s);
        if (r == cudaSuccess) r = cudaEventSynchronize(t1);
        if (r == cudaSuccess) r = cudaEventElapsedTime(elapsed, t0, t1);
        return r;
    };
    float cal = 0.f, el = 0.f;
    int iters = 256;
    if (e == cudaSuccess) e = run(iters, &cal);  // warm-up and calibration
    if (e == cudaSuccess) e = run(iters, &cal);
    if (e == cudaSuccess) {
        const double scale = ms / (cal > 1e-3f ? cal : 1e-3f);
        const double want = iters * scale;
        iters = want < 256.0 ? 256 : (want > 2e8 ? 200000000 : (int)want);
        e = run(iters, &el);
    }
    if (sink) cudaFreeAsync(sink, s);
    if (t0) cudaEventDestroy(t0);
    if (t1) cudaEventDestroy(t1);
    if (e != cudaSuccess) return cuda_fail(e, "integer issue microbenchmark");
    const double ops = (double)blocks * kThreads * (double)iters * kRounds * kChains;
    *out_ops_per_s = ops / (el * 1e-3);
    if (out_ops) *out_ops = ops;
    return FWBF_OK;
}
