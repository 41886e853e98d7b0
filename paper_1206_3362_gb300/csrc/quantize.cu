// int8 quantisation of channel values for the integer decoder:
//   q = saturate_{[-127,127]}(round_half_to_even(16 y)), NaN -> 0.
// 16*y is exact in float32 (or overflows to +-inf, which saturates);
// cvt.rni.s32.f32 rounds half to even, saturates out-of-range values and maps
// NaN to 0, so the clamp to +-127 completes the definition.
#include "fwbf_internal.h"

namespace fwbf {

__device__ __forceinline__ int8_t quantize_one(float v) {
    int r = __float2int_rn(v * 16.0f);
    r = r > 127 ? 127 : (r < -127 ? -127 : r);
    return (int8_t)r;
}

// count/4 groups of four: float4 in, char4 out (both pointers aligned)
__global__ void quantize4_kernel(const float4 *__restrict__ y, char4 *__restrict__ q, int64_t groups) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < groups;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float4 v = __ldcs(y + i);
        char4 o;
        o.x = quantize_one(v.x);
        o.y = quantize_one(v.y);
        o.z = quantize_one(v.z);
        o.w = quantize_one(v.w);
        q[i] = o;
    }
}

__global__ void quantize1_kernel(const float *__restrict__ y, int8_t *__restrict__ q, int64_t count) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * blockDim.x)
        q[i] = quantize_one(y[i]);
}

int launch_quantize(const float *y, int8_t *q, int64_t count, cudaStream_t s) {
    if (count == 0) return 0;
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return cuda_fail(e, "device query");
    const int threads = 256;
    const bool vec = (reinterpret_cast<uintptr_t>(y) % 16 == 0) && (reinterpret_cast<uintptr_t>(q) % 4 == 0);
    const int64_t groups = vec ? count / 4 : 0;
    if (groups > 0) {
        int64_t blocks = (groups + threads - 1) / threads;
        if (blocks > (int64_t)sms * 16) blocks = (int64_t)sms * 16;
        quantize4_kernel<<<(unsigned)blocks, threads, 0, s>>>(reinterpret_cast<const float4 *>(y),
                                                              reinterpret_cast<char4 *>(q), groups);
    }
    const int64_t done = groups * 4;
    if (count > done) {
        const int64_t rest = count - done;
        int64_t blocks = (rest + threads - 1) / threads;
        if (blocks > (int64_t)sms * 16) blocks = (int64_t)sms * 16;
        quantize1_kernel<<<(unsigned)blocks, threads, 0, s>>>(y + done, q + done, rest);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "quantize launch");
    return 0;
}

}  // namespace fwbf
