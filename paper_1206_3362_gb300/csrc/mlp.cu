// Training and inference kernels of the learned schedule network
// (8 -> 64 -> 64 -> 2, ReLU hidden layers, linear outputs; BF16 weights with
// FP32 arithmetic).  The decoder evaluates the same network per frame and pass
// (mlp_device.cuh); these kernels fit it to (features, label) pairs produced by
// plain FWBF.
//
// Loss: mean over samples of the squared error of both outputs.  Gradients are
// taken with respect to the BF16-rounded weights the forward pass uses; the
// optimiser (Adam) updates float32 master weights and rewrites the BF16 blob.
#include <cuda_bf16.h>

#include "fwbf_internal.h"
#include "mlp_device.cuh"

namespace fwbf {

constexpr int kIn = FWBF_MLP_IN, kHid = FWBF_MLP_HIDDEN, kOut = FWBF_MLP_OUT;
constexpr int kSamples = 32;  // samples per block of the gradient kernel

// master weight i (i < kPB1) as the blob holds it (bf16, widened)
__device__ __forceinline__ float blob_w(const unsigned char *blob, int i) {
    const uint16_t h = reinterpret_cast<const uint16_t *>(blob)[mlp_blob_index(i)];
    return __uint_as_float((uint32_t)h << 16);
}

// float32 master parameters -> BF16/FP32 blob (round to nearest even)
__global__ void mlp_pack_kernel(const float *__restrict__ master, unsigned char *__restrict__ blob) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < FWBF_MLP_PARAMS) {
        const float v = master[i];
        if (i < kPB1) {
            const uint16_t h = __bfloat16_as_ushort(__float2bfloat16_rn(v));
            reinterpret_cast<uint16_t *>(blob)[mlp_blob_index(i)] = h;  // W1, W2, W3 from offset 0
        } else {
            reinterpret_cast<float *>(blob + kMlpB1)[i - kPB1] = v;  // b1, b2, b3 contiguous
        }
    }
}

// one thread per sample
__global__ void mlp_forward_kernel(const unsigned char *__restrict__ blob, const float *__restrict__ x,
                                   float *__restrict__ out, int64_t n) {
    const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (s >= n) return;
    float in[kIn], h1[kHid];
    for (int i = 0; i < kIn; ++i) in[i] = x[s * kIn + i];
    const float *b1 = reinterpret_cast<const float *>(blob + kMlpB1);
    const float *b2 = reinterpret_cast<const float *>(blob + kMlpB2);
    const float *b3 = reinterpret_cast<const float *>(blob + kMlpB3);
    for (int j = 0; j < kHid; ++j) {
        float a = b1[j];
        for (int i = 0; i < kIn; ++i) a = fmaf(blob_w(blob, kPW1 + j * kIn + i), in[i], a);
        h1[j] = fmaxf(a, 0.0f);
    }
    float o[kOut] = {b3[0], b3[1]};
    for (int j = 0; j < kHid; ++j) {
        float a = b2[j];
        for (int i = 0; i < kHid; ++i) a = fmaf(blob_w(blob, kPW2 + j * kHid + i), h1[i], a);
        a = fmaxf(a, 0.0f);
        for (int k = 0; k < kOut; ++k) o[k] = fmaf(blob_w(blob, kPW3 + k * kHid + j), a, o[k]);
    }
    for (int k = 0; k < kOut; ++k) out[s * kOut + k] = o[k];
}

// Gradient of sum_s ||net(x_s) - t_s||^2 / n_total over one block of samples,
// added into grad (float32, master order; one atomic per parameter and block)
// and the loss into *loss.
__global__ void __launch_bounds__(256) mlp_grad_kernel(const unsigned char *__restrict__ blob,
                                                       const float *__restrict__ x, const float *__restrict__ t,
                                                       int64_t n, float inv_total, float *__restrict__ grad,
                                                       float *__restrict__ loss) {
    __shared__ float W1[kHid * kIn], W2[kHid * kHid], W3[kOut * kHid], B1[kHid], B2[kHid], B3[kOut];
    __shared__ float X[kSamples][kIn], H1[kSamples][kHid], H2[kSamples][kHid], D2[kSamples][kHid];
    __shared__ float DO[kSamples][kOut];
    __shared__ float L;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int64_t s0 = blockIdx.x * (int64_t)kSamples;
    const int ns = (int)min((int64_t)kSamples, n - s0);
    for (int i = tid; i < kHid * kIn; i += nt) W1[i] = blob_w(blob, kPW1 + i);
    for (int i = tid; i < kHid * kHid; i += nt) W2[i] = blob_w(blob, kPW2 + i);
    for (int i = tid; i < kOut * kHid; i += nt) W3[i] = blob_w(blob, kPW3 + i);
    for (int i = tid; i < kHid; i += nt) {
        B1[i] = reinterpret_cast<const float *>(blob + kMlpB1)[i];
        B2[i] = reinterpret_cast<const float *>(blob + kMlpB2)[i];
    }
    if (tid < kOut) B3[tid] = reinterpret_cast<const float *>(blob + kMlpB3)[tid];
    if (tid == 0) L = 0.0f;
    for (int i = tid; i < kSamples * kIn; i += nt) {
        const int s = i / kIn, c = i % kIn;
        X[s][c] = s < ns ? x[(s0 + s) * kIn + c] : 0.0f;
    }
    __syncthreads();
    // forward
    for (int i = tid; i < kSamples * kHid; i += nt) {
        const int s = i / kHid, j = i % kHid;
        float a = B1[j];
        for (int c = 0; c < kIn; ++c) a = fmaf(W1[j * kIn + c], X[s][c], a);
        H1[s][j] = fmaxf(a, 0.0f);
    }
    __syncthreads();
    for (int i = tid; i < kSamples * kHid; i += nt) {
        const int s = i / kHid, j = i % kHid;
        float a = B2[j];
        for (int c = 0; c < kHid; ++c) a = fmaf(W2[j * kHid + c], H1[s][c], a);
        H2[s][j] = fmaxf(a, 0.0f);
    }
    __syncthreads();
    for (int i = tid; i < kSamples * kOut; i += nt) {
        const int s = i / kOut, k = i % kOut;
        float o = B3[k];
        for (int c = 0; c < kHid; ++c) o = fmaf(W3[k * kHid + c], H2[s][c], o);
        float d = 0.0f;
        if (s < ns) {
            const float e = o - t[(s0 + s) * kOut + k];
            atomicAdd(&L, e * e * inv_total);
            d = 2.0f * e * inv_total;
        }
        DO[s][k] = d;
    }
    __syncthreads();
    // backward: output layer
    for (int i = tid; i < kOut * kHid; i += nt) {
        const int k = i / kHid, c = i % kHid;
        float g = 0.0f;
        for (int s = 0; s < kSamples; ++s) g = fmaf(DO[s][k], H2[s][c], g);
        atomicAdd(&grad[kPW3 + i], g);
    }
    if (tid < kOut) {
        float g = 0.0f;
        for (int s = 0; s < kSamples; ++s) g += DO[s][tid];
        atomicAdd(&grad[kPB3 + tid], g);
    }
    for (int i = tid; i < kSamples * kHid; i += nt) {
        const int s = i / kHid, j = i % kHid;
        float d = 0.0f;
        for (int k = 0; k < kOut; ++k) d = fmaf(W3[k * kHid + j], DO[s][k], d);
        D2[s][j] = H2[s][j] > 0.0f ? d : 0.0f;
    }
    __syncthreads();
    // second layer
    for (int i = tid; i < kHid * kHid; i += nt) {
        const int j = i / kHid, c = i % kHid;
        float g = 0.0f;
        for (int s = 0; s < kSamples; ++s) g = fmaf(D2[s][j], H1[s][c], g);
        atomicAdd(&grad[kPW2 + i], g);
    }
    for (int j = tid; j < kHid; j += nt) {
        float g = 0.0f;
        for (int s = 0; s < kSamples; ++s) g += D2[s][j];
        atomicAdd(&grad[kPB2 + j], g);
    }
    __syncthreads();
    // first layer: reuse H2 for the hidden-1 deltas
    for (int i = tid; i < kSamples * kHid; i += nt) {
        const int s = i / kHid, c = i % kHid;
        float d = 0.0f;
        for (int j = 0; j < kHid; ++j) d = fmaf(W2[j * kHid + c], D2[s][j], d);
        H2[s][c] = H1[s][c] > 0.0f ? d : 0.0f;
    }
    __syncthreads();
    for (int i = tid; i < kHid * kIn; i += nt) {
        const int j = i / kIn, c = i % kIn;
        float g = 0.0f;
        for (int s = 0; s < kSamples; ++s) g = fmaf(H2[s][j], X[s][c], g);
        atomicAdd(&grad[kPW1 + i], g);
    }
    for (int j = tid; j < kHid; j += nt) {
        float g = 0.0f;
        for (int s = 0; s < kSamples; ++s) g += H2[s][j];
        atomicAdd(&grad[kPB1 + j], g);
    }
    __syncthreads();
    if (tid == 0) atomicAdd(loss, L);
}

// Adam on the float32 master weights; rewrites the blob, clears the gradient.
__global__ void mlp_adam_kernel(float *__restrict__ master, unsigned char *__restrict__ blob,
                                float *__restrict__ grad, float *__restrict__ m, float *__restrict__ v, float lr,
                                float beta1, float beta2, float eps, float bc1, float bc2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= FWBF_MLP_PARAMS) return;
    const float g = grad[i];
    const float mi = beta1 * m[i] + (1.0f - beta1) * g;
    const float vi = beta2 * v[i] + (1.0f - beta2) * g * g;
    m[i] = mi;
    v[i] = vi;
    const float w = master[i] - lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
    master[i] = w;
    grad[i] = 0.0f;
    if (i < kPB1)
        reinterpret_cast<uint16_t *>(blob)[mlp_blob_index(i)] = __bfloat16_as_ushort(__float2bfloat16_rn(w));
    else
        reinterpret_cast<float *>(blob + kMlpB1)[i - kPB1] = w;
}

}  // namespace fwbf

using namespace fwbf;

extern "C" {

static int blob_ok(const void *blob) {
    if (!blob) return fail(FWBF_EINVAL, "blob is NULL");
    if (reinterpret_cast<uintptr_t>(blob) % 16) return fail(FWBF_EINVAL, "blob must be 16-byte aligned");
    return FWBF_OK;
}

int fwbf_mlp_pack(const float *master, void *blob, void *stream) {
    int rc = blob_ok(blob);
    if (rc) return rc;
    if (!master) return fail(FWBF_EINVAL, "master is NULL");
    mlp_pack_kernel<<<(FWBF_MLP_PARAMS + 255) / 256, 256, 0, static_cast<cudaStream_t>(stream)>>>(
        master, static_cast<unsigned char *>(blob));
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? FWBF_OK : cuda_fail(e, "mlp_pack launch");
}

int fwbf_mlp_forward(const void *blob, const float *x, int64_t n, float *out, void *stream) {
    int rc = blob_ok(blob);
    if (rc) return rc;
    if (n < 0 || (n > 0 && (!x || !out))) return fail(FWBF_EINVAL, "bad x/out/n");
    if (n == 0) return FWBF_OK;
    const int64_t blocks = (n + 127) / 128;
    mlp_forward_kernel<<<(unsigned)blocks, 128, 0, static_cast<cudaStream_t>(stream)>>>(
        static_cast<const unsigned char *>(blob), x, out, n);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? FWBF_OK : cuda_fail(e, "mlp_forward launch");
}

int fwbf_mlp_grad(const void *blob, const float *x, const float *target, int64_t n, int64_t n_total, float *grad,
                  float *loss, void *stream) {
    int rc = blob_ok(blob);
    if (rc) return rc;
    if (n < 0 || n_total < 1 || (n > 0 && (!x || !target || !grad || !loss)))
        return fail(FWBF_EINVAL, "bad arguments");
    if (n == 0) return FWBF_OK;
    const int64_t blocks = (n + kSamples - 1) / kSamples;
    mlp_grad_kernel<<<(unsigned)blocks, 256, 0, static_cast<cudaStream_t>(stream)>>>(
        static_cast<const unsigned char *>(blob), x, target, n, 1.0f / (float)n_total, grad, loss);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? FWBF_OK : cuda_fail(e, "mlp_grad launch");
}

int fwbf_mlp_adam(float *master, void *blob, float *grad, float *m, float *v, int64_t step, float lr, float beta1,
                  float beta2, float eps, void *stream) {
    int rc = blob_ok(blob);
    if (rc) return rc;
    if (!master || !grad || !m || !v || step < 1) return fail(FWBF_EINVAL, "bad arguments");
    const float bc1 = 1.0f - powf(beta1, (float)step), bc2 = 1.0f - powf(beta2, (float)step);
    mlp_adam_kernel<<<(FWBF_MLP_PARAMS + 255) / 256, 256, 0, static_cast<cudaStream_t>(stream)>>>(
        master, static_cast<unsigned char *>(blob), grad, m, v, lr, beta1, beta2, eps, bc1, bc2);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? FWBF_OK : cuda_fail(e, "mlp_adam launch");
}

}  // extern "C"
