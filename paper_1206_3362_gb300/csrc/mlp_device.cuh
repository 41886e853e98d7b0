// The learned schedule network (8 -> 64 -> 64 -> 2, ReLU, BF16 weights, FP32
// arithmetic) as used inside the decoding kernels: one warp evaluates it for
// its frame, lane l owning hidden units l and l + 32.
//
// Weight blob (device, 16-byte aligned, FWBF_MLP_BLOB_BYTES):
//   [0, 1024)      W1  bf16 [64][8]   (row = hidden unit)
//   [1024, 9216)   W2  bf16 [64][64]
//   [9216, 9472)   W3  bf16 [2][64]
//   [9472, 9728)   b1  f32  [64]
//   [9728, 9984)   b2  f32  [64]
//   [9984, 9992)   b3  f32  [2]
// The float32 master parameters used by training follow the same order:
// W1 (512), W2 (4096), W3 (128), b1 (64), b2 (64), b3 (2) = FWBF_MLP_PARAMS.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "fwbf.h"

namespace fwbf {

constexpr int kMlpW1 = 0, kMlpW2 = 1024, kMlpW3 = 9216, kMlpB1 = 9472, kMlpB2 = 9728, kMlpB3 = 9984;
// offsets of the parameters in the float32 master vector
constexpr int kPW1 = 0, kPW2 = 512, kPW3 = 4608, kPB1 = 4736, kPB2 = 4800, kPB3 = 4864;

__device__ __forceinline__ float bf16_lo(uint32_t w) { return __uint_as_float(w << 16); }
__device__ __forceinline__ float bf16_hi(uint32_t w) { return __uint_as_float(w & 0xffff0000u); }

// out0, out1 = network(feat) for the whole warp (feat identical in every lane)
__device__ __forceinline__ void mlp_eval(const unsigned char *blob, const float *feat, int lane, float &out0,
                                         float &out1) {
    const uint32_t *W1 = reinterpret_cast<const uint32_t *>(blob + kMlpW1);
    const uint32_t *W2 = reinterpret_cast<const uint32_t *>(blob + kMlpW2);
    const uint32_t *W3 = reinterpret_cast<const uint32_t *>(blob + kMlpW3);
    const float *b1 = reinterpret_cast<const float *>(blob + kMlpB1);
    const float *b2 = reinterpret_cast<const float *>(blob + kMlpB2);
    const float *b3 = reinterpret_cast<const float *>(blob + kMlpB3);
    float ha = __ldg(b1 + lane), hb = __ldg(b1 + lane + 32);
#pragma unroll
    for (int w = 0; w < 4; ++w) {
        const uint32_t wa = __ldg(W1 + lane * 4 + w), wb = __ldg(W1 + (lane + 32) * 4 + w);
        ha = fmaf(bf16_lo(wa), feat[2 * w], ha);
        ha = fmaf(bf16_hi(wa), feat[2 * w + 1], ha);
        hb = fmaf(bf16_lo(wb), feat[2 * w], hb);
        hb = fmaf(bf16_hi(wb), feat[2 * w + 1], hb);
    }
    ha = fmaxf(ha, 0.0f);
    hb = fmaxf(hb, 0.0f);
    float ga = __ldg(b2 + lane), gb = __ldg(b2 + lane + 32);
#pragma unroll 4
    for (int w = 0; w < 32; ++w) {  // inputs 2w, 2w + 1
        const float src = w < 16 ? ha : hb;
        const int l0 = (2 * w) & 31;
        const float x0 = __shfl_sync(0xffffffffu, src, l0), x1 = __shfl_sync(0xffffffffu, src, l0 + 1);
        const uint32_t wa = __ldg(W2 + lane * 32 + w), wb = __ldg(W2 + (lane + 32) * 32 + w);
        ga = fmaf(bf16_lo(wa), x0, ga);
        ga = fmaf(bf16_hi(wa), x1, ga);
        gb = fmaf(bf16_lo(wb), x0, gb);
        gb = fmaf(bf16_hi(wb), x1, gb);
    }
    ga = fmaxf(ga, 0.0f);
    gb = fmaxf(gb, 0.0f);
    const uint32_t r0a = __ldg(W3 + (lane >> 1)), r0b = __ldg(W3 + 16 + (lane >> 1));
    const uint32_t r1a = __ldg(W3 + 32 + (lane >> 1)), r1b = __ldg(W3 + 48 + (lane >> 1));
    const bool odd = lane & 1;
    float p0 = (odd ? bf16_hi(r0a) : bf16_lo(r0a)) * ga + (odd ? bf16_hi(r0b) : bf16_lo(r0b)) * gb;
    float p1 = (odd ? bf16_hi(r1a) : bf16_lo(r1a)) * ga + (odd ? bf16_hi(r1b) : bf16_lo(r1b)) * gb;
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
        p0 += __shfl_xor_sync(0xffffffffu, p0, d);
        p1 += __shfl_xor_sync(0xffffffffu, p1, d);
    }
    out0 = p0 + __ldg(b3);
    out1 = p1 + __ldg(b3 + 1);
}

}  // namespace fwbf
