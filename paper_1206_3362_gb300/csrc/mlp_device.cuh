// The learned schedule network (8 -> 64 -> 64 -> 2, ReLU, BF16 weights, FP32
// arithmetic) as used inside the decoding kernels, evaluated for one frame by
// the warps that decode it (mlp_eval).
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

#include "device_common.cuh"
#include "fwbf.h"

namespace fwbf {

constexpr int kMlpW1 = 0, kMlpW2 = 1024, kMlpW3 = 9216, kMlpB1 = 9472, kMlpB2 = 9728, kMlpB3 = 9984;
// offsets of the parameters in the float32 master vector
constexpr int kPW1 = 0, kPW2 = 512, kPW3 = 4608, kPB1 = 4736, kPB2 = 4800, kPB3 = 4864;

__device__ __forceinline__ float bf16_lo(uint32_t w) { return __uint_as_float(w << 16); }
__device__ __forceinline__ float bf16_hi(uint32_t w) { return __uint_as_float(w & 0xffff0000u); }

// Layer 1 for the calling warp (feat identical in every lane): ha, hb =
// ReLU(W1 feat + b1) of hidden units lane and lane + 32.
__device__ __forceinline__ void mlp_layer1(const unsigned char *blob, const float *feat, int lane, float &ha,
                                           float &hb) {
    const uint32_t *W1 = reinterpret_cast<const uint32_t *>(blob + kMlpW1);
    const float *b1 = reinterpret_cast<const float *>(blob + kMlpB1);
    const uint4 w1a = __ldg(reinterpret_cast<const uint4 *>(W1) + lane);
    const uint4 w1b = __ldg(reinterpret_cast<const uint4 *>(W1) + lane + 32);
    ha = __ldg(b1 + lane);
    hb = __ldg(b1 + lane + 32);
    float ta = bf16_lo(w1a.x) * feat[0], tb = bf16_lo(w1b.x) * feat[0];
    ha = fmaf(bf16_hi(w1a.x), feat[1], ha);
    hb = fmaf(bf16_hi(w1b.x), feat[1], hb);
    ta = fmaf(bf16_lo(w1a.y), feat[2], ta);
    tb = fmaf(bf16_lo(w1b.y), feat[2], tb);
    ha = fmaf(bf16_hi(w1a.y), feat[3], ha);
    hb = fmaf(bf16_hi(w1b.y), feat[3], hb);
    ta = fmaf(bf16_lo(w1a.z), feat[4], ta);
    tb = fmaf(bf16_lo(w1b.z), feat[4], tb);
    ha = fmaf(bf16_hi(w1a.z), feat[5], ha);
    hb = fmaf(bf16_hi(w1b.z), feat[5], hb);
    ta = fmaf(bf16_lo(w1a.w), feat[6], ta);
    tb = fmaf(bf16_lo(w1b.w), feat[6], tb);
    ha = fmaf(bf16_hi(w1a.w), feat[7], ha);
    hb = fmaf(bf16_hi(w1b.w), feat[7], hb);
    ha = fmaxf(ha + ta, 0.0f);
    hb = fmaxf(hb + tb, 0.0f);
}

// W3[j][u] (bf16 [2][64], two per word)
__device__ __forceinline__ float mlp_w3(const unsigned char *blob, int j, int u) {
    const uint32_t w = __ldg(reinterpret_cast<const uint32_t *>(blob + kMlpW3) + ((j * 64 + u) >> 1));
    return (u & 1) ? bf16_hi(w) : bf16_lo(w);
}

// sum over the warp, the same butterfly (and so the same float result) in every lane
__device__ __forceinline__ float mlp_warp_sum(float v) {
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) v += __shfl_xor_sync(0xffffffffu, v, d);
    return v;
}

// Arithmetic order, identical for every group size: each layer-2 unit keeps
// four partial sums over its inputs (input 8v + 2t + {0, 1} into sum t, v
// ascending), ((s0 + s1) + (s2 + s3)) then ReLU; each output j is
// (butterfly sum over units 0..31 + butterfly sum over units 32..63) + b3[j].
//
// out0, out1 = network(feat) for a group of WPF warps deciding one frame (feat
// identical in every lane): one warp computes all 64 layer-2 units (lane l:
// units l and l + 32); with WPF > 1, warp 0 computes units 0..31 and warp 1
// units 32..63, the two halves of each output meet through slot (4 floats of
// the group's shared memory) and barrier bar_id.  Layer 2 reads its inputs by
// shuffles and its weight rows as 128-bit loads (8 bf16).
template <int WPF>
__device__ __forceinline__ void mlp_eval(const unsigned char *blob, const float *feat, int lane, int gw, float *slot,
                                         int bar_id, float &out0, float &out1) {
    const uint4 *W2 = reinterpret_cast<const uint4 *>(blob + kMlpW2);  // 8 uint4 per row
    const float *b2 = reinterpret_cast<const float *>(blob + kMlpB2);
    const float *b3 = reinterpret_cast<const float *>(blob + kMlpB3);
    if constexpr (WPF == 1) {
        float ha, hb;
        mlp_layer1(blob, feat, lane, ha, hb);
        float ga[4] = {__ldg(b2 + lane), 0.0f, 0.0f, 0.0f};
        float gb[4] = {__ldg(b2 + lane + 32), 0.0f, 0.0f, 0.0f};
#pragma unroll
        for (int v = 0; v < 8; ++v) {  // inputs 8v .. 8v + 7
            const uint4 wa = __ldg(W2 + lane * 8 + v), wb = __ldg(W2 + (lane + 32) * 8 + v);
            const float src = v < 4 ? ha : hb;
            float x[8];
#pragma unroll
            for (int t = 0; t < 8; ++t) x[t] = __shfl_sync(0xffffffffu, src, (8 * v + t) & 31);
            const uint32_t aw[4] = {wa.x, wa.y, wa.z, wa.w}, bw[4] = {wb.x, wb.y, wb.z, wb.w};
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                ga[t] = fmaf(bf16_lo(aw[t]), x[2 * t], ga[t]);
                ga[t] = fmaf(bf16_hi(aw[t]), x[2 * t + 1], ga[t]);
                gb[t] = fmaf(bf16_lo(bw[t]), x[2 * t], gb[t]);
                gb[t] = fmaf(bf16_hi(bw[t]), x[2 * t + 1], gb[t]);
            }
        }
        const float g1 = fmaxf((ga[0] + ga[1]) + (ga[2] + ga[3]), 0.0f);
        const float g2 = fmaxf((gb[0] + gb[1]) + (gb[2] + gb[3]), 0.0f);
        const float p0a = mlp_warp_sum(mlp_w3(blob, 0, lane) * g1), p0b = mlp_warp_sum(mlp_w3(blob, 0, lane + 32) * g2);
        const float p1a = mlp_warp_sum(mlp_w3(blob, 1, lane) * g1), p1b = mlp_warp_sum(mlp_w3(blob, 1, lane + 32) * g2);
        out0 = (p0a + p0b) + __ldg(b3);
        out1 = (p1a + p1b) + __ldg(b3 + 1);
    } else {
        if (gw < 2) {
            float ha, hb;
            mlp_layer1(blob, feat, lane, ha, hb);
            const int u = 32 * gw + lane;
            float ga[4] = {__ldg(b2 + u), 0.0f, 0.0f, 0.0f};
#pragma unroll
            for (int v = 0; v < 8; ++v) {
                const uint4 wa = __ldg(W2 + u * 8 + v);
                const float src = v < 4 ? ha : hb;
                float x[8];
#pragma unroll
                for (int t = 0; t < 8; ++t) x[t] = __shfl_sync(0xffffffffu, src, (8 * v + t) & 31);
                const uint32_t aw[4] = {wa.x, wa.y, wa.z, wa.w};
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    ga[t] = fmaf(bf16_lo(aw[t]), x[2 * t], ga[t]);
                    ga[t] = fmaf(bf16_hi(aw[t]), x[2 * t + 1], ga[t]);
                }
            }
            const float g = fmaxf((ga[0] + ga[1]) + (ga[2] + ga[3]), 0.0f);
            const float p0 = mlp_warp_sum(mlp_w3(blob, 0, u) * g), p1 = mlp_warp_sum(mlp_w3(blob, 1, u) * g);
            if (lane == 0) {
                slot[2 * gw] = p0;
                slot[2 * gw + 1] = p1;
            }
        }
        group_sync<WPF>(bar_id);
        out0 = (slot[0] + slot[2]) + __ldg(b3);
        out1 = (slot[1] + slot[3]) + __ldg(b3 + 1);
    }
}

}  // namespace fwbf
