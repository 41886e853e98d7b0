// The learned schedule network (8 -> 64 -> 64 -> 2, ReLU, BF16 weights, FP32
// arithmetic) as used inside the decoding kernels, evaluated for one frame by
// the warps that decode it (mlp_eval).
//
// Weight blob (device, 16-byte aligned, FWBF_MLP_BLOB_BYTES):
//   [0, 1024)      W1  bf16 [64][8]   (row = hidden unit)
//   [1024, 9216)   W2  bf16, 512 groups of 16 bytes: group 64 v + u holds
//                  W2[u][8v .. 8v + 7] (unit u, inputs 8v..8v+7), so a warp
//                  whose lanes take consecutive units reads 512 contiguous bytes
//   [9216, 9472)   W3  bf16 [2][64]
//   [9472, 9728)   b1  f32  [64]
//   [9728, 9984)   b2  f32  [64]
//   [9984, 9992)   b3  f32  [2]
// The float32 master parameters used by training are in plain row-major order:
// W1 (512), W2 (4096), W3 (128), b1 (64), b2 (64), b3 (2) = FWBF_MLP_PARAMS;
// mlp_blob_index maps a master weight to its bf16 slot in the blob.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "device_common.cuh"
#include "fwbf.h"

namespace fwbf {

constexpr int kMlpW1 = 0, kMlpW2 = 1024, kMlpW3 = 9216, kMlpB1 = 9472, kMlpB2 = 9728, kMlpB3 = 9984;
static_assert(kMlpB3 + 8 <= FWBF_MLP_BLOB_BYTES, "blob layout");
// offsets of the parameters in the float32 master vector
constexpr int kPW1 = 0, kPW2 = 512, kPW3 = 4608, kPB1 = 4736, kPB2 = 4800, kPB3 = 4864;

// bf16 slot in the blob of master weight i (i < kPB1; W1 and W3 keep their
// order, W2[u][c] goes to group 64 (c / 8) + u, element c % 8)
__host__ __device__ __forceinline__ int mlp_blob_index(int i) {
    if (i < kPW2 || i >= kPW3) return i;
    const int j = i - kPW2, u = j >> 6, c = j & 63;
    return kPW2 + ((c >> 3) << 9) + (u << 3) + (c & 7);
}


__device__ __forceinline__ float bf16_lo(uint32_t w) { return __uint_as_float(w << 16); }
__device__ __forceinline__ float bf16_hi(uint32_t w) { return __uint_as_float(w & 0xffff0000u); }

// Hidden unit u of layer 1: ReLU(W1[u] feat + b1[u]), two partial sums
// (even inputs from 0, odd inputs from b1) added at the end.
__device__ __forceinline__ float mlp_unit1(const unsigned char *blob, float4 fa, float4 fb, int u) {
    const uint4 w = __ldg(reinterpret_cast<const uint4 *>(blob + kMlpW1) + u);
    float h = __ldg(reinterpret_cast<const float *>(blob + kMlpB1) + u);
    float t = bf16_lo(w.x) * fa.x;
    h = fmaf(bf16_hi(w.x), fa.y, h);
    t = fmaf(bf16_lo(w.y), fa.z, t);
    h = fmaf(bf16_hi(w.y), fa.w, h);
    t = fmaf(bf16_lo(w.z), fb.x, t);
    h = fmaf(bf16_hi(w.z), fb.y, h);
    t = fmaf(bf16_lo(w.w), fb.z, t);
    h = fmaf(bf16_hi(w.w), fb.w, h);
    return fmaxf(h + t, 0.0f);
}

// Hidden unit u of layer 2 from the 64 layer-1 outputs h (shared memory, read
// as broadcast 16-byte loads): four partial sums, input 8v + 2t + {0, 1} into
// sum t for v ascending, then ((s0 + s1) + (s2 + s3)) and ReLU.
// (a loop unrolled twice: a small body for the instruction cache, 2 % faster
// learned decoding on EG(1023) than unrolled fully)
__device__ __forceinline__ float mlp_unit2(const unsigned char *blob, const float4 *h4, int u) {
    const uint4 *W2 = reinterpret_cast<const uint4 *>(blob + kMlpW2);
    float g0 = __ldg(reinterpret_cast<const float *>(blob + kMlpB2) + u), g1 = 0.0f, g2 = 0.0f, g3 = 0.0f;
#pragma unroll 2
    for (int v = 0; v < 8; ++v) {
        const uint4 w = __ldg(W2 + 64 * v + u);
        const float4 xa = h4[2 * v], xb = h4[2 * v + 1];
        g0 = fmaf(bf16_lo(w.x), xa.x, g0);
        g0 = fmaf(bf16_hi(w.x), xa.y, g0);
        g1 = fmaf(bf16_lo(w.y), xa.z, g1);
        g1 = fmaf(bf16_hi(w.y), xa.w, g1);
        g2 = fmaf(bf16_lo(w.z), xb.x, g2);
        g2 = fmaf(bf16_hi(w.z), xb.y, g2);
        g3 = fmaf(bf16_lo(w.w), xb.z, g3);
        g3 = fmaf(bf16_hi(w.w), xb.w, g3);
    }
    return fmaxf((g0 + g1) + (g2 + g3), 0.0f);
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

// network(feat) for a group of WPF warps deciding one frame (features fa =
// feat[0..3], fb = feat[4..7], identical in every lane).  h: 64 floats of the frame's shared memory
// (16-byte aligned) holding the layer-1 outputs; slot: 4 floats of it (WPF > 1).
// One warp computes every unit (lane l: units l and l + 32); with WPF > 1,
// warp 0 computes units 0..31 of both layers and warp 1 units 32..63, and the
// group meets twice (after layer 1 and before the outputs).  Each output j is
// (butterfly sum over units 0..31 + butterfly sum over units 32..63) + b3[j]:
// the arithmetic, and so every result, is the same for every group size.
template <int WPF>
__device__ __forceinline__ float2 mlp_eval(const unsigned char *blob, float4 fa, float4 fb, int lane, int gw,
                                           float *h, float *slot, int bar_id) {
    const float *b3 = reinterpret_cast<const float *>(blob + kMlpB3);
    const float4 *h4 = reinterpret_cast<const float4 *>(h);
    if constexpr (WPF == 1) {
        h[lane] = mlp_unit1(blob, fa, fb, lane);
        h[lane + 32] = mlp_unit1(blob, fa, fb, lane + 32);
        __syncwarp();
        const float g1 = mlp_unit2(blob, h4, lane), g2 = mlp_unit2(blob, h4, lane + 32);
        const float p0a = mlp_warp_sum(mlp_w3(blob, 0, lane) * g1), p0b = mlp_warp_sum(mlp_w3(blob, 0, lane + 32) * g2);
        const float p1a = mlp_warp_sum(mlp_w3(blob, 1, lane) * g1), p1b = mlp_warp_sum(mlp_w3(blob, 1, lane + 32) * g2);
        const float2 out = make_float2((p0a + p0b) + __ldg(b3), (p1a + p1b) + __ldg(b3 + 1));
        __syncwarp();  // every lane has read h before the next evaluation rewrites it
        return out;
    } else {
        const int u = 32 * gw + lane;
        if (gw < 2) h[u] = mlp_unit1(blob, fa, fb, u);
        group_sync<WPF>(bar_id);
        if (gw < 2) {
            const float g = mlp_unit2(blob, h4, u);
            const float p0 = mlp_warp_sum(mlp_w3(blob, 0, u) * g), p1 = mlp_warp_sum(mlp_w3(blob, 1, u) * g);
            if (lane == 0) {
                slot[2 * gw] = p0;
                slot[2 * gw + 1] = p1;
            }
        }
        group_sync<WPF>(bar_id);
        return make_float2((slot[0] + slot[2]) + __ldg(b3), (slot[1] + slot[3]) + __ldg(b3 + 1));
    }
}

}  // namespace fwbf
