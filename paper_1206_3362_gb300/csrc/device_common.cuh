// Device helpers shared by the decoding kernels: division by small runtime
// constants, circulant index arithmetic, and the bulk-copy (TMA) staging of
// the code tables into shared memory with a bounded mbarrier wait.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace fwbf {

constexpr unsigned FULL = 0xffffffffu;

// x / d for x < 65536 and 1 <= d <= 65535, with magic = ceil(2^32 / d) (d > 1)
__device__ __forceinline__ uint32_t div_small(uint32_t x, uint32_t d, uint32_t magic) {
    return d == 1 ? x : __umulhi(x, magic);
}

// bit of check (block row entry ent, offset i):  C*Z + ((i + t) mod Z)
__device__ __forceinline__ uint32_t circ_index(uint32_t ent, uint32_t i, uint32_t Z) {
    uint32_t j = i + (ent & 0xffffu);
    j = j >= Z ? j - Z : j;
    return (ent >> 16) * Z + j;
}

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Ends the barrier object (before its shared memory is used for anything
// else; no phase may be pending)
__device__ __forceinline__ void mbar_inval(uint64_t *bar) {
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

// global -> shared bulk copy (TMA, 1-D): 16-byte aligned addresses, size % 16 == 0
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return done != 0;
}

// Waits for phase `parity` of the barrier for at most limit_ns nanoseconds.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, uint64_t limit_ns) {
    const uint64_t t0 = global_ns();
    while (!mbar_try_wait(bar, parity)) {
        if (global_ns() - t0 > limit_ns) return false;
    }
    return true;
}

constexpr uint64_t kWaitLimitNs = 1000000000ull;  // 1 s
constexpr uint32_t kBulkChunk = 65536;

// Stages `words` uint32 of the global table into shared memory with bulk
// copies, the whole CTA waiting on one mbarrier.  Returns false for every
// thread of the CTA if the copy did not complete within the wait limit (the
// caller then records the timeout and leaves).
__device__ __forceinline__ bool stage_table(uint32_t *dst, const uint32_t *src, uint32_t words, uint64_t *bar,
                                            int *flag) {
    const uint32_t bytes = words * 4u;
    if (threadIdx.x == 0) {
        *flag = 0;
        mbar_init(bar, 1);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        // The region may have been read and written through the generic proxy
        // (a previous job's frame slices and tables); the barrier above orders
        // those accesses before this thread, and the fence orders them before
        // the bulk copies (async proxy) that overwrite the region.
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_expect_tx(bar, bytes);
        for (uint32_t off = 0; off < bytes; off += kBulkChunk) {
            uint32_t n = bytes - off < kBulkChunk ? bytes - off : kBulkChunk;
            bulk_g2s(reinterpret_cast<char *>(dst) + off, reinterpret_cast<const char *>(src) + off, n, bar);
        }
    }
    bool ok = mbar_wait_bounded(bar, 0, kWaitLimitNs);
    if (!ok) {
        // let the copies in flight land before the CTA leaves
        mbar_wait_bounded(bar, 0, kWaitLimitNs);
        atomicOr(flag, 1);
    }
    __syncthreads();
    return *flag == 0;
}

__device__ __forceinline__ int warp_sum(int v) { return __reduce_add_sync(FULL, v); }

// Sixteen int8 channel values with -128 replaced by -127: the decoders take
// int8 values in the quantiser's symmetric range, and -128 decodes as -127.
__device__ __forceinline__ uint4 clamp_m127(uint4 v) {
    const uint32_t m = 0x81818181u;  // -127 in every byte
    return make_uint4(__vmaxs4(v.x, m), __vmaxs4(v.y, m), __vmaxs4(v.z, m), __vmaxs4(v.w, m));
}

// The WPF warps that decode one frame meet here: the warp itself, or a named
// barrier (id bar_id, WPF * 32 threads) that also orders their shared memory.
template <int WPF>
__device__ __forceinline__ void group_sync(int bar_id) {
    if constexpr (WPF == 1) {
        __syncwarp();
    } else {
        asm volatile("bar.sync %0, %1;" ::"r"(bar_id), "n"(32 * WPF) : "memory");
    }
}

// Sums of three warp-uniform values over the group's warps, through a
// scratch of 2 x 4 x WPF ints used in alternate halves (a half is rewritten
// only after the group has met again, so no reader can still be on it).
template <int WPF>
__device__ __forceinline__ int3 group_sum3(int3 v, int *red, int &half, int lane, int gw, int bar_id) {
    if constexpr (WPF == 1) {
        return v;
    } else {
        int *r = red + half * 4 * WPF;
        half ^= 1;
        if (lane == 0) {
            r[4 * gw] = v.x;
            r[4 * gw + 1] = v.y;
            r[4 * gw + 2] = v.z;
        }
        group_sync<WPF>(bar_id);
        int3 s = make_int3(0, 0, 0);
#pragma unroll
        for (int w = 0; w < WPF; ++w) {
            s.x += r[4 * w];
            s.y += r[4 * w + 1];
            s.z += r[4 * w + 2];
        }
        return s;
    }
}

}  // namespace fwbf
