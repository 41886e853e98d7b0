// Internal declarations shared by the C-ABI layer and the kernel translation
// units of libfwbf.so.  Not part of the public interface (see include/fwbf.h).
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include "fwbf.h"
#include <stdint.h>

#include <mutex>
#include <string>
#include <utility>
#include <vector>

// Frame work counters (8 bytes of device memory each) owned by a code handle,
// one per stream the handle decodes on: calls on one stream are ordered, so
// they share its counter; the handle frees them.
struct StreamCounters {
    std::mutex mu;
    std::vector<std::pair<cudaStream_t, unsigned long long *>> by_stream;
};

// Index tables of H in circulant form (Z = 1: plain CSR/CSC).
//   A check m = R*Z + i (block row R, offset i) has, for every entry (C, t) of
//   block row R, the bit n = C*Z + ((i + t) mod Z).
//   A bit n = C*Z + j has, for every entry (R, u) of block column C, the check
//   m = R*Z + ((j + u) mod Z), u = (Z - t) mod Z.
// Device blob of uint32 words: rptr[MB+1] | rent[..] | cptr[NB+1] | cent[..],
// entries packed as (block index << 16) | shift.
struct fwbf_code_s {
    int N, M;
    int64_t nnz;
    int Z, MB, NB;
    int dv_max, dc_max;
    int max_row_overlap;        // most bits two checks share (RC constraint iff <= 1)
    int p, B;
    uint32_t p_magic, z_magic;  // ceil(2^32 / d) for exact x / d with x < 65536
    uint32_t rptr_off, rent_off, cptr_off, cent_off;
    uint32_t table_words;       // multiple of 4 (16-byte granules)
    uint32_t *d_table;
    int device;
    int num_sms;
    int smem_optin;             // max dynamic shared memory per block
    mutable StreamCounters counters;
};

namespace fwbf {

// An NVTX range over an entry point's host-side work (argument checks, set-up,
// queueing), named after it, for timeline profilers; header-only NVTX costs a
// few nanoseconds when no profiler is attached.
struct TraceRange {
    explicit TraceRange(const char *name) { nvtxRangePushA(name); }
    ~TraceRange() { nvtxRangePop(); }
    TraceRange(const TraceRange &) = delete;
    TraceRange &operator=(const TraceRange &) = delete;
};

// thread-local detail message for fwbf_last_error()
void set_error(const std::string &msg);
int fail(int status, const std::string &msg);
int cuda_fail(cudaError_t e, const char *what);

// A zeroed frame work counter for a decode on stream s: the handle's counter
// for s, created by the first call on s; a first call made under stream
// capture takes a stream-ordered allocation instead (owned = true), which
// release_counter frees after the launch.
struct CounterLease {
    unsigned long long *ptr = nullptr;
    bool owned = false;
};
int acquire_counter(const fwbf_code_s *c, cudaStream_t s, CounterLease *out);
int release_counter(const CounterLease &lease, cudaStream_t s);
// frees the handle's counters (after the device has finished with them)
void free_counters(const fwbf_code_s *c);

// status word of bounded waits: kernels OR a non-zero value into it
int read_and_clear_status_i8(cudaStream_t s, int *out);
int read_and_clear_status_f32(cudaStream_t s, int *out);

int launch_quantize(const float *y, int8_t *q, int64_t count, cudaStream_t s);
int launch_decode_i8(const fwbf_code_s *c, const int8_t *y, int64_t n_frames, int max_iter,
                     int alpha_q, int theta_q, uint32_t *out_bits, int32_t *out_iters,
                     cudaStream_t s);
bool cyclic_eligible(const fwbf_code_s *c);
int read_and_clear_status_i8_cyclic(cudaStream_t s, int *out);
bool qc_eligible(const fwbf_code_s *c);
int read_and_clear_status_i8_qc(cudaStream_t s, int *out);
int launch_decode_i8_qc(const fwbf_code_s *c, const int8_t *y, int64_t n_frames, int max_iter, int alpha_q,
                        int theta_q, uint32_t *out_bits, int32_t *out_iters, unsigned long long *counter,
                        cudaStream_t s);
// per-pass parameters of the cyclic decoder (mode 0: fixed, 1: schedule arrays,
// 2: learned network with plain fallback)
struct CyclicModes {
    int mode = 0;
    const int32_t *sched_a = nullptr, *sched_t = nullptr;
    long long sched_stride = 0;
    const unsigned char *mlp = nullptr;
    int k_learn = 0;
    int gate_dv = 0;
    int32_t *out_sched = nullptr;
    float *out_feat = nullptr;
    int feat_passes = 0;
};
int launch_decode_i8_cyclic(const fwbf_code_s *c, const int8_t *y, int64_t n_frames, int max_iter, int alpha_q,
                            int theta_q, uint32_t *out_bits, int32_t *out_iters, unsigned long long *counter,
                            cudaStream_t s, const CyclicModes *modes = nullptr);
int launch_decode_i8_modes(const fwbf_code_s *c, const int8_t *y, int64_t n_frames, int max_iter, int alpha_q,
                           uint32_t *out_bits, int32_t *out_iters, const CyclicModes &modes, cudaStream_t s);
// fwbf_decode's launch with a frame counter the caller provides (cleared here)
int launch_decode_i8_with(const fwbf_code_s *c, const int8_t *y, int64_t n_frames, int max_iter, int alpha_q,
                          int theta_q, uint32_t *out_bits, int32_t *out_iters, unsigned long long *counter,
                          cudaStream_t s);
int launch_decode_i8_noalloc(const fwbf_code_s *c, const int8_t *y, int64_t n_frames, int max_iter,
                             int alpha_q, int theta_q, uint32_t *out_bits, int32_t *out_iters,
                             cudaStream_t s);
int launch_decode_i8_lambda(const fwbf_code_s *c, const int8_t *y, int64_t n_frames, int max_iter, int alpha_q,
                            int lambda, uint32_t *out_bits, int32_t *out_iters, cudaStream_t s);
int launch_decode_f32(const fwbf_code_s *c, const float *y, int64_t n_frames, int max_iter,
                      float alpha, float theta, uint32_t *out_bits, int32_t *out_iters,
                      float *out_E, cudaStream_t s);

}  // namespace fwbf
