// Internal declarations shared by the C-ABI layer and the kernel translation
// units of libfwbf.so.  Not part of the public interface (see include/fwbf.h).
#pragma once

#include <cuda_runtime.h>

#include "fwbf.h"
#include <stdint.h>

#include <string>

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
};

namespace fwbf {

// thread-local detail message for fwbf_last_error()
void set_error(const std::string &msg);
int fail(int status, const std::string &msg);
int cuda_fail(cudaError_t e, const char *what);

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
int launch_decode_i8_noalloc(const fwbf_code_s *c, const int8_t *y, int64_t n_frames, int max_iter,
                             int alpha_q, int theta_q, uint32_t *out_bits, int32_t *out_iters,
                             cudaStream_t s);
int launch_decode_i8_lambda(const fwbf_code_s *c, const int8_t *y, int64_t n_frames, int max_iter, int alpha_q,
                            int lambda, uint32_t *out_bits, int32_t *out_iters, cudaStream_t s);
int launch_decode_f32(const fwbf_code_s *c, const float *y, int64_t n_frames, int max_iter,
                      float alpha, float theta, uint32_t *out_bits, int32_t *out_iters,
                      float *out_E, cudaStream_t s);

}  // namespace fwbf
