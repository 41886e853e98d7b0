// C ABI of libfwbf.so (declared in include/fwbf.h): argument checking, code
// handles, and the launches of the decoding kernels.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <numeric>
#include <string>
#include <unordered_map>
#include <vector>

#include "fwbf.h"
#include "fwbf_internal.h"

namespace fwbf {

static thread_local std::string g_last_error;

void set_error(const std::string &msg) { g_last_error = msg; }

int fail(int status, const std::string &msg) {
    g_last_error = msg;
    return status;
}

int cuda_fail(cudaError_t e, const char *what) {
    g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
    return FWBF_ECUDA;
}

static uint32_t magic_for(uint32_t d) {
    // ceil(2^32 / d); x / d == umulhi(x, magic) for every x < 65536 when d <= 65536
    return d <= 1 ? 0u : (uint32_t)((0x100000000ull + d - 1) / d);
}

// Largest Z dividing gcd(N, M) such that every Z x Z block of H is a sum of
// distinct circulant permutations: each (block row, block column, shift) triple
// then occurs exactly Z times.
static int detect_circulant(int N, int M, int64_t nnz, const int32_t *rows, const int32_t *cols) {
    const int g = std::gcd(N, M);
    std::vector<int> divs;
    for (int d = 1; d <= g; ++d)
        if (g % d == 0) divs.push_back(d);
    std::sort(divs.rbegin(), divs.rend());
    for (int Z : divs) {
        if (Z == 1) return 1;
        if (nnz % Z) continue;
        std::unordered_map<uint64_t, uint32_t> cnt;
        cnt.reserve((size_t)(nnz / Z) * 2 + 16);
        bool ok = true;
        for (int64_t e = 0; e < nnz && ok; ++e) {
            const uint32_t R = rows[e] / Z, C = cols[e] / Z;
            const uint32_t t = (uint32_t)(((cols[e] % Z) - (rows[e] % Z) + Z) % Z);
            const uint64_t key = ((uint64_t)R << 32) | ((uint64_t)C << 16) | t;
            if (++cnt[key] > (uint32_t)Z) ok = false;
        }
        if (!ok) continue;
        for (auto &kv : cnt)
            if (kv.second != (uint32_t)Z) {
                ok = false;
                break;
            }
        if (ok) return Z;
    }
    return 1;
}

}  // namespace fwbf

using namespace fwbf;

namespace fwbf {

int acquire_counter(const fwbf_code_s *c, cudaStream_t s, CounterLease *out) {
    *out = CounterLease{};
    {
        std::lock_guard<std::mutex> lock(c->counters.mu);
        for (const auto &kv : c->counters.by_stream)
            if (kv.first == s) out->ptr = kv.second;
        if (!out->ptr) {
            cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
            if (cudaStreamIsCapturing(s, &st) != cudaSuccess) {
                cudaGetLastError();
                st = cudaStreamCaptureStatusActive;  // unknown: take the capturable path
            }
            if (st == cudaStreamCaptureStatusNone) {
                unsigned long long *p = nullptr;
                cudaError_t e = cudaMalloc(reinterpret_cast<void **>(&p), sizeof(unsigned long long));
                if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(frame counter)");
                c->counters.by_stream.emplace_back(s, p);
                out->ptr = p;
            }
        }
    }
    if (!out->ptr) {
        cudaError_t e = cudaMallocAsync(reinterpret_cast<void **>(&out->ptr), sizeof(unsigned long long), s);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMallocAsync(frame counter)");
        out->owned = true;
    }
    cudaError_t e = cudaMemsetAsync(out->ptr, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) {
        release_counter(*out, s);
        return cuda_fail(e, "cudaMemsetAsync(frame counter)");
    }
    return FWBF_OK;
}

int release_counter(const CounterLease &lease, cudaStream_t s) {
    if (!lease.owned) return FWBF_OK;
    cudaError_t e = cudaFreeAsync(lease.ptr, s);
    return e == cudaSuccess ? FWBF_OK : cuda_fail(e, "cudaFreeAsync(frame counter)");
}

void free_counters(const fwbf_code_s *c) {
    std::lock_guard<std::mutex> lock(c->counters.mu);
    for (const auto &kv : c->counters.by_stream) cudaFree(kv.second);
    c->counters.by_stream.clear();
}

}  // namespace fwbf

extern "C" {

const char *fwbf_strerror(int status) {
    switch (status) {
        case FWBF_OK: return "ok";
        case FWBF_EINVAL: return "invalid argument";
        case FWBF_ENOMEM: return "out of memory";
        case FWBF_ECUDA: return "CUDA runtime error";
        case FWBF_EUNSUPPORTED: return "unsupported input";
        case FWBF_ETIMEOUT: return "a kernel gave up a bounded wait";
        default: return "unknown status";
    }
}

const char *fwbf_last_error(void) { return g_last_error.c_str(); }

int fwbf_code_create(int32_t N, int32_t M, int64_t nnz, const int32_t *row_idx, const int32_t *col_idx,
                     int32_t seg_len, fwbf_code *out) {
    TraceRange trace("fwbf_code_create");
    if (!out) return fail(FWBF_EINVAL, "out is NULL");
    *out = nullptr;
    if (N < 1 || N > 65535 || M < 1 || M > 65535)
        return fail(FWBF_EINVAL, "N and M must be in [1, 65535]");
    if (nnz < 1 || nnz > (int64_t)N * M) return fail(FWBF_EINVAL, "nnz out of range");
    if (!row_idx || !col_idx) return fail(FWBF_EINVAL, "row_idx/col_idx is NULL");
    if (seg_len < 1 || seg_len > N) return fail(FWBF_EINVAL, "seg_len must be in [1, N]");

    std::vector<int32_t> rw(M, 0), cw(N, 0);
    std::vector<uint32_t> keys((size_t)nnz);
    for (int64_t e = 0; e < nnz; ++e) {
        if (row_idx[e] < 0 || row_idx[e] >= M || col_idx[e] < 0 || col_idx[e] >= N)
            return fail(FWBF_EINVAL, "index out of range at entry " + std::to_string(e));
        rw[row_idx[e]]++;
        cw[col_idx[e]]++;
        keys[e] = ((uint32_t)row_idx[e] << 16) | (uint32_t)col_idx[e];
    }
    std::sort(keys.begin(), keys.end());
    if (std::adjacent_find(keys.begin(), keys.end()) != keys.end())
        return fail(FWBF_EINVAL, "duplicate entry in H");
    int dc_max = 0, dv_max = 0;
    for (int m = 0; m < M; ++m) {
        if (rw[m] < 2) return fail(FWBF_EUNSUPPORTED, "check " + std::to_string(m) + " has fewer than two bits");
        dc_max = std::max(dc_max, rw[m]);
    }
    for (int n = 0; n < N; ++n) dv_max = std::max(dv_max, cw[n]);
    if (dc_max > 255 || dv_max > 255) return fail(FWBF_EUNSUPPORTED, "row or column weight above 255");

    // RC constraint (Sec. II): the most bits two checks share, by counting for
    // each check m the later checks met through each of its bits
    int max_overlap = 0;
    {
        std::vector<int32_t> cptr(N + 1, 0), crow((size_t)nnz), rptr(M + 1, 0), rcol((size_t)nnz);
        for (int n = 0; n < N; ++n) cptr[n + 1] = cptr[n] + cw[n];
        for (int m = 0; m < M; ++m) rptr[m + 1] = rptr[m] + rw[m];
        std::vector<int32_t> cf(cptr.begin(), cptr.end() - 1), rf(rptr.begin(), rptr.end() - 1);
        for (uint32_t k : keys) {  // sorted by (row, column)
            const int m = (int)(k >> 16), n = (int)(k & 0xffffu);
            crow[cf[n]++] = m;
            rcol[rf[m]++] = n;
        }
        std::vector<int32_t> cnt(M, 0), touched;
        for (int m = 0; m < M; ++m) {
            touched.clear();
            for (int32_t e = rptr[m]; e < rptr[m + 1]; ++e) {
                const int n = rcol[e];
                for (int32_t f = cptr[n]; f < cptr[n + 1]; ++f) {
                    const int r = crow[f];
                    if (r <= m) continue;
                    if (cnt[r]++ == 0) touched.push_back(r);
                    max_overlap = std::max(max_overlap, cnt[r]);
                }
            }
            for (int r : touched) cnt[r] = 0;
        }
    }

    const int Z = detect_circulant(N, M, nnz, row_idx, col_idx);
    const int MB = M / Z, NB = N / Z;
    // circulant entries per block row / block column
    std::vector<std::vector<uint32_t>> rows_of(MB), cols_of(NB);
    {
        std::vector<uint64_t> trip;
        trip.reserve((size_t)(nnz / Z));
        for (int64_t e = 0; e < nnz; ++e) {
            if (Z > 1 && row_idx[e] % Z != 0) continue;  // one representative per circulant
            const uint32_t R = row_idx[e] / Z, C = col_idx[e] / Z;
            const uint32_t t = (uint32_t)((col_idx[e] % Z - row_idx[e] % Z + Z) % Z);
            trip.push_back(((uint64_t)R << 32) | ((uint64_t)C << 16) | t);
        }
        std::sort(trip.begin(), trip.end());
        for (uint64_t k : trip) {
            const uint32_t R = (uint32_t)(k >> 32), C = (uint32_t)(k >> 16) & 0xffffu, t = (uint32_t)k & 0xffffu;
            rows_of[R].push_back((C << 16) | t);
            cols_of[C].push_back((R << 16) | ((Z - t) % Z));
        }
        for (auto &v : cols_of) std::sort(v.begin(), v.end());
    }
    std::vector<uint32_t> blob;
    auto fill = [&](const std::vector<std::vector<uint32_t>> &lists, uint32_t &ptr_off, uint32_t &ent_off) {
        ptr_off = (uint32_t)blob.size();
        uint32_t acc = 0;
        blob.push_back(0);
        for (auto &l : lists) {
            acc += (uint32_t)l.size();
            blob.push_back(acc);
        }
        ent_off = (uint32_t)blob.size();
        for (auto &l : lists) blob.insert(blob.end(), l.begin(), l.end());
    };
    fwbf_code_s *c = new (std::nothrow) fwbf_code_s();
    if (!c) return fail(FWBF_ENOMEM, "host allocation");
    fill(rows_of, c->rptr_off, c->rent_off);
    fill(cols_of, c->cptr_off, c->cent_off);
    while (blob.size() % 4) blob.push_back(0);

    c->N = N;
    c->M = M;
    c->nnz = nnz;
    c->Z = Z;
    c->MB = MB;
    c->NB = NB;
    c->dv_max = dv_max;
    c->dc_max = dc_max;
    c->max_row_overlap = max_overlap;
    c->p = seg_len;
    c->B = (N + seg_len - 1) / seg_len;
    c->p_magic = magic_for((uint32_t)seg_len);
    c->z_magic = magic_for((uint32_t)Z);
    c->table_words = (uint32_t)blob.size();

    cudaError_t e = cudaGetDevice(&c->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device);
    if (e == cudaSuccess)
        e = cudaDeviceGetAttribute(&c->smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->device);
    if (e != cudaSuccess) {
        delete c;
        return cuda_fail(e, "device query");
    }
    e = cudaMalloc(reinterpret_cast<void **>(&c->d_table), blob.size() * sizeof(uint32_t));
    if (e != cudaSuccess) {
        delete c;
        return e == cudaErrorMemoryAllocation ? fail(FWBF_ENOMEM, "cudaMalloc(table)") : cuda_fail(e, "cudaMalloc");
    }
    e = cudaMemcpy(c->d_table, blob.data(), blob.size() * sizeof(uint32_t), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(c->d_table);
        delete c;
        return cuda_fail(e, "cudaMemcpy(table)");
    }
    *out = c;
    return FWBF_OK;
}

int fwbf_destroy(fwbf_code c) {
    if (!c) return FWBF_OK;
    cudaError_t e = cudaDeviceSynchronize();
    free_counters(c);
    cudaError_t e2 = cudaFree(c->d_table);
    delete c;
    if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceSynchronize");
    if (e2 != cudaSuccess) return cuda_fail(e2, "cudaFree");
    return FWBF_OK;
}

int fwbf_code_query(fwbf_code c, fwbf_code_info *out) {
    if (!c || !out) return fail(FWBF_EINVAL, "NULL argument");
    out->N = c->N;
    out->M = c->M;
    out->nnz = c->nnz;
    out->Z = c->Z;
    out->dv_max = c->dv_max;
    out->dc_max = c->dc_max;
    out->seg_len = c->p;
    out->n_blocks = c->B;
    out->table_bytes = (int64_t)c->table_words * 4;
    out->max_row_overlap = c->max_row_overlap;
    out->decoder = cyclic_eligible(c) ? FWBF_DECODER_CYCLIC : qc_eligible(c) ? FWBF_DECODER_QC : FWBF_DECODER_LIST;
    return FWBF_OK;
}

int fwbf_quantize(const float *y, int8_t *q, int64_t count, void *stream) {
    if (count < 0) return fail(FWBF_EINVAL, "count < 0");
    if (count > 0 && (!y || !q)) return fail(FWBF_EINVAL, "NULL buffer");
    return launch_quantize(y, q, count, static_cast<cudaStream_t>(stream));
}

static int check_decode_args(fwbf_code c, const void *y, int64_t n_frames, int32_t max_iter, float alpha,
                             const void *out_bits, const void *out_iters) {
    if (!c) return fail(FWBF_EINVAL, "code is NULL");
    if (n_frames < 0) return fail(FWBF_EINVAL, "n_frames < 0");
    if (max_iter < 1) return fail(FWBF_EINVAL, "max_iter must be >= 1");
    if (!(alpha >= 0.0f && alpha <= 64.0f)) return fail(FWBF_EINVAL, "alpha must be in [0, 64]");
    if (n_frames > 0 && (!y || !out_bits || !out_iters)) return fail(FWBF_EINVAL, "NULL buffer");
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev != c->device) return fail(FWBF_EINVAL, "code was created on another device");
    return FWBF_OK;
}

int fwbf_decode(fwbf_code c, const int8_t *y, int64_t n_frames, int32_t max_iter, float alpha,
                uint32_t *out_bits, int32_t *out_iters, void *stream) {
    TraceRange trace("fwbf_decode");
    int rc = check_decode_args(c, y, n_frames, max_iter, alpha, out_bits, out_iters);
    if (rc) return rc;
    if (reinterpret_cast<uintptr_t>(y) % 16) return fail(FWBF_EINVAL, "y must be 16-byte aligned");
    if (n_frames == 0) return FWBF_OK;
    const int alpha_q = (int)nearbyint((double)alpha * 256.0);
    return launch_decode_i8(c, y, n_frames, max_iter, alpha_q, 0, out_bits, out_iters,
                            static_cast<cudaStream_t>(stream));
}

int fwbf_decode_noalloc(fwbf_code c, const int8_t *y, int64_t n_frames, int32_t max_iter, float alpha,
                        uint32_t *out_bits, int32_t *out_iters, void *stream) {
    TraceRange trace("fwbf_decode_noalloc");
    int rc = check_decode_args(c, y, n_frames, max_iter, alpha, out_bits, out_iters);
    if (rc) return rc;
    if (reinterpret_cast<uintptr_t>(y) % 16) return fail(FWBF_EINVAL, "y must be 16-byte aligned");
    if (n_frames == 0) return FWBF_OK;
    const int alpha_q = (int)nearbyint((double)alpha * 256.0);
    return launch_decode_i8_noalloc(c, y, n_frames, max_iter, alpha_q, 0, out_bits, out_iters,
                                    static_cast<cudaStream_t>(stream));
}

int fwbf_decode_sched(fwbf_code c, const int8_t *y, int64_t n_frames, int32_t max_iter, const int32_t *alpha_q,
                      const int32_t *theta_q, int64_t sched_stride, uint32_t *out_bits, int32_t *out_iters,
                      float *out_feat, int32_t feat_passes, void *stream) {
    TraceRange trace("fwbf_decode_sched");
    int rc = check_decode_args(c, y, n_frames, max_iter, 1.0f, out_bits, out_iters);
    if (rc) return rc;
    if (reinterpret_cast<uintptr_t>(y) % 16) return fail(FWBF_EINVAL, "y must be 16-byte aligned");
    if (n_frames > 0 && (!alpha_q || !theta_q)) return fail(FWBF_EINVAL, "schedule is NULL");
    if (sched_stride != 0 && sched_stride < max_iter) return fail(FWBF_EINVAL, "sched_stride < max_iter");
    if (out_feat && feat_passes < 1) return fail(FWBF_EINVAL, "feat_passes < 1");
    if (n_frames == 0) return FWBF_OK;
    CyclicModes m;
    m.mode = 1;
    m.sched_a = alpha_q;
    m.sched_t = theta_q;
    m.sched_stride = sched_stride;
    m.out_feat = out_feat;
    m.feat_passes = out_feat ? feat_passes : 0;
    return launch_decode_i8_modes(c, y, n_frames, max_iter, 0, out_bits, out_iters, m,
                                  static_cast<cudaStream_t>(stream));
}

int fwbf_decode_learned(fwbf_code c, const int8_t *y, int64_t n_frames, int32_t max_iter, int32_t k_learn,
                        int32_t gate_dv, float alpha_fallback, const void *mlp, uint32_t *out_bits, int32_t *out_iters,
                        int32_t *out_sched, float *out_feat, int32_t feat_passes, void *stream) {
    TraceRange trace("fwbf_decode_learned");
    int rc = check_decode_args(c, y, n_frames, max_iter, alpha_fallback, out_bits, out_iters);
    if (rc) return rc;
    if (reinterpret_cast<uintptr_t>(y) % 16) return fail(FWBF_EINVAL, "y must be 16-byte aligned");
    if (k_learn < 1) return fail(FWBF_EINVAL, "k_learn must be >= 1");
    if (gate_dv < 0 || gate_dv > 65535) return fail(FWBF_EINVAL, "gate_dv must be in [0, 65535]");
    if (!mlp || reinterpret_cast<uintptr_t>(mlp) % 16) return fail(FWBF_EINVAL, "mlp blob NULL or unaligned");
    if (out_feat && feat_passes < 1) return fail(FWBF_EINVAL, "feat_passes < 1");
    if (n_frames == 0) return FWBF_OK;
    CyclicModes m;
    m.mode = 2;
    m.mlp = static_cast<const unsigned char *>(mlp);
    m.k_learn = k_learn;
    m.gate_dv = gate_dv;
    m.out_sched = out_sched;
    m.out_feat = out_feat;
    m.feat_passes = out_feat ? feat_passes : 0;
    const int aq = (int)nearbyint((double)alpha_fallback * 256.0);
    return launch_decode_i8_modes(c, y, n_frames, max_iter, aq, out_bits, out_iters, m,
                                  static_cast<cudaStream_t>(stream));
}

int fwbf_decode_host(fwbf_code c, const float *y_host, int64_t n_frames, int32_t max_iter, float alpha,
                     uint32_t *bits_host, int32_t *iters_host, int64_t chunk_frames, void *stream) {
    TraceRange trace("fwbf_decode_host");
    int rc = check_decode_args(c, y_host, n_frames, max_iter, alpha, bits_host, iters_host);
    if (rc) return rc;
    if (chunk_frames < 1) return fail(FWBF_EINVAL, "chunk_frames must be >= 1");
    if (n_frames == 0) return FWBF_OK;
    cudaStream_t caller = static_cast<cudaStream_t>(stream);
    const int64_t N = c->N, words = (N + 31) / 32;
    const int64_t chunk = chunk_frames < n_frames ? chunk_frames : n_frames;
    // per buffer: float y | int8 q (16-byte aligned) | bits | iters | frame counter
    // (the pipeline's streams are its own, so are their counters)
    const size_t y_bytes = (size_t)(chunk * N) * 4, q_off = (y_bytes + 255) & ~(size_t)255;
    const size_t b_off = (q_off + (size_t)(chunk * N) + 255) & ~(size_t)255;
    const size_t i_off = (b_off + (size_t)(chunk * words) * 4 + 255) & ~(size_t)255;
    const size_t c_off = (i_off + (size_t)chunk * 4 + 255) & ~(size_t)255;
    const size_t buf_bytes = c_off + 256;
    char *dev = nullptr;
    cudaStream_t st[2] = {nullptr, nullptr};
    cudaEvent_t ev_start = nullptr, ev_done[2] = {nullptr, nullptr};
    cudaError_t e = cudaMallocAsync(reinterpret_cast<void **>(&dev), 2 * buf_bytes, caller);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMallocAsync(host pipeline buffers)");
    for (int b = 0; b < 2 && e == cudaSuccess; ++b) {
        e = cudaStreamCreateWithFlags(&st[b], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev_done[b], cudaEventDisableTiming);
    }
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev_start, cudaEventDisableTiming);
    // the pipeline starts after the caller's earlier work (and the allocation)
    if (e == cudaSuccess) e = cudaEventRecord(ev_start, caller);
    for (int b = 0; b < 2 && e == cudaSuccess; ++b) e = cudaStreamWaitEvent(st[b], ev_start, 0);
    int64_t i = 0;
    for (int64_t f0 = 0; f0 < n_frames && e == cudaSuccess && rc == 0; f0 += chunk, ++i) {
        const int b = (int)(i & 1);
        const int64_t nf = (n_frames - f0) < chunk ? (n_frames - f0) : chunk;
        char *base = dev + (size_t)b * buf_bytes;
        float *yd = reinterpret_cast<float *>(base);
        int8_t *qd = reinterpret_cast<int8_t *>(base + q_off);
        uint32_t *bd = reinterpret_cast<uint32_t *>(base + b_off);
        int32_t *id = reinterpret_cast<int32_t *>(base + i_off);
        unsigned long long *cd = reinterpret_cast<unsigned long long *>(base + c_off);
        e = cudaMemcpyAsync(yd, y_host + f0 * N, (size_t)(nf * N) * 4, cudaMemcpyHostToDevice, st[b]);
        if (e != cudaSuccess) break;
        rc = launch_quantize(yd, qd, nf * N, st[b]);
        if (rc) break;
        rc = launch_decode_i8_with(c, qd, nf, max_iter, (int)nearbyint((double)alpha * 256.0), 0, bd, id, cd, st[b]);
        if (rc) break;
        e = cudaMemcpyAsync(bits_host + f0 * words, bd, (size_t)(nf * words) * 4, cudaMemcpyDeviceToHost, st[b]);
        if (e == cudaSuccess) e = cudaMemcpyAsync(iters_host + f0, id, (size_t)nf * 4, cudaMemcpyDeviceToHost, st[b]);
    }
    // join both streams back into the caller's stream, then release
    for (int b = 0; b < 2; ++b) {
        if (st[b] && ev_done[b]) {
            cudaEventRecord(ev_done[b], st[b]);
            cudaStreamWaitEvent(caller, ev_done[b], 0);
        }
    }
    cudaFreeAsync(dev, caller);
    for (int b = 0; b < 2; ++b) {
        if (ev_done[b]) cudaEventDestroy(ev_done[b]);
        if (st[b]) cudaStreamDestroy(st[b]);
    }
    if (ev_start) cudaEventDestroy(ev_start);
    if (rc) return rc;
    return e == cudaSuccess ? FWBF_OK : cuda_fail(e, "host pipeline");
}

int fwbf_decode_lambda(fwbf_code c, const int8_t *y, int64_t n_frames, int32_t max_iter, float alpha,
                       int32_t lambda, uint32_t *out_bits, int32_t *out_iters, void *stream) {
    TraceRange trace("fwbf_decode_lambda");
    int rc = check_decode_args(c, y, n_frames, max_iter, alpha, out_bits, out_iters);
    if (rc) return rc;
    if (reinterpret_cast<uintptr_t>(y) % 16) return fail(FWBF_EINVAL, "y must be 16-byte aligned");
    if (lambda < 1) return fail(FWBF_EINVAL, "lambda must be >= 1");
    if (lambda > c->N) lambda = c->N;
    if (n_frames == 0) return FWBF_OK;
    const int alpha_q = (int)nearbyint((double)alpha * 256.0);
    return launch_decode_i8_lambda(c, y, n_frames, max_iter, alpha_q, lambda, out_bits, out_iters,
                                   static_cast<cudaStream_t>(stream));
}

int fwbf_decode_f32(fwbf_code c, const float *y, int64_t n_frames, int32_t max_iter, float alpha,
                    uint32_t *out_bits, int32_t *out_iters, void *stream) {
    TraceRange trace("fwbf_decode_f32");
    int rc = check_decode_args(c, y, n_frames, max_iter, alpha, out_bits, out_iters);
    if (rc) return rc;
    if (reinterpret_cast<uintptr_t>(y) % 4) return fail(FWBF_EINVAL, "y must be 4-byte aligned");
    if (n_frames == 0) return FWBF_OK;
    return launch_decode_f32(c, y, n_frames, max_iter, alpha, 0.0f, out_bits, out_iters, nullptr,
                             static_cast<cudaStream_t>(stream));
}

int fwbf_metric_f32(fwbf_code c, const float *y, int64_t n_frames, float alpha, float *out_E, void *stream) {
    if (!c) return fail(FWBF_EINVAL, "code is NULL");
    if (n_frames < 0) return fail(FWBF_EINVAL, "n_frames < 0");
    if (!(alpha >= 0.0f && alpha <= 64.0f)) return fail(FWBF_EINVAL, "alpha must be in [0, 64]");
    if (n_frames > 0 && (!y || !out_E)) return fail(FWBF_EINVAL, "NULL buffer");
    if (reinterpret_cast<uintptr_t>(y) % 4) return fail(FWBF_EINVAL, "y must be 4-byte aligned");
    if (n_frames == 0) return FWBF_OK;
    return launch_decode_f32(c, y, n_frames, 1, alpha, 0.0f, nullptr, nullptr, out_E,
                             static_cast<cudaStream_t>(stream));
}

int fwbf_last_status(void *stream) {
    int a = 0, b = 0, c = 0, d = 0;
    int rc = read_and_clear_status_i8(static_cast<cudaStream_t>(stream), &a);
    if (rc) return rc;
    rc = read_and_clear_status_f32(static_cast<cudaStream_t>(stream), &b);
    if (rc) return rc;
    rc = read_and_clear_status_i8_cyclic(static_cast<cudaStream_t>(stream), &c);
    if (rc) return rc;
    rc = read_and_clear_status_i8_qc(static_cast<cudaStream_t>(stream), &d);
    if (rc) return rc;
    return (a || b || c || d) ? fail(FWBF_ETIMEOUT, "a kernel gave up waiting for its table copy") : FWBF_OK;
}

}  // extern "C"
