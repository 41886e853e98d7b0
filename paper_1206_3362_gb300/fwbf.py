"""ctypes binding of libfwbf.so with the C ABI's entry-point names.

Argument marshalling only: every step of decoding runs in the library's CUDA
kernels.  Tensors are PyTorch CUDA tensors (used for device memory and
streams); the calls pass ``tensor.data_ptr()`` and the current stream.  There
is no fallback: if the library is missing or a call fails, an exception is
raised.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libfwbf.so")

FWBF_OK = 0
FWBF_EINVAL = -1
FWBF_ENOMEM = -2
FWBF_ECUDA = -3
FWBF_EUNSUPPORTED = -4
FWBF_ETIMEOUT = -5

# CodeInfo.decoder: the kernel fwbf_decode runs for the code
FWBF_DECODER_LIST = 0
FWBF_DECODER_CYCLIC = 1
FWBF_DECODER_QC = 2


class FwbfError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{msg} (status {status})")
        self.status = status


class BatchJobInfo(ctypes.Structure):
    _fields_ = [("decoder", ctypes.c_int32), ("warps_per_frame", ctypes.c_int32),
                ("frames_per_cta", ctypes.c_int32), ("grouped", ctypes.c_int32)]


class BatchJob(ctypes.Structure):
    _fields_ = [("code", ctypes.c_void_p), ("y", ctypes.c_void_p), ("n_frames", ctypes.c_int64),
                ("max_iter", ctypes.c_int32), ("alpha", ctypes.c_float), ("out_bits", ctypes.c_void_p),
                ("out_iters", ctypes.c_void_p), ("mlp", ctypes.c_void_p), ("k_learn", ctypes.c_int32),
                ("gate_dv", ctypes.c_int32)]


class CodeInfo(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int32), ("M", ctypes.c_int32), ("nnz", ctypes.c_int64),
                ("Z", ctypes.c_int32), ("dv_max", ctypes.c_int32), ("dc_max", ctypes.c_int32),
                ("seg_len", ctypes.c_int32), ("n_blocks", ctypes.c_int32),
                ("table_bytes", ctypes.c_int64), ("max_row_overlap", ctypes.c_int32), ("decoder", ctypes.c_int32)]


_lib = None


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    """Loads libfwbf.so (built by ``__graft_entry__.build()``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with __graft_entry__.build()")
    lib = ctypes.CDLL(path)
    P, i32, i64, f32 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_float
    sig = {
        "fwbf_code_create": ([i32, i32, i64, P, P, i32, ctypes.POINTER(P)], ctypes.c_int),
        "fwbf_destroy": ([P], ctypes.c_int),
        "fwbf_code_query": ([P, ctypes.POINTER(CodeInfo)], ctypes.c_int),
        "fwbf_quantize": ([P, P, i64, P], ctypes.c_int),
        "fwbf_decode": ([P, P, i64, i32, f32, P, P, P], ctypes.c_int),
        "fwbf_decode_noalloc": ([P, P, i64, i32, f32, P, P, P], ctypes.c_int),
        "fwbf_decode_f32": ([P, P, i64, i32, f32, P, P, P], ctypes.c_int),
        "fwbf_decode_lambda": ([P, P, i64, i32, f32, i32, P, P, P], ctypes.c_int),
        "fwbf_decode_host": ([P, P, i64, i32, f32, P, P, i64, P], ctypes.c_int),
        "fwbf_peak_int_issue": ([ctypes.c_int, ctypes.c_double, P, P, P], ctypes.c_int),
        "fwbf_probe_bounded_wait": ([ctypes.c_uint32, P, P], ctypes.c_int),
        "fwbf_metric_f32": ([P, P, i64, f32, P, P], ctypes.c_int),
        "fwbf_decode_sched": ([P, P, i64, i32, P, P, i64, P, P, P, i32, P], ctypes.c_int),
        "fwbf_decode_learned": ([P, P, i64, i32, i32, i32, f32, P, P, P, P, P, i32, P], ctypes.c_int),
        "fwbf_mlp_pack": ([P, P, P], ctypes.c_int),
        "fwbf_mlp_forward": ([P, P, i64, P, P], ctypes.c_int),
        "fwbf_mlp_grad": ([P, P, P, i64, i64, P, P, P], ctypes.c_int),
        "fwbf_mlp_adam": ([P, P, P, P, P, i64, f32, f32, f32, f32, P], ctypes.c_int),
        "fwbf_batch_create": ([P, i32, i32, i32, ctypes.POINTER(P)], ctypes.c_int),
        "fwbf_batch_query": ([P, i32, ctypes.POINTER(BatchJobInfo)], ctypes.c_int),
        "fwbf_decode_batch": ([P, P], ctypes.c_int),
        "fwbf_batch_status": ([P], ctypes.c_int),
        "fwbf_batch_destroy": ([P], ctypes.c_int),
        "fwbf_last_status": ([P], ctypes.c_int),
        "fwbf_strerror": ([ctypes.c_int], ctypes.c_char_p),
        "fwbf_last_error": ([], ctypes.c_char_p),
    }
    for name, (argt, rest) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = argt
        fn.restype = rest
    _lib = lib
    return lib


def _check(rc: int):
    if rc != FWBF_OK:
        lib = load_library()
        raise FwbfError(rc, f"{lib.fwbf_strerror(rc).decode()}: {lib.fwbf_last_error().decode()}")


def _stream(stream):
    if stream is None:
        import torch

        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _dev(t, dtype, name):
    import torch

    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return ctypes.c_void_p(t.data_ptr())


# ---------------------------------------------------------------------------
# entry points (same names as the C ABI)
# ---------------------------------------------------------------------------

def fwbf_code_create(N: int, M: int, row_idx, col_idx, seg_len: int) -> ctypes.c_void_p:
    lib = load_library()
    rows = np.ascontiguousarray(row_idx, dtype=np.int32)
    cols = np.ascontiguousarray(col_idx, dtype=np.int32)
    if rows.shape != cols.shape:
        raise ValueError("row_idx and col_idx differ in length")
    h = ctypes.c_void_p()
    _check(lib.fwbf_code_create(int(N), int(M), rows.size, rows.ctypes.data_as(ctypes.c_void_p),
                                cols.ctypes.data_as(ctypes.c_void_p), int(seg_len), ctypes.byref(h)))
    return h


def fwbf_destroy(code) -> None:
    _check(load_library().fwbf_destroy(code))


def fwbf_code_query(code) -> CodeInfo:
    info = CodeInfo()
    _check(load_library().fwbf_code_query(code, ctypes.byref(info)))
    return info


def fwbf_quantize(y, q, stream=None) -> None:
    import torch

    if y.numel() != q.numel():
        raise ValueError("y and q differ in size")
    _check(load_library().fwbf_quantize(_dev(y, torch.float32, "y"), _dev(q, torch.int8, "q"), y.numel(),
                                        _stream(stream)))


def _frames(y, N):
    if y.dim() != 2 or y.shape[1] != N:
        raise ValueError(f"y must have shape [n_frames, {N}]")
    return y.shape[0]


def _need(t, n: int, name: str) -> None:
    """t (a tensor, or None for an absent optional output) must hold at least
    n elements: the kernels read or write exactly n, and nothing below the C
    ABI can check the size behind a pointer."""
    if t is not None and t.numel() < n:
        raise ValueError(f"{name} holds {t.numel()} elements, needs {n}")


def _outputs(F: int, N: int, out_bits, out_iters) -> None:
    _need(out_bits, F * ((N + 31) // 32), "out_bits")
    _need(out_iters, F, "out_iters")


def _feat(F: int, out_feat) -> int:
    """Passes recorded by an optional out_feat [n_frames][P][8]."""
    if out_feat is None:
        return 0
    if out_feat.dim() != 3 or out_feat.shape[0] < F or out_feat.shape[2] != MLP_IN:
        raise ValueError(f"out_feat must have shape [{F}, passes, {MLP_IN}]")
    return out_feat.shape[1]


def fwbf_decode(code, y, max_iter: int, alpha: float, out_bits, out_iters, stream=None) -> None:
    import torch

    info = fwbf_code_query(code)
    F = _frames(y, info.N)
    _outputs(F, info.N, out_bits, out_iters)
    _check(load_library().fwbf_decode(code, _dev(y, torch.int8, "y"), F, int(max_iter), float(alpha),
                                      _dev(out_bits, torch.int32, "out_bits"),
                                      _dev(out_iters, torch.int32, "out_iters"), _stream(stream)))


def fwbf_decode_noalloc(code, y, max_iter: int, alpha: float, out_bits, out_iters, stream=None) -> None:
    """fwbf_decode for callers that cannot allocate device memory: the frame
    counter lives in a fixed array of the library (see include/fwbf.h); calls
    overlapping on the GPU must not share it."""
    import torch

    info = fwbf_code_query(code)
    F = _frames(y, info.N)
    _outputs(F, info.N, out_bits, out_iters)
    _check(load_library().fwbf_decode_noalloc(code, _dev(y, torch.int8, "y"), F, int(max_iter), float(alpha),
                                              _dev(out_bits, torch.int32, "out_bits"),
                                              _dev(out_iters, torch.int32, "out_iters"), _stream(stream)))


def _host(t, dtype, name):
    import torch

    if not isinstance(t, torch.Tensor) or t.is_cuda:
        raise TypeError(f"{name} must be a host tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return ctypes.c_void_p(t.data_ptr())


def fwbf_decode_host(code, y_host, max_iter: int, alpha: float, bits_host, iters_host,
                     chunk_frames: int = 1 << 15, stream=None) -> None:
    """Host float frames -> host decisions, pipelined in chunks over two
    streams (pinned host tensors give overlapped copies)."""
    import torch

    info = fwbf_code_query(code)
    F = _frames(y_host, info.N)
    _outputs(F, info.N, bits_host, iters_host)
    _check(load_library().fwbf_decode_host(code, _host(y_host, torch.float32, "y_host"), F, int(max_iter),
                                           float(alpha), _host(bits_host, torch.int32, "bits_host"),
                                           _host(iters_host, torch.int32, "iters_host"), int(chunk_frames),
                                           _stream(stream)))


def fwbf_peak_int_issue(mix: int, ms: float = 200.0, stream=None) -> float:
    """Measured integer issue rate of the current GPU, lane-operations per
    second (mix 0: logic ops only; mix 1: logic ops and multiply-adds)."""
    r = ctypes.c_double(0.0)
    _check(load_library().fwbf_peak_int_issue(int(mix), float(ms), _stream(stream), ctypes.byref(r), None))
    return r.value


def fwbf_probe_bounded_wait(expect_bytes: int, stream=None) -> int:
    """Runs the decoders' bounded table-staging wait on a barrier expecting
    expect_bytes that no copy delivers; returns FWBF_OK or FWBF_ETIMEOUT."""
    st = ctypes.c_int(-1)
    _check(load_library().fwbf_probe_bounded_wait(int(expect_bytes), _stream(stream), ctypes.byref(st)))
    return st.value


def fwbf_decode_lambda(code, y, max_iter: int, alpha: float, lam: int, out_bits, out_iters, stream=None) -> None:
    """lambda-largest selection per pass with the IMWBF metric (comparison rule)."""
    import torch

    info = fwbf_code_query(code)
    F = _frames(y, info.N)
    _outputs(F, info.N, out_bits, out_iters)
    _check(load_library().fwbf_decode_lambda(code, _dev(y, torch.int8, "y"), F, int(max_iter), float(alpha),
                                             int(lam), _dev(out_bits, torch.int32, "out_bits"),
                                             _dev(out_iters, torch.int32, "out_iters"), _stream(stream)))


def fwbf_decode_f32(code, y, max_iter: int, alpha: float, out_bits, out_iters, stream=None) -> None:
    import torch

    info = fwbf_code_query(code)
    F = _frames(y, info.N)
    _outputs(F, info.N, out_bits, out_iters)
    _check(load_library().fwbf_decode_f32(code, _dev(y, torch.float32, "y"), F, int(max_iter), float(alpha),
                                          _dev(out_bits, torch.int32, "out_bits"),
                                          _dev(out_iters, torch.int32, "out_iters"), _stream(stream)))


def fwbf_metric_f32(code, y, alpha: float, out_E, stream=None) -> None:
    import torch

    info = fwbf_code_query(code)
    F = _frames(y, info.N)
    _need(out_E, F * info.N, "out_E")
    _check(load_library().fwbf_metric_f32(code, _dev(y, torch.float32, "y"), F, float(alpha),
                                          _dev(out_E, torch.float32, "out_E"), _stream(stream)))


MLP_IN, MLP_HIDDEN, MLP_OUT, MLP_PARAMS, MLP_BLOB_BYTES = 8, 64, 2, 4866, 10000


def _opt(t, dtype, name):
    return None if t is None else _dev(t, dtype, name)


def fwbf_decode_sched(code, y, max_iter: int, alpha_q, theta_q, out_bits, out_iters, out_feat=None,
                      stream=None) -> None:
    """Per-pass schedule: alpha_q/theta_q int32 CUDA tensors [n_frames][max_iter]
    (or [max_iter], shared by all frames); out_feat float32 [n_frames][P][8]."""
    import torch

    info = fwbf_code_query(code)
    F = _frames(y, info.N)
    stride = max_iter if alpha_q.dim() == 2 else 0
    if alpha_q.shape != theta_q.shape or alpha_q.shape[-1] != max_iter or alpha_q.dim() > 2 \
            or (alpha_q.dim() == 2 and alpha_q.shape[0] < F):
        raise ValueError("schedules must be [n_frames][max_iter] or [max_iter]")
    _outputs(F, info.N, out_bits, out_iters)
    fp = _feat(F, out_feat)
    _check(load_library().fwbf_decode_sched(code, _dev(y, torch.int8, "y"), F, int(max_iter),
                                            _dev(alpha_q, torch.int32, "alpha_q"), _dev(theta_q, torch.int32, "theta_q"),
                                            stride, _dev(out_bits, torch.int32, "out_bits"),
                                            _dev(out_iters, torch.int32, "out_iters"),
                                            _opt(out_feat, torch.float32, "out_feat"), fp, _stream(stream)))


def fwbf_decode_learned(code, y, max_iter: int, k_learn: int, alpha_fallback: float, mlp_blob, out_bits,
                        out_iters, out_sched=None, out_feat=None, stream=None, gate_dv: int = 6) -> None:
    """Learned per-pass schedule (network blob: uint8 CUDA tensor of
    MLP_BLOB_BYTES), consulted on passes with W_k >= gate_dv d_v, plain FWBF
    fallback after k_learn passes."""
    import torch

    info = fwbf_code_query(code)
    F = _frames(y, info.N)
    _outputs(F, info.N, out_bits, out_iters)
    _need(mlp_blob, MLP_BLOB_BYTES, "mlp_blob")
    _need(out_sched, F * int(k_learn) * 2, "out_sched")
    fp = _feat(F, out_feat)
    _check(load_library().fwbf_decode_learned(code, _dev(y, torch.int8, "y"), F, int(max_iter), int(k_learn),
                                              int(gate_dv), float(alpha_fallback), _dev(mlp_blob, torch.uint8, "mlp_blob"),
                                              _dev(out_bits, torch.int32, "out_bits"),
                                              _dev(out_iters, torch.int32, "out_iters"),
                                              _opt(out_sched, torch.int32, "out_sched"),
                                              _opt(out_feat, torch.float32, "out_feat"), fp, _stream(stream)))


def fwbf_mlp_pack(master, blob, stream=None) -> None:
    import torch

    _need(master, MLP_PARAMS, "master")
    _need(blob, MLP_BLOB_BYTES, "blob")
    _check(load_library().fwbf_mlp_pack(_dev(master, torch.float32, "master"), _dev(blob, torch.uint8, "blob"),
                                        _stream(stream)))


def fwbf_mlp_forward(blob, x, out, stream=None) -> None:
    import torch

    if x.dim() != 2 or x.shape[1] != MLP_IN:
        raise ValueError(f"x must have shape [samples, {MLP_IN}]")
    _need(blob, MLP_BLOB_BYTES, "blob")
    _need(out, x.shape[0] * MLP_OUT, "out")
    _check(load_library().fwbf_mlp_forward(_dev(blob, torch.uint8, "blob"), _dev(x, torch.float32, "x"), x.shape[0],
                                           _dev(out, torch.float32, "out"), _stream(stream)))


def fwbf_mlp_grad(blob, x, target, n_total: int, grad, loss, stream=None) -> None:
    import torch

    if x.dim() != 2 or x.shape[1] != MLP_IN:
        raise ValueError(f"x must have shape [samples, {MLP_IN}]")
    _need(blob, MLP_BLOB_BYTES, "blob")
    _need(target, x.shape[0] * MLP_OUT, "target")
    _need(grad, MLP_PARAMS, "grad")
    _need(loss, 1, "loss")
    _check(load_library().fwbf_mlp_grad(_dev(blob, torch.uint8, "blob"), _dev(x, torch.float32, "x"),
                                        _dev(target, torch.float32, "target"), x.shape[0], int(n_total),
                                        _dev(grad, torch.float32, "grad"), _dev(loss, torch.float32, "loss"),
                                        _stream(stream)))


def fwbf_mlp_adam(master, blob, grad, m, v, step: int, lr: float, beta1=0.9, beta2=0.999, eps=1e-8,
                  stream=None) -> None:
    import torch

    for t, name in ((master, "master"), (grad, "grad"), (m, "m"), (v, "v")):
        _need(t, MLP_PARAMS, name)
    _need(blob, MLP_BLOB_BYTES, "blob")
    _check(load_library().fwbf_mlp_adam(_dev(master, torch.float32, "master"), _dev(blob, torch.uint8, "blob"),
                                        _dev(grad, torch.float32, "grad"), _dev(m, torch.float32, "m"),
                                        _dev(v, torch.float32, "v"), int(step), float(lr), float(beta1),
                                        float(beta2), float(eps), _stream(stream)))


def fwbf_batch_create(jobs, warps_per_cta: int = 16, packed: int = 1) -> ctypes.c_void_p:
    """jobs: list of (code handle, y int8 [F][N], max_iter, alpha, out_bits,
    out_iters[, mlp blob uint8 tensor, k_learn[, gate_dv (default 6)]])."""
    import torch

    arr = (BatchJob * len(jobs))()
    for i, job in enumerate(jobs):
        code, y, max_iter, alpha, bits, iters = job[:6]
        if len(job) > 6 and job[6] is not None:
            arr[i].mlp = _dev(job[6], torch.uint8, "mlp").value
            arr[i].k_learn = int(job[7])
            arr[i].gate_dv = int(job[8]) if len(job) > 8 else 6
        arr[i].code = code.value if isinstance(code, ctypes.c_void_p) else code
        N = fwbf_code_query(code).N
        F = _frames(y, N)
        _outputs(F, N, bits, iters)
        if len(job) > 6 and job[6] is not None:
            _need(job[6], MLP_BLOB_BYTES, "mlp")
        arr[i].y = _dev(y, torch.int8, "y").value
        arr[i].n_frames = F
        arr[i].max_iter = int(max_iter)
        arr[i].alpha = float(alpha)
        arr[i].out_bits = _dev(bits, torch.int32, "out_bits").value
        arr[i].out_iters = _dev(iters, torch.int32, "out_iters").value
    h = ctypes.c_void_p()
    _check(load_library().fwbf_batch_create(ctypes.cast(arr, ctypes.c_void_p), len(jobs), int(warps_per_cta),
                                            int(packed), ctypes.byref(h)))
    return h


def fwbf_decode_batch(batch, stream=None) -> None:
    _check(load_library().fwbf_decode_batch(batch, _stream(stream)))


def fwbf_batch_query(batch, job: int) -> BatchJobInfo:
    """How the batch decodes job `job` (decoder, warps per frame, frames per
    CTA, grouped kernel or not)."""
    out = BatchJobInfo()
    _check(load_library().fwbf_batch_query(batch, int(job), ctypes.byref(out)))
    return out


def fwbf_batch_status(stream=None) -> int:
    return load_library().fwbf_batch_status(_stream(stream))


def fwbf_batch_destroy(batch) -> None:
    _check(load_library().fwbf_batch_destroy(batch))


def fwbf_last_status(stream=None) -> int:
    return load_library().fwbf_last_status(_stream(stream))


# ---------------------------------------------------------------------------
# convenience wrapper
# ---------------------------------------------------------------------------

class Code:
    """Owns a code handle; decode helpers allocate the outputs."""

    def __init__(self, N: int, M: int, row_idx, col_idx, seg_len: int):
        self.handle = fwbf_code_create(N, M, row_idx, col_idx, seg_len)
        self.info = fwbf_code_query(self.handle)
        self.N, self.M = N, M
        self.words = (N + 31) // 32

    @classmethod
    def from_parity_check(cls, h, seg_len: int, require_rc: bool = False) -> "Code":
        """Handle for ParityCheck h.  A code that breaks the RC constraint (two
        checks sharing two or more bits, i.e. 4-cycles) gets a warning, or with
        require_rc=True a ValueError."""
        code = cls(h.N, h.M, h.rows, h.cols, seg_len)
        overlap = code.info.max_row_overlap
        if overlap > 1:
            if require_rc:
                code.close()
                raise ValueError(f"H breaks the RC constraint: two checks share {overlap} bits")
            import warnings

            warnings.warn(f"H breaks the RC constraint: two checks share {overlap} bits", stacklevel=2)
        return code

    def close(self):
        if self.handle:
            fwbf_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def outputs(self, F: int, device="cuda"):
        import torch

        return (torch.empty((F, self.words), dtype=torch.int32, device=device),
                torch.empty(F, dtype=torch.int32, device=device))

    def decode(self, y, max_iter: int, alpha: float, stream=None):
        bits, iters = self.outputs(y.shape[0], y.device)
        fwbf_decode(self.handle, y, max_iter, alpha, bits, iters, stream)
        return bits, iters

    def decode_f32(self, y, max_iter: int, alpha: float, stream=None):
        bits, iters = self.outputs(y.shape[0], y.device)
        fwbf_decode_f32(self.handle, y, max_iter, alpha, bits, iters, stream)
        return bits, iters

    def metric_f32(self, y, alpha: float, stream=None):
        import torch

        out = torch.empty_like(y)
        fwbf_metric_f32(self.handle, y, alpha, out, stream)
        return out


def quantize(y, stream=None):
    import torch

    q = torch.empty(y.shape, dtype=torch.int8, device=y.device)
    fwbf_quantize(y, q, stream)
    return q
