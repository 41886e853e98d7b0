"""CPU oracle for FWBF decoding (ctypes wrapper of ``fwbf_oracle.c``).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg may import this package.  The decoding library and
its Python binding never do, and nothing here is shared with the CUDA path.

Every function follows the paper's steps directly (Sec. II, Eq. 1, Sec. III);
the C file's header lists the readings taken where the paper is silent.

Parity status: every function here is pinned by ``tests/test_oracle_pins.py``
(closed forms, hand-traced golden frames, code invariants, the p = N special
case against the separately written single-flip routine).  The only unpinned
part is the statistical agreement with the paper's Tab. 1 averages, which can
only be checked within a band because the paper does not state alpha or its
noise seeds.
"""
from __future__ import annotations

import concurrent.futures
import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fwbf_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle into liboracle.so next to its source (gcc -O2)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            P = ctypes.c_void_p
            i32, i64, f64 = ctypes.c_int32, ctypes.c_int64, ctypes.c_double
            lib.oracle_quantize.argtypes = [P, P, i64]
            lib.oracle_alpha_q.argtypes = [f64]
            lib.oracle_alpha_q.restype = i32
            lib.oracle_fwbf_i8.argtypes = [i32, i32, i64, P, P, i32, P, i64, i32, P, P, i64,
                                           P, P, P, P, P]
            lib.oracle_fwbf_f64.argtypes = [i32, i32, i64, P, P, i32, P, i64, i32, f64, f64,
                                            P, P, P, P]
            lib.oracle_single_flip_i8.argtypes = [i32, i32, i64, P, P, P, i64, i32, i32, i32, P, P]
            lib.oracle_lambda_i8.argtypes = [i32, i32, i64, P, P, i32, P, i64, i32, i32, i32, P, P]
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def _check(rc: int):
    if rc != 0:
        raise RuntimeError(f"oracle error {rc}")


def _coo(code):
    return (np.ascontiguousarray(code.rows, dtype=np.int32),
            np.ascontiguousarray(code.cols, dtype=np.int32))


def quantize(y: np.ndarray) -> np.ndarray:
    """int8 channel values: saturate_{+-127}(round_half_even(16 y)), NaN -> 0."""
    y = np.ascontiguousarray(y, dtype=np.float32)
    q = np.empty(y.shape, dtype=np.int8)
    _check(_load().oracle_quantize(_ptr(y), _ptr(q), y.size))
    return q


def alpha_q(alpha: float) -> int:
    """Fixed-point weighting factor round_half_even(256 alpha)."""
    return int(_load().oracle_alpha_q(float(alpha)))


def fwbf_i8(code, p: int, q: np.ndarray, max_iter: int, alpha: float = 1.0,
            theta_q: int = 0, alpha_sched=None, theta_sched=None, trace: bool = False):
    """FWBF on int8 frames q[F][N] (Sec. III).

    Returns (bits uint32 [F][ceil(N/32)], iters int32 [F]) and, with trace=True
    (one frame), a dict with the syndrome, metric and flips of every pass.
    ``alpha_sched``/``theta_sched`` (int32 [F][max_iter] or [max_iter]) give a
    per-pass fixed-point alpha_q / theta_q in place of the constant ones.
    """
    lib = _load()
    q = np.ascontiguousarray(q, dtype=np.int8).reshape(-1, code.N)
    F = q.shape[0]
    rows, cols = _coo(code)
    if alpha_sched is None:
        asch = np.full(max_iter, alpha_q(alpha), dtype=np.int32)
    else:
        asch = np.ascontiguousarray(alpha_sched, dtype=np.int32)
    if theta_sched is None:
        tsch = np.full(asch.shape, theta_q, dtype=np.int32)
    else:
        tsch = np.ascontiguousarray(theta_sched, dtype=np.int32)
    stride = max_iter if asch.ndim == 2 else 0
    assert asch.shape == tsch.shape and asch.shape[-1] == max_iter
    words = (code.N + 31) // 32
    bits = np.zeros((F, words), dtype=np.uint32)
    iters = np.zeros(F, dtype=np.int32)
    tr = None
    if trace:
        assert F == 1
        tr = dict(s=np.zeros((max_iter + 1, code.M), dtype=np.uint8),
                  E=np.zeros((max_iter, code.N), dtype=np.int64),
                  flip=np.zeros((max_iter, code.N), dtype=np.uint8))
    _check(lib.oracle_fwbf_i8(code.N, code.M, rows.size, _ptr(rows), _ptr(cols), int(p), _ptr(q), F,
                              int(max_iter), _ptr(asch), _ptr(tsch), stride, _ptr(bits), _ptr(iters),
                              _ptr(tr["s"]) if tr else None, _ptr(tr["E"]) if tr else None,
                              _ptr(tr["flip"]) if tr else None))
    if trace:
        return bits, iters, tr
    return bits, iters


def fwbf_f64(code, p: int, y: np.ndarray, max_iter: int, alpha: float = 1.0, theta: float = 0.0,
             want_E0: bool = False):
    """FWBF on real channel values in double precision.

    Returns (bits, iters, margin[F]) and, with want_E0, the first-pass metric
    E0 float64 [F][N]."""
    lib = _load()
    y = np.ascontiguousarray(y, dtype=np.float32).reshape(-1, code.N)
    F = y.shape[0]
    rows, cols = _coo(code)
    words = (code.N + 31) // 32
    bits = np.zeros((F, words), dtype=np.uint32)
    iters = np.zeros(F, dtype=np.int32)
    margin = np.zeros(F, dtype=np.float64)
    e0 = np.zeros((F, code.N), dtype=np.float64) if want_E0 else None
    _check(lib.oracle_fwbf_f64(code.N, code.M, rows.size, _ptr(rows), _ptr(cols), int(p), _ptr(y), F,
                               int(max_iter), float(alpha), float(theta), _ptr(bits), _ptr(iters),
                               _ptr(margin), _ptr(e0)))
    if want_E0:
        return bits, iters, margin, e0
    return bits, iters, margin


def single_flip_i8(code, q: np.ndarray, max_iter: int, alpha: float = 1.0, theta_q: int = 0):
    """Separately written global single-bit flipping (FWBF with p = N)."""
    lib = _load()
    q = np.ascontiguousarray(q, dtype=np.int8).reshape(-1, code.N)
    F = q.shape[0]
    rows, cols = _coo(code)
    bits = np.zeros((F, (code.N + 31) // 32), dtype=np.uint32)
    iters = np.zeros(F, dtype=np.int32)
    _check(lib.oracle_single_flip_i8(code.N, code.M, rows.size, _ptr(rows), _ptr(cols), _ptr(q), F,
                                     int(max_iter), alpha_q(alpha), int(theta_q), _ptr(bits), _ptr(iters)))
    return bits, iters


def lambda_i8(code, lam: int, q: np.ndarray, max_iter: int, alpha: float = 1.0, theta_q: int = 0):
    """lambda-largest selection per pass (MLP-WBF's bit-choose) with the
    IMWBF metric, written separately from fwbf_i8."""
    lib = _load()
    q = np.ascontiguousarray(q, dtype=np.int8).reshape(-1, code.N)
    F = q.shape[0]
    rows, cols = _coo(code)
    bits = np.zeros((F, (code.N + 31) // 32), dtype=np.uint32)
    iters = np.zeros(F, dtype=np.int32)
    _check(lib.oracle_lambda_i8(code.N, code.M, rows.size, _ptr(rows), _ptr(cols), int(lam), _ptr(q), F,
                                int(max_iter), alpha_q(alpha), int(theta_q), _ptr(bits), _ptr(iters)))
    return bits, iters


def fwbf_i8_threaded(code, p: int, q: np.ndarray, max_iter: int, alpha: float = 1.0,
                     threads: int | None = None):
    """fwbf_i8 over frame chunks on a thread pool (the C call releases the GIL).
    Returns (bits, iters, threads_used)."""
    q = np.ascontiguousarray(q, dtype=np.int8).reshape(-1, code.N)
    F = q.shape[0]
    threads = threads or os.cpu_count() or 1
    threads = max(1, min(threads, F))
    bounds = np.linspace(0, F, threads + 1).astype(int)
    bits = np.zeros((F, (code.N + 31) // 32), dtype=np.uint32)
    iters = np.zeros(F, dtype=np.int32)

    def run(i):
        lo, hi = bounds[i], bounds[i + 1]
        if hi > lo:
            b, it = fwbf_i8(code, p, q[lo:hi], max_iter, alpha)
            bits[lo:hi] = b
            iters[lo:hi] = it

    _load()
    with concurrent.futures.ThreadPoolExecutor(threads) as ex:
        list(ex.map(run, range(threads)))
    return bits, iters, threads


def unpack_bits(bits: np.ndarray, N: int) -> np.ndarray:
    """uint32 [F][ceil(N/32)] -> uint8 [F][N] (bit n = word n/32, bit n%32)."""
    b = np.ascontiguousarray(bits, dtype=np.uint32)
    u8 = np.unpackbits(b.view(np.uint8), axis=-1, bitorder="little")
    return u8[..., :N]
