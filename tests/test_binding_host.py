"""The Python binding's marshalling, with the C library replaced by a
recorder (no GPU): every entry point passes the frame count, sizes and pass
counts the C ABI expects, and refuses buffers too small for what the kernels
would read or write."""
import ctypes

import pytest

torch = pytest.importorskip("torch")

from paper_1206_3362_gb300 import fwbf  # noqa: E402

N = 255
WORDS = (N + 31) // 32


class _Recorder:
    def __init__(self):
        self.calls = []

    def __getattr__(self, name):
        def call(*args):
            if name == "fwbf_batch_create":  # copy the job table while the caller still owns it
                jobs = ctypes.cast(args[0], ctypes.POINTER(fwbf.BatchJob))
                self.jobs = [(jobs[i].n_frames, jobs[i].max_iter, jobs[i].k_learn, jobs[i].gate_dv)
                             for i in range(args[1])]
            self.calls.append((name, args))
            return 0
        return call


@pytest.fixture
def lib(monkeypatch):
    rec = _Recorder()
    info = fwbf.CodeInfo()
    info.N = N

    def dev(t, dtype, name):  # the device check, minus the device
        if t.dtype != dtype or not t.is_contiguous():
            raise TypeError(name)
        return ctypes.c_void_p(t.data_ptr())

    monkeypatch.setattr(fwbf, "load_library", lambda *a: rec)
    monkeypatch.setattr(fwbf, "fwbf_code_query", lambda code: info)
    monkeypatch.setattr(fwbf, "_dev", dev)
    monkeypatch.setattr(fwbf, "_stream", lambda s: None)
    return rec


def _io(F):
    return (torch.zeros((F, N), dtype=torch.int8), torch.zeros((F, WORDS), dtype=torch.int32),
            torch.zeros(F, dtype=torch.int32))


def test_decode_family(lib):
    y, bits, iters = _io(7)
    for fn in (fwbf.fwbf_decode, fwbf.fwbf_decode_noalloc):
        fn(1, y, 10, 1.5, bits, iters)
    fwbf.fwbf_decode_lambda(1, y, 10, 1.5, 3, bits, iters)
    fwbf.fwbf_decode_f32(1, y.float(), 10, 1.5, bits, iters)
    fwbf.fwbf_metric_f32(1, y.float(), 1.5, torch.zeros((7, N)))
    fwbf.fwbf_decode_host(1, y.float(), 10, 1.5, bits, iters, chunk_frames=4)
    assert [c[0] for c in lib.calls] == ["fwbf_decode", "fwbf_decode_noalloc", "fwbf_decode_lambda",
                                         "fwbf_decode_f32", "fwbf_metric_f32", "fwbf_decode_host"]
    assert all(c[1][2] == 7 for c in lib.calls)  # n_frames
    with pytest.raises(ValueError, match="out_bits"):
        fwbf.fwbf_decode(1, y, 10, 1.5, bits[:6], iters)
    with pytest.raises(ValueError, match="out_iters"):
        fwbf.fwbf_decode_host(1, y.float(), 10, 1.5, bits, iters[:6])
    with pytest.raises(ValueError, match="out_E"):
        fwbf.fwbf_metric_f32(1, y.float(), 1.5, torch.zeros((7, N - 1)))
    y0, b0, i0 = _io(0)
    fwbf.fwbf_decode(1, y0, 10, 1.5, b0, i0)


def test_schedules_and_learned(lib):
    F, K = 6, 12
    y, bits, iters = _io(F)
    A = torch.zeros((F, K), dtype=torch.int32)
    feat = torch.zeros((F, 4, 8))
    fwbf.fwbf_decode_sched(1, y, K, A, A.clone(), bits, iters, out_feat=feat)
    name, args = lib.calls[-1]
    assert name == "fwbf_decode_sched" and args[6] == K and args[10] == 4  # stride, feat passes
    fwbf.fwbf_decode_sched(1, y, K, A[0].clone(), A[0].clone(), bits, iters)
    assert lib.calls[-1][1][6] == 0  # one schedule shared by every frame
    with pytest.raises(ValueError, match="schedules"):
        fwbf.fwbf_decode_sched(1, y, K, A[:5].clone(), A[:5].clone(), bits, iters)
    blob = torch.zeros(fwbf.MLP_BLOB_BYTES, dtype=torch.uint8)
    sched = torch.zeros((F, 3, 2), dtype=torch.int32)
    fwbf.fwbf_decode_learned(1, y, K, 3, 1.5, blob, bits, iters, out_sched=sched, out_feat=feat)
    name, args = lib.calls[-1]
    assert name == "fwbf_decode_learned" and args[4:7] == (3, 6, 1.5) and args[12] == 4  # k_learn, gate, alpha
    fwbf.fwbf_decode_learned(1, y, K, 3, 1.5, blob, bits, iters, gate_dv=0)
    assert lib.calls[-1][1][5] == 0
    with pytest.raises(ValueError, match="out_sched"):
        fwbf.fwbf_decode_learned(1, y, K, 4, 1.5, blob, bits, iters, out_sched=sched)
    with pytest.raises(ValueError, match="mlp_blob"):
        fwbf.fwbf_decode_learned(1, y, K, 3, 1.5, blob[:100], bits, iters)


def test_network_kernels(lib):
    blob = torch.zeros(fwbf.MLP_BLOB_BYTES, dtype=torch.uint8)
    master = torch.zeros(fwbf.MLP_PARAMS)
    x, out = torch.zeros((33, 8)), torch.zeros((33, 2))
    fwbf.fwbf_mlp_pack(master, blob)
    fwbf.fwbf_mlp_forward(blob, x, out)
    fwbf.fwbf_mlp_grad(blob, x, out, 33, torch.zeros(fwbf.MLP_PARAMS), torch.zeros(1))
    fwbf.fwbf_mlp_adam(master, blob, torch.zeros(fwbf.MLP_PARAMS), torch.zeros(fwbf.MLP_PARAMS),
                       torch.zeros(fwbf.MLP_PARAMS), 1, 1e-3)
    assert [c[0] for c in lib.calls] == ["fwbf_mlp_pack", "fwbf_mlp_forward", "fwbf_mlp_grad", "fwbf_mlp_adam"]
    assert lib.calls[1][1][2] == 33
    with pytest.raises(ValueError, match="out"):
        fwbf.fwbf_mlp_forward(blob, x, out[:32])
    with pytest.raises(ValueError, match="x must"):
        fwbf.fwbf_mlp_forward(blob, torch.zeros((33, 7)), out)
    with pytest.raises(ValueError, match="grad"):
        fwbf.fwbf_mlp_grad(blob, x, out, 33, torch.zeros(10), torch.zeros(1))


def test_batch_jobs(lib):
    y, bits, iters = _io(9)
    blob = torch.zeros(fwbf.MLP_BLOB_BYTES, dtype=torch.uint8)
    fwbf.fwbf_batch_create([(ctypes.c_void_p(1), y, 10, 1.5, bits, iters),
                            (ctypes.c_void_p(2), y[:4], 20, 2.0, bits[:4], iters[:4], blob, 5),
                            (ctypes.c_void_p(3), y[:2], 20, 2.0, bits[:2], iters[:2], blob, 4, 12)], 16, 2)
    name, args = lib.calls[-1]
    assert name == "fwbf_batch_create" and args[1:4] == (3, 16, 2)
    assert lib.jobs == [(9, 10, 0, 0), (4, 20, 5, 6), (2, 20, 4, 12)]
    with pytest.raises(ValueError, match="out_bits"):
        fwbf.fwbf_batch_create([(ctypes.c_void_p(1), y, 10, 1.5, bits[:8], iters)])
    with pytest.raises(ValueError, match="mlp"):
        fwbf.fwbf_batch_create([(ctypes.c_void_p(1), y, 10, 1.5, bits, iters, blob[:8], 5)])
