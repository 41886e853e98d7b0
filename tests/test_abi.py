"""The C-ABI library loads and exports every symbol its header declares; host
argument checks reject bad input before touching a GPU."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", h) for h in os.listdir(os.path.join(ROOT, "include")) if h.endswith(".h")]


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__

    __graft_entry__.build()
    from paper_1206_3362_gb300 import fwbf

    return fwbf.load_library()


def _declared():
    names = set()
    for h in HEADERS:
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(fwbf_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return names


def test_header_declares_entry_points():
    names = _declared()
    for required in ("fwbf_code_create", "fwbf_decode", "fwbf_destroy", "fwbf_quantize",
                     "fwbf_decode_f32", "fwbf_metric_f32", "fwbf_strerror"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    from paper_1206_3362_gb300 import fwbf

    out = subprocess.run(["nm", "-D", "--defined-only", fwbf.LIB_PATH], capture_output=True, text=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if line.strip()}
    missing = _declared() - exported
    assert not missing, missing
    for name in _declared():
        assert hasattr(lib, name)


def test_header_constants_match_binding():
    """Status codes, decoder kinds and network sizes: the same values in the
    header and in the Python binding."""
    from paper_1206_3362_gb300 import fwbf

    text = open(os.path.join(ROOT, "include", "fwbf.h")).read()
    defines = {m.group(1): int(m.group(2)) for m in re.finditer(r"^#define (FWBF_\w+)\s+(-?\d+)", text, flags=re.M)}
    names = [n for n in defines if re.match(r"FWBF_(OK|E[A-Z]+|DECODER_\w+)$", n)]
    assert {"FWBF_OK", "FWBF_ETIMEOUT", "FWBF_DECODER_LIST", "FWBF_DECODER_CYCLIC", "FWBF_DECODER_QC"} <= set(names)
    for n in names:
        assert getattr(fwbf, n) == defines[n], n
    assert [f[0] for f in fwbf.CodeInfo._fields_][-2:] == ["max_row_overlap", "decoder"]
    assert ctypes.sizeof(fwbf.CodeInfo) == 56


def test_strerror(lib):
    from paper_1206_3362_gb300 import fwbf

    assert lib.fwbf_strerror(fwbf.FWBF_OK) == b"ok"
    for code in (fwbf.FWBF_EINVAL, fwbf.FWBF_ENOMEM, fwbf.FWBF_ECUDA, fwbf.FWBF_EUNSUPPORTED, fwbf.FWBF_ETIMEOUT):
        assert lib.fwbf_strerror(code) not in (b"ok", b"unknown status")


@pytest.mark.parametrize("case", ["range", "dup", "weight1", "seg", "size"])
def test_code_create_rejects_bad_input(lib, case):
    from paper_1206_3362_gb300 import fwbf

    rows = np.array([0, 0, 1, 1], dtype=np.int32)
    cols = np.array([0, 1, 1, 2], dtype=np.int32)
    N, M, seg = 3, 2, 1
    want = fwbf.FWBF_EINVAL
    if case == "range":
        cols = np.array([0, 1, 1, 3], dtype=np.int32)
    elif case == "dup":
        cols = np.array([0, 1, 1, 1], dtype=np.int32)
    elif case == "weight1":
        rows = np.array([0, 0, 1], dtype=np.int32)
        cols = np.array([0, 1, 1], dtype=np.int32)
        want = fwbf.FWBF_EUNSUPPORTED
    elif case == "seg":
        seg = 4
    elif case == "size":
        N = 70000
    with pytest.raises(fwbf.FwbfError) as ei:
        fwbf.fwbf_code_create(N, M, rows, cols, seg)
    assert ei.value.status == want


def test_decode_rejects_null_code(lib):
    from paper_1206_3362_gb300 import fwbf

    rc = lib.fwbf_decode(None, None, 0, 10, ctypes.c_float(1.0), None, None, None)
    assert rc == fwbf.FWBF_EINVAL
    assert lib.fwbf_quantize(None, None, -1, None) == fwbf.FWBF_EINVAL


def test_division_magic():
    """The kernels divide by p and Z with umulhi(x, ceil(2^32/d)); exact for
    every x < 65536 and 2 <= d <= 65535."""
    x = np.arange(65536, dtype=np.uint64)
    for d in list(range(2, 300)) + [1023, 4095, 16383, 32767, 65535]:
        magic = np.uint64(((1 << 32) + d - 1) // d)
        assert np.array_equal((x * magic) >> np.uint64(32), x // np.uint64(d))


def test_binding_fails_loudly_without_library(tmp_path):
    from paper_1206_3362_gb300 import fwbf

    saved = fwbf._lib
    fwbf._lib = None
    try:
        with pytest.raises(ImportError):
            fwbf.load_library(str(tmp_path / "missing.so"))
    finally:
        fwbf._lib = saved


def test_peak_probe_rejects_bad_arguments(lib):
    """The integer issue-rate microbenchmark validates its arguments on the
    host before any CUDA call."""
    from paper_1206_3362_gb300 import fwbf

    r = ctypes.c_double(0.0)
    assert lib.fwbf_peak_int_issue(2, 100.0, None, ctypes.byref(r), None) == fwbf.FWBF_EINVAL
    assert lib.fwbf_peak_int_issue(1, 0.5, None, ctypes.byref(r), None) == fwbf.FWBF_EINVAL
    assert lib.fwbf_peak_int_issue(1, 100.0, None, None, None) == fwbf.FWBF_EINVAL


def test_bounded_wait_probe_rejects_bad_arguments(lib):
    from paper_1206_3362_gb300 import fwbf

    st = ctypes.c_int(0)
    assert lib.fwbf_probe_bounded_wait(65537, None, ctypes.byref(st)) == fwbf.FWBF_EINVAL
    assert lib.fwbf_probe_bounded_wait(16, None, None) == fwbf.FWBF_EINVAL


def test_binding_refuses_short_buffers():
    """The binding checks every buffer's size against what the kernels will
    read or write before any call crosses the C ABI (which cannot see sizes)."""
    import torch

    from paper_1206_3362_gb300 import fwbf

    F, N = 5, 1023  # 32 words of decisions per frame
    fwbf._outputs(F, N, torch.empty((F, 32), dtype=torch.int32), torch.empty(F, dtype=torch.int32))
    fwbf._outputs(0, N, torch.empty((0, 32), dtype=torch.int32), torch.empty(0, dtype=torch.int32))
    with pytest.raises(ValueError, match="out_bits"):
        fwbf._outputs(F, N, torch.empty((F, 31), dtype=torch.int32), torch.empty(F, dtype=torch.int32))
    with pytest.raises(ValueError, match="out_iters"):
        fwbf._outputs(F, N, torch.empty((F, 32), dtype=torch.int32), torch.empty(F - 1, dtype=torch.int32))
    fwbf._need(None, 10, "optional")
    with pytest.raises(ValueError, match="blob"):
        fwbf._need(torch.empty(fwbf.MLP_BLOB_BYTES - 1, dtype=torch.uint8), fwbf.MLP_BLOB_BYTES, "blob")
    assert fwbf._feat(F, None) == 0
    assert fwbf._feat(F, torch.empty((F, 6, 8))) == 6
    for bad in (torch.empty((F - 1, 6, 8)), torch.empty((F, 6, 7)), torch.empty((F, 48))):
        with pytest.raises(ValueError, match="out_feat"):
            fwbf._feat(F, bad)
