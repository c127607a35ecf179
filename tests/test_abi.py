"""CPU-side checks of the boundary: the CUDA library builds for sm_103a, loads
without a GPU, exports every symbol include/cupc.h declares, and its host
logic (workspace sizing, status strings) behaves. No kernels run here."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "cupc.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(cupc_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def C():
    from paper_2509_14433_gb300 import build
    build.build()
    from paper_2509_14433_gb300 import cupc
    return cupc


def test_library_exports_every_declared_symbol(C):
    syms = declared_symbols()
    assert len(syms) >= 15
    lib = ctypes.CDLL(C.LIB_PATH)
    for s in syms:
        assert hasattr(lib, s), s
    assert set(syms) == set(C.EXPORTED)
    out = subprocess.run(["nm", "-D", "--defined-only", C.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\b(cupc_[a-z_0-9]+)\b", out))
    assert set(syms) <= exported


def test_workspace_bytes(C):
    assert C.cupc_workspace_bytes(1) == 0
    assert C.cupc_workspace_bytes(0) == 0
    for V, (L, W) in {1024: (12, 141), 16384: (16, 197), 131072: (19, 239)}.items():
        b = C.cupc_workspace_bytes(V)
        sketch = L * V * W * 16
        assert sketch < b < 2.2 * sketch + (64 << 20)
        assert b % 256 == 0
    assert C.cupc_workspace_bytes(1000, (0, 32, 0, 0)) == 0  # C > 31
    assert C.cupc_workspace_bytes(1000, (0, 0, 64, 0)) == 0  # D > 63
    assert C.cupc_workspace_bytes(1000, (0, 31, 30, 0)) == 0  # W > 256
    assert C.cupc_workspace_bytes(1000, (3, 2, 5, 100)) > 0
    assert C.cupc_workspace_bytes(1000, (64, 16, 2, 0)) == 0  # 64 layers x 32 lanes > 1024 threads
    assert C.cupc_workspace_bytes(1000, (32, 16, 2, 0)) > 0
    assert C.cupc_workspace_bytes(1 << 21, (0, 0, 8, 1 << 10)) > 0
    assert C.cupc_workspace_bytes((1 << 21) + 1, (0, 0, 8, 1 << 10)) == 0  # edge and vertex id share a key
    assert C.cupc_workspace_bytes(1000, (0, 0, 0, 1 << 20)) > C.cupc_workspace_bytes(1000, (0, 0, 0, 1 << 10))


def test_status_strings_and_null_handles(C):
    for s in range(6):
        assert C.cupc_status_string(s).startswith("CUPC_")
    assert "unknown" in C.cupc_status_string(99)
    assert C.cupc_update_batch(None, None, None, 0) == C.CUPC_EINVAL
    assert C.cupc_sync(None) == C.CUPC_EINVAL
    assert C.cupc_init(1, 0)[0] == C.CUPC_EINVAL
    assert C.cupc_set_writeback_bucket(None, 10, C.CUPC_WRITEBACK_ATOMIC) == C.CUPC_EINVAL
    C.cupc_destroy(None)
