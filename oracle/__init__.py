"""CPU oracle for sketch-based connectivity (arXiv 2509.14433).

TEST INFRASTRUCTURE ONLY. The plain C implementation in ``cupc_oracle.c`` is
what the CUDA library is checked against. Only the test suite, the smoke
check and the CPU-baseline leg of ``bench.py`` may import this module. It
shares no code with the CUDA path and never calls it.

``build()`` compiles the C source with gcc into ``oracle/_build``; the
ctypes wrapper below only marshals arguments.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cupc_oracle.c")
_LIB = os.path.join(_HERE, "_build", "libcupc_oracle.so")

OK, EINVAL, ENOMEM, EINCOMPLETE = 0, 1, 2, 3
ZERO, GOOD, FAIL = 0, 1, 2

_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle (plain C, no threads) and return the .so path."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    stale = (not os.path.exists(_LIB)) or any(
        os.path.getmtime(os.path.join(_HERE, f)) > os.path.getmtime(_LIB)
        for f in ("cupc_oracle.c", "cupc_oracle.h"))
    if force or stale:
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-Wall", "-shared", "-fPIC",
                               "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = ctypes.CDLL(build())
    P, u32, u64, sz = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_size_t
    sig = {
        "orc_mix64": (u64, [u64]),
        "orc_keys": (None, [u64, P, sz]),
        "orc_params": (None, [u32, P, P, P]),
        "orc_hash_bits": (u32, [u32]),
        "orc_mas_depth": (u32, [u64, u64, u64, u64, u32, u32, u64]),
        "orc_create": (P, [u32, u64, u32, u32, u32]),
        "orc_destroy": (None, [P]),
        "orc_get_params": (None, [P, P]),
        "orc_update_batch": (ctypes.c_int, [P, P, P, sz]),
        "orc_sync": (ctypes.c_int, [P]),
        "orc_recover": (ctypes.c_int, [P]),
        "orc_query": (ctypes.c_int, [P, P, sz, P]),
        "orc_spanning_forest": (ctypes.c_int, [P, P, sz, P]),
        "orc_labels": (None, [P, P]),
        "orc_stats": (None, [P, P]),
        "orc_round_log": (None, [P, P, P, P]),
        "orc_export": (None, [P, P]),
        "orc_import": (None, [P, P]),
        "orc_sketch_sum": (None, [P, P, sz, u32, P]),
        "orc_sample": (ctypes.c_int, [P, P, u32, P]),
        "orc_vertex_sketch": (None, [u32, u64, u32, u32, u32, u32, P, sz, P]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def mix64(z: int) -> int:
    return int(_load().orc_mix64(z & (2**64 - 1)))


def keys(seed: int, n: int) -> np.ndarray:
    out = np.zeros(n, dtype=np.uint64)
    _load().orc_keys(seed & (2**64 - 1), _ptr(out), n)
    return out


def params(V: int, L: int = 0, C: int = 0, D: int = 0):
    a = [ctypes.c_uint32(x) for x in (L, C, D)]
    _load().orc_params(V, *[ctypes.byref(x) for x in a])
    L, C, D = (x.value for x in a)
    return L, C, D, 1 + C * D


def hash_bits(V: int) -> int:
    return int(_load().orc_hash_bits(V))


def mas_depth(a: int, b: int, a2: int, b2: int, ell: int, D: int, x: int) -> int:
    m = 2**64 - 1
    return int(_load().orc_mas_depth(a & m, b & m, a2 & m, b2 & m, ell, D, x & m))


def vertex_sketch(V: int, seed: int, w: int, nbrs, L=0, C=0, D=0) -> np.ndarray:
    """Sketch of one vertex from its neighbour set: array [L][W][2] u64."""
    L, C, D, W = params(V, L, C, D)
    nb = np.ascontiguousarray(np.asarray(nbrs, dtype=np.uint32))
    out = np.zeros((L, W, 2), dtype=np.uint64)
    _load().orc_vertex_sketch(V, seed, L, C, D, w, _ptr(nb), nb.size, _ptr(out))
    return out


class Graph:
    """One oracle instance: V vertices, sketches seeded by ``seed``."""

    def __init__(self, V: int, seed: int, L: int = 0, C: int = 0, D: int = 0):
        lib = _load()
        self._h = lib.orc_create(V, seed & (2**64 - 1), L, C, D)
        if not self._h:
            raise MemoryError("oracle graph allocation failed")
        p = np.zeros(4, dtype=np.uint32)
        lib.orc_get_params(self._h, _ptr(p))
        self.V = V
        self.seed = seed
        self.L, self.C, self.D, self.W = (int(x) for x in p)

    def close(self):
        if self._h:
            _load().orc_destroy(self._h)
            self._h = None

    __del__ = close

    def update(self, edges: np.ndarray, ops: np.ndarray | None = None) -> int:
        e = np.ascontiguousarray(edges, dtype=np.uint32).reshape(-1)
        n = e.size // 2
        o = np.ones(n, dtype=np.int8) if ops is None else np.ascontiguousarray(ops, dtype=np.int8)
        return int(_load().orc_update_batch(self._h, _ptr(e), _ptr(o), n))

    def sync(self) -> int:
        return int(_load().orc_sync(self._h))

    def recover(self) -> int:
        return int(_load().orc_recover(self._h))

    def query(self, pairs: np.ndarray):
        p = np.ascontiguousarray(pairs, dtype=np.uint32).reshape(-1)
        out = np.zeros(p.size // 2, dtype=np.uint8)
        s = int(_load().orc_query(self._h, _ptr(p), p.size // 2, _ptr(out)))
        return s, out

    def spanning_forest(self):
        out = np.zeros(self.V, dtype=np.uint64)
        n = ctypes.c_size_t(0)
        s = int(_load().orc_spanning_forest(self._h, _ptr(out), self.V, ctypes.byref(n)))
        return s, out[: n.value].copy()

    def labels(self) -> np.ndarray:
        out = np.zeros(self.V, dtype=np.uint32)
        _load().orc_labels(self._h, _ptr(out))
        return out

    def stats(self) -> dict:
        s = np.zeros(5, dtype=np.uint64)
        _load().orc_stats(self._h, _ptr(s))
        return {"rounds": int(s[0]), "fail": int(s[1]), "false_pos": int(s[2]),
                "complete": bool(s[3]), "n_logged": int(s[4])}

    def round_log(self):
        st = self.stats()
        R = st["rounds"]
        live = np.zeros(max(R, 1), dtype=np.uint32)
        ncand = np.zeros(max(R, 1), dtype=np.uint32)
        ids = np.zeros(max(st["n_logged"], 1), dtype=np.uint64)
        _load().orc_round_log(self._h, _ptr(live), _ptr(ncand), _ptr(ids))
        out, k = [], 0
        for r in range(R):
            out.append((int(live[r]), ids[k:k + int(ncand[r])].copy()))
            k += int(ncand[r])
        return out

    def export(self) -> np.ndarray:
        """All sketches as [L][V][W][2] u64 (alpha, gamma)."""
        out = np.zeros((self.L, self.V, self.W, 2), dtype=np.uint64)
        _load().orc_export(self._h, _ptr(out))
        return out

    def import_(self, sk: np.ndarray) -> None:
        """Overwrite every sketch word from a [L][V][W][2] u64 array."""
        a = np.ascontiguousarray(sk, dtype=np.uint64)
        assert a.shape == (self.L, self.V, self.W, 2)
        _load().orc_import(self._h, _ptr(a))

    def sketch_sum(self, verts, r: int) -> np.ndarray:
        v = np.ascontiguousarray(np.asarray(verts, dtype=np.uint32))
        out = np.zeros((self.W, 2), dtype=np.uint64)
        _load().orc_sketch_sum(self._h, _ptr(v), v.size, r, _ptr(out))
        return out

    def sample(self, layer: np.ndarray, r: int):
        lay = np.ascontiguousarray(layer, dtype=np.uint64)
        e = ctypes.c_uint64(0)
        res = int(_load().orc_sample(self._h, _ptr(lay), r, ctypes.byref(e)))
        return res, int(e.value)
