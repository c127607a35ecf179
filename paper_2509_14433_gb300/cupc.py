"""Thin ctypes binding of libcupc (include/cupc.h): argument marshalling only.

Every function has the C name and returns the C status. Pointer arguments
accept a torch tensor (its data_ptr), a numpy array (host memory), an int
address or None. Stream arguments accept a torch.cuda.Stream, an int handle
or None (the legacy default stream).

Importing this module loads the CUDA library and raises ImportError if it
has not been built: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libcupc.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"libcupc.so is not built ({LIB_PATH}); run __graft_entry__.build() first")

_lib = ctypes.CDLL(LIB_PATH)

CUPC_OK, CUPC_EINVAL, CUPC_ENOMEM, CUPC_EINCOMPLETE, CUPC_ECUDA, CUPC_ETIMEOUT = range(6)

_P, _u32, _u64, _sz = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_size_t


class cupc_params(ctypes.Structure):
    _fields_ = [("rounds", _u32), ("columns", _u32), ("rows", _u32), ("max_batch", _u32)]


_SIGS = {
    "cupc_workspace_bytes": (_sz, [_u32, _P]),
    "cupc_init": (ctypes.c_int, [_u32, _u64, _P, _P, _P, _P]),
    "cupc_reset": (ctypes.c_int, [_P, _P]),
    "cupc_update_batch": (ctypes.c_int, [_P, _P, _P, _sz, _P]),
    "cupc_query": (ctypes.c_int, [_P, _P, _sz, _P, _P]),
    "cupc_spanning_forest": (ctypes.c_int, [_P, _P, _sz, _P, _P]),
    "cupc_labels": (ctypes.c_int, [_P, _P, _P]),
    "cupc_sync": (ctypes.c_int, [_P, _P]),
    "cupc_export_sketches": (ctypes.c_int, [_P, _P, _sz, _P]),
    "cupc_import_sketches": (ctypes.c_int, [_P, _P, _sz, _P]),
    "cupc_stats": (ctypes.c_int, [_P, _P, _P]),
    "cupc_round_log": (ctypes.c_int, [_P, _P, _P, _P, _sz, _P, _P]),
    "cupc_get_params": (ctypes.c_int, [_P, _P]),
    "cupc_set_tuning": (ctypes.c_int, [_P, _u32, _u32, _u32]),
    "cupc_set_tuning_bucket": (ctypes.c_int, [_P, _u32, _u32, _u32, _u32]),
    "cupc_set_writeback_bucket": (ctypes.c_int, [_P, _u32, _u32]),
    "cupc_set_incremental": (ctypes.c_int, [_P, ctypes.c_int, _P]),
    "cupc_update_batches": (ctypes.c_int, [_P, _P, _P, _P, _sz, _P]),
    "cupc_batcher_create": (ctypes.c_int, [_u32, ctypes.c_int, _P]),
    "cupc_batcher_update": (ctypes.c_int, [_P, _P, _P, _P, _P, _u32, _P]),
    "cupc_batcher_destroy": (None, [_P]),
    "cupc_server_create": (ctypes.c_int, [_P, _P]),
    "cupc_server_open": (ctypes.c_int, [_P, _u32, _u64, _P]),
    "cupc_server_update": (ctypes.c_int, [_P, _u64, _P, _P, _sz, _P]),
    "cupc_server_query": (ctypes.c_int, [_P, _u64, _P, _sz, _P, _P]),
    "cupc_server_close": (ctypes.c_int, [_P, _u64, _P]),
    "cupc_server_wait": (ctypes.c_int, [_P, _u64, _u32, _P]),
    "cupc_server_export": (ctypes.c_int, [_P, _u64, _P, _sz]),
    "cupc_server_stats": (ctypes.c_int, [_P, _P]),
    "cupc_server_destroy": (None, [_P]),
    "cupc_get_tuning": (ctypes.c_int, [_P, _P]),
    "cupc_profile_enable": (ctypes.c_int, [_P, ctypes.c_int]),
    "cupc_profile_read": (ctypes.c_int, [_P, _P, _P, _sz]),
    "cupc_destroy": (None, [_P]),
    "cupc_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "cupc_selftest_wait_timeout": (ctypes.c_int, [_u32, _u32, ctypes.c_int, _P]),
    "cupc_build_info": (ctypes.c_int, [_P, _P]),
    "cupc_cutset_create": (ctypes.c_int, [_P, _P, _P]),
    "cupc_cutset_apply": (ctypes.c_int, [_P, _P, _sz, _P, _P]),
    "cupc_cutset_connected": (ctypes.c_int, [_P, _u32, _u32, _P]),
    "cupc_cutset_tree_sketch": (ctypes.c_int, [_P, _u32, _P, _P]),
    "cupc_cutset_query": (ctypes.c_int, [_P, _u32, _u32, _P, _P, _P]),
    "cupc_cutset_stats": (ctypes.c_int, [_P, _P]),
    "cupc_cutset_destroy": (None, [_P]),
    "cupc_update_sketch_static": (ctypes.c_int, [_P, _u32, _u64, _P, _P, _sz, _P, _P]),
}
for _name, (_res, _args) in _SIGS.items():
    _fn = getattr(_lib, _name)
    _fn.restype = _res
    _fn.argtypes = _args

EXPORTED = tuple(_SIGS)


def ptr(x) -> int | None:
    """Address of a torch tensor / numpy array / int (None stays None)."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if hasattr(x, "ctypes"):
        return x.ctypes.data
    raise TypeError(f"cannot take the address of {type(x)}")


def stream_handle(s) -> int | None:
    if s is None or isinstance(s, int):
        return s
    return s.cuda_stream


def _params(p):
    if p is None:
        return None
    if isinstance(p, cupc_params):
        return ctypes.byref(p)
    return ctypes.byref(cupc_params(*p))


def cupc_workspace_bytes(V: int, params=None) -> int:
    return int(_lib.cupc_workspace_bytes(V, _params(params)))


def cupc_init(V: int, seed: int, params=None, workspace=None, stream=None):
    """Returns (status, handle)."""
    h = ctypes.c_void_p(0)
    st = _lib.cupc_init(V, seed & (2**64 - 1), _params(params), ptr(workspace), stream_handle(stream),
                        ctypes.byref(h))
    return st, h.value


def cupc_reset(g, stream=None) -> int:
    return _lib.cupc_reset(g, stream_handle(stream))


def cupc_update_batch(g, edges, ops, n: int, stream=None) -> int:
    return _lib.cupc_update_batch(g, ptr(edges), ptr(ops), n, stream_handle(stream))


def cupc_query(g, pairs, m: int, out, stream=None) -> int:
    return _lib.cupc_query(g, ptr(pairs), m, ptr(out), stream_handle(stream))


def cupc_spanning_forest(g, out, cap: int, stream=None):
    """Returns (status, n)."""
    n = ctypes.c_size_t(0)
    st = _lib.cupc_spanning_forest(g, ptr(out), cap, ctypes.byref(n), stream_handle(stream))
    return st, n.value


def cupc_labels(g, out, stream=None) -> int:
    return _lib.cupc_labels(g, ptr(out), stream_handle(stream))


def cupc_sync(g, stream=None) -> int:
    return _lib.cupc_sync(g, stream_handle(stream))


def cupc_export_sketches(g, dst, nbytes: int, stream=None) -> int:
    return _lib.cupc_export_sketches(g, ptr(dst), nbytes, stream_handle(stream))


def cupc_import_sketches(g, src, nbytes: int, stream=None) -> int:
    return _lib.cupc_import_sketches(g, ptr(src), nbytes, stream_handle(stream))


def cupc_stats(g, out8, stream=None) -> int:
    return _lib.cupc_stats(g, ptr(out8), stream_handle(stream))


def cupc_round_log(g, live, ncand, ids, cap: int, stream=None):
    """Returns (status, rounds)."""
    nr = ctypes.c_uint32(0)
    st = _lib.cupc_round_log(g, ptr(live), ptr(ncand), ptr(ids), cap, ctypes.byref(nr), stream_handle(stream))
    return st, nr.value


def cupc_get_params(g, out4) -> int:
    return _lib.cupc_get_params(g, ptr(out4))


def cupc_update_batches(g, edges, ops, offsets, k: int, stream=None) -> int:
    """offsets: host uint64 array of k+1 entries."""
    return _lib.cupc_update_batches(g, ptr(edges), ptr(ops), ptr(offsets), k, stream_handle(stream))


def cupc_batcher_create(max_graphs: int, use_cuda_graph: bool = True):
    """Returns (status, handle)."""
    h = ctypes.c_void_p(0)
    st = _lib.cupc_batcher_create(max_graphs, 1 if use_cuda_graph else 0, ctypes.byref(h))
    return st, h.value


def cupc_batcher_update(b, graphs, edges, ops, ns, stream=None) -> int:
    """graphs: handles; edges/ops: device tensors or addresses; ns: sizes."""
    k = len(graphs)
    G = (ctypes.c_void_p * k)(*graphs)
    E = (ctypes.c_void_p * k)(*[ptr(e) for e in edges])
    O = (ctypes.c_void_p * k)(*[ptr(o) for o in ops])
    N = (ctypes.c_size_t * k)(*ns)
    return _lib.cupc_batcher_update(b, G, E, O, N, k, stream_handle(stream))


def cupc_batcher_destroy(b) -> None:
    _lib.cupc_batcher_destroy(b)


class cupc_server_config(ctypes.Structure):
    _fields_ = [("mem_bytes", _sz), ("max_graphs", _u32), ("max_batch", _u32), ("query_streams", _u32),
                ("pinned_bytes", _sz)]


def cupc_server_create(mem_bytes: int, max_graphs: int, max_batch: int = 0, query_streams: int = 0,
                       pinned_bytes: int = 0):
    """Returns (status, handle)."""
    cfg = cupc_server_config(mem_bytes, max_graphs, max_batch, query_streams, pinned_bytes)
    h = ctypes.c_void_p(0)
    st = _lib.cupc_server_create(ctypes.byref(cfg), ctypes.byref(h))
    return st, h.value


def cupc_server_open(s, V: int, seed: int):
    i = ctypes.c_uint64(0)
    st = _lib.cupc_server_open(s, V, seed & (2**64 - 1), ctypes.byref(i))
    return st, i.value


def cupc_server_update(s, gid: int, edges, ops, n: int):
    t = ctypes.c_uint64(0)
    st = _lib.cupc_server_update(s, gid, ptr(edges), ptr(ops), n, ctypes.byref(t))
    return st, t.value


def cupc_server_query(s, gid: int, pairs, m: int, out):
    t = ctypes.c_uint64(0)
    st = _lib.cupc_server_query(s, gid, ptr(pairs), m, ptr(out), ctypes.byref(t))
    return st, t.value


def cupc_server_close(s, gid: int):
    t = ctypes.c_uint64(0)
    st = _lib.cupc_server_close(s, gid, ctypes.byref(t))
    return st, t.value


def cupc_server_wait(s, ticket: int, timeout_ms: int = 60000):
    """Returns (status, latency_us)."""
    lat = ctypes.c_double(0.0)
    st = _lib.cupc_server_wait(s, ticket, timeout_ms, ctypes.byref(lat))
    return st, lat.value


def cupc_server_export(s, gid: int, dst, nbytes: int) -> int:
    return _lib.cupc_server_export(s, gid, ptr(dst), nbytes)


def cupc_server_stats(s, out8) -> int:
    return _lib.cupc_server_stats(s, ptr(out8))


def cupc_server_destroy(s) -> None:
    _lib.cupc_server_destroy(s)


def cupc_set_tuning(g, item_records: int, smem_rows: int, ctas_per_sm: int) -> int:
    return _lib.cupc_set_tuning(g, item_records, smem_rows, ctas_per_sm)


def cupc_set_tuning_bucket(g, bucket: int, item_records: int, smem_rows: int, ctas_per_sm: int) -> int:
    return _lib.cupc_set_tuning_bucket(g, bucket, item_records, smem_rows, ctas_per_sm)


def cupc_set_writeback_bucket(g, bucket: int, mode: int) -> int:
    return _lib.cupc_set_writeback_bucket(g, bucket, mode)


def cupc_set_incremental(g, on: int, stream=None) -> int:
    return _lib.cupc_set_incremental(g, on, stream_handle(stream))


def cupc_get_tuning(g, out4) -> int:
    return _lib.cupc_get_tuning(g, ptr(out4))


def cupc_profile_enable(g, on: int) -> int:
    return _lib.cupc_profile_enable(g, on)


def cupc_profile_read(g, ms, launches, n: int) -> int:
    return _lib.cupc_profile_read(g, ptr(ms), ptr(launches), n)


def cupc_destroy(g) -> None:
    _lib.cupc_destroy(g)


def cupc_selftest_wait_timeout(ctas: int, limit_us: int, absent_cta: int, stream=None) -> int:
    return _lib.cupc_selftest_wait_timeout(ctas, limit_us, absent_cta, stream_handle(stream))


CUPC_CUTSET_LINK, CUPC_CUTSET_CUT, CUPC_CUTSET_REFRESH = 1, 2, 3
CUPC_WRITEBACK_AUTO, CUPC_WRITEBACK_LOAD_STORE, CUPC_WRITEBACK_ATOMIC = 0, 1, 2


def cupc_cutset_create(g, stream=None):
    """Returns (status, handle)."""
    h = ctypes.c_void_p(0)
    st = _lib.cupc_cutset_create(g, stream_handle(stream), ctypes.byref(h))
    return st, h.value


def cupc_cutset_apply(c, ops, stream=None):
    """ops: host uint32 array of {kind, u, v} triples. Returns (status, applied)."""
    n = ctypes.c_size_t(0)
    st = _lib.cupc_cutset_apply(c, ptr(ops), len(ops) // 3, ctypes.byref(n), stream_handle(stream))
    return st, n.value


def cupc_cutset_connected(c, u: int, v: int):
    out = ctypes.c_int(0)
    st = _lib.cupc_cutset_connected(c, u, v, ctypes.byref(out))
    return st, bool(out.value)


def cupc_cutset_tree_sketch(c, w: int, dst, stream=None) -> int:
    return _lib.cupc_cutset_tree_sketch(c, w, ptr(dst), stream_handle(stream))


def cupc_cutset_query(c, w: int, r: int, stream=None):
    """Returns (status, result 0/1/2, edge)."""
    res, e = ctypes.c_uint32(0), ctypes.c_uint64(0)
    st = _lib.cupc_cutset_query(c, w, r, ctypes.byref(res), ctypes.byref(e), stream_handle(stream))
    return st, res.value, e.value


def cupc_cutset_stats(c, out4) -> int:
    return _lib.cupc_cutset_stats(c, ptr(out4))


def cupc_cutset_destroy(c) -> None:
    _lib.cupc_cutset_destroy(c)


def cupc_build_info():
    """Returns (status, binary_version, ptx_version) of the update kernel."""
    b, p = ctypes.c_int(0), ctypes.c_int(0)
    st = _lib.cupc_build_info(ctypes.byref(b), ctypes.byref(p))
    return st, b.value, p.value


def cupc_status_string(st: int) -> str:
    return _lib.cupc_status_string(st).decode()


CUPC_STATIC_MAX_V = 65536
CUPC_STATIC_MAX_EDGES = 65536


def cupc_update_sketch_static(sketch, V: int, seed: int, edges, ops, n: int, status_out=None, stream=None) -> int:
    return _lib.cupc_update_sketch_static(ptr(sketch), V, seed & (2**64 - 1), ptr(edges), ptr(ops), n,
                                          ptr(status_out), stream_handle(stream))


class CupcError(RuntimeError):
    def __init__(self, st: int, what: str):
        super().__init__(f"{what}: {cupc_status_string(st)}")
        self.status = st


def check(st: int, what: str = "cupc", ok=(CUPC_OK,)) -> int:
    if st not in ok:
        raise CupcError(st, what)
    return st
