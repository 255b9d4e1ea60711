"""Python binding of the GB300 EMD lower-bound library (include/emd.h).

Argument marshalling only: every step of the computation runs in the CUDA library
`_build/libemd_gb300.so`.  There is no Python or CPU fallback; if the library has not
been built, loading it raises.  Host arrays are numpy; device arrays are torch CUDA
tensors (PyTorch owns device memory and streams, nothing more).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import _build

__all__ = [
    "EmdError", "emd_db_options_default", "emd_db_create", "emd_db_destroy", "emd_db_info_get",
    "emd_query_batch", "emd_topk", "emd_query_batch_device", "emd_topk_device",
    "emd_db_check_device_errors", "emd_phase1_table", "emd_db_set_profiling", "emd_topk_select_static",
    "emd_db_profile_get", "emd_db_profile_reset", "emd_last_error", "emd_version",
    "emd_server_options_default", "emd_server_create", "emd_server_submit", "emd_server_poll",
    "emd_server_stats_get", "emd_server_stats_reset", "emd_server_destroy", "EmdError", "emd_all_pairs_topk",
    "emd_baseline_batch", "emd_baseline_topk", "emd_topk_merge",
    "MEASURES", "DIRECTIONS", "PRECISIONS", "PHASES", "library_path", "load",
]

MEASURES = {"rwmd": 0, "omr": 1, "act": 2, "ict": 3}
DIRECTIONS = {"fwd": 0, "rev": 1, "max": 2}
PRECISIONS = {"fp32": 0, "bf16": 1, "fp8": 2, "fp32_tc": 3}
PHASES = ("stage", "distance", "table", "fwd", "rev", "topk", "other")
STATUS = {0: "OK", 1: "INVALID_ARG", 2: "OUT_OF_MEMORY", 3: "CUDA", 4: "TIMEOUT", 5: "BUSY",
          6: "SHUTDOWN", 7: "UNSUPPORTED"}


class EmdError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status
        self.name = STATUS.get(status, str(status))


class emd_db_options(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("rerank_margin", ctypes.c_int32), ("max_query_h", ctypes.c_int32),
                ("max_table_k", ctypes.c_int32), ("max_batch", ctypes.c_int32),
                ("prune_topk", ctypes.c_int32), ("lanes", ctypes.c_int32), ("batched", ctypes.c_int32),
                ("batch_columns", ctypes.c_int32), ("graphs", ctypes.c_int32), ("autotune", ctypes.c_int32),
                ("fused_phase1", ctypes.c_int32), ("fwd_kernel", ctypes.c_int32), ("tc_pair", ctypes.c_int32)]


class emd_db_info(ctypes.Structure):
    _fields_ = [("v", ctypes.c_int64), ("v_used", ctypes.c_int64), ("n_docs", ctypes.c_int64),
                ("nnz", ctypes.c_int64), ("m", ctypes.c_int32), ("cost_matrix_mode", ctypes.c_int32),
                ("device_bytes", ctypes.c_int64), ("autotuned", ctypes.c_int32), ("tc_group_mult", ctypes.c_int32),
                ("tc_stages", ctypes.c_int32), ("rev_warps", ctypes.c_int32), ("fwd_kernel", ctypes.c_int32),
                ("tc_pair", ctypes.c_int32)]


class emd_queries(ctypes.Structure):
    _fields_ = [("n_queries", ctypes.c_int64), ("row_ptr", ctypes.c_void_p),
                ("idx", ctypes.c_void_p), ("w", ctypes.c_void_p)]


class emd_profile(ctypes.Structure):
    _fields_ = [("ms", ctypes.c_double * 7), ("launches", ctypes.c_int64 * 7),
                ("total_launches", ctypes.c_int64), ("pruned_queries", ctypes.c_int64),
                ("prune_fallbacks", ctypes.c_int64), ("graph_launches", ctypes.c_int64),
                ("ict_wide", ctypes.c_int64), ("fused_retries", ctypes.c_int64)]


class emd_server_options(ctypes.Structure):
    _fields_ = [("max_inflight", ctypes.c_int32), ("queue_capacity", ctypes.c_int32),
                ("workspace_bytes", ctypes.c_int64), ("max_query_h", ctypes.c_int32)]


class emd_server_stats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int64) for n in ("submitted", "completed", "rejected_busy", "failed",
                                              "prune_fallbacks", "queued", "in_flight", "max_in_flight",
                                              "pool_bytes", "pool_used_max")] + \
               [(n, ctypes.c_double) for n in ("qps", "latency_p50_us", "latency_p99_us", "latency_mean_us",
                                               "latency_max_us")]


_lib = None


def library_path() -> str:
    return _build.LIB


def load():
    """Load the CUDA library; raise if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_build.LIB):
        raise ImportError(f"CUDA library {_build.LIB} is missing: build it first "
                          "(python -c 'import __graft_entry__ as g; g.build()')")
    L = ctypes.CDLL(_build.LIB)
    P, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
    L.emd_db_options_default.argtypes = [ctypes.POINTER(emd_db_options)]
    L.emd_db_options_default.restype = None
    L.emd_db_create.argtypes = [P, i64, i32, P, P, P, P, i64, ctypes.POINTER(emd_db_options),
                                ctypes.POINTER(P)]
    L.emd_db_destroy.argtypes = [P]
    L.emd_db_info_get.argtypes = [P, ctypes.POINTER(emd_db_info)]
    L.emd_query_batch.argtypes = [P, ctypes.POINTER(emd_queries), i32, i32, i32, P]
    L.emd_topk.argtypes = [P, ctypes.POINTER(emd_queries), i32, i32, i32, i32, P, P]
    L.emd_query_batch_device.argtypes = [P, i64, P, P, P, i32, i32, i32, P, P]
    L.emd_topk_device.argtypes = [P, i64, P, P, P, i32, i32, i32, i32, P, P, P]
    L.emd_db_check_device_errors.argtypes = [P]
    L.emd_topk_select_static.argtypes = [P, i64, i64, i32, P, P, P]
    L.emd_phase1_table.argtypes = [P, P, P, i32, i32, P, P, P, P]
    L.emd_db_set_profiling.argtypes = [P, i32]
    L.emd_db_profile_get.argtypes = [P, ctypes.POINTER(emd_profile)]
    L.emd_db_profile_reset.argtypes = [P]
    L.emd_all_pairs_topk.argtypes = [P, i32, i32, i32, P, P]
    L.emd_topk_merge.argtypes = [i32, P, P, P, i64, i32, i32, P, P]
    L.emd_baseline_batch.argtypes = [P, P, i32, P]
    L.emd_baseline_topk.argtypes = [P, P, i32, i32, P, P]
    L.emd_server_options_default.argtypes = [ctypes.POINTER(emd_server_options)]
    L.emd_server_options_default.restype = None
    L.emd_server_create.argtypes = [P, ctypes.POINTER(emd_server_options), ctypes.POINTER(P)]
    L.emd_server_submit.argtypes = [P, P, P, i32, i32, i32, i32, ctypes.POINTER(ctypes.c_uint64)]
    L.emd_server_poll.argtypes = [P, ctypes.c_uint64, i32, P, P]
    L.emd_server_stats_get.argtypes = [P, ctypes.POINTER(emd_server_stats)]
    L.emd_server_stats_reset.argtypes = [P]
    L.emd_server_destroy.argtypes = [P]
    L.emd_last_error.restype = ctypes.c_char_p
    L.emd_version.restype = ctypes.c_char_p
    for name in ("emd_db_create", "emd_db_destroy", "emd_db_info_get", "emd_query_batch", "emd_topk",
                 "emd_query_batch_device", "emd_topk_device", "emd_db_check_device_errors",
                 "emd_phase1_table", "emd_db_set_profiling", "emd_db_profile_get", "emd_topk_select_static",
                 "emd_db_profile_reset", "emd_all_pairs_topk", "emd_baseline_batch",
                 "emd_baseline_topk", "emd_topk_merge", "emd_server_create", "emd_server_submit", "emd_server_poll",
                 "emd_server_stats_get", "emd_server_stats_reset", "emd_server_destroy"):
        getattr(L, name).restype = ctypes.c_int
    _lib = L
    return L


def _check(status: int):
    if status != 0:
        raise EmdError(status, load().emd_last_error().decode())


def _np(a, dtype):
    a = np.ascontiguousarray(a, dtype=dtype)
    return a, a.ctypes.data_as(ctypes.c_void_p)


def _dev(t, dtype_name: str):
    if t is None:
        return None
    if not (hasattr(t, "is_cuda") and t.is_cuda):
        raise TypeError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("device tensor must be contiguous")
    if str(t.dtype) != f"torch.{dtype_name}":
        raise TypeError(f"expected torch.{dtype_name}, got {t.dtype}")
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    """cudaStream_t handle: an int (torch's `cuda_stream`; 0 is the default stream) or None
    (also the default stream)."""
    return ctypes.c_void_p(int(stream)) if stream is not None else None


def _code(table, x):
    return table[x] if isinstance(x, str) else int(x)


# ------------------------------------------------------------------------ API

def emd_version() -> str:
    return load().emd_version().decode()


def emd_last_error() -> str:
    return load().emd_last_error().decode()


def emd_db_options_default(**over) -> emd_db_options:
    o = emd_db_options()
    load().emd_db_options_default(ctypes.byref(o))
    names = {f[0] for f in emd_db_options._fields_}
    for k, v in over.items():
        if k not in names:
            raise TypeError(f"unknown option {k!r}")
        setattr(o, k, _code(PRECISIONS, v) if k == "precision" else int(v))
    return o


def emd_db_create(emb, cost_matrix, row_ptr, col, val, options: emd_db_options | None = None,
                  v: int | None = None):
    """emb: float32 [v, m] or None; cost_matrix: float32 [v, v] or None."""
    L = load()
    keep = []
    if emb is not None:
        e, pe = _np(emb, np.float32); keep.append(e)
        vv, m = e.shape
    else:
        pe, m = None, 0
    if cost_matrix is not None:
        c, pc = _np(cost_matrix, np.float32); keep.append(c)
        vv = c.shape[0]
    else:
        pc = None
    if v is not None:
        vv = v
    rp, prp = _np(row_ptr, np.int64)
    cl, pcl = _np(col, np.int32)
    vl, pvl = _np(val, np.float32)
    out = ctypes.c_void_p()
    _check(L.emd_db_create(pe, vv, m, pc, prp, pcl, pvl, len(rp) - 1,
                           ctypes.byref(options) if options is not None else None, ctypes.byref(out)))
    return out


def emd_db_destroy(db):
    if db:
        _check(load().emd_db_destroy(db))


def emd_db_info_get(db) -> dict:
    info = emd_db_info()
    _check(load().emd_db_info_get(db, ctypes.byref(info)))
    return {f: getattr(info, f) for f, _ in info._fields_}


def _queries(row_ptr, idx, w):
    rp, prp = _np(row_ptr, np.int64)
    ix, pix = _np(idx, np.int32)
    ww, pw = _np(w, np.float32)
    q = emd_queries(len(rp) - 1, prp, pix, pw)
    return q, (rp, ix, ww)


def emd_query_batch(db, q_row_ptr, q_idx, q_w, meas="act", k: int = 1, dir="max", n_docs=None):
    q, keep = _queries(q_row_ptr, q_idx, q_w)
    n = n_docs if n_docs is not None else emd_db_info_get(db)["n_docs"]
    out = np.empty((q.n_queries, n), dtype=np.float32)
    _check(load().emd_query_batch(db, ctypes.byref(q), _code(MEASURES, meas), int(k),
                                  _code(DIRECTIONS, dir), out.ctypes.data_as(ctypes.c_void_p)))
    return out


def emd_topk(db, q_row_ptr, q_idx, q_w, meas="act", k: int = 1, dir="max", K: int = 16,
             out_idx=None, out_dist=None):
    """Host variant; out_idx/out_dist may be caller-owned (e.g. pinned) numpy arrays."""
    q, keep = _queries(q_row_ptr, q_idx, q_w)
    if out_idx is None:
        out_idx = np.empty((q.n_queries, K), dtype=np.int64)
    if out_dist is None:
        out_dist = np.empty((q.n_queries, K), dtype=np.float32)
    _check(load().emd_topk(db, ctypes.byref(q), _code(MEASURES, meas), int(k), _code(DIRECTIONS, dir),
                           int(K), out_idx.ctypes.data_as(ctypes.c_void_p),
                           out_dist.ctypes.data_as(ctypes.c_void_p)))
    return out_idx, out_dist


def emd_query_batch_device(db, q_row_ptr_host, q_idx_dev, q_w_dev, out_dev, meas="act", k: int = 1,
                           dir="max", stream=None):
    rp, prp = _np(q_row_ptr_host, np.int64)
    _check(load().emd_query_batch_device(db, len(rp) - 1, prp, _dev(q_idx_dev, "int32"),
                                         _dev(q_w_dev, "float32"), _code(MEASURES, meas), int(k),
                                         _code(DIRECTIONS, dir), _dev(out_dev, "float32"),
                                         _stream(stream)))


def emd_topk_device(db, q_row_ptr_host, q_idx_dev, q_w_dev, out_idx_dev, out_dist_dev, meas="act",
                    k: int = 1, dir="max", K: int = 16, stream=None):
    rp, prp = _np(q_row_ptr_host, np.int64)
    _check(load().emd_topk_device(db, len(rp) - 1, prp, _dev(q_idx_dev, "int32"),
                                  _dev(q_w_dev, "float32"), _code(MEASURES, meas), int(k),
                                  _code(DIRECTIONS, dir), int(K), _dev(out_idx_dev, "int64"),
                                  _dev(out_dist_dev, "float32"),
                                  _stream(stream)))


def emd_topk_select_static(t_dev, K: int, out_idx_dev, out_dist_dev, stream=None):
    """Top-K of each row of a device distance matrix [n_rows, n], without any allocation
    (scratch is a fixed array inside the library; see include/emd.h)."""
    if t_dev.dim() not in (1, 2):
        raise ValueError("t_dev must be 1-D (one row) or 2-D [n_rows, n]")
    n_rows, n = (t_dev.shape[0], t_dev.shape[1]) if t_dev.dim() == 2 else (1, t_dev.shape[0])
    for name, o in (("out_idx_dev", out_idx_dev), ("out_dist_dev", out_dist_dev)):
        if o.numel() < n_rows * int(K):
            raise ValueError(f"{name} holds {o.numel()} elements, fewer than n_rows * K = {n_rows * int(K)}")
    _check(load().emd_topk_select_static(_dev(t_dev, "float32"), n_rows, n, int(K),
                                         _dev(out_idx_dev, "int64"), _dev(out_dist_dev, "float32"),
                                         _stream(stream)))


def emd_db_check_device_errors(db):
    _check(load().emd_db_check_device_errors(db))


def emd_phase1_table(db, q_idx, q_w, k: int):
    ix, pix = _np(q_idx, np.int32)
    ww, pw = _np(q_w, np.float32)
    vu = emd_db_info_get(db)["v_used"]
    used = np.empty(vu, dtype=np.int32)
    z = np.empty((vu, k), dtype=np.float32)
    s = np.empty((vu, k), dtype=np.int32)
    w = np.empty((vu, k), dtype=np.float32)
    _check(load().emd_phase1_table(db, pix, pw, len(ix), int(k), used.ctypes.data_as(ctypes.c_void_p),
                                   z.ctypes.data_as(ctypes.c_void_p), s.ctypes.data_as(ctypes.c_void_p),
                                   w.ctypes.data_as(ctypes.c_void_p)))
    return used, z, s, w


def emd_db_set_profiling(db, on: bool = True):
    _check(load().emd_db_set_profiling(db, 1 if on else 0))


def emd_db_profile_get(db) -> dict:
    p = emd_profile()
    _check(load().emd_db_profile_get(db, ctypes.byref(p)))
    return {"ms": dict(zip(PHASES, list(p.ms))), "launches": dict(zip(PHASES, list(p.launches))),
            "total_launches": int(p.total_launches), "pruned_queries": int(p.pruned_queries),
            "prune_fallbacks": int(p.prune_fallbacks), "graph_launches": int(p.graph_launches),
            "ict_wide": int(p.ict_wide), "fused_retries": int(p.fused_retries)}


def emd_db_profile_reset(db):
    _check(load().emd_db_profile_reset(db))


def emd_all_pairs_topk(db, meas="act", k: int = 1, K: int = 16):
    """Each database histogram against all others (no self-match): (idx int64[n, K],
    dist float32[n, K]) of the K smallest symmetric bounds."""
    n = emd_db_info_get(db)["n_docs"]
    out_idx = np.empty((n, K), dtype=np.int64)
    out_dist = np.empty((n, K), dtype=np.float32)
    _check(load().emd_all_pairs_topk(db, _code(MEASURES, meas), int(k), int(K),
                                     out_idx.ctypes.data_as(ctypes.c_void_p), out_dist.ctypes.data_as(ctypes.c_void_p)))
    return out_idx, out_dist


def emd_topk_merge(shards, id_offsets, K: int):
    """Exact global top-K from per-shard results: shards = [(idx int64[nq, Ks], dist
    float32[nq, Ks]), ...] with local ids, id_offsets = each shard's first global id."""
    n = len(shards)
    if n < 1:
        raise ValueError("no shard")
    idx = [np.ascontiguousarray(s[0], dtype=np.int64) for s in shards]
    dist = [np.ascontiguousarray(s[1], dtype=np.float32) for s in shards]
    nq, ks = idx[0].shape
    if any(a.shape != (nq, ks) for a in idx + dist):
        raise ValueError("shard results must all be n_queries x K_shard")
    pi = (ctypes.c_void_p * n)(*[a.ctypes.data for a in idx])
    pd = (ctypes.c_void_p * n)(*[a.ctypes.data for a in dist])
    offs = np.ascontiguousarray(id_offsets, dtype=np.int64)
    out_idx = np.empty((nq, K), dtype=np.int64)
    out_dist = np.empty((nq, K), dtype=np.float32)
    _check(load().emd_topk_merge(n, ctypes.cast(pi, ctypes.c_void_p), ctypes.cast(pd, ctypes.c_void_p),
                                 offs.ctypes.data_as(ctypes.c_void_p), nq, ks, int(K),
                                 out_idx.ctypes.data_as(ctypes.c_void_p), out_dist.ctypes.data_as(ctypes.c_void_p)))
    return out_idx, out_dist


BASELINES = {"bow": 0, "wcd": 1}


def emd_baseline_batch(db, q_row_ptr, q_idx, q_w, kind="bow", n_docs=None):
    """Section 6 baselines: BoW cosine similarity ("bow") or word centroid distance ("wcd"),
    float32[n_queries, n_docs]."""
    n = n_docs if n_docs is not None else emd_db_info_get(db)["n_docs"]
    q, keep = _queries(q_row_ptr, q_idx, q_w)
    out = np.empty((q.n_queries, n), dtype=np.float32)
    _check(load().emd_baseline_batch(db, ctypes.byref(q), _code(BASELINES, kind),
                                     out.ctypes.data_as(ctypes.c_void_p)))
    return out


def emd_baseline_topk(db, q_row_ptr, q_idx, q_w, kind="bow", K: int = 16):
    """K nearest documents by 1 - cosine ("bow") or by word centroid distance ("wcd")."""
    q, keep = _queries(q_row_ptr, q_idx, q_w)
    out_idx = np.empty((q.n_queries, K), dtype=np.int64)
    out_dist = np.empty((q.n_queries, K), dtype=np.float32)
    _check(load().emd_baseline_topk(db, ctypes.byref(q), _code(BASELINES, kind), int(K),
                                    out_idx.ctypes.data_as(ctypes.c_void_p),
                                    out_dist.ctypes.data_as(ctypes.c_void_p)))
    return out_idx, out_dist


# ------------------------------------------------------------------------ serving

def emd_server_options_default(**over) -> emd_server_options:
    o = emd_server_options()
    load().emd_server_options_default(ctypes.byref(o))
    names = {f[0] for f in emd_server_options._fields_}
    for k, v in over.items():
        if k not in names:
            raise TypeError(f"unknown option {k!r}")
        setattr(o, k, int(v))
    return o


def emd_server_create(db, options: emd_server_options | None = None):
    h = ctypes.c_void_p()
    _check(load().emd_server_create(db, ctypes.byref(options) if options is not None else None,
                                    ctypes.byref(h)))
    return h


def emd_server_submit(server, idx, w, meas="act", k: int = 1, K: int = 16) -> int:
    """Queue one query (vocabulary ids idx, weights w); returns its ticket.  Raises EmdError
    (name "BUSY" when the queue is full)."""
    i, pi = _np(idx, np.int32)
    ww, pw = _np(w, np.float32)
    if i.shape != ww.shape or i.ndim != 1:
        raise ValueError("idx and w must be 1-D of the same length")
    t = ctypes.c_uint64()
    _check(load().emd_server_submit(server, pi, pw, int(i.shape[0]), _code(MEASURES, meas), int(k), int(K),
                                    ctypes.byref(t)))
    return int(t.value)


def emd_server_poll(server, ticket: int, timeout_ms: int, out_idx, out_dist) -> bool:
    """Wait up to timeout_ms (-1: no limit) for a result; writes out_idx (int64[K]) and
    out_dist (float32[K]) and returns True when ready, False on timeout."""
    if out_idx.dtype != np.int64 or out_dist.dtype != np.float32:
        raise TypeError("out_idx must be int64 and out_dist float32")
    if not (out_idx.flags.c_contiguous and out_dist.flags.c_contiguous):
        raise ValueError("outputs must be contiguous")
    st = load().emd_server_poll(server, ctypes.c_uint64(ticket), int(timeout_ms),
                                out_idx.ctypes.data_as(ctypes.c_void_p), out_dist.ctypes.data_as(ctypes.c_void_p))
    if st == 4:  # TIMEOUT
        return False
    _check(st)
    return True


def emd_server_stats_get(server) -> dict:
    st = emd_server_stats()
    _check(load().emd_server_stats_get(server, ctypes.byref(st)))
    return {f[0]: (float if f[1] is ctypes.c_double else int)(getattr(st, f[0])) for f in emd_server_stats._fields_}


def emd_server_stats_reset(server):
    _check(load().emd_server_stats_reset(server))


def emd_server_destroy(server):
    _check(load().emd_server_destroy(server))
