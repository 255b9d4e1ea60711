"""FP64 CPU oracle (test infrastructure only).

Only the tests, the smoke check and the benchmark's CPU-baseline leg import this
package.  The product path (the CUDA library and its binding) never loads it.

`emd_oracle.c` implements, in plain FP64 C:
  * Algorithms 1-3 of the paper (OMR, ICT, ACT) and the one-directional RWMD relaxation
    (Section 2.1) for a given cost matrix;
  * exact EMD (Eq. 1-3) by a small min-cost-flow solver, for tiny histograms;
  * the per-pair definition for one query against a whole database (both directions);
  * the linear-complexity form of Section 5 (Phase 1, Eq. 6-8, Eq. 9) for the forward
    direction, with the reverse direction gathered from the Phase-1 distances;
  * the two cheap baselines of Section 6: bag-of-words cosine similarity and the word
    centroid distance.
This module compiles it with gcc on first use and wraps it with ctypes.
"""
from __future__ import annotations

import concurrent.futures
import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "emd_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libemd_oracle.so")

MEASURES = {"rwmd": 0, "omr": 1, "act": 2, "ict": 3}

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle into oracle/_build/libemd_oracle.so (gcc, -O2, no -march)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fno-fast-math",
                               "-ffp-contract=off", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            P = ctypes.c_void_p
            i32, i64, dbl = ctypes.c_int32, ctypes.c_int64, ctypes.c_double
            for name in ("oracle_rwmd", "oracle_omr", "oracle_ict", "oracle_emd"):
                f = getattr(L, name)
                f.argtypes = [P, i32, P, i32, P]
                f.restype = dbl
            L.oracle_act.argtypes = [P, i32, P, i32, P, i32]
            L.oracle_act.restype = dbl
            L.oracle_measure.argtypes = [i32, P, i32, P, i32, P, i32]
            L.oracle_measure.restype = dbl
            L.oracle_cost_block.argtypes = [P, i32, P, i64, P, i32, P, i32, P]
            L.oracle_cost_block.restype = None
            for name in ("oracle_pair_db", "oracle_lc_query"):
                f = getattr(L, name)
                f.argtypes = [P, i32, P, i64, P, P, P, i64, P, P, i32, i32, i32, P, P]
                f.restype = i32
            L.oracle_phase1.argtypes = [P, i32, P, i64, P, i64, P, P, i32, i32, P, P, P]
            L.oracle_phase1.restype = None
            L.oracle_bow_db.argtypes = [i64, P, P, P, i64, P, P, i32, P]
            L.oracle_bow_db.restype = i32
            L.oracle_wcd_db.argtypes = [P, i32, P, P, P, i64, P, P, i32, P]
            L.oracle_wcd_db.restype = i32
            _lib = L
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


# ----------------------------------------------------------------- pairwise

def rwmd(p, q, C) -> float:
    p, q, C = _f64(p), _f64(q), _f64(C)
    return lib().oracle_rwmd(_p(p), len(p), _p(q), len(q), _p(C))


def omr(p, q, C) -> float:
    p, q, C = _f64(p), _f64(q), _f64(C)
    return lib().oracle_omr(_p(p), len(p), _p(q), len(q), _p(C))


def ict(p, q, C) -> float:
    p, q, C = _f64(p), _f64(q), _f64(C)
    return lib().oracle_ict(_p(p), len(p), _p(q), len(q), _p(C))


def act(p, q, C, k: int) -> float:
    p, q, C = _f64(p), _f64(q), _f64(C)
    return lib().oracle_act(_p(p), len(p), _p(q), len(q), _p(C), int(k))


def emd(p, q, C) -> float:
    p, q, C = _f64(p), _f64(q), _f64(C)
    return lib().oracle_emd(_p(p), len(p), _p(q), len(q), _p(C))


def measure(name: str, p, q, C, k: int = 1) -> float:
    p, q, C = _f64(p), _f64(q), _f64(C)
    return lib().oracle_measure(MEASURES[name], _p(p), len(p), _p(q), len(q), _p(C), int(k))


def cost_block(emb, cost, ia, ib) -> np.ndarray:
    emb = np.ascontiguousarray(emb, dtype=np.float32)
    cost = None if cost is None else np.ascontiguousarray(cost, dtype=np.float32)
    ia = np.ascontiguousarray(ia, dtype=np.int32)
    ib = np.ascontiguousarray(ib, dtype=np.int32)
    out = np.empty((len(ia), len(ib)), dtype=np.float64)
    lib().oracle_cost_block(_p(emb), emb.shape[1], _p(cost), emb.shape[0], _p(ia), len(ia),
                            _p(ib), len(ib), _p(out))
    return out


# ----------------------------------------------------------------- one query vs database

def _db_args(emb, cost, db):
    emb = np.ascontiguousarray(emb, dtype=np.float32)
    cost = None if cost is None else np.ascontiguousarray(cost, dtype=np.float32)
    return (emb, cost, np.ascontiguousarray(db.row_ptr, dtype=np.int64),
            np.ascontiguousarray(db.col, dtype=np.int32),
            np.ascontiguousarray(db.val, dtype=np.float32))


def _run(fn_name, emb, cost, db, q_idx, q_w, meas, k, fwd, rev):
    emb, cost, rp, col, val = _db_args(emb, cost, db)
    q_idx = np.ascontiguousarray(q_idx, dtype=np.int32)
    q_w = np.ascontiguousarray(q_w, dtype=np.float32)
    n = len(rp) - 1
    tf = np.empty(n, dtype=np.float64) if fwd else None
    tr = np.empty(n, dtype=np.float64) if rev else None
    rc = getattr(lib(), fn_name)(_p(emb), emb.shape[1], _p(cost), emb.shape[0], _p(rp), _p(col),
                                 _p(val), n, _p(q_idx), _p(q_w), len(q_idx), MEASURES[meas],
                                 int(k), _p(tf), _p(tr))
    if rc != 0:
        raise MemoryError("oracle allocation failed")
    return tf, tr


def pair_db(emb, cost, db, q_idx, q_w, meas: str, k: int = 1, fwd=True, rev=True):
    """Per-pair definition (Algorithms 1-3 on a fresh cost block per document)."""
    return _run("oracle_pair_db", emb, cost, db, q_idx, q_w, meas, k, fwd, rev)


def lc_query(emb, cost, db, q_idx, q_w, meas: str, k: int = 1, fwd=True, rev=True):
    """Linear-complexity form (Section 5) for one query."""
    return _run("oracle_lc_query", emb, cost, db, q_idx, q_w, meas, k, fwd, rev)


def phase1(emb, cost, rows, q_idx, q_w, kk: int):
    emb = np.ascontiguousarray(emb, dtype=np.float32)
    cost = None if cost is None else np.ascontiguousarray(cost, dtype=np.float32)
    rows = np.ascontiguousarray(rows, dtype=np.int32)
    q_idx = np.ascontiguousarray(q_idx, dtype=np.int32)
    q_w = np.ascontiguousarray(q_w, dtype=np.float32)
    Z = np.empty((len(rows), kk)); W = np.empty((len(rows), kk))
    S = np.empty((len(rows), kk), dtype=np.int32)
    lib().oracle_phase1(_p(emb), emb.shape[1], _p(cost), emb.shape[0], _p(rows), len(rows),
                        _p(q_idx), _p(q_w), len(q_idx), kk, _p(Z), _p(S), _p(W))
    return Z, S, W


def symmetric(t_fwd, t_rev):
    """Section 6: the symmetric measure is the maximum of the two directions."""
    return np.maximum(t_fwd, t_rev)


def topk(t, K: int):
    """The K smallest distances ordered by (distance, document id)."""
    t = np.asarray(t)
    order = np.lexsort((np.arange(len(t)), t))[:K]
    return order.astype(np.int64), t[order]


def lc_queries(emb, cost, db, queries, qids, meas: str, k: int, fwd=True, rev=True,
               threads: int | None = None):
    """lc_query over several queries on a thread pool (the C calls release the GIL)."""
    threads = threads or os.cpu_count() or 1
    lib()

    def one(qi):
        qi_idx, qi_w = queries.row(int(qi))
        return lc_query(emb, cost, db, qi_idx, qi_w, meas, k, fwd, rev)

    with concurrent.futures.ThreadPoolExecutor(max_workers=threads) as ex:
        return list(ex.map(one, list(qids)))


def _slice(db, d0: int, d1: int):
    """Documents d0..d1-1 of a CSR set as a view (no copy of col/val)."""
    a, b = int(db.row_ptr[d0]), int(db.row_ptr[d1])

    class _S:
        pass
    s = _S()
    s.row_ptr = db.row_ptr[d0:d1 + 1] - a
    s.col = db.col[a:b]
    s.val = db.val[a:b]
    return s


def lc_query_split(emb, cost, db, q_idx, q_w, meas: str, k: int = 1, fwd=True, rev=True,
                   threads: int | None = None):
    """lc_query for one query, with the database cut into `threads` contiguous document
    slices evaluated concurrently.  Each slice runs the unchanged oracle on its own used
    vocabulary; every document's value is computed exactly as in one call, so the
    concatenation equals lc_query on the whole database."""
    threads = max(1, min(threads or os.cpu_count() or 1, db.n if hasattr(db, "n") else len(db.row_ptr) - 1))
    n = len(db.row_ptr) - 1
    bounds = np.linspace(0, n, threads + 1).astype(np.int64)
    lib()

    def one(i):
        return lc_query(emb, cost, _slice(db, bounds[i], bounds[i + 1]), q_idx, q_w, meas, k, fwd, rev)

    with concurrent.futures.ThreadPoolExecutor(max_workers=threads) as ex:
        parts = list(ex.map(one, range(threads)))
    tf = np.concatenate([p[0] for p in parts]) if fwd else None
    tr = np.concatenate([p[1] for p in parts]) if rev else None
    return tf, tr


# ----------------------------------------------------------------- Section 6 baselines

def bow_cosine(v: int, db, q_idx, q_w) -> np.ndarray:
    """Bag-of-words cosine similarity of one query with every database histogram."""
    rp = np.ascontiguousarray(db.row_ptr, dtype=np.int64)
    col = np.ascontiguousarray(db.col, dtype=np.int32)
    val = np.ascontiguousarray(db.val, dtype=np.float32)
    q_idx = np.ascontiguousarray(q_idx, dtype=np.int32)
    q_w = np.ascontiguousarray(q_w, dtype=np.float32)
    out = np.empty(len(rp) - 1, dtype=np.float64)
    if lib().oracle_bow_db(int(v), _p(rp), _p(col), _p(val), len(rp) - 1, _p(q_idx), _p(q_w), len(q_idx),
                           _p(out)) != 0:
        raise MemoryError("oracle allocation failed")
    return out


def wcd(emb, db, q_idx, q_w) -> np.ndarray:
    """Word centroid distance of one query to every database histogram."""
    emb = np.ascontiguousarray(emb, dtype=np.float32)
    rp = np.ascontiguousarray(db.row_ptr, dtype=np.int64)
    col = np.ascontiguousarray(db.col, dtype=np.int32)
    val = np.ascontiguousarray(db.val, dtype=np.float32)
    q_idx = np.ascontiguousarray(q_idx, dtype=np.int32)
    q_w = np.ascontiguousarray(q_w, dtype=np.float32)
    out = np.empty(len(rp) - 1, dtype=np.float64)
    if lib().oracle_wcd_db(_p(emb), emb.shape[1], _p(rp), _p(col), _p(val), len(rp) - 1, _p(q_idx), _p(q_w),
                           len(q_idx), _p(out)) != 0:
        raise MemoryError("oracle allocation failed")
    return out
