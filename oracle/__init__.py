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
            L.oracle_lc_phase23.argtypes = [P, P, P, i64, P, P, P, i32, i32, i32, P]
            L.oracle_lc_phase23.restype = i32
            L.oracle_lc_rev.argtypes = [P, P, P, i64, P, P, P, i32, i32, i32, P]
            L.oracle_lc_rev.restype = i32
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


def table_width(meas: str, k: int, hq: int) -> int:
    """Columns of the Phase-1 tables of a query with hq bins (as oracle_lc_query sizes them)."""
    kk = {"rwmd": 1, "omr": 2, "ict": hq}.get(meas, min(k, hq))
    return min(kk, hq)


class LcPrep:
    """What the split forms reuse across queries of one database: contiguous copies of
    its arrays, the used vocabulary (ascending ids, Section 2.2) and the table row of
    every vocabulary id."""

    def __init__(self, emb, cost, db):
        self.emb, self.cost, self.rp, self.col, self.val = _db_args(emb, cost, db)
        self.used = np.unique(self.col).astype(np.int32)
        self.v = self.emb.shape[0] if self.cost is None else self.cost.shape[0]
        self.row_of_id = np.full(self.v, -1, dtype=np.int64)
        self.row_of_id[self.used] = np.arange(len(self.used))
        self.n = len(self.rp) - 1


def prepare(emb, cost, db) -> LcPrep:
    return LcPrep(emb, cost, db)


def _phase23(P, Z, W, kk, meas, hq, threads):
    """Phase 2 and 3 (oracle_lc_phase23) on document slices, on threads."""
    L = lib()
    bounds = np.linspace(0, P.n, threads + 1).astype(np.int64)
    tf = np.empty(P.n)

    def one(i):
        d0, d1 = int(bounds[i]), int(bounds[i + 1])
        if d1 > d0:
            a = int(P.rp[d0])
            sub_rp = np.ascontiguousarray(P.rp[d0:d1 + 1] - a)
            out = np.empty(d1 - d0)
            if L.oracle_lc_phase23(_p(sub_rp), _p(P.col[a:]), _p(P.val[a:]), d1 - d0, _p(P.row_of_id), _p(Z), _p(W),
                                   kk, MEASURES[meas], hq, _p(out)) != 0:
                raise MemoryError("oracle allocation failed")
            tf[d0:d1] = out

    with concurrent.futures.ThreadPoolExecutor(max_workers=threads) as ex:
        list(ex.map(one, range(threads)))
    return tf


def lc_forward_split(emb, cost, db, q_idx, q_w, meas: str, k: int = 1, threads: int | None = None,
                     prep: LcPrep | None = None):
    """Forward values (Section 5: Phase 1, then Phase 2 and 3) of one query against the
    whole database, the work spread over threads without changing any value: Phase 1
    (oracle_phase1) on slices of the used vocabulary's rows, then Phase 2 and 3
    (oracle_lc_phase23) on slices of the documents.  Each table row and each document is
    computed by the same steps as in oracle_lc_query, so the values are identical to its
    forward output (tests/test_oracle_lc.py)."""
    threads = max(1, threads or os.cpu_count() or 1)
    P = prep or LcPrep(emb, cost, db)
    q_idx = np.ascontiguousarray(q_idx, dtype=np.int32)
    q_w = np.ascontiguousarray(q_w, dtype=np.float32)
    hq = len(q_idx)
    kk = table_width(meas, k, hq)
    vu = len(P.used)
    Z = np.empty((vu, kk)); W = np.empty((vu, kk)); S = np.empty((vu, kk), dtype=np.int32)
    m = P.emb.shape[1]
    L = lib()
    rb = np.linspace(0, vu, threads + 1).astype(np.int64)

    def p1(i):
        a, b = int(rb[i]), int(rb[i + 1])
        if b > a:
            L.oracle_phase1(_p(P.emb), m, _p(P.cost), P.v, _p(P.used[a:b]), b - a, _p(q_idx), _p(q_w), hq, kk,
                            _p(Z[a:b]), _p(S[a:b]), _p(W[a:b]))

    with concurrent.futures.ThreadPoolExecutor(max_workers=threads) as ex:
        list(ex.map(p1, range(threads)))
    return _phase23(P, Z, W, kk, meas, hq, threads)


def lc_query_full_split(emb, cost, db, q_idx, q_w, meas: str, k: int = 1, threads: int | None = None,
                        prep: LcPrep | None = None):
    """Both directions for every document, as oracle_lc_query computes them, spread over
    threads: the Phase-1 block D (oracle_cost_block on slices of the used vocabulary's
    rows), each row's first kk entries in (distance, position) order (a stable sort),
    Phase 2 and 3 (oracle_lc_phase23) and the reverse direction (oracle_lc_rev) on slices
    of the documents.  Identical to oracle_lc_query (tests/test_oracle_lc.py)."""
    threads = max(1, threads or os.cpu_count() or 1)
    P = prep or LcPrep(emb, cost, db)
    q_idx = np.ascontiguousarray(q_idx, dtype=np.int32)
    q_w = np.ascontiguousarray(q_w, dtype=np.float32)
    hq = len(q_idx)
    kk = table_width(meas, k, hq)
    vu = len(P.used)
    D = np.empty((vu, hq))
    Z = np.empty((vu, kk)); W = np.empty((vu, kk))
    qw64 = q_w.astype(np.float64)
    m = P.emb.shape[1]
    L = lib()
    rb = np.linspace(0, vu, threads + 1).astype(np.int64)

    def p1(i):
        a, b = int(rb[i]), int(rb[i + 1])
        if b > a:
            L.oracle_cost_block(_p(P.emb), m, _p(P.cost), P.v, _p(P.used[a:b]), b - a, _p(q_idx), hq, _p(D[a:b]))
            order = np.argsort(D[a:b], axis=1, kind="stable")[:, :kk]
            Z[a:b] = np.take_along_axis(D[a:b], order, axis=1)
            W[a:b] = qw64[order]

    with concurrent.futures.ThreadPoolExecutor(max_workers=threads) as ex:
        list(ex.map(p1, range(threads)))
    tf = _phase23(P, Z, W, kk, meas, hq, threads)
    tr = np.empty(P.n)
    bounds = np.linspace(0, P.n, threads + 1).astype(np.int64)

    def rev(i):
        d0, d1 = int(bounds[i]), int(bounds[i + 1])
        if d1 > d0:
            a = int(P.rp[d0])
            sub_rp = np.ascontiguousarray(P.rp[d0:d1 + 1] - a)
            out = np.empty(d1 - d0)
            if L.oracle_lc_rev(_p(sub_rp), _p(P.col[a:]), _p(P.val[a:]), d1 - d0, _p(P.row_of_id), _p(D), _p(q_w), hq,
                               MEASURES[meas], int(k), _p(out)) != 0:
                raise MemoryError("oracle allocation failed")
            tr[d0:d1] = out

    with concurrent.futures.ThreadPoolExecutor(max_workers=threads) as ex:
        list(ex.map(rev, range(threads)))
    return tf, tr


class SymTopK:
    """Exact top-K of max(fwd, rev) for one query (Section 6: top-l search with the
    symmetric bound), from oracle routines only: the forward values of every document
    (lc_forward_split), then the reverse values by the per-pair definition (pair_db on one
    document) in ascending forward order.  Since max(fwd, rev) >= fwd, once the next
    forward value exceeds the K-th smallest symmetric value found so far, no remaining
    document can enter the top-K (strictly larger, so not even by the id order)."""

    def __init__(self, emb, cost, db, q_idx, q_w, meas: str, k: int, K: int, threads: int | None = None,
                 prep: LcPrep | None = None):
        self.args = (emb, cost, db, np.asarray(q_idx), np.asarray(q_w), meas, k)
        self.threads = max(1, threads or os.cpu_count() or 1)
        self.fwd = lc_forward_split(emb, cost, db, q_idx, q_w, meas, k, self.threads, prep)
        self.rev = {}
        n = len(self.fwd)
        order = np.lexsort((np.arange(n), self.fwd))
        pos, chunk = 0, 4 * self.threads
        while pos < n:
            kth = self.kth(K)
            take = [int(d) for d in order[pos:pos + chunk] if self.fwd[d] <= kth]
            if not take:
                break
            self.reverse(take)
            pos += chunk
        keys = sorted((self.sym(d), d) for d in self.rev)
        self.idx = np.array([d for _, d in keys[:K]], dtype=np.int64)
        self.dist = np.array([v for v, _ in keys[:K]])

    def kth(self, K):
        vals = sorted(self.sym(d) for d in self.rev)
        return vals[K - 1] if len(vals) >= K else np.inf

    def sym(self, d: int) -> float:
        return max(self.fwd[d], self.rev[d])

    def reverse(self, docs):
        """Reverse values (per-pair definition) of the given documents, on threads."""
        emb, cost, db, q_idx, q_w, meas, k = self.args
        docs = [int(d) for d in docs if int(d) not in self.rev]

        def one(d):
            return d, pair_db(emb, cost, _slice(db, d, d + 1), q_idx, q_w, meas, k, fwd=False, rev=True)[1][0]

        with concurrent.futures.ThreadPoolExecutor(max_workers=self.threads) as ex:
            for d, r in ex.map(one, docs):
                self.rev[d] = r

    def sym_of(self, docs) -> np.ndarray:
        """Symmetric values of any documents (reverse values computed where missing)."""
        self.reverse(docs)
        return np.array([self.sym(int(d)) for d in docs])


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
