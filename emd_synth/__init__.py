"""Seeded synthetic inputs shaped like the paper's workloads (Table 3: 20 Newsgroups
with Word2Vec, MNIST).  The real datasets are not used; these generators stand in for
them with the same shapes, sizes and value distributions.

This module holds input generation only: random histograms, embeddings, the pixel
grid and its ground-cost matrix.  It contains none of the EMD relaxations themselves
and is the one module that both the FP64 oracle side and the CUDA side read.

Recipe (all numpy PCG64):
  * Text vocabulary: rank r = 1..V is vocabulary id r-1 with P(r) proportional to
    r^-1.1 (Zipf 1.1).  A histogram of size h is h distinct ids drawn by successive
    sampling without replacement in proportion to P (draw with replacement, keep first
    occurrences), stored sorted by id.
  * Term counts are uniform integers 1..5, L1-normalised in FP64, stored as FP32.
  * Embeddings: i.i.d. N(0,1) rows, L2-normalised in FP64, stored as FP32.
  * Histogram sizes: uniform 10..40 (tiny), log-normal with median 100 and sigma 0.5
    (natural log) rounded and clipped to 10..1000 (text at scale), log-uniform 5..2000
    (batched / serving queries).
  * Images: 28x28 grid, each image the clipped sum of 3..6 Gaussian strokes (segments
    with endpoints uniform in [9,18]^2 and sigma ~ U[1,2] px), pixels below 0.1 set to
    zero, L1-normalised: about 19% nonzeros (h ~ 146, MNIST's is 149.9).  Coordinates
    are (row, col) pixel positions, not normalised; the ground cost is their Euclidean
    distance, computed in FP64 and stored FP32 with an exact zero diagonal.
"""
from __future__ import annotations

import ctypes
import dataclasses
import hashlib
import os
import subprocess

import numpy as np

BASE_SEED = 1812020910
QUERY_SEED_OFFSET = 100


@dataclasses.dataclass
class Histograms:
    """A set of L1-normalised sparse histograms in CSR form (row = histogram)."""
    row_ptr: np.ndarray  # int64 [n+1]
    col: np.ndarray      # int32 [nnz], vocabulary ids, strictly increasing per row
    val: np.ndarray      # float32 [nnz], > 0, each row sums to 1 (FP64-normalised)

    @property
    def n(self) -> int:
        return int(self.row_ptr.shape[0] - 1)

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    def row(self, i: int):
        a, b = int(self.row_ptr[i]), int(self.row_ptr[i + 1])
        return self.col[a:b], self.val[a:b]

    def subset(self, rows) -> "Histograms":
        rows = np.asarray(rows, dtype=np.int64)
        lens = self.row_ptr[rows + 1] - self.row_ptr[rows]
        rp = np.zeros(len(rows) + 1, dtype=np.int64)
        np.cumsum(lens, out=rp[1:])
        cols = [self.col[self.row_ptr[r]:self.row_ptr[r + 1]] for r in rows]
        vals = [self.val[self.row_ptr[r]:self.row_ptr[r + 1]] for r in rows]
        return Histograms(rp,
                          np.concatenate(cols).astype(np.int32) if cols else np.zeros(0, np.int32),
                          np.concatenate(vals).astype(np.float32) if vals else np.zeros(0, np.float32))


@dataclasses.dataclass
class Workload:
    name: str
    v: int                       # vocabulary size
    m: int                       # embedding dimension
    emb: np.ndarray              # float32 [v, m]
    cost: np.ndarray | None      # float32 [v, v] ground-cost matrix (image mode) or None
    db: Histograms
    queries: Histograms
    k_list: tuple
    top_k: int


# --------------------------------------------------------------------------- sizes

def _lengths(rng, n, law):
    kind = law[0]
    if kind == "uniform":
        lo, hi = law[1], law[2]
        return rng.integers(lo, hi + 1, size=n).astype(np.int64)
    if kind == "lognormal":
        median, sigma, lo, hi = law[1:]
        x = np.exp(np.log(median) + sigma * rng.standard_normal(n))
        return np.clip(np.rint(x), lo, hi).astype(np.int64)
    if kind == "loguniform":
        lo, hi = law[1], law[2]
        x = np.exp(rng.uniform(np.log(lo), np.log(hi), size=n))
        return np.clip(np.rint(x), lo, hi).astype(np.int64)
    raise ValueError(law)


# --------------------------------------------------------------------------- text

def zipf_cdf(V: int, s: float = 1.1) -> np.ndarray:
    p = np.arange(1, V + 1, dtype=np.float64) ** (-s)
    c = np.cumsum(p)
    return c / c[-1]


def _zipf_sets_chunk(rng, cdf, lengths):
    """Distinct ids per row: draw with replacement from the Zipf law and keep the first
    `length` distinct values in draw order (successive sampling without replacement)."""
    V = cdf.shape[0]
    n = lengths.shape[0]
    result = [None] * n
    todo = np.arange(n)
    factor = 2.0
    while todo.size:
        lens = lengths[todo]
        draws = np.ceil(lens * factor).astype(np.int64) + 8
        total = int(draws.sum())
        owner = np.repeat(np.arange(todo.size), draws)
        pos = np.arange(total) - np.repeat(np.cumsum(draws) - draws, draws)
        ids = np.searchsorted(cdf, rng.random(total), side="right")
        ids = np.minimum(ids, V - 1)
        order = np.lexsort((pos, ids, owner))
        o, i, p = owner[order], ids[order], pos[order]
        first = np.ones(total, dtype=bool)
        first[1:] = (o[1:] != o[:-1]) | (i[1:] != i[:-1])
        o, i, p = o[first], i[first], p[first]
        order2 = np.lexsort((p, o))
        o, i = o[order2], i[order2]
        start = np.searchsorted(o, np.arange(todo.size), side="left")
        end = np.searchsorted(o, np.arange(todo.size), side="right")
        failed = []
        for t in range(todo.size):
            L = int(lens[t])
            if end[t] - start[t] >= L:
                result[todo[t]] = np.sort(i[start[t]:start[t] + L])
            else:
                failed.append(todo[t])
        todo = np.asarray(failed, dtype=np.int64)
        factor *= 2.0
    return result


_HELPER_SRC = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_zipf.c")
_HELPER_LIB = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "libzipf.so")
_helper = None


def _zipf_helper():
    """The C form of the per-row selection (emd_synth/_zipf.c, compiled with gcc on first
    use), or None when no C compiler is available (the numpy form is used then)."""
    global _helper
    if _helper is not None:
        return _helper or None
    try:
        os.makedirs(os.path.dirname(_HELPER_LIB), exist_ok=True)
        if not os.path.exists(_HELPER_LIB) or os.path.getmtime(_HELPER_LIB) < os.path.getmtime(_HELPER_SRC):
            tmp = _HELPER_LIB + f".tmp{os.getpid()}"
            subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, _HELPER_SRC],
                                  stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
            os.replace(tmp, _HELPER_LIB)
        L = ctypes.CDLL(_HELPER_LIB)
        P, i64 = ctypes.c_void_p, ctypes.c_int64
        L.zipf_first_distinct.argtypes = [P, i64, P, P, P, i64, P, i64, P, P, P, P]
        L.zipf_first_distinct.restype = None
        _helper = L
    except (OSError, subprocess.CalledProcessError):
        _helper = False
    return _helper or None


def _zipf_rows_c(L, rng, cdf, lengths, col, offsets, stamp, tag):
    """Same rows, same random draws as _zipf_sets_chunk, with the per-row selection in C;
    rows are written into col at their offsets.  Returns the next free stamp tag."""
    p = lambda a: a.ctypes.data_as(ctypes.c_void_p)  # noqa: E731
    V = cdf.shape[0]
    todo = np.arange(lengths.shape[0])
    factor = 2.0
    buf = np.empty(max(1, int(lengths.max()) if lengths.size else 1), dtype=np.int32)
    while todo.size:
        lens = np.ascontiguousarray(lengths[todo], dtype=np.int64)
        draws = np.ceil(lens * factor).astype(np.int64) + 8
        u = rng.random(int(draws.sum()))
        off = np.ascontiguousarray(offsets[todo], dtype=np.int64)
        ok = np.zeros(todo.size, dtype=np.uint8)
        L.zipf_first_distinct(p(cdf), V, p(u), p(draws), p(lens), todo.size, p(stamp), tag, p(col), p(off), p(ok),
                              p(buf))
        tag += todo.size
        todo = todo[ok == 0]
        factor *= 2.0
    return tag


def zipf_histograms(rng, V: int, lengths: np.ndarray, s: float = 1.1, chunk: int = 50000,
                    use_c: bool = True) -> Histograms:
    if np.any(lengths > V):
        raise ValueError("histogram longer than the vocabulary")
    cdf = zipf_cdf(V, s)
    n = lengths.shape[0]
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(lengths, out=row_ptr[1:])
    col = np.empty(int(row_ptr[-1]), dtype=np.int32)
    L = _zipf_helper() if use_c else None
    stamp = np.full(V, -1, dtype=np.int64) if L else None
    tag = 0
    for a in range(0, n, chunk):
        b = min(n, a + chunk)
        if L:
            tag = _zipf_rows_c(L, rng, cdf, lengths[a:b], col, row_ptr[a:b], stamp, tag)
        else:
            sets = _zipf_sets_chunk(rng, cdf, lengths[a:b])
            col[row_ptr[a]:row_ptr[b]] = np.concatenate(sets)
    counts = rng.integers(1, 6, size=col.shape[0]).astype(np.float64)
    sums = np.add.reduceat(counts, row_ptr[:-1]) if n else np.zeros(0)
    val = (counts / np.repeat(sums, lengths)).astype(np.float32)
    return Histograms(row_ptr, col, val)


def unit_embeddings(rng, V: int, m: int) -> np.ndarray:
    x = rng.standard_normal((V, m))
    x /= np.linalg.norm(x, axis=1, keepdims=True)
    e = x.astype(np.float32)
    # distinct coordinates: zero ground distance must mean "same vocabulary id"
    digests = {hashlib.blake2b(r.tobytes(), digest_size=16).digest() for r in e}
    assert len(digests) == V, "duplicate embedding rows"
    return e


# --------------------------------------------------------------------------- images

GRID = 28


def pixel_coords() -> np.ndarray:
    r, c = np.divmod(np.arange(GRID * GRID), GRID)
    return np.stack([r, c], axis=1).astype(np.float32)


def pixel_cost_matrix() -> np.ndarray:
    xy = pixel_coords().astype(np.float64)
    d = np.sqrt(((xy[:, None, :] - xy[None, :, :]) ** 2).sum(-1))
    np.fill_diagonal(d, 0.0)
    return d.astype(np.float32)


def stroke_images(rng, n: int, box=(9.0, 18.0), chunk: int = 4096) -> Histograms:
    xy = pixel_coords().astype(np.float64)  # [784, 2]
    rows, vals, lens = [], [], []
    for a in range(0, n, chunk):
        b = min(n, a + chunk)
        cnt = b - a
        img = np.zeros((cnt, GRID * GRID))
        nstrokes = rng.integers(3, 7, size=cnt)
        for s in range(6):
            active = nstrokes > s
            p0 = rng.uniform(box[0], box[1], size=(cnt, 2))
            p1 = rng.uniform(box[0], box[1], size=(cnt, 2))
            sigma = rng.uniform(1.0, 2.0, size=cnt)
            d = p1 - p0
            L2 = np.maximum((d ** 2).sum(1), 1e-12)
            t = ((xy[None, :, :] - p0[:, None, :]) * d[:, None, :]).sum(-1) / L2[:, None]
            t = np.clip(t, 0.0, 1.0)
            proj = p0[:, None, :] + t[..., None] * d[:, None, :]
            dist2 = ((xy[None, :, :] - proj) ** 2).sum(-1)
            img += active[:, None] * np.exp(-dist2 / (2.0 * sigma[:, None] ** 2))
        img = np.clip(img, 0.0, 1.0)
        img[img < 0.1] = 0.0
        img /= img.sum(1, keepdims=True)
        for i in range(cnt):
            nz = np.nonzero(img[i])[0]
            rows.append(nz.astype(np.int32))
            vals.append(img[i, nz].astype(np.float32))
            lens.append(nz.shape[0])
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(np.asarray(lens, dtype=np.int64), out=row_ptr[1:])
    return Histograms(row_ptr, np.concatenate(rows), np.concatenate(vals))


# --------------------------------------------------------------------------- configs

TEXT_LEN_TINY = ("uniform", 10, 40)
TEXT_LEN_SCALE = ("lognormal", 100.0, 0.5, 10, 1000)
QUERY_LEN_MIXED = ("loguniform", 5, 2000)


def text_workload(name, seed, V, m, n, doc_law, n_queries, query_law, k_list, top_k,
                  query_seed=None, query_limit=None) -> Workload:
    rng = np.random.Generator(np.random.PCG64(seed))
    emb = unit_embeddings(rng, V, m)
    db = zipf_histograms(rng, V, _lengths(rng, n, doc_law))
    queries = text_queries(V, n_queries, query_law, query_seed if query_seed is not None
                           else seed + QUERY_SEED_OFFSET, query_limit)
    return Workload(name, V, m, emb, None, db, queries, tuple(k_list), top_k)


def text_queries(V, n_queries, query_law, query_seed, query_limit=None) -> Histograms:
    qrng = np.random.Generator(np.random.PCG64(query_seed))
    nq = n_queries if query_limit is None else min(n_queries, query_limit)
    qlens = _lengths(qrng, n_queries, query_law)[:nq]
    return zipf_histograms(qrng, V, qlens)


def mixed_queries(query_limit: int | None = None) -> Histograms:
    """The queries of workload 4 (h_q log-uniform 5..2000 over the vocabulary of workload 2)
    without generating its database, which is workload 2's."""
    return text_queries(100000, 4096, QUERY_LEN_MIXED, BASE_SEED + 4 + QUERY_SEED_OFFSET, query_limit)


def image_workload(name, seed, n, n_queries, k_list, top_k, query_limit=None) -> Workload:
    rng = np.random.Generator(np.random.PCG64(seed))
    db = stroke_images(rng, n)
    qrng = np.random.Generator(np.random.PCG64(seed + QUERY_SEED_OFFSET))
    nq = n_queries if query_limit is None else min(n_queries, query_limit)
    queries = stroke_images(qrng, nq)
    return Workload(name, GRID * GRID, 2, pixel_coords(), pixel_cost_matrix(), db, queries,
                    tuple(k_list), top_k)


def config(cid: int, query_limit: int | None = None, n_docs: int | None = None) -> Workload:
    """The five workloads: 1 tiny text, 2 text at scale, 3 images, 4 mixed-size queries on
    the database of 2, 5 serving-size database.  `n_docs` shrinks the database (tests)."""
    s = BASE_SEED + cid
    if cid == 1:
        return text_workload("tiny-text V=2000 m=64 n=1000", s, 2000, 64, n_docs or 1000,
                             TEXT_LEN_TINY, 10, TEXT_LEN_TINY, (1, 2, 3, 4), 10,
                             query_limit=query_limit)
    if cid == 2:
        return text_workload("text V=100000 m=300 n=20000", s, 100000, 300, n_docs or 20000,
                             TEXT_LEN_SCALE, 1000, TEXT_LEN_SCALE, (1, 2, 4, 8, 16), 16,
                             query_limit=query_limit)
    if cid == 3:
        return image_workload("image 28x28 n=60000", s, n_docs or 60000, 10000,
                              tuple(range(1, 17)), 16, query_limit=query_limit)
    if cid == 4:
        return text_workload("mixed-h text V=100000 m=300 n=20000", BASE_SEED + 2, 100000, 300,
                             n_docs or 20000, TEXT_LEN_SCALE, 4096, QUERY_LEN_MIXED,
                             (4,), 16, query_seed=s + QUERY_SEED_OFFSET, query_limit=query_limit)
    if cid == 5:
        return text_workload("serving V=200000 m=300 n=1000000", s, 200000, 300, n_docs or 1000000,
                             TEXT_LEN_SCALE, 100000, QUERY_LEN_MIXED, (4,), 16,
                             query_limit=query_limit)
    raise ValueError(cid)


def small_text(seed: int, V: int, m: int, n: int, n_queries: int, lo: int, hi: int,
               qlo: int | None = None, qhi: int | None = None) -> Workload:
    """A small text-like workload with chosen sizes (parity cases that span several tiles
    and a ragged tail)."""
    return text_workload(f"text V={V} m={m} n={n}", seed, V, m, n, ("uniform", lo, hi),
                         n_queries, ("uniform", qlo or lo, qhi or hi), (1, 2, 4), 10)
