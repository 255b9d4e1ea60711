"""Parity at the configs' full query sizes: workload 4 (the text database of workload 2,
V = 1e5, m = 300, n = 2e4, with queries of h_q log-uniform in 5..2000) on a seeded subset
of 32 queries stratified by size -- the pool's longest query, at least four with
h_q > 1000, eight with 300 < h_q <= 1000, the rest shorter -- in every Phase-1 arithmetic,
through the C ABI, against the FP64 oracle (lc_query_full_split: the oracle's own steps
on threads, identical to oracle_lc_query).

These queries span up to 16 column tiles of 128 in the tensor-core kernels, table rows
scanned over ~2000 columns, reverse passes with long query lists and re-ranked rows of the
approximate forms.

FP32 forms (plain SIMT and the FP32-grade FP16 split): every distance of every document in
each direction within 1e-5 relative (+1e-7 absolute), and the top-16 identical to the
oracle's outside the tie group of the 16th distance (|d - d_16| <= 1e-5 d_16 + 1e-9, the
oracle's own distances).

Approximate forms (BF16, FP8-E4M3 products with per-row scales, exact FP32 re-rank of each
row's k + 8 candidates): reverse distances within the operand-rounding bound of R15
(unit roundoff u: 2^-8 BF16, 2^-4 E4M3; |d(a.b)| <= (2u + u^2)|a||b| for unit rows, so a
squared distance moves by at most 2(2u + u^2) and a reverse value, the row cost being
1-Lipschitz per unit mass, by at most (2u + u^2)/d_min relative with d_min >= 1 here);
forward distances exact wherever the true nearest entries were among the re-ranked
candidates, otherwise within twice that bound (a table entry can be replaced only by one
whose approximate value was no larger); top-16 recall against the oracle under the same tie
rule, reported and held to a floor.
"""
import os

import numpy as np
import pytest

import emd_synth
import oracle

pytestmark = pytest.mark.gpu

RTOL, ATOL = 1e-5, 1e-7
BOUND = {"bf16": 2 * 2.0 ** -8 + 2.0 ** -16, "fp8": 2 * 2.0 ** -4 + 2.0 ** -8}
K = 16
KW = 4  # LC-ACT k of the workload


def stratified_subset(hs: np.ndarray, seed: int = 44) -> np.ndarray:
    rng = np.random.default_rng(seed)
    longest = int(np.argmax(hs))
    long_ = np.setdiff1d(np.nonzero(hs > 1000)[0], [longest])
    mid = np.nonzero((hs > 300) & (hs <= 1000))[0]
    short = np.nonzero(hs <= 300)[0]
    pick = np.concatenate([[longest], rng.choice(long_, 4, replace=False), rng.choice(mid, 8, replace=False),
                           rng.choice(short, 19, replace=False)])
    return np.sort(pick).astype(np.int64)


@pytest.fixture(scope="module")
def emd():
    import paper_1812_02091_gb300 as m
    from paper_1812_02091_gb300 import _build
    _build.build()
    m.load()
    return m


@pytest.fixture(scope="module")
def work():
    w = emd_synth.config(2, query_limit=1)
    pool = emd_synth.mixed_queries()
    sub = stratified_subset(np.diff(pool.row_ptr))
    return w, pool.subset(sub)


@pytest.fixture(scope="module")
def want(work):
    w, q = work
    prep = oracle.prepare(w.emb, None, w.db)
    threads = os.cpu_count() or 1
    return [oracle.lc_query_full_split(w.emb, None, w.db, *q.row(i), "act", KW, threads=threads, prep=prep)
            for i in range(q.n)]


def test_subset_covers_the_long_queries(work):
    _, q = work
    hs = np.diff(q.row_ptr)
    assert q.n == 32 and (hs > 1000).sum() >= 5 and hs.max() > 1900 and hs.min() < 50


def make_db(emd, w, precision):
    return emd.emd_db_create(w.emb, None, w.db.row_ptr, w.db.col, w.db.val,
                             emd.emd_db_options_default(precision=precision, max_query_h=2048), v=w.v)


def oracle_topk_sets(ref, K):
    order = np.lexsort((np.arange(len(ref)), ref))
    dK = ref[order[K - 1]]
    tie = np.abs(ref - dK) <= 1e-5 * dK + 1e-9
    return order, dK, tie


@pytest.mark.parametrize("precision", ["fp32", "fp32_tc"])
def test_fp32_forms_every_distance(emd, work, want, precision):
    w, q = work
    db = make_db(emd, w, precision)
    try:
        for d in ("fwd", "rev", "max"):
            got = emd.emd_query_batch(db, q.row_ptr, q.col, q.val, "act", KW, d)
            for i in range(q.n):
                tf, tr = want[i]
                ref = tf if d == "fwd" else tr if d == "rev" else np.maximum(tf, tr)
                np.testing.assert_allclose(got[i], ref, rtol=RTOL, atol=ATOL,
                                           err_msg=f"{precision} {d} query {i} h={q.row_ptr[i + 1] - q.row_ptr[i]}")
        gi, gd = emd.emd_topk(db, q.row_ptr, q.col, q.val, "act", KW, "max", K)
        for i in range(q.n):
            ref = np.maximum(*want[i])
            order, dK, tie = oracle_topk_sets(ref, K)
            assert {int(j) for j in order[:K] if not tie[j]} == {int(j) for j in gi[i] if not tie[j]}, i
            np.testing.assert_allclose(gd[i], ref[gi[i]], rtol=RTOL, atol=ATOL)
            keys = list(zip(gd[i].tolist(), gi[i].tolist()))
            assert keys == sorted(keys)
        emd.emd_db_check_device_errors(db)
    finally:
        emd.emd_db_destroy(db)


RECALL_FLOOR = {"bf16": 0.9, "fp8": 0.5}


@pytest.mark.parametrize("precision", ["bf16", "fp8"])
def test_approximate_forms_against_oracle(emd, work, want, precision):
    w, q = work
    b = BOUND[precision]
    db = make_db(emd, w, precision)
    try:
        fwd = emd.emd_query_batch(db, q.row_ptr, q.col, q.val, "act", KW, "fwd")
        rev = emd.emd_query_batch(db, q.row_ptr, q.col, q.val, "act", KW, "rev")
        exact_frac = []
        for i in range(q.n):
            tf, tr = want[i]
            rf = np.abs(fwd[i] - tf) / tf
            exact_frac.append(float(np.mean(rf <= RTOL)))
            assert rf.max() <= 2 * b, (i, rf.max())
            assert (np.abs(rev[i] - tr) / tr).max() <= b, i
        gi, gd = emd.emd_topk(db, q.row_ptr, q.col, q.val, "act", KW, "max", K)
        recalls = []
        for i in range(q.n):
            ref = np.maximum(*want[i])
            order, dK, tie = oracle_topk_sets(ref, K)
            truth = {int(j) for j in order[:K]}
            recalls.append(sum(1 for j in gi[i] if int(j) in truth or tie[int(j)]) / K)
            assert (np.abs(gd[i] - ref[gi[i]]) / ref[gi[i]]).max() <= 2 * b
        print(f"{precision}: forward values exact at 1e-5: {np.mean(exact_frac):.6f}; "
              f"top-{K} recall {np.mean(recalls):.4f} (min {np.min(recalls):.4f}) over {q.n} queries")
        assert np.mean(recalls) >= RECALL_FLOOR[precision]
        emd.emd_db_check_device_errors(db)
    finally:
        emd.emd_db_destroy(db)
