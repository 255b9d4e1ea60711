"""Parity of the tensor-core Phase-1 path (precision EMD_PREC_FP32_TC: FP16 split operands,
three tcgen05 products, FP32 accumulators in TMEM) with the FP64 oracle, at the same
tolerance as the plain FP32 path: 1e-5 relative."""
import numpy as np
import pytest

import emd_synth
import oracle

pytestmark = pytest.mark.gpu

RTOL, ATOL = 1e-5, 1e-7


@pytest.fixture(scope="module")
def emd():
    import paper_1812_02091_gb300 as m
    from paper_1812_02091_gb300 import _build
    _build.build()
    m.load()
    return m


def make_db(emd, w, **opt):
    return emd.emd_db_create(w.emb, None, w.db.row_ptr, w.db.col, w.db.val,
                             emd.emd_db_options_default(precision="fp32_tc", **opt), v=w.v)


def oracle_dir(w, qi, meas, k, direction):
    qidx, qw = w.queries.row(qi)
    tf, tr = oracle.lc_query(w.emb, None, w.db, qidx, qw, meas, k,
                             fwd=direction != "rev", rev=direction != "fwd")
    return tf if direction == "fwd" else tr if direction == "rev" else np.maximum(tf, tr)


@pytest.fixture(scope="module")
def tiny(emd):
    w = emd_synth.config(1)
    db = make_db(emd, w, max_query_h=64)
    yield w, db
    emd.emd_db_destroy(db)


def test_tc_phase1_table_matches_oracle(emd, tiny):
    w, db = tiny
    for qi in range(3):
        qidx, qw = w.queries.row(qi)
        used, z, s, wt = emd.emd_phase1_table(db, qidx, qw, 4)
        Z, S, W = oracle.phase1(w.emb, None, used, qidx, qw, 4)
        np.testing.assert_allclose(z, Z, rtol=RTOL, atol=ATOL)
        np.testing.assert_array_equal(s, S)


@pytest.mark.parametrize("meas,k", [("rwmd", 1), ("omr", 1), ("act", 2), ("act", 4), ("ict", 1)])
def test_tc_tiny_all_queries(emd, tiny, meas, k):
    w, db = tiny
    q = w.queries
    for direction in ("fwd", "rev", "max"):
        got = emd.emd_query_batch(db, q.row_ptr, q.col, q.val, meas, k, direction)
        for qi in range(q.n):
            np.testing.assert_allclose(got[qi], oracle_dir(w, qi, meas, k, direction), rtol=RTOL, atol=ATOL)


def test_tc_several_column_tiles_and_odd_m(emd):
    """m = 37 (K padded to 64), queries of 100..300 bins (up to three 128-column tiles, a
    ragged last tile), more than one 128-row vocabulary tile with a ragged tail."""
    w = emd_synth.small_text(5150, V=3000, m=37, n=300, n_queries=4, lo=5, hi=60, qlo=100, qhi=300)
    db = make_db(emd, w, max_query_h=320)
    try:
        q = w.queries
        got = emd.emd_query_batch(db, q.row_ptr, q.col, q.val, "act", 3, "max")
        for qi in range(q.n):
            np.testing.assert_allclose(got[qi], oracle_dir(w, qi, "act", 3, "max"), rtol=RTOL, atol=ATOL)
        qidx, qw = q.row(0)
        used, z, s, wt = emd.emd_phase1_table(db, qidx, qw, 8)
        Z, S, W = oracle.phase1(w.emb, None, used, qidx, qw, 8)
        np.testing.assert_allclose(z, Z, rtol=RTOL, atol=ATOL)
    finally:
        emd.emd_db_destroy(db)


def test_tc_full_size_text(emd):
    w = emd_synth.config(2, query_limit=3)
    db = make_db(emd, w, max_query_h=1024, max_batch=8)
    try:
        q = w.queries
        got = emd.emd_query_batch(db, q.row_ptr, q.col, q.val, "act", 4, "max")
        idx, dist = emd.emd_topk(db, q.row_ptr, q.col, q.val, "act", 4, "max", 16)
        for qi in range(q.n):
            qidx, qw = q.row(qi)
            tf, tr = oracle.lc_query_split(w.emb, None, w.db, qidx, qw, "act", 4)
            want = np.maximum(tf, tr)
            np.testing.assert_allclose(got[qi], want, rtol=RTOL, atol=ATOL)
            order = np.lexsort((np.arange(w.db.n), want))[:16]
            dK = want[order[15]]
            tie = np.abs(want - dK) <= 1e-5 * dK + 1e-9
            assert {int(i) for i in order if not tie[i]} == {int(i) for i in idx[qi] if not tie[i]}
        emd.emd_db_check_device_errors(db)
    finally:
        emd.emd_db_destroy(db)
