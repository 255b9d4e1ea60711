"""The linear-complexity form (Section 5: Phase 1, Eq. 6-8, Eq. 9) reaches the per-pair
definition (Algorithms 1-3) exactly: a vocabulary row's top-k over the query is the same
set whether computed once for the vocabulary or per pair (Section 2.2).  Only the
summation order differs, so the two agree to FP64 round-off."""
import numpy as np
import pytest

import emd_synth
import oracle


@pytest.fixture(scope="module")
def tiny():
    return emd_synth.config(1)


@pytest.fixture(scope="module")
def image_small():
    return emd_synth.config(3, query_limit=3, n_docs=300)


MEAS = [("rwmd", 1), ("omr", 1), ("act", 1), ("act", 2), ("act", 3), ("act", 4), ("act", 7),
        ("ict", 1)]


@pytest.mark.parametrize("meas,k", MEAS)
def test_lc_form_equals_pairwise_text(tiny, meas, k):
    for qi in range(0, tiny.queries.n, 3):
        qidx, qw = tiny.queries.row(qi)
        pf, pr = oracle.pair_db(tiny.emb, None, tiny.db, qidx, qw, meas, k)
        lf, lr = oracle.lc_query(tiny.emb, None, tiny.db, qidx, qw, meas, k)
        np.testing.assert_allclose(lf, pf, rtol=1e-12, atol=0)
        np.testing.assert_allclose(lr, pr, rtol=1e-12, atol=0)


@pytest.mark.parametrize("meas,k", [("rwmd", 1), ("omr", 1), ("act", 2), ("act", 16), ("ict", 1)])
def test_lc_form_equals_pairwise_image(image_small, meas, k):
    w = image_small
    for qi in range(w.queries.n):
        qidx, qw = w.queries.row(qi)
        pf, pr = oracle.pair_db(w.emb, w.cost, w.db, qidx, qw, meas, k)
        lf, lr = oracle.lc_query(w.emb, w.cost, w.db, qidx, qw, meas, k)
        np.testing.assert_allclose(lf, pf, rtol=1e-12, atol=1e-15)
        np.testing.assert_allclose(lr, pr, rtol=1e-12, atol=1e-15)


def test_image_rwmd_vanishes_on_full_overlap(image_small):
    """Section 4 / Table 5: a query whose support equals a document's support has RWMD 0
    to that document in both directions, while OMR stays positive."""
    w = image_small
    cols, vals = w.db.row(0)
    rng = np.random.default_rng(7)
    qw = (vals.astype(np.float64) * rng.uniform(0.5, 1.5, len(vals)))
    qw = (qw / qw.sum()).astype(np.float32)
    one = emd_synth.Histograms(np.array([0, len(cols)], np.int64), cols, vals)
    rf, rr = oracle.lc_query(w.emb, w.cost, one, cols, qw, "rwmd")
    of, orr = oracle.lc_query(w.emb, w.cost, one, cols, qw, "omr")
    assert rf[0] == 0.0 and rr[0] == 0.0
    assert of[0] > 0.0 and orr[0] > 0.0


def test_phase1_tables_match_sorted_rows(tiny):
    qidx, qw = tiny.queries.row(0)
    rows = np.unique(tiny.db.col)[:50]
    Z, S, W = oracle.phase1(tiny.emb, None, rows, qidx, qw, 4)
    C = oracle.cost_block(tiny.emb, None, rows, qidx)
    for r in range(len(rows)):
        order = np.lexsort((np.arange(len(qidx)), C[r]))[:4]
        np.testing.assert_array_equal(S[r], order)
        np.testing.assert_array_equal(Z[r], C[r, order])
        np.testing.assert_array_equal(W[r], qw[order].astype(np.float64))
