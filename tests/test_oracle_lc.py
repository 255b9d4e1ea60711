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


@pytest.mark.parametrize("meas,k", [("rwmd", 1), ("omr", 1), ("act", 2), ("act", 4), ("act", 9), ("ict", 1)])
def test_split_forward_equals_lc_query(tiny, meas, k):
    """lc_forward_split (Phase 1 on vocabulary-row slices, Phase 2 and 3 on document
    slices, on threads) takes the same steps per table row and per document as
    oracle_lc_query, so its forward values are identical."""
    for qi in (0, 4, 9):
        qidx, qw = tiny.queries.row(qi)
        lf, _ = oracle.lc_query(tiny.emb, None, tiny.db, qidx, qw, meas, k, rev=False)
        for threads in (1, 3, 8):
            sf = oracle.lc_forward_split(tiny.emb, None, tiny.db, qidx, qw, meas, k, threads=threads)
            np.testing.assert_array_equal(sf, lf)


def test_split_forward_equals_lc_query_images(image_small):
    w = image_small
    qidx, qw = w.queries.row(1)
    for meas, k in (("act", 3), ("omr", 1)):
        lf, _ = oracle.lc_query(w.emb, w.cost, w.db, qidx, qw, meas, k, rev=False)
        np.testing.assert_array_equal(oracle.lc_forward_split(w.emb, w.cost, w.db, qidx, qw, meas, k, threads=4), lf)


@pytest.mark.parametrize("meas,k,K", [("act", 2, 10), ("act", 4, 16), ("omr", 1, 5), ("ict", 1, 16), ("rwmd", 1, 1)])
def test_certified_symmetric_topk_equals_brute_force(tiny, meas, k, K):
    """SymTopK evaluates the reverse direction only in ascending forward order until the
    certificate holds; its top-K equals the top-K of max(fwd, rev) over all documents
    (per-pair definition), ids in (distance, id) order, distances to FP64 round-off."""
    for qi in range(tiny.queries.n):
        qidx, qw = tiny.queries.row(qi)
        pf, pr = oracle.pair_db(tiny.emb, None, tiny.db, qidx, qw, meas, k)
        want_i, want_d = oracle.topk(np.maximum(pf, pr), K)
        got = oracle.SymTopK(tiny.emb, None, tiny.db, qidx, qw, meas, k, K, threads=4)
        np.testing.assert_array_equal(got.idx, want_i)
        np.testing.assert_allclose(got.dist, want_d, rtol=1e-12, atol=0)
        assert len(got.rev) < tiny.db.n  # the certificate stopped the scan early
        extra = [3, 500, 999]
        np.testing.assert_allclose(got.sym_of(extra), np.maximum(pf, pr)[extra], rtol=1e-12, atol=0)


@pytest.mark.parametrize("meas,k", [("rwmd", 1), ("omr", 1), ("act", 3), ("act", 40), ("ict", 1)])
def test_full_split_equals_lc_query(tiny, meas, k):
    """lc_query_full_split (cost block on row slices, stable sort of each row, Phase 2 and 3
    and the reverse direction on document slices) equals oracle_lc_query bit for bit."""
    prep = oracle.prepare(tiny.emb, None, tiny.db)
    for qi in (1, 5, 8):
        qidx, qw = tiny.queries.row(qi)
        lf, lr = oracle.lc_query(tiny.emb, None, tiny.db, qidx, qw, meas, k)
        for threads in (1, 5):
            sf, sr = oracle.lc_query_full_split(tiny.emb, None, tiny.db, qidx, qw, meas, k, threads=threads, prep=prep)
            np.testing.assert_array_equal(sf, lf)
            np.testing.assert_array_equal(sr, lr)


def test_full_split_equals_lc_query_images(image_small):
    w = image_small
    qidx, qw = w.queries.row(2)
    for meas, k in (("act", 5), ("ict", 1)):
        lf, lr = oracle.lc_query(w.emb, w.cost, w.db, qidx, qw, meas, k)
        sf, sr = oracle.lc_query_full_split(w.emb, w.cost, w.db, qidx, qw, meas, k, threads=3)
        np.testing.assert_array_equal(sf, lf)
        np.testing.assert_array_equal(sr, lr)
