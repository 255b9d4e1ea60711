"""The Section 6 baselines on the device (bag-of-words cosine similarity, word centroid
distance) against the FP64 oracle."""
import numpy as np
import pytest

import emd_synth
import oracle

pytestmark = pytest.mark.gpu

RTOL, ATOL = 1e-5, 1e-6


@pytest.fixture(scope="module")
def emd():
    import paper_1812_02091_gb300 as m
    from paper_1812_02091_gb300 import _build
    _build.build()
    m.load()
    return m


@pytest.fixture(scope="module")
def work():
    # 21 queries: two full groups of eight and a ragged one; 3..180 bins, some ids unused
    return emd_synth.small_text(612, 3000, 96, 2600, 21, 5, 60, 3, 180)


def make_db(emd, w, **opt):
    return emd.emd_db_create(w.emb if w.cost is None else None, w.cost, w.db.row_ptr, w.db.col, w.db.val,
                             emd.emd_db_options_default(**opt), v=w.v)


def check_topk(gi, gd, want, K):
    order = np.lexsort((np.arange(len(want)), want))
    dK = want[order[K - 1]]
    tie = np.abs(want - dK) <= 1e-5 * abs(dK) + 1e-6
    assert {int(i) for i in order[:K] if not tie[i]} == {int(i) for i in gi if not tie[i]}
    np.testing.assert_allclose(gd, want[gi], rtol=RTOL, atol=ATOL)


@pytest.mark.parametrize("max_batch", [64, 8])
def test_bow_against_oracle(emd, work, max_batch):
    w = work
    q = w.queries
    db = make_db(emd, w, max_query_h=256, max_batch=max_batch)
    try:
        got = emd.emd_baseline_batch(db, q.row_ptr, q.col, q.val, "bow")
        want = [oracle.bow_cosine(w.v, w.db, *q.row(i)) for i in range(q.n)]
        for i in range(q.n):
            np.testing.assert_allclose(got[i], want[i], rtol=RTOL, atol=ATOL)
        gi, gd = emd.emd_baseline_topk(db, q.row_ptr, q.col, q.val, "bow", 12)
        for i in range(q.n):
            check_topk(gi[i], gd[i], np.maximum(1.0 - want[i], 0.0), 12)
        # the dense query vectors are cleared after each batch: a second, different batch
        # gives what it gives alone
        sub = q.subset(np.arange(5, 9))
        again = emd.emd_baseline_batch(db, sub.row_ptr, sub.col, sub.val, "bow")
        assert np.array_equal(again, got[5:9])
    finally:
        emd.emd_db_destroy(db)


@pytest.mark.parametrize("max_batch", [64, 8])
def test_wcd_against_oracle(emd, work, max_batch):
    w = work
    q = w.queries
    db = make_db(emd, w, max_query_h=256, max_batch=max_batch)
    try:
        got = emd.emd_baseline_batch(db, q.row_ptr, q.col, q.val, "wcd")
        want = [oracle.wcd(w.emb, w.db, *q.row(i)) for i in range(q.n)]
        for i in range(q.n):
            np.testing.assert_allclose(got[i], want[i], rtol=RTOL, atol=ATOL)
        gi, gd = emd.emd_baseline_topk(db, q.row_ptr, q.col, q.val, "wcd", 12)
        for i in range(q.n):
            check_topk(gi[i], gd[i], want[i], 12)
    finally:
        emd.emd_db_destroy(db)


def test_wcd_self_zero_and_symmetric(emd, work):
    """Database histograms as queries: WCD(p, p) = 0 and WCD(p, q) = WCD(q, p)."""
    w = work
    db = make_db(emd, w, max_query_h=256)
    try:
        sub = w.db.subset(np.arange(0, 40))
        got = emd.emd_baseline_batch(db, sub.row_ptr, sub.col, sub.val, "wcd")
        assert np.all(np.abs(got[np.arange(40), np.arange(40)]) <= 1e-6)
        np.testing.assert_allclose(got[:, :40], got[:, :40].T, rtol=RTOL, atol=ATOL)
    finally:
        emd.emd_db_destroy(db)


def test_baselines_cost_matrix_mode(emd):
    w = emd_synth.config(3, query_limit=5, n_docs=700)
    q = w.queries
    db = make_db(emd, w, max_query_h=784)
    try:
        got = emd.emd_baseline_batch(db, q.row_ptr, q.col, q.val, "bow")
        for i in range(q.n):
            np.testing.assert_allclose(got[i], oracle.bow_cosine(w.v, w.db, *q.row(i)), rtol=RTOL, atol=ATOL)
        with pytest.raises(emd.EmdError, match="UNSUPPORTED"):
            emd.emd_baseline_batch(db, q.row_ptr, q.col, q.val, "wcd")
        with pytest.raises(emd.EmdError, match="INVALID_ARG"):
            emd.emd_baseline_topk(db, q.row_ptr, q.col, q.val, "bow", 65)
    finally:
        emd.emd_db_destroy(db)
