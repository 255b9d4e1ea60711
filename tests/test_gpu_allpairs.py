"""All-pairs top-K over the database itself (emd_all_pairs_topk): every histogram ranked
against all others, as in the evaluation of Section 6, against the oracle.

The device computes one forward pass per histogram and takes the reverse bound of a pair
as the forward bound of the transposed pair; the oracle computes both directions of each
sampled row directly, so the two share neither the reverse arithmetic nor the order of
summation (FP32 tolerance)."""
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
    return emd.emd_db_create(w.emb if w.cost is None else None, w.cost, w.db.row_ptr, w.db.col,
                             w.db.val, emd.emd_db_options_default(**opt), v=w.v)


def check_rows(w, idx, dist, rows, meas, k, K):
    n = w.db.n
    for a in rows:
        tf, tr = oracle.lc_query(w.emb, w.cost, w.db, *w.db.row(a), meas, k)
        want = np.maximum(tf, tr)
        want[a] = np.inf
        assert a not in set(idx[a].tolist())
        order = np.lexsort((np.arange(n), want))
        dK = want[order[K - 1]]
        tie = np.abs(want - dK) <= 1e-5 * dK + 1e-9
        assert {int(i) for i in order[:K] if not tie[i]} == {int(i) for i in idx[a] if not tie[i]}, a
        np.testing.assert_allclose(dist[a], want[idx[a]], rtol=RTOL, atol=ATOL)


@pytest.mark.parametrize("precision", ["fp32", "fp32_tc"])
@pytest.mark.parametrize("meas,k", [("act", 4), ("omr", 1), ("rwmd", 1)])
def test_all_pairs_text(emd, precision, meas, k):
    # 301 histograms (ten batches of 32 and a ragged one; ten 32-row tiles and a tail)
    w = emd_synth.small_text(1812, 2500, 48, 301, 1, 3, 70)
    K = 10
    db = make_db(emd, w, precision=precision, max_query_h=128, max_batch=32)
    try:
        idx, dist = emd.emd_all_pairs_topk(db, meas, k, K)
        assert idx.shape == (w.db.n, K)
        assert np.all(np.diff(dist, axis=1) >= 0)
        check_rows(w, idx, dist, [0, 1, 31, 32, 150, 299, 300], meas, k, K)
        # the symmetric bound of a pair is one number: both rows that hold it agree bit for bit
        pos = {(a, int(b)): float(d) for a in range(w.db.n) for b, d in zip(idx[a], dist[a])}
        both = [(a, b) for (a, b) in pos if (b, a) in pos]
        assert both
        assert all(pos[(a, b)] == pos[(b, a)] for a, b in both)
    finally:
        emd.emd_db_destroy(db)


def test_all_pairs_images(emd):
    """Cost-matrix mode (28 x 28 pixel grid, Section 6 image workload)."""
    w = emd_synth.config(3, query_limit=1, n_docs=200)
    db = make_db(emd, w, max_query_h=784)
    try:
        idx, dist = emd.emd_all_pairs_topk(db, "act", 2, 16)
        check_rows(w, idx, dist, [0, 77, 199], "act", 2, 16)
    finally:
        emd.emd_db_destroy(db)


def test_all_pairs_unbatched_equals_batched(emd):
    w = emd_synth.small_text(7, 1500, 32, 130, 1, 3, 40)
    db_a = make_db(emd, w, precision="fp32_tc", max_query_h=64, batched=0)
    db_b = make_db(emd, w, precision="fp32_tc", max_query_h=64, max_batch=16)
    try:
        ia, da = emd.emd_all_pairs_topk(db_a, "act", 3, 8)
        ib, db_ = emd.emd_all_pairs_topk(db_b, "act", 3, 8)
        assert np.array_equal(ia, ib) and np.array_equal(da, db_)
    finally:
        emd.emd_db_destroy(db_a)
        emd.emd_db_destroy(db_b)


def test_all_pairs_limits(emd):
    w = emd_synth.small_text(8, 800, 32, 40, 1, 3, 40)
    db = make_db(emd, w, max_query_h=16)
    try:
        with pytest.raises(emd.EmdError, match="INVALID_ARG"):  # histograms above max_query_h bins
            emd.emd_all_pairs_topk(db, "act", 2, 4)
    finally:
        emd.emd_db_destroy(db)
    db = make_db(emd, w, max_query_h=64)
    try:
        with pytest.raises(emd.EmdError, match="INVALID_ARG"):  # K must leave out the histogram itself
            emd.emd_all_pairs_topk(db, "act", 2, 40)
        idx, dist = emd.emd_all_pairs_topk(db, "act", 2, 39)   # every other histogram
        for a in range(w.db.n):
            assert sorted(idx[a].tolist()) == [b for b in range(w.db.n) if b != a]
    finally:
        emd.emd_db_destroy(db)
