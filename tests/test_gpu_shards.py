"""Database sharding on the device: two databases holding contiguous halves of the
documents, each queried with emd_topk, merged with emd_topk_merge, equal the unsharded
database's top-K bit for bit (every per-document value is computed the same way whatever
other documents share its database)."""
import numpy as np
import pytest

import emd_synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def emd():
    import paper_1812_02091_gb300 as m
    from paper_1812_02091_gb300 import _build
    _build.build()
    m.load()
    return m


@pytest.mark.parametrize("precision,meas,k", [("fp32_tc", "act", 4), ("fp32", "omr", 1), ("fp32_tc", "ict", 1)])
def test_sharded_topk_equals_whole(emd, precision, meas, k):
    w = emd_synth.small_text(8080, 3000, 64, 1700, 19, 4, 60, 3, 150)
    q = w.queries
    K = 16
    bounds = [0, 777, 1700]
    dbs = []
    try:
        whole = emd.emd_db_create(w.emb, None, w.db.row_ptr, w.db.col, w.db.val,
                                  emd.emd_db_options_default(precision=precision, max_query_h=256), v=w.v)
        dbs.append(whole)
        ref = emd.emd_topk(whole, q.row_ptr, q.col, q.val, meas, k, "max", K)
        shards = []
        for s in range(2):
            part = w.db.subset(np.arange(bounds[s], bounds[s + 1]))
            db = emd.emd_db_create(w.emb, None, part.row_ptr, part.col, part.val,
                                   emd.emd_db_options_default(precision=precision, max_query_h=256), v=w.v)
            dbs.append(db)
            shards.append(emd.emd_topk(db, q.row_ptr, q.col, q.val, meas, k, "max", K))
        mi, md = emd.emd_topk_merge(shards, bounds[:2], K)
        assert np.array_equal(mi, ref[0]) and np.array_equal(md, ref[1])
    finally:
        for db in dbs:
            emd.emd_db_destroy(db)


@pytest.mark.parametrize("precision,meas,k", [("fp32_tc", "act", 4), ("fp32", "act", 2)])
def test_sharded_topk_against_oracle(emd, precision, meas, k):
    """Three shards of unequal size, each its own database: the merged top-K equals the FP64
    oracle's top-K over the whole database outside the tie group of the K-th distance, with
    each returned distance the oracle's value of that document (1e-5 relative)."""
    import oracle
    w = emd_synth.small_text(9191, 3000, 64, 2100, 8, 4, 60, 3, 300)
    q = w.queries
    K = 16
    bounds = [0, 500, 1320, 2100]
    shards, dbs = [], []
    try:
        for s in range(3):
            part = w.db.subset(np.arange(bounds[s], bounds[s + 1]))
            db = emd.emd_db_create(w.emb, None, part.row_ptr, part.col, part.val,
                                   emd.emd_db_options_default(precision=precision, max_query_h=512), v=w.v)
            dbs.append(db)
            shards.append(emd.emd_topk(db, q.row_ptr, q.col, q.val, meas, k, "max", K))
        mi, md = emd.emd_topk_merge(shards, bounds[:3], K)
    finally:
        for db in dbs:
            emd.emd_db_destroy(db)
    for i in range(q.n):
        tf, tr = oracle.lc_query(w.emb, None, w.db, *q.row(i), meas, k)
        ref = np.maximum(tf, tr)
        order = np.lexsort((np.arange(len(ref)), ref))
        dK = ref[order[K - 1]]
        tie = np.abs(ref - dK) <= 1e-5 * dK + 1e-9
        assert {int(j) for j in order[:K] if not tie[j]} == {int(j) for j in mi[i] if not tie[j]}, i
        np.testing.assert_allclose(md[i], ref[mi[i]], rtol=1e-5, atol=1e-7)
