"""ICT (Section 4.2, Algorithm 2) at full query sizes, against the oracle.

The forward table of a vocabulary row holds the row's nearest query bins in ascending
order only as far as the largest database weight of that row needs (its residual reaches
0), at most max_table_k entries; a query for which some row needs more is recomputed with
tables of full width h.  Either way the forward values are those of Algorithm 2 with every
destination available, so they are checked against the oracle's ICT at the FP32
tolerance, and the narrow and full-width forms against each other bit for bit."""
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


@pytest.fixture(scope="module")
def work():
    # queries of 3..300 bins (beyond max_table_k), documents of 5..60 bins
    return emd_synth.small_text(360, 3000, 64, 1500, 12, 5, 60, 3, 300)


@pytest.fixture(scope="module")
def want(work):
    w = work
    return [oracle.lc_query(w.emb, None, w.db, *w.queries.row(i), "ict") for i in range(w.queries.n)]


def make_db(emd, w, **opt):
    return emd.emd_db_create(w.emb if w.cost is None else None, w.cost, w.db.row_ptr, w.db.col, w.db.val,
                             emd.emd_db_options_default(**opt), v=w.v)


def run_dirs(emd, db, q):
    return {d: emd.emd_query_batch(db, q.row_ptr, q.col, q.val, "ict", 1, d) for d in ("fwd", "rev", "max")}


@pytest.mark.parametrize("precision,batched", [("fp32", 1), ("fp32_tc", 1), ("fp32_tc", 0)])
def test_ict_directions_against_oracle(emd, work, want, precision, batched):
    w = work
    db = make_db(emd, w, precision=precision, max_query_h=512, batched=batched)
    try:
        got = run_dirs(emd, db, w.queries)
        for qi in range(w.queries.n):
            tf, tr = want[qi]
            np.testing.assert_allclose(got["fwd"][qi], tf, rtol=RTOL, atol=ATOL)
            np.testing.assert_allclose(got["rev"][qi], tr, rtol=RTOL, atol=ATOL)
            np.testing.assert_allclose(got["max"][qi], np.maximum(tf, tr), rtol=RTOL, atol=ATOL)
    finally:
        emd.emd_db_destroy(db)


@pytest.mark.parametrize("batched", [1, 0])
def test_ict_overflow_recomputed_exactly(emd, work, batched):
    """max_table_k = 4: most queries need longer rows and are recomputed with full-width
    tables; the values equal those of a database whose tables may always be h wide
    (max_table_k 512 >= every h) bit for bit."""
    w = work
    db_w = make_db(emd, w, precision="fp32_tc", max_query_h=512, max_table_k=512)
    db_n = make_db(emd, w, precision="fp32_tc", max_query_h=512, max_table_k=4, batched=batched)
    try:
        ref = run_dirs(emd, db_w, w.queries)
        assert emd.emd_db_profile_get(db_w)["ict_wide"] == 0
        got = run_dirs(emd, db_n, w.queries)
        for d in ("fwd", "max"):
            assert np.array_equal(got[d], ref[d]), d
        assert emd.emd_db_profile_get(db_n)["ict_wide"] > 0
        ti, td = emd.emd_topk(db_w, w.queries.row_ptr, w.queries.col, w.queries.val, "ict", 1, "max", 10)
        ni, nd = emd.emd_topk(db_n, w.queries.row_ptr, w.queries.col, w.queries.val, "ict", 1, "max", 10)
        assert np.array_equal(ti, ni) and np.array_equal(td, nd)
    finally:
        emd.emd_db_destroy(db_w)
        emd.emd_db_destroy(db_n)


def test_ict_topk_pruned(emd, work, want):
    """Pruned symmetric top-K (reverse on the forward candidates only) against the oracle,
    and bit-identical to the unpruned path."""
    w = work
    K = 10
    db = make_db(emd, w, precision="fp32_tc", max_query_h=512)
    db_u = make_db(emd, w, precision="fp32_tc", max_query_h=512, prune_topk=0)
    try:
        gi, gd = emd.emd_topk(db, w.queries.row_ptr, w.queries.col, w.queries.val, "ict", 1, "max", K)
        assert emd.emd_db_profile_get(db)["pruned_queries"] == w.queries.n
        ui, ud = emd.emd_topk(db_u, w.queries.row_ptr, w.queries.col, w.queries.val, "ict", 1, "max", K)
        assert np.array_equal(gi, ui) and np.array_equal(gd, ud)
        for qi in range(w.queries.n):
            ref = np.maximum(*want[qi])
            order = np.lexsort((np.arange(len(ref)), ref))
            dK = ref[order[K - 1]]
            tie = np.abs(ref - dK) <= 1e-5 * dK + 1e-9
            assert {int(i) for i in order[:K] if not tie[i]} == {int(i) for i in gi[qi] if not tie[i]}
            np.testing.assert_allclose(gd[qi], ref[gi[qi]], rtol=RTOL, atol=ATOL)
    finally:
        emd.emd_db_destroy(db)
        emd.emd_db_destroy(db_u)


def test_ict_above_act(emd, work):
    """ACT is non-decreasing in k and reaches ICT at k = h (Section 4.2): on the device,
    forward ICT >= forward ACT for k = 1, 4, 16 within rounding."""
    w = work
    db = make_db(emd, w, precision="fp32_tc", max_query_h=512)
    try:
        q = w.queries
        ict = emd.emd_query_batch(db, q.row_ptr, q.col, q.val, "ict", 1, "fwd")
        prev = None
        for k in (1, 4, 16):
            act = emd.emd_query_batch(db, q.row_ptr, q.col, q.val, "act", k, "fwd")
            assert np.all(ict >= act * (1 - 1e-6) - 1e-7)
            if prev is not None:
                assert np.all(act >= prev * (1 - 1e-6) - 1e-7)
            prev = act
    finally:
        emd.emd_db_destroy(db)


def test_ict_images(emd):
    """Cost-matrix mode: 28 x 28 pixel images, queries of up to a few hundred pixels."""
    w = emd_synth.config(3, query_limit=4, n_docs=500)
    db = make_db(emd, w, max_query_h=784, max_table_k=16)
    try:
        got = run_dirs(emd, db, w.queries)
        for qi in range(w.queries.n):
            tf, tr = oracle.lc_query(w.emb, w.cost, w.db, *w.queries.row(qi), "ict")
            np.testing.assert_allclose(got["fwd"][qi], tf, rtol=RTOL, atol=ATOL)
            np.testing.assert_allclose(got["max"][qi], np.maximum(tf, tr), rtol=RTOL, atol=ATOL)
    finally:
        emd.emd_db_destroy(db)


def test_ict_served(emd, work):
    w = work
    db = make_db(emd, w, precision="fp32_tc", max_query_h=512, max_table_k=8)
    srv = emd.emd_server_create(db)
    try:
        tickets = [emd.emd_server_submit(srv, *w.queries.row(i), meas="ict", k=1, K=10) for i in range(w.queries.n)]
        ti, td = emd.emd_topk(db, w.queries.row_ptr, w.queries.col, w.queries.val, "ict", 1, "max", 10)
        for i, t in enumerate(tickets):
            oi, od = np.empty(10, np.int64), np.empty(10, np.float32)
            assert emd.emd_server_poll(srv, t, -1, oi, od)
            assert np.array_equal(oi, ti[i]) and np.array_equal(od, td[i])
        assert emd.emd_server_stats_get(srv)["failed"] == 0
    finally:
        emd.emd_server_destroy(srv)
        emd.emd_db_destroy(db)
