"""The fused form of the batched pruned top-K path (precision FP32_TC): the Phase-1 table is
taken in the tensor-core product's epilogue and the reverse direction reads an exact
distance block over the candidate documents' rows only, so no v_used x h_q matrix is
written.  Every distance it uses is computed by the same operands, MMA order and epilogue
arithmetic as the full matrix's entry, and the table keeps the k smallest by (value, bin)
as the table kernel does, so the answers must be bit-identical to the materialized form
(fused_phase1 = 0), which the other tests check against the FP64 oracle; the oracle
comparison at full query sizes runs through this path too (test_gpu_mixed)."""
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


def pair(emd, w, **opt):
    base = dict(precision="fp32_tc", autotune=0, **opt)
    f = emd.emd_db_create(w.emb, None, w.db.row_ptr, w.db.col, w.db.val,
                          emd.emd_db_options_default(fused_phase1=1, **base), v=w.v)
    m = emd.emd_db_create(w.emb, None, w.db.row_ptr, w.db.col, w.db.val,
                          emd.emd_db_options_default(fused_phase1=0, **base), v=w.v)
    return f, m


def same_topk(emd, f, m, q, meas, k, K):
    """Equal answers, and equal certificate decisions: the queries the fused form leaves
    uncertified (recomputed over all documents) are those the materialized form does."""
    emd.emd_db_profile_reset(f)
    emd.emd_db_profile_reset(m)
    a = emd.emd_topk(f, q.row_ptr, q.col, q.val, meas, k, "max", K)
    b = emd.emd_topk(m, q.row_ptr, q.col, q.val, meas, k, "max", K)
    np.testing.assert_array_equal(a[0], b[0])
    np.testing.assert_array_equal(a[1], b[1])
    pf, pm = emd.emd_db_profile_get(f), emd.emd_db_profile_get(m)
    assert pf["pruned_queries"] == pm["pruned_queries"] == q.n
    assert pf["prune_fallbacks"] == pm["prune_fallbacks"], (pf["prune_fallbacks"], pm["prune_fallbacks"])
    return a


@pytest.fixture(scope="module")
def text():
    w = emd_synth.config(2, query_limit=48)
    return w


@pytest.mark.parametrize("meas,k", [("act", 1), ("act", 2), ("act", 3), ("act", 4), ("act", 8), ("act", 16),
                                    ("rwmd", 1), ("omr", 1)])
def test_fused_equals_materialized_text(emd, text, meas, k):
    f, m = pair(emd, text, max_query_h=1024)
    try:
        same_topk(emd, f, m, text.queries, meas, k, 16)
        emd.emd_db_check_device_errors(f)
    finally:
        emd.emd_db_destroy(f)
        emd.emd_db_destroy(m)


def test_fused_equals_materialized_mixed_sizes(emd):
    """Queries of h_q 5..2000 (up to 16 column tiles, several sub-batches per call, both
    tile streams of the fused kernel busy with queries of very different lengths)."""
    w = emd_synth.config(2, query_limit=1)
    q = emd_synth.mixed_queries(80)
    f, m = pair(emd, w, max_query_h=2048, batch_columns=8192)
    try:
        for K in (16, 5):
            same_topk(emd, f, m, q, "act", 4, K)
        emd.emd_db_check_device_errors(f)
    finally:
        emd.emd_db_destroy(f)
        emd.emd_db_destroy(m)


def test_fused_small_ragged(emd):
    """Embedding width 37 (one 64-wide K chunk), query sizes 1..150 (one or two column
    tiles with ragged tails), batches of 1..13 queries, every K up to 16."""
    w = emd_synth.small_text(5150, 1500, 37, 900, 13, 1, 60, 1, 150)
    f, m = pair(emd, w, max_query_h=256)
    try:
        for K in (1, 7, 16):
            for nq in (1, 5, 13):
                sub = w.queries.subset(np.arange(nq))
                same_topk(emd, f, m, sub, "act", 3, K)
        emd.emd_db_check_device_errors(f)
    finally:
        emd.emd_db_destroy(f)
        emd.emd_db_destroy(m)


def test_fused_candidate_row_overflow(emd):
    """Forty documents of 1000 distinct vocabulary rows each, all on a circle at the same
    distance from the query's single bin: every document is a candidate and together they
    hold 40000 distinct rows, more than the candidate block holds (kCandRows = 32768).  The
    query is rerun with the full distance matrix (a retry, not a recompute over all
    documents: the forty candidates certify there) and the answer equals the materialized
    form's."""
    per, ndoc = 1000, 40
    V = per * ndoc + 1
    t = np.arange(V - 1) * (2 * np.pi / (V - 1))
    emb = np.zeros((V, 3), np.float32)
    emb[:-1, 0] = 0.6 * np.cos(t)
    emb[:-1, 1] = 0.6 * np.sin(t)
    emb[:-1, 2] = 0.8
    emb[-1] = (0.0, 0.0, 1.0)  # the query's bin
    rp = np.arange(ndoc + 1, dtype=np.int64) * per
    col = np.arange(ndoc * per, dtype=np.int32)
    rng = np.random.default_rng(3)
    val = rng.integers(1, 6, ndoc * per).astype(np.float64)
    val = (val / np.repeat(np.add.reduceat(val, rp[:-1]), per)).astype(np.float32)
    db_hist = emd_synth.Histograms(rp, col, val)
    w = emd_synth.Workload("circle", V, 3, emb, None, db_hist, db_hist, (1,), 16)
    q = emd_synth.Histograms(np.array([0, 1], np.int64), np.array([V - 1], np.int32), np.array([1.0], np.float32))
    f, m = pair(emd, w, max_query_h=32)
    try:
        emd.emd_db_profile_reset(f)
        emd.emd_db_profile_reset(m)
        a = emd.emd_topk(f, q.row_ptr, q.col, q.val, "act", 2, "max", 16)
        b = emd.emd_topk(m, q.row_ptr, q.col, q.val, "act", 2, "max", 16)
        np.testing.assert_array_equal(a[0], b[0])
        np.testing.assert_array_equal(a[1], b[1])
        pf, pm = emd.emd_db_profile_get(f), emd.emd_db_profile_get(m)
        assert pf["fused_retries"] == 1 and pf["prune_fallbacks"] == 0  # the block overflowed, the retry certified
        assert pm["fused_retries"] == 0 and pm["prune_fallbacks"] == 0
        emd.emd_db_check_device_errors(f)
    finally:
        emd.emd_db_destroy(f)
        emd.emd_db_destroy(m)


def test_forward_sweep_forms_bit_identical(emd):
    """The four forms of the grouped forward sweep (fwd_kernel 1..4; their table layouts
    differ) give the same forward values and the same pruned top-K, bit for bit."""
    w = emd_synth.small_text(6161, 2500, 48, 1500, 19, 2, 200, 1, 300)
    q = w.queries
    outs = []
    for fk in (1, 2, 3, 4):
        db = emd.emd_db_create(w.emb, None, w.db.row_ptr, w.db.col, w.db.val,
                               emd.emd_db_options_default(precision="fp32_tc", max_query_h=512, autotune=0,
                                                          fwd_kernel=fk), v=w.v)
        try:
            assert emd.emd_db_info_get(db)["fwd_kernel"] == fk
            res = []
            for meas, k in (("act", 4), ("act", 16), ("act", 7), ("omr", 1), ("rwmd", 1)):
                res.append(emd.emd_query_batch(db, q.row_ptr, q.col, q.val, meas, k, "fwd"))
                res.extend(emd.emd_topk(db, q.row_ptr, q.col, q.val, meas, k, "max", 16))
            outs.append(res)
        finally:
            emd.emd_db_destroy(db)
    for other in outs[1:]:
        for a, b in zip(outs[0], other):
            np.testing.assert_array_equal(a, b)


@pytest.mark.parametrize("precision", ["bf16", "fp8"])
def test_fused_approximate_forms_against_oracle(emd, precision):
    """Fused pruned top-K in the approximate formats on the text workload (V = 1e5, m = 300):
    the product's epilogue keeps each row's k + 8 smallest approximate distances, the table
    is their exact FP32 re-rank, and the reverse direction reads the exact FP16-split block
    of the candidate rows.  BF16 certifies every row (or recomputes it over all bins), so its
    top-16 meets the FP32 tolerance: identical to the oracle's outside the tie group of the
    16th distance, every returned distance within 1e-5.  E4M3's bound is too wide for the
    certificate; its returned distances are held to the forward rounding bound of R15 and
    its recall against the oracle is reported."""
    import os
    import oracle
    w = emd_synth.config(2, query_limit=24)
    q = w.queries
    K = 16
    db = emd.emd_db_create(w.emb, None, w.db.row_ptr, w.db.col, w.db.val,
                           emd.emd_db_options_default(precision=precision, max_query_h=1024, fused_phase1=2), v=w.v)
    try:
        gi, gd = emd.emd_topk(db, q.row_ptr, q.col, q.val, "act", 4, "max", K)
        emd.emd_db_check_device_errors(db)
    finally:
        emd.emd_db_destroy(db)
    prep = oracle.prepare(w.emb, None, w.db)
    threads = os.cpu_count() or 1
    recalls = []
    for i in range(q.n):
        ref = oracle.SymTopK(w.emb, None, w.db, *q.row(i), "act", 4, K, threads=threads, prep=prep)
        dK = ref.dist[K - 1]
        got_sym = ref.sym_of(gi[i])
        tie = np.abs(got_sym - dK) <= 1e-5 * dK + 1e-9
        truth = set(int(d) for d in ref.idx)
        hits = sum(1 for d, t in zip(gi[i], tie) if int(d) in truth or t)
        recalls.append(hits / K)
        rel = np.abs(gd[i] - got_sym) / got_sym
        if precision == "bf16":
            ref_tie = np.abs(ref.dist - dK) <= 1e-5 * dK + 1e-9
            assert {int(d) for d, t in zip(ref.idx, ref_tie) if not t} <= {int(d) for d in gi[i]}, i
            assert rel.max() <= 1e-5, (i, rel.max())
        else:
            assert rel.max() <= 2 * (2 * 2.0 ** -4 + 2.0 ** -8), (i, rel.max())
    print(f"{precision} fused: top-{K} recall {np.mean(recalls):.4f} (min {np.min(recalls):.4f}) over {q.n} queries")
    assert np.mean(recalls) >= (1.0 if precision == "bf16" else 0.9)
