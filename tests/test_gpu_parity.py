"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerance: distances within 1e-5 relative in the FP32 form (plus 1e-7 absolute for exact
zeros).  Neighbour lists: identical to the oracle's after removing the tie group around
the K-th distance (|d - d_K| <= 1e-5 d_K + 1e-9); the order outside ties is the
(distance, document id) order.
"""
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


def oracle_dir(w, qi, meas, k, direction):
    qidx, qw = w.queries.row(qi)
    tf, tr = oracle.lc_query(w.emb, w.cost, w.db, qidx, qw, meas, k,
                             fwd=direction != "rev", rev=direction != "fwd")
    if direction == "fwd":
        return tf
    if direction == "rev":
        return tr
    return np.maximum(tf, tr)


def assert_topk_matches(gpu_idx, gpu_dist, want, K):
    """A12: identical outside the tie group of the K-th distance."""
    order = np.lexsort((np.arange(len(want)), want))
    dK = want[order[K - 1]]
    tie = np.abs(want - dK) <= 1e-5 * dK + 1e-9
    want_set = {int(i) for i in order[:K] if not tie[i]}
    got_set = {int(i) for i in gpu_idx if not tie[i]}
    assert want_set == got_set
    # every reported id is valid and carries its own distance
    np.testing.assert_allclose(gpu_dist, want[gpu_idx], rtol=RTOL, atol=ATOL)
    # reported order is (distance, id)
    keys = list(zip(gpu_dist.tolist(), gpu_idx.tolist()))
    assert keys == sorted(keys)


# --------------------------------------------------------------------- tiny text (config 1)

@pytest.fixture(scope="module")
def tiny(emd):
    w = emd_synth.config(1)
    db = make_db(emd, w, max_query_h=64)
    yield w, db
    emd.emd_db_destroy(db)


TINY_CASES = [("rwmd", 1), ("omr", 1), ("act", 1), ("act", 2), ("act", 3), ("act", 4), ("ict", 1)]


@pytest.mark.parametrize("meas,k", TINY_CASES)
@pytest.mark.parametrize("direction", ["fwd", "rev", "max"])
def test_tiny_all_queries(emd, tiny, meas, k, direction):
    w, db = tiny
    q = w.queries
    got = emd.emd_query_batch(db, q.row_ptr, q.col, q.val, meas, k, direction)
    for qi in range(q.n):
        np.testing.assert_allclose(got[qi], oracle_dir(w, qi, meas, k, direction), rtol=RTOL, atol=ATOL)


@pytest.mark.parametrize("meas,k", [("act", 2), ("omr", 1), ("ict", 1)])
def test_tiny_top10(emd, tiny, meas, k):
    w, db = tiny
    q = w.queries
    idx, dist = emd.emd_topk(db, q.row_ptr, q.col, q.val, meas, k, "max", 10)
    for qi in range(q.n):
        assert_topk_matches(idx[qi], dist[qi], oracle_dir(w, qi, meas, k, "max"), 10)


def test_tiny_phase1_table(emd, tiny):
    w, db = tiny
    qidx, qw = w.queries.row(0)
    used, z, s, wt = emd.emd_phase1_table(db, qidx, qw, 4)
    np.testing.assert_array_equal(used, np.unique(w.db.col))
    Z, S, W = oracle.phase1(w.emb, None, used, qidx, qw, 4)
    np.testing.assert_allclose(z, Z, rtol=RTOL, atol=ATOL)
    np.testing.assert_array_equal(s, S)  # random embeddings: no ties
    np.testing.assert_array_equal(wt, W.astype(np.float32))


# --------------------------------------------------------------------- ragged sizes

@pytest.fixture(scope="module")
def ragged(emd):
    """Odd m (row padding), queries of 1..70 bins (one and several 32-lane chunks, more
    than one 64-column tile), documents of 1..70 bins (several 32-nonzero chunks)."""
    w = emd_synth.small_text(9001, V=3000, m=37, n=700, n_queries=6, lo=1, hi=70)
    # force the degenerate sizes: a one-bin query and a one-bin document exist
    qlens = np.diff(w.queries.row_ptr)
    assert qlens.min() <= 70
    db = make_db(emd, w, max_query_h=128, max_table_k=80)
    yield w, db
    emd.emd_db_destroy(db)


@pytest.mark.parametrize("meas,k", [("rwmd", 1), ("omr", 1), ("act", 3), ("act", 5), ("act", 16),
                                    ("act", 17), ("act", 40), ("ict", 1)])
def test_ragged_both_directions(emd, ragged, meas, k):
    w, db = ragged
    q = w.queries
    for direction in ("fwd", "rev", "max"):
        got = emd.emd_query_batch(db, q.row_ptr, q.col, q.val, meas, k, direction)
        for qi in range(q.n):
            np.testing.assert_allclose(got[qi], oracle_dir(w, qi, meas, k, direction), rtol=RTOL, atol=ATOL)


def test_single_bin_query_and_documents(emd):
    rng = np.random.default_rng(5)
    V, m = 200, 16
    emb = emd_synth.unit_embeddings(rng, V, m)
    # documents: 40 single-bin docs plus 40 two-bin docs
    cols, vals, rp = [], [], [0]
    for d in range(80):
        h = 1 if d < 40 else 2
        c = np.sort(rng.choice(V, h, replace=False)).astype(np.int32)
        x = np.full(h, 1.0 / h, dtype=np.float32)
        cols.append(c); vals.append(x); rp.append(rp[-1] + h)
    db_h = emd_synth.Histograms(np.array(rp, np.int64), np.concatenate(cols), np.concatenate(vals))
    queries = emd_synth.Histograms(np.array([0, 1, 3], np.int64), np.array([7, 3, 150], np.int32),
                                   np.array([1.0, 0.25, 0.75], np.float32))
    w = emd_synth.Workload("edge", V, m, emb, None, db_h, queries, (1, 2, 4), 5)
    db = make_db(emd, w, max_query_h=8)
    try:
        for meas, k in [("rwmd", 1), ("omr", 1), ("act", 2), ("act", 4), ("ict", 1)]:
            for direction in ("fwd", "rev", "max"):
                got = emd.emd_query_batch(db, queries.row_ptr, queries.col, queries.val, meas, k, direction)
                for qi in range(2):
                    np.testing.assert_allclose(got[qi], oracle_dir(w, qi, meas, k, direction), rtol=RTOL, atol=ATOL)
    finally:
        emd.emd_db_destroy(db)


def test_identical_histogram_is_at_zero(emd, tiny):
    """p = q gives 0 for every measure (exact zeros from identical coordinates)."""
    w, db = tiny
    c, x = w.db.row(17)
    rp = np.array([0, len(c)], np.int64)
    for meas, k in [("omr", 1), ("act", 3), ("ict", 1)]:
        got = emd.emd_query_batch(db, rp, c, x, meas, k, "max")
        assert got[0, 17] == 0.0
        idx, dist = emd.emd_topk(db, rp, c, x, meas, k, "max", 1)
        assert idx[0, 0] == 17 and dist[0, 0] == 0.0


def test_full_overlap_rwmd_zero_omr_positive(emd):
    """Section 4 / Table 5: same support, different weights -> RWMD 0, OMR > 0."""
    w = emd_synth.config(3, query_limit=1, n_docs=64)
    db = make_db(emd, w, max_query_h=784)
    try:
        c, x = w.db.row(5)
        qw = (x.astype(np.float64) * np.linspace(0.5, 1.5, len(x)))
        qw = (qw / qw.sum()).astype(np.float32)
        rp = np.array([0, len(c)], np.int64)
        r = emd.emd_query_batch(db, rp, c, qw, "rwmd", 1, "max")
        o = emd.emd_query_batch(db, rp, c, qw, "omr", 1, "max")
        assert r[0, 5] == 0.0 and o[0, 5] > 0.0
        one = emd_synth.Workload("q", w.v, w.m, w.emb, w.cost, w.db,
                                 emd_synth.Histograms(rp, c, qw), (), 1)
        np.testing.assert_allclose(o[0], oracle_dir(one, 0, "omr", 1, "max"), rtol=RTOL, atol=ATOL)
    finally:
        emd.emd_db_destroy(db)


# --------------------------------------------------------------------- image mode

@pytest.mark.parametrize("meas,k", [("rwmd", 1), ("omr", 1), ("act", 2), ("act", 8), ("act", 16)])
def test_image_mode(emd, meas, k):
    w = emd_synth.config(3, query_limit=3, n_docs=400)
    db = make_db(emd, w, max_query_h=784)
    try:
        q = w.queries
        got = emd.emd_query_batch(db, q.row_ptr, q.col, q.val, meas, k, "max")
        for qi in range(q.n):
            np.testing.assert_allclose(got[qi], oracle_dir(w, qi, meas, k, "max"), rtol=RTOL, atol=ATOL)
        idx, dist = emd.emd_topk(db, q.row_ptr, q.col, q.val, meas, k, "max", 16)
        for qi in range(q.n):
            assert_topk_matches(idx[qi], dist[qi], oracle_dir(w, qi, meas, k, "max"), 16)
    finally:
        emd.emd_db_destroy(db)


# --------------------------------------------------------------------- device variants

def test_device_entry_points_match_host(emd, tiny):
    import torch
    w, db = tiny
    q = w.queries
    host = emd.emd_query_batch(db, q.row_ptr, q.col, q.val, "act", 3, "max")
    hidx, hdist = emd.emd_topk(db, q.row_ptr, q.col, q.val, "act", 3, "max", 10)
    qi = torch.from_numpy(q.col).cuda()
    qw = torch.from_numpy(q.val).cuda()
    out = torch.empty((q.n, w.db.n), dtype=torch.float32, device="cuda")
    oi = torch.empty((q.n, 10), dtype=torch.int64, device="cuda")
    od = torch.empty((q.n, 10), dtype=torch.float32, device="cuda")
    s = torch.cuda.current_stream().cuda_stream
    emd.emd_query_batch_device(db, q.row_ptr, qi, qw, out, "act", 3, "max", stream=s)
    emd.emd_topk_device(db, q.row_ptr, qi, qw, oi, od, "act", 3, "max", 10, stream=s)
    torch.cuda.synchronize()
    emd.emd_db_check_device_errors(db)
    np.testing.assert_array_equal(out.cpu().numpy(), host)
    np.testing.assert_array_equal(oi.cpu().numpy(), hidx)
    np.testing.assert_array_equal(od.cpu().numpy(), hdist)


def test_device_bad_index_is_latched_not_faulted(emd, tiny):
    import torch
    w, db = tiny
    qi = torch.tensor([5, w.v + 10, 9], dtype=torch.int32, device="cuda")
    qw = torch.tensor([0.5, 0.25, 0.25], dtype=torch.float32, device="cuda")
    out = torch.empty((1, w.db.n), dtype=torch.float32, device="cuda")
    emd.emd_query_batch_device(db, np.array([0, 3]), qi, qw, out, "act", 2, "max",
                               stream=torch.cuda.current_stream().cuda_stream)
    with pytest.raises(emd.EmdError) as e:
        emd.emd_db_check_device_errors(db)
    assert e.value.name == "INVALID_ARG"
    emd.emd_db_check_device_errors(db)  # latch cleared


# --------------------------------------------------------------------- argument checks

def test_invalid_queries_rejected(emd, tiny):
    w, db = tiny
    c, x = w.queries.row(0)
    rp = np.array([0, len(c)], np.int64)
    bad = [
        (rp, c, x * 2),                                    # sum != 1
        (rp, np.where(np.arange(len(c)) == 0, w.v, c), x),  # id out of range
        (rp, np.concatenate([c[:1], c[:-1]]), x),          # repeated id
        (np.array([0, 0], np.int64), c[:0], x[:0]),         # empty query
    ]
    for r, cc, xx in bad:
        with pytest.raises(emd.EmdError) as e:
            emd.emd_query_batch(db, r, cc, xx, "act", 2, "max")
        assert e.value.name == "INVALID_ARG"
    with pytest.raises(emd.EmdError) as e:
        emd.emd_topk(db, rp, c, x, "act", 2, "max", w.db.n + 1)
    assert e.value.name == "INVALID_ARG"
    with pytest.raises(emd.EmdError) as e:
        emd.emd_query_batch(db, rp, c, x, "act", 0, "max")
    assert e.value.name == "INVALID_ARG"
    # zero queries: a no-op
    out = emd.emd_query_batch(db, np.array([0], np.int64), c[:0], x[:0], "act", 2, "max")
    assert out.shape == (0, w.db.n)


def test_invalid_database_rejected(emd):
    rng = np.random.default_rng(1)
    emb = emd_synth.unit_embeddings(rng, 50, 8)
    rp = np.array([0, 2, 2, 3], np.int64)  # empty document 1
    col = np.array([1, 2, 3], np.int32)
    val = np.array([0.5, 0.5, 1.0], np.float32)
    with pytest.raises(emd.EmdError) as e:
        emd.emd_db_create(emb, None, rp, col, val)
    assert e.value.name == "INVALID_ARG"
    with pytest.raises(emd.EmdError):
        emd.emd_db_create(emb, None, np.array([0, 2], np.int64), col[:2], np.array([0.5, 0.6], np.float32))


def test_query_above_max_query_h_is_rejected(emd, tiny):
    w, db = tiny  # max_query_h = 64
    rng = np.random.default_rng(3)
    c = np.sort(rng.choice(w.v, 70, replace=False)).astype(np.int32)
    x = np.full(70, 1 / 70, np.float32)
    with pytest.raises(emd.EmdError) as e:
        emd.emd_query_batch(db, np.array([0, 70]), c, x, "ict", 1, "max")
    assert e.value.name == "INVALID_ARG"


# --------------------------------------------------------------------- full size (config 2)

@pytest.fixture(scope="module")
def text_full(emd):
    w = emd_synth.config(2, query_limit=6)
    db = make_db(emd, w, max_query_h=1024, max_batch=8)
    yield w, db
    emd.emd_db_destroy(db)


def test_text_full_size_sampled(emd, text_full):
    """Full-size text database (V=1e5, m=300, n=2e4) in the benchmark's launch
    configuration: every distance of 3 queries against the oracle, and top-16."""
    w, db = text_full
    q = w.queries.subset([0, 1, 2])
    got = emd.emd_query_batch(db, q.row_ptr, q.col, q.val, "act", 4, "max")
    idx, dist = emd.emd_topk(db, q.row_ptr, q.col, q.val, "act", 4, "max", 16)
    for qi in range(q.n):
        qidx, qw = q.row(qi)
        tf, tr = oracle.lc_query_split(w.emb, None, w.db, qidx, qw, "act", 4)
        want = np.maximum(tf, tr)
        np.testing.assert_allclose(got[qi], want, rtol=RTOL, atol=ATOL)
        assert_topk_matches(idx[qi], dist[qi], want, 16)


@pytest.mark.parametrize("meas,k", [("omr", 1), ("act", 16)])
def test_text_full_size_forward_sampled_docs(emd, text_full, meas, k):
    """Other measures at full size, checked on 300 sampled documents with the per-pair
    definition (one document at a time)."""
    w, db = text_full
    q = w.queries.subset([3])
    qidx, qw = q.row(0)
    got = emd.emd_query_batch(db, q.row_ptr, q.col, q.val, meas, k, "max")[0]
    docs = np.random.default_rng(11).choice(w.db.n, 300, replace=False)
    sub = w.db.subset(docs)
    tf, tr = oracle.pair_db(w.emb, None, sub, qidx, qw, meas, k)
    np.testing.assert_allclose(got[docs], np.maximum(tf, tr), rtol=RTOL, atol=ATOL)


# --------------------------------------------------------------------- pruned symmetric top-K

def test_pruned_topk_equals_unpruned_full_size(emd, text_full):
    """max(fwd, rev) >= fwd: the pruned top-K (reverse pass on the forward candidates only)
    must equal the top-K over all documents."""
    w, db = text_full
    q = w.queries
    emd.emd_db_profile_reset(db)
    for K in (1, 10, 16):
        for meas, k in (("act", 4), ("omr", 1), ("act", 2)):
            pi, pd = emd.emd_topk(db, q.row_ptr, q.col, q.val, meas, k, "max", K)
            full = emd.emd_query_batch(db, q.row_ptr, q.col, q.val, meas, k, "max")
            for r in range(q.n):
                order = np.lexsort((np.arange(w.db.n), full[r]))[:K]
                np.testing.assert_array_equal(pi[r], order)
                np.testing.assert_array_equal(pd[r], full[r][order])
    prof = emd.emd_db_profile_get(db)
    assert prof["pruned_queries"] >= 9 * q.n


def test_pruning_fallback_on_ties(emd):
    """Identical documents tie at every distance, so every one of them is a candidate;
    more candidates than the pruned path holds (256) means no certificate, and the query
    is recomputed over all documents.  The answer is the lowest ids either way."""
    rng = np.random.default_rng(12)
    emb = emd_synth.unit_embeddings(rng, 300, 16)
    c = np.sort(rng.choice(300, 12, replace=False)).astype(np.int32)
    x = np.full(12, 1 / 12, np.float32)
    n = 300
    rp = np.arange(n + 1, dtype=np.int64) * 12
    db = emd.emd_db_create(emb, None, rp, np.tile(c, n), np.tile(x, n), emd.emd_db_options_default(max_query_h=32))
    try:
        qc = np.sort(rng.choice(300, 9, replace=False)).astype(np.int32)
        qw = np.full(9, 1 / 9, np.float32)
        emd.emd_db_profile_reset(db)
        idx, dist = emd.emd_topk(db, np.array([0, 9]), qc, qw, "act", 3, "max", 10)
        np.testing.assert_array_equal(idx[0], np.arange(10))
        assert np.all(dist[0] == dist[0][0])
        prof = emd.emd_db_profile_get(db)
        assert prof["prune_fallbacks"] == 1 and prof["pruned_queries"] == 1
    finally:
        emd.emd_db_destroy(db)


def test_device_topk_is_ordered_on_the_callers_stream(emd, text_full):
    """Results of the device entry point are visible to later work on the same stream
    without any explicit synchronisation (torch's current stream, here the default one)."""
    import torch
    w, db = text_full
    q = w.queries
    qi = torch.from_numpy(q.col).cuda()
    qw = torch.from_numpy(q.val).cuda()
    for K in (16, 32):  # 16: pruned path; 32: all documents, fully asynchronous
        hi, hd = emd.emd_topk(db, q.row_ptr, q.col, q.val, "act", 4, "max", K)
        for s in (torch.cuda.current_stream(), torch.cuda.Stream()):
            with torch.cuda.stream(s):
                oi = torch.full((q.n, K), -5, dtype=torch.int64, device="cuda")
                od = torch.full((q.n, K), -5.0, dtype=torch.float32, device="cuda")
                emd.emd_topk_device(db, q.row_ptr, qi, qw, oi, od, "act", 4, "max", K, stream=s.cuda_stream)
                ci, cd = oi.clone(), od.clone()  # same stream, no synchronize in between
            torch.cuda.synchronize()
            np.testing.assert_array_equal(ci.cpu().numpy(), hi)
            np.testing.assert_array_equal(cd.cpu().numpy(), hd)


@pytest.mark.parametrize("meas,k", [("rwmd", 1), ("omr", 1), ("act", 2), ("act", 4), ("act", 16)])
def test_pruned_topk_equals_unpruned_small_queries(emd, meas, k):
    """Queries of 5..45 bins (one 32-bin chunk or several), where the reverse and forward
    bounds differ most; every K up to the pruning limit."""
    w = emd_synth.small_text(4242, V=600, m=48, n=300, n_queries=6, lo=5, hi=45)
    q = w.queries
    dbp = make_db(emd, w, max_query_h=64)
    dbf = make_db(emd, w, max_query_h=64, prune_topk=0)
    try:
        for K in (1, 8, 16):
            pi, pd = emd.emd_topk(dbp, q.row_ptr, q.col, q.val, meas, k, "max", K)
            fi, fd = emd.emd_topk(dbf, q.row_ptr, q.col, q.val, meas, k, "max", K)
            np.testing.assert_array_equal(pi, fi)
            np.testing.assert_array_equal(pd, fd)
        for qi in range(q.n):
            assert_topk_matches(pi[qi], pd[qi], oracle_dir(w, qi, meas, k, "max"), 16)
    finally:
        emd.emd_db_destroy(dbp)
        emd.emd_db_destroy(dbf)


# --------------------------------------------------------------------- batched form

@pytest.mark.parametrize("precision", ["fp32", "fp32_tc", "bf16"])
def test_batched_equals_per_query(emd, precision):
    """One launch per step over a batch (batched=1) against the per-query kernels
    (batched=0): the same device bodies, so every distance and top-K is bit-identical,
    with the autotuned parameters and graph replay (db_b) as with fixed defaults and
    direct launches (db_c).  A small batch_columns forces several sub-batches per call."""
    w = emd_synth.small_text(99, 2500, 48, 900, 23, 4, 50, 1, 150)
    rp, qi, qw = w.queries.row_ptr, w.queries.col, w.queries.val
    # the fused pruned path of the approximate formats (fused_phase1 = 2) computes its reverse
    # distances exactly, not from the approximate matrix, so it is held to the oracle instead
    # (test_gpu_fused); here the default (fused only for FP32_TC, bit-identical) runs
    fused = 1
    db_q = make_db(emd, w, precision=precision, max_query_h=160, max_table_k=160, batched=0)
    db_b = make_db(emd, w, precision=precision, max_query_h=160, max_table_k=160, batch_columns=512, max_batch=8,
                   fused_phase1=fused)
    db_c = make_db(emd, w, precision=precision, max_query_h=160, max_table_k=160, batch_columns=512, max_batch=8,
                   graphs=0, autotune=0, fused_phase1=fused)
    info_b, info_c = emd.emd_db_info_get(db_b), emd.emd_db_info_get(db_c)
    assert info_b["autotuned"] == 1 and info_c["autotuned"] == 0
    assert info_b["rev_warps"] in (2, 4, 8) and info_b["tc_group_mult"] in (1, 2, 4)
    try:
        cases = [("rwmd", 1), ("omr", 1), ("act", 2), ("act", 4), ("act", 8)]
        if precision != "bf16":
            cases += [("act", 16), ("ict", 1)]
        for meas, k in cases:
            dirs = ("fwd", "rev", "max") if not (meas == "ict" and precision == "bf16") else ("rev",)
            for d in dirs:
                a = emd.emd_query_batch(db_q, rp, qi, qw, meas, k, d)
                for dbx in (db_b, db_c, db_b):  # graph captured, direct launches, graph replayed
                    b = emd.emd_query_batch(dbx, rp, qi, qw, meas, k, d)
                    assert np.array_equal(a, b), (meas, k, d)
            for K in (10, 32):
                ai, ad = emd.emd_topk(db_q, rp, qi, qw, meas, k, "max", K)
                for dbx in (db_b, db_c, db_b):
                    bi, bd = emd.emd_topk(dbx, rp, qi, qw, meas, k, "max", K)
                    assert np.array_equal(ai, bi) and np.array_equal(ad, bd), (meas, k, K)
        assert emd.emd_db_profile_get(db_b)["graph_launches"] > 0
        assert emd.emd_db_profile_get(db_c)["graph_launches"] == 0
    finally:
        emd.emd_db_destroy(db_q)
        emd.emd_db_destroy(db_b)
        emd.emd_db_destroy(db_c)


def test_pruned_topk_over_several_sub_batches(emd):
    """A batch split into several sub-batches (small batch workspace), called repeatedly:
    every sub-batch's candidate counts start from zero, so the pruned top-K equals the
    unpruned one bit for bit on every call."""
    w = emd_synth.small_text(515, 2500, 48, 1200, 40, 4, 50, 20, 200)
    q = w.queries
    db_p = make_db(emd, w, precision="fp32_tc", max_query_h=256, batch_columns=768, max_batch=32)
    db_u = make_db(emd, w, precision="fp32_tc", max_query_h=256, prune_topk=0)
    try:
        ui, ud = emd.emd_topk(db_u, q.row_ptr, q.col, q.val, "act", 4, "max", 12)
        for _ in range(3):
            pi, pd = emd.emd_topk(db_p, q.row_ptr, q.col, q.val, "act", 4, "max", 12)
            assert np.array_equal(pi, ui) and np.array_equal(pd, ud)
        assert emd.emd_db_profile_get(db_p)["pruned_queries"] == 3 * q.n
    finally:
        emd.emd_db_destroy(db_p)
        emd.emd_db_destroy(db_u)
