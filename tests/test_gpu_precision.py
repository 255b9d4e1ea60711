"""The approximate Phase-1 forms (BF16 and FP8-E4M3 tensor-core products with per-row
absmax scales) against the FP64 oracle.

The table kernel re-ranks each row's k + margin smallest approximate distances with exact
FP32 sums of squared differences, so forward distances and the Phase-1 table are expected
at the FP32 tolerance (1e-5 relative) whenever a row's true k nearest lie among those
candidates.  Reverse distances use the approximate matrix.  Their bound follows from the
operand rounding: with unit roundoff u per stored element (2^-8 BF16: 8 significant bits;
2^-4 E4M3: 4 significant bits; round to nearest), |d(a.b)| <= (2u + u^2) sum|a_i b_i| <= (2u + u^2) |a||b|; for unit
embeddings the squared distance moves by at most 2(2u + u^2) and, since the row cost is
1-Lipschitz in the distances, a reverse value by at most 2(2u + u^2) / (2 d_min) per unit
mass.  With d >= 1 in these workloads (random unit vectors in 64+ dimensions; identical ids
give an exact 0 on both sides) that is 7.8e-3 (BF16) and 0.13 (E4M3) relative; the tests
take those bounds (E4M3 values below the normal range only add absolute errors far below
them).
"""
import numpy as np
import pytest

import emd_synth
import oracle

pytestmark = pytest.mark.gpu

RTOL, ATOL = 1e-5, 1e-7
BOUND = {"bf16": 2 * 2.0 ** -8 + 2.0 ** -16, "fp8": 2 * 2.0 ** -4 + 2.0 ** -8}


@pytest.fixture(scope="module")
def emd():
    import paper_1812_02091_gb300 as m
    from paper_1812_02091_gb300 import _build
    _build.build()
    m.load()
    return m


@pytest.fixture(scope="module")
def work():
    return emd_synth.small_text(4321, 3000, 64, 1200, 10, 5, 60, 3, 180)


@pytest.fixture(scope="module")
def want(work):
    w = work
    return [oracle.lc_query(w.emb, None, w.db, *w.queries.row(i), "act", 4) for i in range(w.queries.n)]


def make_db(emd, w, **opt):
    return emd.emd_db_create(w.emb, None, w.db.row_ptr, w.db.col, w.db.val,
                             emd.emd_db_options_default(**opt), v=w.v)


def entries_match_up_to_ties(s, z, oz2, os2, k, rtol=2e-6):
    """Table row check where the order of entries whose distances differ by less than the
    FP32 resolution is not fixed (the device orders by its FP32 squared distance, the
    oracle by the FP64 distance, both then by column): every device entry l must be one of
    the oracle's entries tied with the oracle's l-th (oracle table taken k + 8 wide, so a
    tie group that crosses the k-th entry is seen whole), and no column may repeat."""
    if len(set(s.tolist())) != len(s):
        return False
    n2 = len(oz2)
    for l in range(k):
        lo = l
        while lo > 0 and abs(oz2[lo - 1] - oz2[l]) <= rtol * max(oz2[l], 1e-30):
            lo -= 1
        hi = l
        while hi + 1 < n2 and abs(oz2[hi + 1] - oz2[l]) <= rtol * max(oz2[l], 1e-30):
            hi += 1
        if s[l] not in set(os2[lo:hi + 1].tolist()):
            return False
    return True


@pytest.mark.parametrize("precision", ["bf16", "fp8"])
def test_table_reranked_exact(emd, work, precision):
    w = work
    db = make_db(emd, w, precision=precision, max_query_h=256)
    try:
        for qi in range(w.queries.n):
            qidx, qw = w.queries.row(qi)
            for k in (1, 4, 16):
                used, z, s, wt = emd.emd_phase1_table(db, qidx, qw, k)
                k2 = min(k + 8, len(qidx))
                oz2, os2, _ = oracle.phase1(w.emb, None, used, qidx, qw, k2)
                oz = oz2[:, :k]
                bad = ~np.isclose(z, oz, rtol=RTOL, atol=ATOL).all(1)
                assert bad.mean() <= 1e-3, (qi, k, bad.sum())
                for r in np.nonzero(~bad)[0]:
                    assert entries_match_up_to_ties(s[r], z[r], oz2[r], os2[r], k), (qi, k, r)
                    np.testing.assert_array_equal(wt[r], qw[s[r]])
    finally:
        emd.emd_db_destroy(db)


@pytest.mark.parametrize("precision", ["bf16", "fp8"])
def test_directions_against_oracle(emd, work, want, precision):
    w = work
    db = make_db(emd, w, precision=precision, max_query_h=256)
    try:
        for d in ("fwd", "rev", "max"):
            got = emd.emd_query_batch(db, w.queries.row_ptr, w.queries.col, w.queries.val, "act", 4, d)
            for qi in range(w.queries.n):
                tf, tr = want[qi]
                ref = tf if d == "fwd" else tr if d == "rev" else np.maximum(tf, tr)
                rel = np.abs(got[qi] - ref) / np.maximum(ref, 1e-30)
                if d == "fwd":
                    assert np.mean(rel > RTOL) <= 1e-3
                assert rel.max() <= BOUND[precision], (d, qi, rel.max())
    finally:
        emd.emd_db_destroy(db)


@pytest.mark.parametrize("precision", ["bf16", "fp8"])
def test_topk_within_bound(emd, work, want, precision):
    """Top-16 (pruned path): identical to the oracle outside the band of distances the
    reverse error bound cannot separate from the 16th."""
    w = work
    K = 16
    db = make_db(emd, w, precision=precision, max_query_h=256)
    try:
        gi, gd = emd.emd_topk(db, w.queries.row_ptr, w.queries.col, w.queries.val, "act", 4, "max", K)
        b = BOUND[precision]
        for qi in range(w.queries.n):
            ref = np.maximum(*want[qi])
            order = np.lexsort((np.arange(len(ref)), ref))
            dK = ref[order[K - 1]]
            band = np.abs(ref - dK) <= 2 * b * dK + 1e-9
            assert {int(i) for i in order[:K] if not band[i]} == {int(i) for i in gi[qi] if not band[i]}
            rel = np.abs(gd[qi] - ref[gi[qi]]) / ref[gi[qi]]
            assert rel.max() <= b
    finally:
        emd.emd_db_destroy(db)


def test_config2_sample(emd):
    """Embedding width 300 at the text scale (database cut to 3000 documents): BF16 and
    E4M3 forward distances at the FP32 tolerance, reverse within the bound."""
    w = emd_synth.config(2, query_limit=2, n_docs=3000)
    want = [oracle.lc_query(w.emb, None, w.db, *w.queries.row(i), "act", 4) for i in range(w.queries.n)]
    for precision in ("bf16", "fp8"):
        db = make_db(emd, w, precision=precision, max_query_h=1024)
        try:
            fwd = emd.emd_query_batch(db, w.queries.row_ptr, w.queries.col, w.queries.val, "act", 4, "fwd")
            rev = emd.emd_query_batch(db, w.queries.row_ptr, w.queries.col, w.queries.val, "act", 4, "rev")
            for qi in range(w.queries.n):
                tf, tr = want[qi]
                assert np.mean(np.abs(fwd[qi] - tf) > RTOL * tf) <= 1e-3
                assert (np.abs(rev[qi] - tr) / tr).max() <= BOUND[precision]
        finally:
            emd.emd_db_destroy(db)


def test_limits(emd, work):
    w = work
    with pytest.raises(emd.EmdError, match="INVALID_ARG"):
        make_db(emd, w, precision="bf16", rerank_margin=33)
    db = make_db(emd, w, precision="fp8", max_query_h=256)
    try:
        rp = np.array([0, 100], np.int64)
        qidx = np.arange(100, dtype=np.int32)
        qw = np.full(100, 0.01, np.float32)
        with pytest.raises(emd.EmdError, match="UNSUPPORTED"):   # ICT: table width h = 100
            emd.emd_query_batch(db, rp, qidx, qw, "ict", 1, "fwd")
        with pytest.raises(emd.EmdError, match="UNSUPPORTED"):   # k + margin = 33 > 32
            emd.emd_query_batch(db, rp, qidx, qw, "act", 25, "fwd")
        out = emd.emd_query_batch(db, rp, qidx, qw, "act", 24, "fwd")  # k + margin = 32
        assert np.isfinite(out).all()
    finally:
        emd.emd_db_destroy(db)
