"""The fused Phase-1 table on clusters of two SMs (tcgen05.mma.cta_group::2, M = 256 rows per
product, each CTA staging half of every query chunk) against the one-SM form.  Per row the
operands, K order, accumulator split and epilogue arithmetic are those of the one-SM kernel,
so tables, top-K answers and certificate decisions must be bit-identical; the one-SM fused
form is itself bit-identical to the materialized form (test_gpu_fused) and checked against the
FP64 oracle at full query sizes (test_gpu_mixed).  tc_pair = 1 uses 64-column tiles (256 TMEM
columns per CTA), 2 uses 128-column tiles (512)."""
import numpy as np
import pytest

import emd_synth

pytestmark = pytest.mark.gpu

PAIRS = [pytest.param(1, id="pair64"), pytest.param(2, id="pair128")]


@pytest.fixture(scope="module")
def emd():
    import paper_1812_02091_gb300 as m
    from paper_1812_02091_gb300 import _build
    _build.build()
    m.load()
    return m


def make(emd, w, tc_pair, **opt):
    return emd.emd_db_create(w.emb, None, w.db.row_ptr, w.db.col, w.db.val,
                             emd.emd_db_options_default(precision="fp32_tc", autotune=0, fused_phase1=1,
                                                        tc_pair=tc_pair, **opt), v=w.v)


def compare(emd, p, s, q, cases, K=16):
    for meas, k in cases:
        emd.emd_db_profile_reset(p)
        emd.emd_db_profile_reset(s)
        a = emd.emd_topk(p, q.row_ptr, q.col, q.val, meas, k, "max", K)
        b = emd.emd_topk(s, q.row_ptr, q.col, q.val, meas, k, "max", K)
        np.testing.assert_array_equal(a[0], b[0], err_msg=f"{meas} k={k}")
        np.testing.assert_array_equal(a[1], b[1], err_msg=f"{meas} k={k}")
        pp, ps = emd.emd_db_profile_get(p), emd.emd_db_profile_get(s)
        assert pp["prune_fallbacks"] == ps["prune_fallbacks"] and pp["fused_retries"] == ps["fused_retries"]
    emd.emd_db_check_device_errors(p)


@pytest.mark.parametrize("tc_pair", PAIRS)
def test_pair_small_ragged(emd, tc_pair):
    """Embedding width 37 (one 64-wide K chunk), v_used a few thousand (a partial last row
    pair), query sizes 1..150 with ragged column tiles, batches of 1, 5 and 13 queries."""
    w = emd_synth.small_text(5150, 1500, 37, 900, 13, 1, 60, 1, 150)
    p, s = make(emd, w, tc_pair, max_query_h=256), make(emd, w, 0, max_query_h=256)
    try:
        assert emd.emd_db_info_get(p)["tc_pair"] == tc_pair
        assert emd.emd_db_info_get(s)["tc_pair"] == 0
        for nq in (1, 5, 13):
            compare(emd, p, s, w.queries.subset(np.arange(nq)), [("act", 3)], K=7)
    finally:
        emd.emd_db_destroy(p)
        emd.emd_db_destroy(s)


@pytest.mark.parametrize("tc_pair", PAIRS)
def test_pair_text(emd, tc_pair):
    """The text workload (V = 1e5, m = 300): every table width (k = 1..16), RWMD and OMR."""
    w = emd_synth.config(2, query_limit=40)
    p, s = make(emd, w, tc_pair, max_query_h=1024), make(emd, w, 0, max_query_h=1024)
    try:
        compare(emd, p, s, w.queries, [("act", 4), ("act", 1), ("act", 2), ("act", 8), ("act", 16), ("rwmd", 1),
                                       ("omr", 1)])
    finally:
        emd.emd_db_destroy(p)
        emd.emd_db_destroy(s)


@pytest.mark.parametrize("tc_pair", PAIRS)
def test_pair_mixed_sizes(emd, tc_pair):
    """Queries of h_q 5..2000 (up to 32 column tiles of 64), several sub-batches per call."""
    w = emd_synth.config(2, query_limit=1)
    q = emd_synth.mixed_queries(80)
    p = make(emd, w, tc_pair, max_query_h=2048, batch_columns=8192)
    s = make(emd, w, 0, max_query_h=2048, batch_columns=8192)
    try:
        compare(emd, p, s, q, [("act", 4)])
        compare(emd, p, s, q, [("act", 4)], K=5)
    finally:
        emd.emd_db_destroy(p)
        emd.emd_db_destroy(s)
