"""The serving entry points (emd_server_*): parity with the oracle, results that do not
depend on the mix of requests in flight, admission by workspace memory, queue limits and
argument checks.

Each request is the symmetric top-K (max of both directions, Section 6) with the same
kernel sequence as emd_topk, so a result served alone, served among many overlapping
requests, and returned by emd_topk must be bit-identical.
"""
import threading

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
    # query sizes 3..180 (several column tiles, ragged tails), documents 5..60 bins
    return emd_synth.small_text(20261203, 3000, 64, 2500, 40, 5, 60, 3, 180)


def make_db(emd, w, **opt):
    return emd.emd_db_create(w.emb, None, w.db.row_ptr, w.db.col, w.db.val,
                             emd.emd_db_options_default(**opt), v=w.v)


def serve_all(emd, srv, w, ids, meas, k, K):
    tickets = [emd.emd_server_submit(srv, *w.queries.row(i), meas=meas, k=k, K=K) for i in ids]
    out = []
    for t in tickets:
        oi = np.empty(K, np.int64)
        od = np.empty(K, np.float32)
        assert emd.emd_server_poll(srv, t, -1, oi, od)
        out.append((oi, od))
    return out


def serve_alone(emd, srv, w, ids, meas, k, K):
    out = []
    for i in ids:
        t = emd.emd_server_submit(srv, *w.queries.row(i), meas=meas, k=k, K=K)
        oi = np.empty(K, np.int64)
        od = np.empty(K, np.float32)
        assert emd.emd_server_poll(srv, t, -1, oi, od)
        out.append((oi, od))
    return out


@pytest.mark.parametrize("precision", ["fp32", "fp32_tc", "bf16", "fp8"])
def test_alone_equals_mix_equals_topk(emd, work, precision):
    w = work
    db = make_db(emd, w, precision=precision, max_query_h=256)
    srv = emd.emd_server_create(db, emd.emd_server_options_default(max_inflight=6))
    try:
        ids = list(range(w.queries.n))
        for meas, k, K in (("act", 4, 16), ("omr", 1, 10), ("act", 2, 32)):
            alone = serve_alone(emd, srv, w, ids, meas, k, K)
            mix = serve_all(emd, srv, w, ids, meas, k, K)
            ti, td = emd.emd_topk(db, w.queries.row_ptr, w.queries.col, w.queries.val, meas, k, "max", K)
            for i in ids:
                assert np.array_equal(alone[i][0], mix[i][0]) and np.array_equal(alone[i][1], mix[i][1])
                assert np.array_equal(mix[i][0], ti[i]) and np.array_equal(mix[i][1], td[i])
        st = emd.emd_server_stats_get(srv)
        assert st["failed"] == 0 and st["completed"] == st["submitted"] == 6 * w.queries.n
        assert st["max_in_flight"] > 1  # the mixed submissions overlapped on the device
    finally:
        emd.emd_server_destroy(srv)
        emd.emd_db_destroy(db)


def test_server_matches_oracle(emd, work):
    w = work
    db = make_db(emd, w, precision="fp32_tc", max_query_h=256)
    srv = emd.emd_server_create(db)
    try:
        ids = [0, 7, 19, 33]
        got = serve_all(emd, srv, w, ids, "act", 4, 16)
        for (gi, gd), qi in zip(got, ids):
            qidx, qw = w.queries.row(qi)
            tf, tr = oracle.lc_query(w.emb, None, w.db, qidx, qw, "act", 4)
            want = np.maximum(tf, tr)
            order = np.lexsort((np.arange(len(want)), want))
            dK = want[order[15]]
            tie = np.abs(want - dK) <= 1e-5 * dK + 1e-9
            assert {int(i) for i in order[:16] if not tie[i]} == {int(i) for i in gi if not tie[i]}
            np.testing.assert_allclose(gd, want[gi], rtol=RTOL, atol=ATOL)
    finally:
        emd.emd_server_destroy(srv)
        emd.emd_db_destroy(db)


def test_admission_by_workspace(emd, work):
    """Executors of 512 distance-matrix columns each (a few requests of the workload): every
    batch stays within its executor's columns, everything completes bit-identical to
    emd_topk, and a pool too small for one request is refused."""
    w = work
    db = make_db(emd, w, precision="fp32_tc", max_query_h=256)
    vu = emd.emd_db_info_get(db)["v_used"]
    col = 4 * vu
    with pytest.raises(emd.EmdError, match="INVALID_ARG"):
        emd.emd_server_create(db, emd.emd_server_options_default(workspace_bytes=2 * 128 * col))
    srv = emd.emd_server_create(db, emd.emd_server_options_default(workspace_bytes=2 * 512 * col))
    try:
        ids = list(range(w.queries.n))
        got = serve_all(emd, srv, w, ids, "act", 4, 16)
        ti, td = emd.emd_topk(db, w.queries.row_ptr, w.queries.col, w.queries.val, "act", 4, "max", 16)
        for i in ids:
            assert np.array_equal(got[i][0], ti[i]) and np.array_equal(got[i][1], td[i])
        st = emd.emd_server_stats_get(srv)
        assert st["completed"] == len(ids) and st["failed"] == 0
        assert st["pool_bytes"] == 2 * 512 * col
        assert 0 < st["pool_used_max"] <= 512 * col
        assert st["max_in_flight"] >= 2
    finally:
        emd.emd_server_destroy(srv)
        emd.emd_db_destroy(db)


def test_queue_full_and_errors(emd, work):
    w = work
    db = make_db(emd, w, precision="fp32_tc", max_query_h=256)
    srv = emd.emd_server_create(db, emd.emd_server_options_default(max_inflight=1, queue_capacity=1))
    try:
        qidx, qw = w.queries.row(int(np.argmax(np.diff(w.queries.row_ptr))))
        tickets, busy = [], 0
        for _ in range(64):
            try:
                tickets.append(emd.emd_server_submit(srv, qidx, qw, "act", 4, 16))
            except emd.EmdError as e:
                assert e.name == "BUSY"
                busy += 1
        assert busy >= 1 and len(tickets) >= 1
        oi, od = np.empty(16, np.int64), np.empty(16, np.float32)
        ref = None
        for t in tickets:
            assert emd.emd_server_poll(srv, t, -1, oi, od)
            ref = (oi.copy(), od.copy()) if ref is None else ref
            assert np.array_equal(oi, ref[0]) and np.array_equal(od, ref[1])
        assert emd.emd_server_stats_get(srv)["rejected_busy"] == busy
        # collected tickets and unknown tickets are invalid
        with pytest.raises(emd.EmdError, match="INVALID_ARG"):
            emd.emd_server_poll(srv, tickets[0], 0, oi, od)
        bad = [(qidx, qw * 2, "act", 4, 16),                    # weights do not sum to 1
               (np.array([1, 1], np.int32), np.array([.5, .5], np.float32), "act", 4, 16),  # repeated id
               (np.array([w.v], np.int32), np.array([1.], np.float32), "act", 4, 16),       # id out of range
               (qidx, qw, "act", 0, 16),                        # k < 1
               (qidx, qw, "act", 4, 65)]                        # K above 64
        for a in bad:
            with pytest.raises(emd.EmdError, match="INVALID_ARG"):
                emd.emd_server_submit(srv, *a)
        with pytest.raises(emd.EmdError, match="BUSY"):
            emd.emd_db_destroy(db)  # a server is attached
    finally:
        emd.emd_server_destroy(srv)
        emd.emd_db_destroy(db)


def test_concurrent_clients_and_drain(emd, work):
    """Several host threads submit and poll at once; destroy with requests still queued
    finishes them without error."""
    w = work
    db = make_db(emd, w, precision="fp32_tc", max_query_h=256)
    srv = emd.emd_server_create(db, emd.emd_server_options_default(max_inflight=4))
    ti, td = emd.emd_topk(db, w.queries.row_ptr, w.queries.col, w.queries.val, "act", 4, "max", 16)
    errors = []

    def client(ids):
        try:
            for i in ids:
                t = emd.emd_server_submit(srv, *w.queries.row(i), meas="act", k=4, K=16)
                oi, od = np.empty(16, np.int64), np.empty(16, np.float32)
                assert emd.emd_server_poll(srv, t, -1, oi, od)
                assert np.array_equal(oi, ti[i]) and np.array_equal(od, td[i])
        except Exception as e:  # noqa: BLE001
            errors.append(e)

    threads = [threading.Thread(target=client, args=(list(range(c, w.queries.n, 4)),)) for c in range(4)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    assert not errors
    for i in range(w.queries.n):
        emd.emd_server_submit(srv, *w.queries.row(i), meas="act", k=4, K=16)
    emd.emd_server_destroy(srv)  # drains the requests just queued
    emd.emd_db_check_device_errors(db)
    emd.emd_db_destroy(db)
