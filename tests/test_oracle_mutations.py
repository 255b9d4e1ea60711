"""The pins catch plausible mistakes: each case below plants one mistake in a private
copy of the oracle source (compiled on the CPU into a temporary library) and checks that
a pin from test_oracle_pins / test_oracle_lc then fails."""
import ctypes
import os
import subprocess

import numpy as np
import pytest

import emd_synth
import oracle
from test_oracle_baselines import BOW_PINS, WCD_PINS
from test_oracle_pins import CASES, lp, nearest_mask, random_pair

SRC = os.path.join(os.path.dirname(oracle.__file__), "emd_oracle.c")

MUTATIONS = {
    "drop_phase3_remainder": ("if (pi != 0.0) t = t + pi * Ci[s[keff - 1]];", "if (pi != 0.0) t = t;"),
    "cost_at_kth_not_lth": ("t = t + r * Ci[s[l]]; /* R1 */", "t = t + r * Ci[s[keff - 1]]; /* R1 */"),
    "capacity_unsorted_index": ("double r = fmin(pi, q[s[l]]);\n            pi = pi - r;\n            t = t + r * Ci[s[l]]; /* R1 */",
                                "double r = fmin(pi, q[l]);\n            pi = pi - r;\n            t = t + r * Ci[s[l]]; /* R1 */"),
    "omr_rest_to_nearest": ("if (hq > 1) t = t + pi * Ci[s[1]];", "if (hq > 1) t = t + pi * Ci[s[0]];"),
    "ict_stops_early": ("while (pi > 0.0 && l < hq) {", "while (pi > 0.0 && l < hq - 1) {"),
    "emd_backward_arc_sign": ("double nd = dist[hp + j] - C[(int64_t)i * hq + j];",
                              "double nd = dist[hp + j] + C[(int64_t)i * hq + j];"),
    "lc_phase2_first_column": ("double y = fmin(X[e], W[u * kk + l]);", "double y = fmin(X[e], W[u * kk]);"),
    "lc_rev_gather_shifted": ("for (int32_t j = 0; j < hq; ++j) CT[(int64_t)j * hd + i] = Du[j];",
                              "for (int32_t j = 0; j < hq; ++j) CT[(int64_t)j * hd + i] = Du[(j + 1) % hq];"),
}


def build_mutant(tmp_path, name):
    """The oracle source with one mistake planted wherever the mutated line occurs (the LC
    steps appear both in oracle_lc_query and in its split forms)."""
    old, new = MUTATIONS[name]
    src = open(SRC).read()
    assert src.count(old) >= 1, name
    path = tmp_path / f"{name}.c"
    path.write_text(src.replace(old, new))
    so = tmp_path / f"lib{name}.so"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", str(so), str(path), "-lm"])
    L = ctypes.CDLL(str(so))
    P, i32, i64, dbl = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
    L.oracle_measure.argtypes = [i32, P, i32, P, i32, P, i32]
    L.oracle_measure.restype = dbl
    L.oracle_emd.argtypes = [P, i32, P, i32, P]
    L.oracle_emd.restype = dbl
    L.oracle_lc_query.argtypes = [P, i32, P, i64, P, P, P, i64, P, P, i32, i32, i32, P, P]
    L.oracle_lc_query.restype = i32
    return L


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def pair_pins_pass(L):
    """True when the mutant passes every pairwise LP pin."""
    for hp, hq, ov, seed in CASES:
        p, q, C = random_pair(np.random.default_rng(seed), hp, hq, ov)
        p, q, C = (np.ascontiguousarray(x, dtype=np.float64) for x in (p, q, C))
        def meas(code, k=1):
            return L.oracle_measure(code, _p(p), hp, _p(q), hq, _p(C), k)
        checks = [(meas(1), lp(C, p, q, C == 0.0)), (meas(3), lp(C, p, q, np.ones_like(C, bool))),
                  (L.oracle_emd(_p(p), hp, _p(q), hq, _p(C)), lp(C, p, q, inflow=True))]
        for k in (2, 3, 5):
            checks.append((meas(2, k), lp(C, p, q, nearest_mask(C, min(k, hq) - 1))))
        for got, want in checks:
            if abs(got - want) > 1e-9 * max(1.0, abs(want)):
                return False
    return True


def lc_pins_pass(L, w):
    for qi in range(w.queries.n):
        qidx, qw = w.queries.row(qi)
        for code, name, k in ((2, "act", 3), (1, "omr", 1)):
            pf, pr = oracle.pair_db(w.emb, None, w.db, qidx, qw, name, k)
            n = w.db.n
            lf, lr = np.empty(n), np.empty(n)
            qidx32 = np.ascontiguousarray(qidx, np.int32); qw32 = np.ascontiguousarray(qw, np.float32)
            L.oracle_lc_query(_p(w.emb), w.emb.shape[1], None, w.emb.shape[0], _p(w.db.row_ptr),
                              _p(w.db.col), _p(w.db.val), n, _p(qidx32), _p(qw32), len(qidx32),
                              code, k, _p(lf), _p(lr))
            if not (np.allclose(lf, pf, rtol=1e-12, atol=0) and np.allclose(lr, pr, rtol=1e-12, atol=0)):
                return False
    return True


def test_unmutated_oracle_passes(tmp_path):
    L = ctypes.CDLL(oracle.build())
    L.oracle_measure.argtypes = [ctypes.c_int32, ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p,
                                 ctypes.c_int32, ctypes.c_void_p, ctypes.c_int32]
    L.oracle_measure.restype = ctypes.c_double
    L.oracle_emd.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p]
    L.oracle_emd.restype = ctypes.c_double
    assert pair_pins_pass(L)


@pytest.mark.parametrize("name", [n for n in MUTATIONS if not n.startswith("lc_")])
def test_pairwise_mutation_is_caught(tmp_path, name):
    assert not pair_pins_pass(build_mutant(tmp_path, name))


@pytest.mark.parametrize("name", [n for n in MUTATIONS if n.startswith("lc_")])
def test_lc_mutation_is_caught(tmp_path, name):
    w = emd_synth.small_text(77, 300, 8, 40, 2, 3, 12)
    assert not lc_pins_pass(build_mutant(tmp_path, name), w)


BASELINE_MUTATIONS = {
    "bow_no_document_norm": ("out[d] = (qn > 0.0 && dn > 0.0) ? dot / (qn * dn) : 0.0;",
                             "out[d] = (qn > 0.0 && dn > 0.0) ? dot / qn : 0.0;"),
    "bow_unsquared_norm": ("dn += (double)val[e] * (double)val[e];", "dn += (double)val[e];"),
    "bow_query_weight_index": ("dense[q_idx[j]] = (double)q_w[j];", "dense[q_idx[j]] = (double)q_w[0];"),
    "wcd_sum_not_difference": ("const double diff = cd[i] / sd - cq[i];", "const double diff = cd[i] / sd + cq[i];"),
    "wcd_query_row_shifted": ("cq[i] += (double)q_w[j] * (double)emb[(int64_t)q_idx[j] * m + i];",
                              "cq[i] += (double)q_w[j] * (double)emb[(int64_t)q_idx[j] * m + (i + 1) % m];"),
    "wcd_no_root": ("out[d] = sqrt(s);", "out[d] = s;"),
}


def build_baseline_mutant(tmp_path, name):
    old, new = BASELINE_MUTATIONS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, name
    path = tmp_path / f"{name}.c"
    path.write_text(src.replace(old, new))
    so = tmp_path / f"lib{name}.so"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", str(so), str(path), "-lm"])
    L = ctypes.CDLL(str(so))
    P, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
    L.oracle_bow_db.argtypes = [i64, P, P, P, i64, P, P, i32, P]
    L.oracle_bow_db.restype = i32
    L.oracle_wcd_db.argtypes = [P, i32, P, P, P, i64, P, P, i32, P]
    L.oracle_wcd_db.restype = i32

    def bow(v, db, qi, qw):
        rp = np.ascontiguousarray(db.row_ptr, np.int64)
        col = np.ascontiguousarray(db.col, np.int32)
        val = np.ascontiguousarray(db.val, np.float32)
        qi = np.ascontiguousarray(qi, np.int32)
        qw = np.ascontiguousarray(qw, np.float32)
        out = np.empty(len(rp) - 1)
        L.oracle_bow_db(int(v), _p(rp), _p(col), _p(val), len(rp) - 1, _p(qi), _p(qw), len(qi), _p(out))
        return out

    def wcd(emb, db, qi, qw):
        emb = np.ascontiguousarray(emb, np.float32)
        rp = np.ascontiguousarray(db.row_ptr, np.int64)
        col = np.ascontiguousarray(db.col, np.int32)
        val = np.ascontiguousarray(db.val, np.float32)
        qi = np.ascontiguousarray(qi, np.int32)
        qw = np.ascontiguousarray(qw, np.float32)
        out = np.empty(len(rp) - 1)
        L.oracle_wcd_db(_p(emb), emb.shape[1], _p(rp), _p(col), _p(val), len(rp) - 1, _p(qi), _p(qw), len(qi),
                        _p(out))
        return out

    return bow, wcd


@pytest.mark.parametrize("name", list(BASELINE_MUTATIONS))
def test_baseline_mutation_is_caught(tmp_path, name):
    bow, wcd = build_baseline_mutant(tmp_path, name)
    if name.startswith("bow_"):
        assert not all(pin(bow) for pin in BOW_PINS)
    else:
        assert not all(pin(wcd) for pin in WCD_PINS)
