"""Pins for the oracle's two Section 6 baselines (bag-of-words cosine similarity, word
centroid distance) against facts that do not come from the oracle:
  * BoW: scipy's cosine distance on dense weight vectors, p = q gives 1, disjoint supports
    give 0, invariance to scaling the weights, a hand-computed value;
  * WCD: one-bin histograms give the Euclidean distance of the two embedding vectors,
    WCD <= EMD (the centroid difference is the flow-weighted sum of displacements; the
    norm of a sum is at most the sum of norms) with EMD from an independent LP solver,
    invariance to translating every embedding, a hand-computed 1-D value.
"""
import types

import numpy as np
import pytest
from scipy.optimize import linprog
from scipy.spatial.distance import cosine as scipy_cosine

import oracle


def csr(rows):
    """[(ids, weights), ...] -> an object with row_ptr / col / val."""
    rp = np.zeros(len(rows) + 1, np.int64)
    for i, (ids, _) in enumerate(rows):
        rp[i + 1] = rp[i] + len(ids)
    col = np.concatenate([np.asarray(r[0], np.int32) for r in rows]) if rows else np.zeros(0, np.int32)
    val = np.concatenate([np.asarray(r[1], np.float32) for r in rows]) if rows else np.zeros(0, np.float32)
    return types.SimpleNamespace(row_ptr=rp, col=col, val=val)


def random_hist(rng, v, lo, hi):
    h = int(rng.integers(lo, hi + 1))
    ids = np.sort(rng.choice(v, h, replace=False)).astype(np.int32)
    w = rng.random(h).astype(np.float32) + np.float32(0.05)
    return ids, (w / w.sum()).astype(np.float32)


def dense(v, ids, w):
    x = np.zeros(v)
    x[ids] = np.asarray(w, np.float64)
    return x


# ----------------------------------------------------------------------- pins as predicates
# (also run against mutated copies of the oracle in test_oracle_mutations)

def lp_emd(C, p, q):
    hp, hq = C.shape
    A, b = [], []
    for i in range(hp):
        r = np.zeros(hp * hq); r[i * hq:(i + 1) * hq] = 1; A.append(r); b.append(p[i])
    for j in range(hq):
        r = np.zeros(hp * hq); r[j::hq] = 1; A.append(r); b.append(q[j])
    res = linprog(C.ravel(), A_eq=np.array(A), b_eq=np.array(b), bounds=[(0, None)] * (hp * hq), method="highs")
    assert res.status == 0
    return res.fun


def bow_scipy_pin(bow) -> bool:
    rng = np.random.default_rng(11)
    v = 60
    rows = [random_hist(rng, v, 1, 20) for _ in range(40)]
    db = csr(rows)
    for _ in range(10):
        qi, qw = random_hist(rng, v, 1, 25)
        got = bow(v, db, qi, qw)
        for d, (ids, w) in enumerate(rows):
            want = 1.0 - scipy_cosine(dense(v, ids, w), dense(v, qi, qw))
            if abs(got[d] - want) > 1e-12:
                return False
    return True


def bow_special_pins(bow) -> bool:
    v = 10
    db = csr([([1, 4, 7], [0.2, 0.3, 0.5]), ([0, 2], [0.5, 0.5]), ([0, 1], [0.5, 0.5])])
    got = bow(v, db, np.array([1, 4, 7], np.int32), np.array([0.2, 0.3, 0.5], np.float32))
    if not (abs(got[0] - 1.0) <= 1e-12 and got[1] == 0.0):
        return False
    # hand value: p = (1/2, 1/2) on ids {0, 1}, q = 1 on id 0: (1/2) / (1/sqrt(2) * 1) = 1/sqrt(2)
    got = bow(v, db, np.array([0], np.int32), np.array([1.0], np.float32))
    if abs(got[2] - 2 ** -0.5) > 1e-12:
        return False
    # scaling the query weights changes nothing
    a = bow(v, db, np.array([0, 1], np.int32), np.array([0.25, 0.75], np.float32))
    b = bow(v, db, np.array([0, 1], np.int32), np.array([0.5, 1.5], np.float32))
    return bool(np.allclose(a, b, rtol=1e-12, atol=0))


def wcd_one_bin_pin(wcd) -> bool:
    rng = np.random.default_rng(5)
    emb = rng.standard_normal((30, 7)).astype(np.float32)
    db = csr([([u], [1.0]) for u in range(30)])
    got = wcd(emb, db, np.array([4], np.int32), np.array([1.0], np.float32))
    want = np.linalg.norm(emb.astype(np.float64) - emb[4].astype(np.float64), axis=1)
    return bool(np.allclose(got, want, rtol=1e-12, atol=1e-15) and got[4] == 0.0)


def wcd_emd_bound_pin(wcd) -> bool:
    rng = np.random.default_rng(6)
    v, m = 40, 5
    emb = rng.standard_normal((v, m)).astype(np.float32)
    rows = [random_hist(rng, v, 1, 8) for _ in range(25)]
    db = csr(rows)
    for _ in range(6):
        qi, qw = random_hist(rng, v, 1, 8)
        got = wcd(emb, db, qi, qw)
        for d, (ids, w) in enumerate(rows):
            C = np.linalg.norm(emb[ids][:, None, :].astype(np.float64) - emb[qi][None, :, :].astype(np.float64), axis=2)
            pw, qq = np.asarray(w, np.float64), np.asarray(qw, np.float64)
            if got[d] > lp_emd(C, pw / pw.sum(), qq / qq.sum()) + 1e-7:
                return False
    return True


def wcd_translation_and_hand_pins(wcd) -> bool:
    rng = np.random.default_rng(7)
    v, m = 25, 6
    emb = rng.standard_normal((v, m)).astype(np.float32)
    rows = [random_hist(rng, v, 1, 6) for _ in range(12)]
    db = csr(rows)
    qi, qw = random_hist(rng, v, 1, 6)
    a = wcd(emb, db, qi, qw)
    b = wcd(emb + np.float32(3.0), db, qi, qw)
    if not np.allclose(a, b, rtol=1e-5, atol=1e-6):
        return False
    # 1-D: coordinates 0, 1, 3; p = (1/2, 1/2) on {0, 1} has centroid 1/2, q = 1 on {2} has 3
    emb1 = np.array([[0.0], [1.0], [3.0]], np.float32)
    got = wcd(emb1, csr([([0, 1], [0.5, 0.5])]), np.array([2], np.int32), np.array([1.0], np.float32))
    return abs(got[0] - 2.5) <= 1e-12


BOW_PINS = (bow_scipy_pin, bow_special_pins)
WCD_PINS = (wcd_one_bin_pin, wcd_emd_bound_pin, wcd_translation_and_hand_pins)


# ----------------------------------------------------------------------- the oracle passes them

@pytest.mark.parametrize("pin", BOW_PINS, ids=lambda f: f.__name__)
def test_bow_pins(pin):
    assert pin(oracle.bow_cosine)


@pytest.mark.parametrize("pin", WCD_PINS, ids=lambda f: f.__name__)
def test_wcd_pins(pin):
    assert pin(oracle.wcd)
