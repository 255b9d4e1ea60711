"""Pins for the FP64 oracle against facts fixed by the paper and by mathematics, not by
the oracle itself:
  * linear-programming optima (scipy HiGHS, an independent solver) of the constrained
    problems that Thm. 1 and Lemma A.2 say Algorithms 2 and 3 solve exactly, and of the
    out-flow-only relaxation of Section 2.1 (RWMD);
  * EMD (Eq. 1-3) against the LP and, in one dimension, against the closed form
    integral |F_p - F_q|;
  * hand-derived worked examples (tests/golden/worked_examples.json);
  * special cases (k = 1 is RWMD, k >= h is ICT, h_q = 1 forces every flow, p = q gives 0)
    and the ordering of Thm. 2, monotonicity in k, and effectiveness (Appendix A).
"""
import json
import os

import numpy as np
import pytest
from scipy.optimize import linprog

import oracle

GOLD = os.path.join(os.path.dirname(__file__), "golden", "worked_examples.json")


def lp(C, p, q, cap_mask=None, inflow=False):
    """min sum F*C s.t. sum_j F_ij = p_i (Eq. 2), F >= 0, optionally F_ij <= q_j where
    cap_mask[i, j] (Eq. 4 imposed selectively) and optionally sum_i F_ij = q_j (Eq. 3)."""
    hp, hq = C.shape
    A_eq, b_eq = [], []
    for i in range(hp):
        r = np.zeros(hp * hq); r[i * hq:(i + 1) * hq] = 1; A_eq.append(r); b_eq.append(p[i])
    if inflow:
        for j in range(hq):
            r = np.zeros(hp * hq); r[j::hq] = 1; A_eq.append(r); b_eq.append(q[j])
    bounds = []
    for i in range(hp):
        for j in range(hq):
            ub = q[j] if (cap_mask is not None and cap_mask[i, j]) else None
            bounds.append((0.0, ub))
    res = linprog(C.ravel(), A_eq=np.array(A_eq), b_eq=np.array(b_eq), bounds=bounds,
                  method="highs")
    assert res.status == 0, res.message
    return res.fun


def random_pair(rng, hp, hq, overlap=0, m=3):
    """Histograms over Euclidean coordinates; the first `overlap` bins of p and q share
    their coordinates (zero ground cost)."""
    P = rng.standard_normal((hp, m))
    Q = rng.standard_normal((hq, m))
    o = min(overlap, hp, hq)
    Q[:o] = P[:o]
    C = np.sqrt(((P[:, None, :] - Q[None, :, :]) ** 2).sum(-1))
    C[np.arange(o), np.arange(o)] = 0.0
    p = rng.random(hp) + 0.05; p /= p.sum()
    q = rng.random(hq) + 0.05; q /= q.sum()
    return p, q, C


def nearest_mask(C, count):
    """mask of the `count` nearest destinations of each row (ties by position)."""
    hp, hq = C.shape
    mask = np.zeros_like(C, dtype=bool)
    for i in range(hp):
        order = np.lexsort((np.arange(hq), C[i]))
        mask[i, order[:count]] = True
    return mask


CASES = [(hp, hq, ov, seed) for seed, (hp, hq, ov) in enumerate(
    [(1, 1, 0), (1, 4, 0), (4, 1, 0), (3, 3, 0), (3, 3, 3), (5, 7, 2), (7, 5, 4), (8, 8, 8),
     (6, 2, 1), (2, 6, 2), (9, 4, 3), (4, 9, 0)])]


@pytest.mark.parametrize("hp,hq,ov,seed", CASES)
def test_emd_equals_transport_lp(hp, hq, ov, seed):
    p, q, C = random_pair(np.random.default_rng(seed), hp, hq, ov)
    assert oracle.emd(p, q, C) == pytest.approx(lp(C, p, q, inflow=True), rel=1e-9, abs=1e-12)


@pytest.mark.parametrize("seed", range(6))
def test_emd_one_dimensional_closed_form(seed):
    rng = np.random.default_rng(100 + seed)
    hp, hq = rng.integers(1, 9, 2)
    x = np.sort(rng.random(hp) * 10)
    y = np.sort(rng.random(hq) * 10)
    p = rng.random(hp) + 0.1; p /= p.sum()
    q = rng.random(hq) + 0.1; q /= q.sum()
    C = np.abs(x[:, None] - y[None, :])
    pts = np.sort(np.concatenate([x, y]))
    Fp = np.array([p[x <= t].sum() for t in pts[:-1]])
    Fq = np.array([q[y <= t].sum() for t in pts[:-1]])
    closed = float((np.abs(Fp - Fq) * np.diff(pts)).sum())
    assert oracle.emd(p, q, C) == pytest.approx(closed, rel=1e-9, abs=1e-12)


@pytest.mark.parametrize("hp,hq,ov,seed", CASES)
def test_ict_is_optimum_of_relaxed_problem(hp, hq, ov, seed):
    """Thm. 1 (i): ICT solves {Eq. 1, Eq. 2, Eq. 4 on all edges}."""
    p, q, C = random_pair(np.random.default_rng(seed), hp, hq, ov)
    assert oracle.ict(p, q, C) == pytest.approx(lp(C, p, q, np.ones_like(C, bool)), rel=1e-9, abs=1e-12)


@pytest.mark.parametrize("hp,hq,ov,seed", CASES)
@pytest.mark.parametrize("k", [1, 2, 3, 5, 12])
def test_act_is_optimum_with_k_minus_1_capped_edges(hp, hq, ov, seed, k):
    """Lemma A.2: ACT_k solves Eq. 1-2 with Eq. 4 imposed on each row's k-1 nearest."""
    p, q, C = random_pair(np.random.default_rng(seed), hp, hq, ov)
    keff = min(k, hq)
    mask = nearest_mask(C, keff - 1)
    assert oracle.act(p, q, C, k) == pytest.approx(lp(C, p, q, mask), rel=1e-9, abs=1e-12)


@pytest.mark.parametrize("hp,hq,ov,seed", CASES)
def test_rwmd_is_outflow_only_optimum(hp, hq, ov, seed):
    """Section 2.1: dropping the in-flow constraints leaves Eq. 1-2."""
    p, q, C = random_pair(np.random.default_rng(seed), hp, hq, ov)
    want = lp(C, p, q)
    assert oracle.rwmd(p, q, C) == pytest.approx(want, rel=1e-9, abs=1e-12)
    assert oracle.act(p, q, C, 1) == pytest.approx(want, rel=1e-9, abs=1e-12)


@pytest.mark.parametrize("hp,hq,ov,seed", CASES)
def test_omr_is_optimum_with_overlap_edges_capped(hp, hq, ov, seed):
    """Section 4.1: OMR imposes Eq. 4 only between overlapping coordinates (C = 0)."""
    p, q, C = random_pair(np.random.default_rng(seed), hp, hq, ov)
    assert oracle.omr(p, q, C) == pytest.approx(lp(C, p, q, C == 0.0), rel=1e-9, abs=1e-12)


@pytest.mark.parametrize("ex", json.load(open(GOLD))["examples"], ids=lambda e: e["name"])
def test_worked_examples(ex):
    p, q, C = np.array(ex["p"]), np.array(ex["q"]), np.array(ex["C"])
    got = {"rwmd": oracle.rwmd(p, q, C), "omr": oracle.omr(p, q, C),
           "act1": oracle.act(p, q, C, 1), "act2": oracle.act(p, q, C, 2),
           "act3": oracle.act(p, q, C, 3), "ict": oracle.ict(p, q, C), "emd": oracle.emd(p, q, C)}
    for key, want in ex["expect"].items():
        assert got[key] == pytest.approx(want, abs=1e-12), key
    if "expect_rev" in ex:
        CT = C.T.copy()
        rev = {"rwmd": oracle.rwmd(q, p, CT), "omr": oracle.omr(q, p, CT),
               "act1": oracle.act(q, p, CT, 1), "act2": oracle.act(q, p, CT, 2),
               "act3": oracle.act(q, p, CT, 3), "ict": oracle.ict(q, p, CT), "emd": oracle.emd(q, p, CT)}
        for key, want in ex["expect_rev"].items():
            assert rev[key] == pytest.approx(want, abs=1e-12), key


@pytest.mark.parametrize("seed", range(40))
def test_ordering_theorem_2(seed):
    rng = np.random.default_rng(1000 + seed)
    hp, hq = rng.integers(1, 10, 2)
    p, q, C = random_pair(rng, hp, hq, overlap=int(rng.integers(0, 6)))
    r, o, i, e = oracle.rwmd(p, q, C), oracle.omr(p, q, C), oracle.ict(p, q, C), oracle.emd(p, q, C)
    acts = [oracle.act(p, q, C, k) for k in range(1, hq + 2)]
    tol = 1e-12
    assert r <= o + tol
    for k, a in enumerate(acts, start=1):
        if k >= 2:
            assert o <= a + tol
        assert a <= i + tol
    assert all(acts[j] <= acts[j + 1] + tol for j in range(len(acts) - 1))
    assert i <= e + tol
    assert acts[0] == pytest.approx(r, abs=1e-15)
    assert acts[-1] == pytest.approx(i, rel=1e-12, abs=1e-15)


@pytest.mark.parametrize("seed", range(5))
def test_single_destination_forces_every_flow(seed):
    rng = np.random.default_rng(2000 + seed)
    p, _, C = random_pair(rng, int(rng.integers(1, 8)), 1)
    q = np.array([1.0])
    want = float((p * C[:, 0]).sum())
    for val in (oracle.rwmd(p, q, C), oracle.omr(p, q, C), oracle.ict(p, q, C), oracle.emd(p, q, C),
                oracle.act(p, q, C, 1), oracle.act(p, q, C, 4)):
        assert val == pytest.approx(want, rel=1e-12)


@pytest.mark.parametrize("seed", range(5))
def test_identical_histograms_are_at_distance_zero(seed):
    rng = np.random.default_rng(3000 + seed)
    h = int(rng.integers(1, 9))
    p, _, C = random_pair(rng, h, h, overlap=h)
    for val in (oracle.rwmd(p, p, C), oracle.omr(p, p, C), oracle.ict(p, p, C), oracle.emd(p, p, C),
                oracle.act(p, p, C, 2), oracle.act(p, p, C, 5)):
        assert val == pytest.approx(0.0, abs=1e-15)


@pytest.mark.parametrize("seed", range(8))
def test_effectiveness_omr_versus_rwmd(seed):
    """Appendix A: with an effective cost, OMR = 0 only for p = q; RWMD is 0 whenever the
    supports coincide (Section 4, Table 5)."""
    rng = np.random.default_rng(4000 + seed)
    h = int(rng.integers(2, 9))
    p, q, C = random_pair(rng, h, h, overlap=h)
    assert not np.allclose(p, q)
    assert oracle.rwmd(p, q, C) == 0.0
    assert oracle.omr(p, q, C) > 1e-6
    assert oracle.act(p, q, C, 3) >= oracle.omr(p, q, C)
