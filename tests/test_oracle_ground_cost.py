"""Pins for the oracle's ground cost (Section 6: the Euclidean distance between two
embedding vectors; Section 2: the h_p x h_q cost block between the bins of two
histograms; cost-matrix mode: the given matrix itself), against references that do not
share the oracle's code:
  * scipy.spatial.distance.cdist on the same FP32 rows promoted to FP64;
  * hand-derived values (a 3-4-5 right triangle, one-dimensional coordinates);
  * an asymmetric cost matrix read back element by element with numpy indexing.
A planted mistake in the oracle's ground cost (square root dropped, FP32 accumulation, a
transposed block, a wrong row stride or a transposed cost-matrix index) must fail one of
these pins (test_ground_cost_mutation_is_caught).
"""
import ctypes
import os
import subprocess

import numpy as np
import pytest
from scipy.spatial.distance import cdist

import oracle

SRC = os.path.join(os.path.dirname(oracle.__file__), "emd_oracle.c")


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _block(fn, emb, cost, ia, ib):
    """Calls an oracle_cost_block implementation (the oracle's or a mutant's)."""
    ia = np.ascontiguousarray(ia, np.int32)
    ib = np.ascontiguousarray(ib, np.int32)
    if cost is not None:
        cost = np.ascontiguousarray(cost, np.float32)
        v, m = cost.shape[0], 0
    else:
        emb = np.ascontiguousarray(emb, np.float32)
        v, m = emb.shape
    out = np.empty((len(ia), len(ib)))
    fn(_p(emb), m, _p(cost), v, _p(ia), len(ia), _p(ib), len(ib), _p(out))
    return out


def _oracle_fn():
    return oracle.lib().oracle_cost_block


def pin_cdist(fn):
    """Unit-norm FP32 embeddings (the text workloads' law), a non-square block with
    repeated and shuffled ids: equal to cdist on the FP64 promotion of the same rows."""
    rng = np.random.default_rng(5)
    x = rng.standard_normal((50, 37))
    emb = (x / np.linalg.norm(x, axis=1, keepdims=True)).astype(np.float32)
    ia = rng.integers(0, 50, 13)
    ib = rng.integers(0, 50, 29)
    got = _block(fn, emb, None, ia, ib)
    want = cdist(emb[ia].astype(np.float64), emb[ib].astype(np.float64))
    return got.shape == want.shape and np.allclose(got, want, rtol=1e-15, atol=0.0)


def pin_wide_rows(fn):
    """Embeddings of width 300 with entries of mixed magnitude: FP32 accumulation of the
    squared differences would be off by ~1e-7 relative."""
    rng = np.random.default_rng(9)
    emb = (rng.standard_normal((20, 300)) * rng.uniform(0.01, 100.0, (20, 1))).astype(np.float32)
    ia, ib = np.arange(0, 20, 2), np.arange(1, 20, 3)
    got = _block(fn, emb, None, ia, ib)
    want = cdist(emb[ia].astype(np.float64), emb[ib].astype(np.float64))
    return np.allclose(got, want, rtol=1e-15, atol=0.0)


def pin_345(fn):
    """Coordinates (0,0), (3,4), (6,8), (3,0): distances 5, 10, 5, 3, 4, 5 by hand."""
    emb = np.array([[0, 0], [3, 4], [6, 8], [3, 0]], np.float32)
    got = _block(fn, emb, None, [0, 1, 3], [1, 2, 0])
    want = np.array([[5.0, 10.0, 0.0],
                     [0.0, 5.0, 5.0],
                     [4.0, np.sqrt(73.0), 3.0]])  # (3,0)-(6,8): sqrt(3^2 + 8^2)
    return np.array_equal(got, want)


def pin_one_dimension(fn):
    """m = 1: the distance is |a - b|, exactly (differences of small integers)."""
    emb = np.array([[-2.0], [0.5], [7.0], [1.25]], np.float32)
    got = _block(fn, emb, None, [3, 0, 2], [1, 2])
    want = np.abs(emb[[3, 0, 2]].astype(np.float64) - emb[[1, 2]].astype(np.float64).T)
    return np.array_equal(got, want)


def pin_cost_matrix(fn):
    """Cost-matrix mode reads C[ia[i], ib[j]] of the given (here asymmetric) matrix."""
    rng = np.random.default_rng(3)
    C = rng.uniform(0.0, 5.0, (9, 9)).astype(np.float32)
    np.fill_diagonal(C, 0.0)
    ia, ib = [4, 0, 8, 2], [1, 7, 3]
    got = _block(fn, None, C, ia, ib)
    want = C[np.ix_(ia, ib)].astype(np.float64)
    return np.array_equal(got, want)


PINS = [pin_cdist, pin_wide_rows, pin_345, pin_one_dimension, pin_cost_matrix]


@pytest.mark.parametrize("pin", PINS, ids=[p.__name__ for p in PINS])
def test_ground_cost_pin(pin):
    assert pin(_oracle_fn())


def test_cost_block_wrapper_matches_cdist():
    rng = np.random.default_rng(11)
    emb = rng.standard_normal((30, 64)).astype(np.float32)
    ia, ib = rng.integers(0, 30, 7), rng.integers(0, 30, 5)
    np.testing.assert_allclose(oracle.cost_block(emb, None, ia, ib),
                               cdist(emb[ia].astype(np.float64), emb[ib].astype(np.float64)), rtol=1e-15, atol=0)


MUTATIONS = {
    "euclid_no_sqrt": ("    return sqrt(s);\n}", "    return s;\n}"),
    "euclid_fp32_accumulation": ("    double s = 0.0;\n    for (int32_t i = 0; i < m; ++i) {\n        double d = (double)a[i] - (double)b[i];",
                                 "    float s = 0.0f;\n    for (int32_t i = 0; i < m; ++i) {\n        double d = (double)a[i] - (double)b[i];"),
    "euclid_drops_last_dimension": ("for (int32_t i = 0; i < m; ++i) {\n        double d = (double)a[i] - (double)b[i];",
                                    "for (int32_t i = 0; i + 1 < m; ++i) {\n        double d = (double)a[i] - (double)b[i];"),
    "row_stride_off_by_one": ("return euclid(emb + (int64_t)a * m, emb + (int64_t)b * m, m);",
                              "return euclid(emb + (int64_t)a * (m > 1 ? m - 1 : m), emb + (int64_t)b * m, m);"),
    "cost_matrix_transposed": ("if (cost) return (double)cost[(int64_t)a * v + b];",
                               "if (cost) return (double)cost[(int64_t)b * v + a];"),
    "block_transposed": ("C[(int64_t)i * hb + j] = ground_cost(emb, m, cost, v, ia[i], ib[j]);",
                         "C[(int64_t)j * ha + i] = ground_cost(emb, m, cost, v, ia[i], ib[j]);"),
}


def build_mutant(tmp_path, name):
    old, new = MUTATIONS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, name
    path = tmp_path / f"{name}.c"
    path.write_text(src.replace(old, new))
    so = tmp_path / f"lib{name}.so"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fno-fast-math", "-ffp-contract=off",
                           "-o", str(so), str(path), "-lm"])
    L = ctypes.CDLL(str(so))
    P, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
    L.oracle_cost_block.argtypes = [P, i32, P, i64, P, i32, P, i32, P]
    L.oracle_cost_block.restype = None
    return L.oracle_cost_block


@pytest.mark.parametrize("name", list(MUTATIONS))
def test_ground_cost_mutation_is_caught(tmp_path, name):
    fn = build_mutant(tmp_path, name)
    assert not all(pin(fn) for pin in PINS)
